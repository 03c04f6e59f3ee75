"""GPU parity of the tensor-core forms (BF16 / FP8 tcgen05 GEMM with the quick
multi-select fused into its epilogue, exact re-rank, fallbacks) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from acceptance import check_exact, check_float
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def graph(X, k, precision="bf16", **kw):
    out = kb.knng_build(dev(X), k, precision=precision, fused=1, return_stats=True, **kw)
    torch.cuda.synchronize()
    return out[0].cpu().numpy(), out[1].cpu().numpy(), out[2]


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_integer_lattice_bit_exact(precision):
    X = inputs.integer_lattice(n=4096, d=128)
    idx, dist, st = graph(X, 16, precision)
    assert st["fused_used"] == 1
    check_exact(idx, dist, *oracle.knng(X, 16))


@pytest.mark.parametrize("n,d,k", [(1000, 37, 7), (300, 200, 64), (257, 64, 1), (5000, 130, 100)])
def test_integer_ragged_bit_exact(n, d, k):
    X = inputs.integer_lattice(n=n, d=d, lo=-6, hi=6, seed=200 + n)
    idx, dist, _ = graph(X, k)
    check_exact(idx, dist, *oracle.knng(X, k))


def test_gaussian_mixture_float():
    X = inputs.gaussian_mixture(n=6000, d=256, components=16)
    idx, dist, st = graph(X, 32)
    rows = inputs.sample_rows(len(X), 200, seed=1)
    ref_idx, ref_dist = oracle.knng(X, 32, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_unit_directions_with_duplicates():
    X, t, s = inputs.unit_directions_with_duplicates(n=20000, d=1024, seed=3)
    idx, dist, st = graph(X, 64)
    assert np.all(dist[t, 0] == 0.0) and np.array_equal(idx[t, 0], s)
    rows = np.concatenate([t[:10], inputs.sample_rows(len(X), 40, seed=5)])
    ref_idx, ref_dist = oracle.knng(X, 64, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_search_separate_sets():
    C = inputs.gaussian_mixture(n=7000, d=96, components=8, seed=5)
    Q = inputs.gaussian_mixture(n=333, d=96, components=8, seed=6)
    idx, dist, st = kb.knn_search(dev(Q), dev(C), 20, precision="bf16", fused=1, return_stats=True)
    ref_idx, ref_dist = oracle.knn(Q, C, 20)
    check_float(Q, C, np.arange(len(Q)), idx.cpu().numpy(), dist.cpu().numpy(), ref_idx, ref_dist, False)


def test_fused_matches_plain_exactly_on_float_data():
    X = inputs.anisotropic_mixture(n=5000, d=192, components=16, seed=8)
    a = graph(X, 24, "bf16")
    b = kb.knng_build(dev(X), 24, precision="fp32")
    # both forms are exact: identical answers (distances may differ only where FP64 decided)
    assert np.array_equal(a[0], b[0].cpu().numpy())
    assert np.allclose(a[1], b[1].cpu().numpy(), rtol=1e-6, atol=0)


def test_tight_threshold_goes_through_the_fallback():
    X = inputs.gaussian_mixture(n=4000, d=64, components=8, seed=13)
    base_i, base_d, _ = graph(X, 16)
    thr = (base_d[:, -1] * 0.5).astype(np.float32)  # too tight: every row misses
    i2, d2, st = graph(X, 16, row_threshold=dev(thr))
    assert st["threshold_misses"] > 0 and st["rows_fallback"] > 0
    assert np.array_equal(i2, base_i) and np.array_equal(d2, base_d)
    thr = (base_d[:, -1] * 1.2 + 1.0).astype(np.float32)  # loose: nothing lost
    i3, d3, st3 = graph(X, 16, row_threshold=dev(thr))
    assert np.array_equal(i3, base_i) and np.array_equal(d3, base_d)


def test_fp8_on_float_data_is_still_exact():
    X = inputs.gaussian_mixture(n=3000, d=128, components=8, seed=21)
    idx, dist, st = graph(X, 10, "fp8")
    ref_idx, ref_dist = oracle.knng(X, 10, rows=np.arange(100))
    check_float(X, X, np.arange(100), idx[:100], dist[:100], ref_idx, ref_dist, exclude_self=True)


@pytest.fixture
def fused_cap_override(monkeypatch):
    def set_cap(cap):
        monkeypatch.setenv("KNN_FUSED_CAP", str(cap))
    return set_cap


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_wide_lists_integer_bit_exact(precision, fused_cap_override):
    # lists of up to 1024 keys (32 per lane in the shrink), more stages traded for list room
    fused_cap_override(1024)
    X = inputs.integer_lattice(n=5000, d=130, lo=-6, hi=6, seed=61)
    idx, dist, st = graph(X, 40, precision)
    assert st["list_capacity"] == 1024 and st["fused_used"] == 1
    check_exact(idx, dist, *oracle.knng(X, 40))


def test_wide_lists_float(fused_cap_override):
    fused_cap_override(640)
    X = inputs.anisotropic_mixture(n=9000, d=200, components=12, seed=62)
    idx, dist, st = graph(X, 100)
    assert st["list_capacity"] == 640
    rows = inputs.sample_rows(len(X), 150, seed=63)
    ref_idx, ref_dist = oracle.knng(X, 100, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_band_probe_on_a_large_graph():
    # 2^34 pairs: the band of sampled rows sizes the lists before the fused launch
    X = inputs.anisotropic_mixture(n=131072, d=256, components=256, seed=64)
    idx, dist, st = graph(X, 100)
    assert 448 <= st["list_capacity"] <= 1024
    assert st["rows_fallback"] <= 0.02 * len(X), st
    rows = inputs.sample_rows(len(X), 64, seed=65)
    ref_idx, ref_dist = oracle.knng(X, 100, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_crowded_band_goes_through_every_fallback():
    # points close together far from the origin: the reduced-precision error bound dwarfs
    # the distances, every band holds the whole set, the lists overflow even at the widest
    # capacity and the rows end in the plain FP32 form (or FP64) -- still exact
    rng = np.random.default_rng(66)
    base = rng.standard_normal(64).astype(np.float32) * 30
    X = (base + 0.05 * rng.standard_normal((3000, 64))).astype(np.float32)
    idx, dist, st = graph(X, 10)
    assert st["rows_fallback"] == len(X)
    rows = inputs.sample_rows(len(X), 100, seed=67)
    ref_idx, ref_dist = oracle.knng(X, 10, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_crowded_long_lists_trimmed_before_any_shrink():
    # a crowded corpus of 690 points and k = 300: the lists (824 keys) never reach their
    # mid-sweep trigger, so the first shrink of a row is the trim before the re-rank, on a
    # list whose threshold is still open and whose band no sample value reaches (the error
    # window dwarfs the distances). The trim must find the ranks exactly and keep only the
    # row's own keys: no index twice in any row, and the answer exact
    rng = np.random.default_rng(68)
    base = rng.standard_normal(64).astype(np.float32) * 30
    C = (base + 0.05 * rng.standard_normal((690, 64))).astype(np.float32)
    Q = (base + 0.05 * rng.standard_normal((96, 64))).astype(np.float32)
    idx, dist, st = kb.knn_search(dev(Q), dev(C), 300, precision="bf16", fused=1, return_stats=True)
    assert st["fused_used"] == 1
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    assert all(len(set(r.tolist())) == 300 for r in idx)
    rows = np.arange(0, 96, 8)
    ref_idx, ref_dist = oracle.knn(Q, C, 300, rows=rows)
    check_float(Q, C, rows, idx[rows], dist[rows], ref_idx, ref_dist, False)


@pytest.fixture
def speculate(monkeypatch):
    def set_spec(on):
        monkeypatch.setenv("KNN_SPECULATE", "1" if on else "0")
    return set_spec


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_speculative_thresholds_integer_bit_exact(precision, speculate):
    # speculation forced on a small graph: mid-sweep shrinks aim at reduced ranks
    speculate(True)
    X = inputs.integer_lattice(n=4096, d=128)
    idx, dist, st = graph(X, 16, precision)
    check_exact(idx, dist, *oracle.knng(X, 16))


def test_speculation_on_ordered_points_falls_back_exactly(speculate):
    # points along a curve in index order: a row's neighbours sit in one or two corpus
    # tiles, so wherever those tiles come early in the sweep a speculative threshold cuts
    # into the answer; those rows must be caught (truncated, certificate, second pass)
    speculate(True)
    n, d = 6144, 64
    t = np.arange(n, dtype=np.float64) * 0.01
    rng = np.random.default_rng(71)
    X = np.zeros((n, d), dtype=np.float64)
    X[:, 0] = np.cos(t) * 3
    X[:, 1] = np.sin(t) * 3
    X[:, 2] = t
    X += 1e-3 * rng.standard_normal((n, d))
    X = X.astype(np.float32)
    idx, dist, st = graph(X, 24)
    rows = np.concatenate([np.arange(0, n, 97), np.arange(n - 40, n)])
    ref_idx, ref_dist = oracle.knng(X, 24, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_speculation_does_not_change_answers(speculate):
    X = inputs.gaussian_mixture(n=20000, d=128, components=32, seed=72)
    speculate(False)
    a = graph(X, 32)
    speculate(True)
    b = graph(X, 32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_integer_ties_on_a_long_sweep_bit_exact():
    # integer points with many equal distances and a sweep long enough for speculation:
    # exact-arithmetic inputs keep the natural tile order, so thresholds that are exact
    # keys (zero error window) never drop a tied key of a smaller index
    X = inputs.integer_lattice(n=20000, d=16, lo=-2, hi=2, seed=73)
    idx, dist, st = graph(X, 24)
    rows = inputs.sample_rows(len(X), 120, seed=74)
    ref_idx, ref_dist = oracle.knng(X, 24, rows=rows)
    check_exact(idx[rows], dist[rows], ref_idx, ref_dist)


def test_large_k_integer_bit_exact():
    # k + m = 632: lists of 1440 keys (48 per lane in the shrink), trimmed before the
    # re-rank, whose longest tier then takes the rows
    X = inputs.integer_lattice(n=3000, d=64, lo=-5, hi=5, seed=75)
    idx, dist, st = graph(X, 600)
    assert st["fused_used"] == 1 and st["list_capacity"] > 1024
    check_exact(idx, dist, *oracle.knng(X, 600))


def test_large_k_float_search():
    C = inputs.gaussian_mixture(n=20000, d=64, components=16, seed=76)
    Q = inputs.gaussian_mixture(n=300, d=64, components=16, seed=77)
    idx, dist, st = kb.knn_search(dev(Q), dev(C), 500, precision="bf16", fused=1, return_stats=True)
    assert st["fused_used"] == 1
    rows = np.arange(0, 300, 10)
    ref_idx, ref_dist = oracle.knn(Q, C, 500, rows=rows)
    check_float(Q, C, rows, idx.cpu().numpy()[rows], dist.cpu().numpy()[rows], ref_idx, ref_dist, False)


@pytest.fixture
def rerank_in_sweep(monkeypatch):
    # the in-sweep re-rank serves the full sweep (a graph this size would otherwise take the
    # symmetric form, whose rows are complete only after the whole launch)
    monkeypatch.setenv("KNN_SYMMETRIC", "0")

    def set_rr(on):
        monkeypatch.setenv("KNN_RERANK_IN_SWEEP", "1" if on else "0")
    return set_rr


def test_rerank_in_sweep_integer_bit_exact(rerank_in_sweep):
    # 313 row blocks: the fused kernel's re-rank warps take the rows of finished row
    # blocks during the sweep, the launch after the kernel the rest
    X = inputs.integer_lattice(n=40000, d=128, seed=81)
    rerank_in_sweep(True)
    a = graph(X, 16)
    assert 0 < a[2]["rows_reranked_in_sweep"] < len(X), a[2]
    rerank_in_sweep(False)
    b = graph(X, 16)
    assert b[2]["rows_reranked_in_sweep"] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    rows = inputs.sample_rows(len(X), 64, seed=82)
    check_exact(a[0][rows], a[1][rows], *oracle.knng(X, 16, rows=rows))


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_rerank_in_sweep_float_identical(precision, rerank_in_sweep):
    X, t, s = inputs.unit_directions_with_duplicates(n=40000, d=256, seed=83)
    rerank_in_sweep(True)
    a = graph(X, 64, precision)
    rerank_in_sweep(False)
    b = graph(X, 64, precision)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2]["rows_uncertified"] == b[2]["rows_uncertified"]
    rows = np.concatenate([t[:8], inputs.sample_rows(len(X), 24, seed=84)])
    ref_idx, ref_dist = oracle.knng(X, 64, rows=rows)
    check_float(X, X, rows, a[0][rows], a[1][rows], ref_idx, ref_dist, exclude_self=True)


@pytest.mark.parametrize("d", [1024, 4096])
@pytest.mark.parametrize("kind", inputs.STRESS_KINDS)
@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_gemm_error_stays_within_its_bound(precision, kind, d):
    # every certificate rests on |approximate - exact| <= E_i for the GEMM's ranking value;
    # the re-rank measures that ratio on every candidate it evaluates
    X = inputs.accumulation_stress(kind, n=2048, d=d)
    idx, dist, st = graph(X, 16, precision)
    ratio = st["max_error_ratio"]
    print(f"{precision} {kind} d={d}: max |approx - exact| / E = {ratio:.4g}")
    assert 0.0 < ratio <= 1.0, st
    rows = inputs.sample_rows(len(X), 16, seed=85)
    ref_idx, ref_dist = oracle.knng(X, 16, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_fp8_certifies_near_duplicate_groups():
    # groups of 128 near-duplicates: the FP8 error bound is far below the gap between groups,
    # so every row is certified by the first pass (no fallback) and the graph is exact
    X = inputs.tight_groups(n=32768, d=256, group=128, seed=86)
    idx, dist, st = graph(X, 64, "fp8")
    assert st["rows_uncertified"] == 0 and st["rows_fallback"] == 0, st
    rows = inputs.sample_rows(len(X), 48, seed=87)
    ref_idx, ref_dist = oracle.knng(X, 64, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)
