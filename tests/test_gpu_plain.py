"""GPU parity of the plain form (FP32 SIMT GEMM -> unfused quick multi-select ->
exact re-rank) against the FP64 oracle, through the C ABI."""
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


def run_graph(X, k, **kw):
    idx, dist = kb.knng_build(dev(X), k, precision="fp32", **kw)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def test_integer_lattice_4096x128_k16_bit_exact():
    X = inputs.integer_lattice(n=4096, d=128)
    idx, dist = run_graph(X, 16)
    ref_idx, ref_dist = oracle.knng(X, 16)
    check_exact(idx, dist, ref_idx, ref_dist)


@pytest.mark.parametrize("n,d,k", [(1000, 37, 7), (129, 5, 128), (517, 64, 1), (2, 3, 1), (33, 1, 32),
                                   (3001, 130, 48)])
def test_integer_ragged_shapes_bit_exact(n, d, k):
    X = inputs.integer_lattice(n=n, d=d, lo=-5, hi=5, seed=100 + n + d)
    idx, dist = run_graph(X, k)
    ref_idx, ref_dist = oracle.knng(X, k)
    check_exact(idx, dist, ref_idx, ref_dist)


def test_integer_heavy_ties_bit_exact():
    # values in {-1, 0, 1} at d = 6: many exact ties at every rank
    X = inputs.integer_lattice(n=2500, d=6, lo=-1, hi=1, seed=7)
    idx, dist = run_graph(X, 40)
    ref_idx, ref_dist = oracle.knng(X, 40)
    check_exact(idx, dist, ref_idx, ref_dist)


def test_all_equal_points():
    X = np.ones((300, 8), dtype=np.float32)
    idx, dist = run_graph(X, 10)
    ref_idx, ref_dist = oracle.knng(X, 10)
    check_exact(idx, dist, ref_idx, ref_dist)


def test_gaussian_mixture_float():
    X = inputs.gaussian_mixture(n=6000, d=256, components=16)
    k = 32
    idx, dist = run_graph(X, k)
    rows = inputs.sample_rows(len(X), 200, seed=1)
    ref_idx, ref_dist = oracle.knng(X, k, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_duplicates_at_distance_zero():
    X, t, s = inputs.unit_directions_with_duplicates(n=4096, d=256, dup_fraction=0.01, seed=11)
    idx, dist = run_graph(X, 10)
    assert np.all(dist[t, 0] == 0.0) and np.array_equal(idx[t, 0], s)
    rows = np.concatenate([t[:20], inputs.sample_rows(len(X), 60, seed=2)])
    ref_idx, ref_dist = oracle.knng(X, 10, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_search_separate_query_set():
    C = inputs.gaussian_mixture(n=5000, d=48, components=8, seed=5)
    Q = inputs.gaussian_mixture(n=777, d=48, components=8, seed=6)
    idx, dist = kb.knn_search(dev(Q), dev(C), 20, precision="fp32")
    ref_idx, ref_dist = oracle.knn(Q, C, 20)
    check_float(Q, C, np.arange(len(Q)), idx.cpu().numpy(), dist.cpu().numpy(), ref_idx, ref_dist, False)


def test_search_query_equal_to_corpus_point_not_excluded():
    C = inputs.integer_lattice(n=500, d=16, seed=3)
    Q = C[:10].copy()
    idx, dist = kb.knn_search(dev(Q), dev(C), 5, precision="fp32")
    idx = idx.cpu().numpy()
    assert np.array_equal(idx[:, 0], np.arange(10)) and np.all(dist.cpu().numpy()[:, 0] == 0)
    check_exact(idx, dist.cpu().numpy(), *oracle.knn(Q, C, 5))


def test_host_arrays_match_device_arrays():
    X = inputs.integer_lattice(n=1500, d=32, seed=9)
    i_host, d_host = kb.knng_build(X, 12, precision="fp32")  # numpy in, numpy out
    i_dev, d_dev = run_graph(X, 12)
    assert np.array_equal(i_host, i_dev) and np.array_equal(d_host, d_dev)


def test_gaussian_mixture_65536x256_sampled_rows():
    X = inputs.gaussian_mixture()
    k = 32
    idx, dist = run_graph(X, k)
    rows = inputs.sample_rows(len(X), 48, seed=4)
    ref_idx, ref_dist = oracle.knng(X, k, rows=rows)
    check_float(X, X, rows, idx[rows], dist[rows], ref_idx, ref_dist, exclude_self=True)


def test_slabs_give_the_same_answer():
    X = inputs.gaussian_mixture(n=3000, d=64, components=8, seed=12)
    a = run_graph(X, 16)
    b = run_graph(X, 16, max_workspace_bytes=2 * 128 * 3008 * 4)  # 128-row slabs
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_threshold_is_only_a_prefilter():
    X = inputs.gaussian_mixture(n=4000, d=64, components=8, seed=13)
    base = run_graph(X, 16)
    ref_idx, ref_dist = oracle.knng(X, 16, rows=np.arange(50))
    for scale in (0.5, 1.0, 1.5, 100.0):  # too tight, about right, loose, useless
        thr = (base[1][:, -1] * scale).astype(np.float32)
        i, d, st = kb.knng_build(dev(X), 16, precision="fp32", row_threshold=dev(thr), return_stats=True)
        assert np.array_equal(i.cpu().numpy(), base[0]) and np.array_equal(d.cpu().numpy(), base[1])
        if scale < 1.0:
            assert st["threshold_misses"] > 0
    check_float(X, X, np.arange(50), base[0][:50], base[1][:50], ref_idx, ref_dist, True)


def test_select_uniform_rows_match_sort():
    D = inputs.uniform_matrix(300, 5000)
    idx, val = kb.knn_select(dev(D), 50)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    for r in range(D.shape[0]):
        order = np.lexsort((np.arange(D.shape[1]), D[r]))[:50]
        assert np.array_equal(idx[r], order) and np.array_equal(val[r], D[r][order])


def test_select_ties_and_ragged_ldd():
    rng_vals = inputs.integer_lattice(n=64, d=1003, lo=0, hi=9, seed=21)
    D = np.zeros((64, 1008), dtype=np.float32)
    D[:, :1003] = rng_vals
    D[:, 1003:] = -100.0  # padding beyond n must be ignored
    idx, val = kb.knn_select(dev(D), 77, n=1003)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    for r in range(64):
        order = np.lexsort((np.arange(1003), rng_vals[r]))[:77]
        assert np.array_equal(idx[r], order)


def _sorted_runs(n, run, seed):
    # concatenated ascending runs of random values (the shape of merged per-segment answers)
    v = inputs.uniform_matrix(1, n, seed=seed)[0]
    return np.concatenate([np.sort(v[i:i + run]) for i in range(0, n, run)])


@pytest.mark.parametrize("pattern", ["ascending", "descending", "constant", "sawtooth", "runs256", "runs2048"])
def test_select_adversarial_orders(pattern):
    n = 20000
    base = np.arange(n, dtype=np.float32)
    row = {"ascending": base, "descending": base[::-1].copy(), "constant": np.zeros(n, np.float32),
           "sawtooth": (base % 97).astype(np.float32), "runs256": _sorted_runs(n, 256, 46),
           "runs2048": _sorted_runs(n, 2048, 47)}[pattern]
    D = np.stack([row, row[::-1].copy()])
    idx, val = kb.knn_select(dev(D), 300)
    idx = idx.cpu().numpy()
    for r in range(2):
        assert np.array_equal(idx[r], np.lexsort((np.arange(n), D[r]))[:300])


def test_errors_are_statuses():
    X = inputs.gaussian_mixture(n=100, d=8, components=2)
    bad = X.copy()
    bad[5, 3] = np.nan
    with pytest.raises(kb.KnnError) as e:
        kb.knng_build(dev(bad), 4, precision="fp32")
    assert e.value.status == kb.KNN_EINVAL
    with pytest.raises(kb.KnnError):
        kb.knng_build(dev(X), 100, precision="fp32")
    D = np.zeros((3, 10), np.float32)
    D[1, 4] = np.nan
    with pytest.raises(kb.KnnError):
        kb.knn_select(dev(D), 2)


@pytest.mark.parametrize("spec", ["0", "1"])
def test_select_speculation_on_off(spec, monkeypatch):
    # uniform rows (speculation pays off) and integer rows with heavy ties, with the
    # speculative shrinks forced on and off: both are exact
    monkeypatch.setenv("KNN_SPECULATE", spec)
    for D in (inputs.uniform_matrix(257, 9000, seed=31),
              inputs.integer_lattice(n=200, d=12000, lo=0, hi=40, seed=32)):
        idx, val = kb.knn_select(dev(D), 64)
        idx, val = idx.cpu().numpy(), val.cpu().numpy()
        for r in range(0, D.shape[0], 7):
            order = np.lexsort((np.arange(D.shape[1]), D[r]))[:64]
            assert np.array_equal(idx[r], order) and np.array_equal(val[r], D[r][order])


def _check_rows_sorted(D, idx, val, k, rows):
    for r in rows:
        order = np.lexsort((np.arange(D.shape[1]), D[r]))[:k]
        assert np.array_equal(idx[r], order) and np.array_equal(val[r], D[r][order]), r


@pytest.mark.parametrize("m,n,k", [(8, 1 << 20, 64), (1, 1 << 20, 1), (37, 1 << 18, 256), (3, 65536 + 256, 16),
                                   (120, 1 << 19, 8), (8, 1 << 20, 1024), (2, 1 << 20, 700), (256, 1 << 20, 1024),
                                   (32, 1 << 20, 128), (64, 1 << 20, 128)])
def test_select_few_long_rows(m, n, k):
    # the paper's selection experiment shape: few rows of up to 2^20 uniform values; rows
    # this few are split into segments selected in parallel and merged (a warp-wide sort for
    # short merges, a select over the concatenated segment answers, split again, for long)
    D = inputs.uniform_matrix(m, n, seed=40 + m)
    idx, val, st = kb.knn_select(dev(D), k, return_stats=True, timing=True)
    _check_rows_sorted(D, idx.cpu().numpy(), val.cpu().numpy(), k, range(0, m, max(1, m // 16)))
    assert st["rows"] == m and st["kernel_launches"] >= 1 and st["ms_select"] > 0
    oi = torch.empty((m, k), dtype=torch.int32, device="cuda")
    ov = torch.empty((m, k), dtype=torch.float32, device="cuda")
    kb.knn_select_noalloc(dev(D), k, oi, ov)
    assert np.array_equal(oi.cpu().numpy(), idx.cpu().numpy())


def test_select_few_long_rows_ties_across_segments():
    # integer values 0..3 over 2^20 columns: the k smallest are all ties at 0, spread over
    # every segment; the merge must keep the lowest column indices
    m, n, k = 4, 1 << 20, 200
    D = inputs.integer_lattice(n=m, d=n, lo=0, hi=3, seed=44)
    D[2, :] = 5.0
    D[2, n - 300:] = 1.0  # the answer sits in the last segment
    idx, val = kb.knn_select(dev(D), k)
    _check_rows_sorted(D, idx.cpu().numpy(), val.cpu().numpy(), k, range(m))


def test_select_few_long_rows_nan_rejected():
    D = inputs.uniform_matrix(2, 1 << 20, seed=45)
    D[1, 700001] = np.nan
    with pytest.raises(kb.KnnError):
        kb.knn_select(dev(D), 4)


@pytest.mark.parametrize("block_k", ["1", "0"])
@pytest.mark.parametrize("m,n,ldd,k,kind", [(40, 4096, 4096, 512, "uniform"), (9, 20000, 20000, 1000, "ints"),
                                          (33, 5003, 5008, 256, "uniform"), (17, 3001, 3001, 5, "ints"),
                                          (5, 70000, 70000, 64, "runs"), (3, 1500, 1500, 1024, "uniform"),
                                          (12, 100000, 100000, 300, "ints")])
def test_select_block_and_warp_kernels(m, n, ldd, k, kind, block_k, monkeypatch):
    # the block-per-row select (forced for every k with 1) and the warp-per-row select
    # (forced with 0) on ragged, strided, tied and sorted-run rows
    monkeypatch.setenv("KNN_SELECT_BLOCK_K", block_k)
    if kind == "uniform":
        V = inputs.uniform_matrix(m, n, seed=60 + m)
    elif kind == "ints":
        V = inputs.integer_lattice(n=m, d=n, lo=0, hi=6, seed=61 + m)
    else:
        V = np.stack([_sorted_runs(n, 512, 62 + r) for r in range(m)])
    D = np.full((m, ldd), -5.0, dtype=np.float32)
    D[:, :n] = V
    idx, val = kb.knn_select(dev(D), k, n=n)
    _check_rows_sorted(V, idx.cpu().numpy(), val.cpu().numpy(), k, range(m))


def test_select_block_kernel_rejects_nan(monkeypatch):
    monkeypatch.setenv("KNN_SELECT_BLOCK_K", "1")
    D = inputs.uniform_matrix(4, 9000, seed=63)
    D[3, 8999] = np.nan
    with pytest.raises(kb.KnnError):
        kb.knn_select(dev(D), 300)
