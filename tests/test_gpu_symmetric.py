"""The symmetric form of the k-NN graph (each pair's product computed once and used for
both of its rows: the transpose reuse of Methods, "Distance calculation") gives the same
graph as the full sweep, through the C ABI, and stays exact where its speculative
threshold or its inboxes fall short (the rows go through the second pass)."""
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


@pytest.fixture
def symmetric(monkeypatch):
    # on: 1 (the probe may keep the full sweep where inboxes would overflow), forced: 2
    def set_sym(on):
        monkeypatch.setenv("KNN_SYMMETRIC", str(int(on)))
    return set_sym


def graph(X, k, precision="bf16"):
    i, d, st = kb.knng_build(dev(X), k, precision=precision, fused=1, return_stats=True)
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy(), st


def both(X, k, symmetric, precision="bf16", forced=False):
    symmetric(2 if forced else 1)
    a = graph(X, k, precision)
    symmetric(False)
    b = graph(X, k, precision)
    assert a[2]["symmetric"] == 1 and b[2]["symmetric"] == 0
    # the symmetric launch computes about half of the distance product
    assert a[2]["gemm_flops"] < 0.55 * b[2]["gemm_flops"], (a[2]["gemm_flops"], b[2]["gemm_flops"])
    return a, b


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_symmetric_integer_bit_exact(precision, symmetric):
    # 2^30 pairs and more: the band probe runs and proposes the threshold of the transposed pairs
    # forced: lattice distances are few integers, so many keys tie below the threshold and the
    # probe alone would keep the full sweep
    X = inputs.integer_lattice(n=33000, d=64, seed=101)
    a, b = both(X, 16, symmetric, precision, forced=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    rows = np.concatenate([np.arange(0, 300), inputs.sample_rows(len(X), 64, seed=102), np.arange(len(X) - 200, len(X))])
    check_exact(a[0][rows], a[1][rows], *oracle.knng(X, 16, rows=rows))


def test_symmetric_unit_directions_identical(symmetric):
    X, t, s = inputs.unit_directions_with_duplicates(n=40000, d=256, seed=103)
    a, b = both(X, 64, symmetric)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.all(a[1][t, 0] == 0.0) and np.array_equal(a[0][t, 0], s)
    rows = np.concatenate([t[:8], inputs.sample_rows(len(X), 32, seed=104)])
    ref_idx, ref_dist = oracle.knng(X, 64, rows=rows)
    check_float(X, X, rows, a[0][rows], a[1][rows], ref_idx, ref_dist, exclude_self=True)


def test_symmetric_clustered_rows_beyond_the_threshold(symmetric):
    # uneven cluster sizes: rows in sparse clusters have k-th distances beyond the sampled
    # threshold; the certificate rejects them and the second pass makes them exact
    X = inputs.anisotropic_mixture(n=36000, d=96, components=40, seed=105)
    a, b = both(X, 32, symmetric, forced=True)
    assert np.array_equal(a[0], b[0])
    assert np.allclose(a[1], b[1], rtol=1e-6, atol=0)
    rows = inputs.sample_rows(len(X), 96, seed=106)
    ref_idx, ref_dist = oracle.knng(X, 32, rows=rows)
    check_float(X, X, rows, a[0][rows], a[1][rows], ref_idx, ref_dist, exclude_self=True)


def test_symmetric_inbox_overflow_is_caught(symmetric):
    # points crowded far from the origin: the reduced-precision bound dwarfs the distances,
    # every transposed pair passes the threshold, the inboxes overflow, and every row is
    # recomputed -- still exact. Left to the probe, the full sweep is taken instead.
    rng = np.random.default_rng(107)
    base = rng.standard_normal(32).astype(np.float32) * 30
    X = (base + 0.05 * rng.standard_normal((33000, 32))).astype(np.float32)
    symmetric(2)  # forced: the probe alone would keep the full sweep here
    i, d, st = graph(X, 8)
    assert st["symmetric"] == 1 and st["rows_fallback"] == len(X)
    symmetric(1)
    assert graph(X, 8)[2]["symmetric"] == 0
    rows = inputs.sample_rows(len(X), 48, seed=108)
    ref_idx, ref_dist = oracle.knng(X, 8, rows=rows)
    check_float(X, X, rows, i[rows], d[rows], ref_idx, ref_dist, exclude_self=True)



def test_headline_graph_full_size_sampled_rows():
    # the bench's workload and launch configuration: 262144 unit directions in d = 1024 with 1%
    # exact duplicates, k = 64, the default form (symmetric fused BF16 with the band probe);
    # sampled rows, duplicate targets among them, against the FP64 oracle
    X, targets, sources = inputs.unit_directions_with_duplicates(n=262144, d=1024)
    i, d, st = kb.knng_build(dev(X), 64, return_stats=True)
    torch.cuda.synchronize()
    assert st["symmetric"] == 1 and st["rows_uncertified"] == 0
    i, d = i.cpu().numpy(), d.cpu().numpy()
    rows = np.unique(np.concatenate([targets[:8], sources[:8], inputs.sample_rows(len(X), 32, seed=96)]))
    ref_idx, ref_dist = oracle.knng(X, 64, rows=rows)
    check_float(X, X, rows, i[rows], d[rows], ref_idx, ref_dist, exclude_self=True)
    # a duplicate pair is each other's nearest neighbour at distance 0
    for t, s in zip(targets[:8], sources[:8]):
        assert i[t, 0] == s and d[t, 0] == 0.0
