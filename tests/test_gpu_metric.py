"""GPU parity of the cosine and Pearson similarity path (unit rows -> Euclidean engine ->
FP64 similarity of the candidates with a certificate -> FP64 fallback) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def nonzero_rows(X, centered):
    keep = [len(set(r.tolist())) > 1 if centered else bool(np.any(r != 0)) for r in X]
    return np.ascontiguousarray(X[np.array(keep)])


def check_sim_exact(idx, val, ref_idx, ref_sim):
    """Integer inputs: the FP64 similarities are computed exactly alike on both sides."""
    assert np.array_equal(idx.astype(np.int64), ref_idx), np.argwhere(idx != ref_idx)[:3]
    assert np.array_equal(val, ref_sim.astype(np.float32))


def check_sim_float(Q, C, rows, idx, val, ref_idx, ref_sim, metric, exclude_self):
    """Float inputs: values within one FP32 ulp of the FP64 similarity of the same pair;
    every oracle neighbour clearly above the k-th similarity reported; nothing reported
    clearly below it; rows descending."""
    for r, i in enumerate(rows):
        gi, gv = idx[r].astype(np.int64), val[r].astype(np.float64)
        assert np.all(np.diff(gv) <= 0), (i, gv)
        assert len(set(gi.tolist())) == len(gi)
        if exclude_self:
            assert i not in gi
        exact = np.array([oracle.similarity(Q[i], C[j], metric) for j in gi])
        ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(gv - exact) <= ulp), (i, np.max(np.abs(gv - exact)))
        kth = ref_sim[r, -1]
        must = ref_idx[r][ref_sim[r] > kth + 1e-12]
        assert set(must.tolist()) <= set(gi.tolist()), (i, set(must.tolist()) - set(gi.tolist()))
        assert np.all(exact >= kth - 1e-12), i


@pytest.mark.parametrize("metric,n,d,k", [("cosine", 3000, 16, 12), ("cosine", 1000, 3, 40), ("pearson", 2500, 16, 20),
                                          ("pearson", 700, 8, 64), ("cosine", 515, 130, 7)])
def test_integer_graph_bit_exact(metric, n, d, k):
    centered = metric == "pearson"
    X = nonzero_rows(inputs.integer_lattice(n=n, d=d, lo=-4, hi=4, seed=70 + n + d), centered)
    idx, val, st = kb.knng_build_metric(dev(X), k, metric, return_stats=True)
    ref_idx, ref_sim = oracle.knng_sim(X, k, metric)
    check_sim_exact(idx.cpu().numpy(), val.cpu().numpy(), ref_idx, ref_sim)


@pytest.mark.parametrize("metric", ["cosine", "pearson"])
def test_float_graph_and_search(metric):
    X = inputs.gaussian_mixture(n=8000, d=96, components=12, seed=71)
    k = 24
    idx, val = kb.knng_build_metric(dev(X), k, metric)
    rows = inputs.sample_rows(len(X), 150, seed=3)
    ref_idx, ref_sim = oracle.knng_sim(X, k, metric, rows=rows)
    check_sim_float(X, X, rows, idx.cpu().numpy()[rows], val.cpu().numpy()[rows], ref_idx, ref_sim, metric, True)
    Q = inputs.gaussian_mixture(n=300, d=96, components=5, seed=72)
    idx, val = kb.knn_search_metric(dev(Q), dev(X), k, metric)
    ref_idx, ref_sim = oracle.knn_sim(Q, X, k, metric)
    check_sim_float(Q, X, range(len(Q)), idx.cpu().numpy(), val.cpu().numpy(), ref_idx, ref_sim, metric, False)


def test_parallel_duplicates_take_the_fallback():
    # every point has 39 power-of-two multiples: exact ties at the top similarity, more of
    # them than the k + m candidates, which no distance gap can certify; the FP64
    # recomputation over the whole corpus orders them by index
    base = nonzero_rows(inputs.integer_lattice(n=30, d=12, lo=-3, hi=3, seed=73), True)
    X = np.concatenate([np.float32(2.0 ** e) * base for e in range(-8, 32)]).astype(np.float32)
    for metric in ("cosine", "pearson"):
        Xm = nonzero_rows(X, metric == "pearson")
        idx, val, st = kb.knng_build_metric(dev(Xm), 6, metric, return_stats=True)
        ref_idx, ref_sim = oracle.knng_sim(Xm, 6, metric)
        assert np.array_equal(idx.cpu().numpy(), ref_idx)
        assert np.array_equal(val.cpu().numpy(), ref_sim.astype(np.float32))
        assert st["rows_uncertified"] > 0 and st["rows_fallback"] >= st["rows_uncertified"]


def test_all_candidates_and_small_shapes():
    X = nonzero_rows(inputs.integer_lattice(n=40, d=5, lo=-3, hi=3, seed=74), False)
    n = len(X)
    idx, val = kb.knng_build_metric(dev(X), n - 1, "cosine")
    ref_idx, ref_sim = oracle.knng_sim(X, n - 1, "cosine")
    check_sim_exact(idx.cpu().numpy(), val.cpu().numpy(), ref_idx, ref_sim)
    Q = X[:3]
    idx, val = kb.knn_search_metric(dev(Q), dev(X), n, "cosine")
    ref_idx, ref_sim = oracle.knn_sim(Q, X, n, "cosine")
    check_sim_exact(idx.cpu().numpy(), val.cpu().numpy(), ref_idx, ref_sim)


def test_euclidean_passthrough():
    X = inputs.integer_lattice(n=900, d=20, seed=75)
    a = kb.knng_build_metric(dev(X), 9, "euclidean")
    b = kb.knng_build(dev(X), 9)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_undefined_similarities_are_rejected():
    X = inputs.gaussian_mixture(n=200, d=8, components=2, seed=76)
    Z = X.copy()
    Z[17] = 0.0
    with pytest.raises(kb.KnnError) as e:
        kb.knng_build_metric(dev(Z), 4, "cosine")
    assert e.value.status == kb.KNN_EINVAL
    P = X.copy()
    P[5] = 3.0  # constant row: zero norm after centring
    kb.knng_build_metric(dev(P), 4, "cosine")
    with pytest.raises(kb.KnnError):
        kb.knng_build_metric(dev(P), 4, "pearson")
    B = X.copy()
    B[9, 2] = np.nan
    with pytest.raises(kb.KnnError):
        kb.knng_build_metric(dev(B), 4, "cosine")


def test_cosine_graph_65536x128_sampled_rows():
    X = inputs.gaussian_mixture(n=65536, d=128, components=32, seed=77)
    k = 32
    idx, val, st = kb.knng_build_metric(dev(X), k, "cosine", return_stats=True)
    rows = inputs.sample_rows(len(X), 64, seed=5)
    ref_idx, ref_sim = oracle.knng_sim(X, k, "cosine", rows=rows)
    check_sim_float(X, X, rows, idx.cpu().numpy()[rows], val.cpu().numpy()[rows], ref_idx, ref_sim, "cosine", True)
    print("cosine 65536x128 stats:", {kk: st[kk] for kk in ("rows_uncertified", "rows_fallback", "candidates",
                                                           "rows_truncated", "precision_used", "list_capacity")})
    assert st["rows_uncertified"] < len(X) // 100


def test_host_arrays_are_staged():
    # numpy inputs and outputs: the library stages them through device memory
    X = nonzero_rows(inputs.integer_lattice(n=800, d=10, lo=-4, hi=4, seed=78), True)
    Q = X[:50]
    for metric in ("cosine", "pearson"):
        idx, val = kb.knn_search_metric(Q, X, 9, metric)
        assert isinstance(idx, np.ndarray) and isinstance(val, np.ndarray)
        ref_idx, ref_sim = oracle.knn_sim(Q, X, 9, metric)
        if metric == "cosine":
            check_sim_exact(idx, val, ref_idx, ref_sim)
        else:
            check_sim_float(Q, X, range(len(Q)), idx, val, ref_idx, ref_sim, metric, False)
