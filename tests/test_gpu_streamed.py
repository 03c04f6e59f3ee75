"""GPU parity of the out-of-core search (corpus read in chunks, each chunk's answer merged by
FP64 distance and global index): identical to the in-core search and to the FP64 oracle."""
import numpy as np
import pytest

import oracle
from acceptance import check_exact
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def same_as_in_core(Q, C, k, chunk_rows, corpus="host"):
    Cs = {"host": np.ascontiguousarray(C), "pinned": torch.from_numpy(np.ascontiguousarray(C)).pin_memory(),
          "device": dev(C)}[corpus]
    si, sd, st = kb.knn_search_streamed(dev(Q), Cs, k, chunk_rows=chunk_rows, return_stats=True)
    ii, idd = kb.knn_search(dev(Q), dev(C), k)
    si, sd = si.cpu().numpy(), sd.cpu().numpy()
    assert np.array_equal(si, ii.cpu().numpy())
    # distances: the FP32 rounding of the pair's FP64 distance (one FP32 ulp of the oracle's
    # FP64 value, summed in another order; within the re-rank's tolerance of the in-core value)
    exact = np.array([[oracle.sqdist(Q[i], C[j]) for j in si[i]] for i in range(0, len(Q), 7)])
    got = sd[::7].astype(np.float64)
    assert np.all(np.abs(got - exact) <= np.spacing(exact.astype(np.float32)).astype(np.float64))
    assert np.allclose(sd, idd.cpu().numpy(), rtol=1e-6, atol=0)
    assert st["gemm_launches"] == -(-C.shape[0] // min(chunk_rows or C.shape[0], C.shape[0])) or chunk_rows == 0
    return si, sd


@pytest.mark.parametrize("chunk_rows", [1000, 4099, 20011, 0])
def test_integer_chunks_bit_exact(chunk_rows):
    C = inputs.integer_lattice(n=20011, d=32, lo=-4, hi=4, seed=80)
    Q = inputs.integer_lattice(n=333, d=32, lo=-4, hi=4, seed=81)
    si, sd = same_as_in_core(Q, C, 17, chunk_rows)
    ref_idx, ref_dist = oracle.knn(Q, C, 17)
    check_exact(si, sd, ref_idx, ref_dist)


def test_chunks_smaller_than_k_and_ties_across_chunks():
    # values in {-1, 0, 1}: many exact ties at every rank, spread over 47 chunks of 13 rows
    C = inputs.integer_lattice(n=600, d=6, lo=-1, hi=1, seed=82)
    Q = inputs.integer_lattice(n=40, d=6, lo=-1, hi=1, seed=83)
    si, sd = same_as_in_core(Q, C, 30, 13)
    ref_idx, ref_dist = oracle.knn(Q, C, 30)
    check_exact(si, sd, ref_idx, ref_dist)


@pytest.mark.parametrize("corpus", ["host", "pinned", "device"])
def test_float_corpus_memory_kinds(corpus):
    C = inputs.gaussian_mixture(n=30000, d=64, components=20, seed=84)
    Q = inputs.gaussian_mixture(n=200, d=64, components=8, seed=85)
    same_as_in_core(Q, C, 32, 7000, corpus)


def test_bad_chunk_rows():
    C = inputs.integer_lattice(n=100, d=4, seed=86)
    with pytest.raises(kb.KnnError):
        kb.knn_search_streamed(dev(C[:5]), C, 3, chunk_rows=-1)


def test_later_chunks_beyond_the_bound():
    # the first chunk holds every query's neighbours, the later chunks lie far away: from the
    # second chunk on the running k-th distance bounds the search, the later chunks' rows keep no
    # point within it, and the answer is the first chunk's
    rng = np.random.default_rng(87)
    near = rng.standard_normal((3000, 48)).astype(np.float32)
    far = (rng.standard_normal((9000, 48)) + 40.0).astype(np.float32)
    C = np.concatenate([near, far])
    Q = rng.standard_normal((300, 48)).astype(np.float32)
    si, sd, st = kb.knn_search_streamed(dev(Q), np.ascontiguousarray(C), 25, chunk_rows=3000, return_stats=True)
    si = si.cpu().numpy()
    assert st["rows_fallback"] == 0
    assert si.max() < 3000
    rows = inputs.sample_rows(len(Q), 40, seed=88)
    ref_idx, _ = oracle.knn(Q, C, 25, rows=rows)
    assert np.array_equal(si[rows], ref_idx)


@pytest.mark.parametrize("data", ["ties", "float"])
def test_bound_on_and_off_identical(monkeypatch, data):
    if data == "ties":
        C = inputs.integer_lattice(n=5000, d=8, lo=-2, hi=2, seed=89)
        Q = inputs.integer_lattice(n=150, d=8, lo=-2, hi=2, seed=90)
    else:
        C = inputs.gaussian_mixture(n=24000, d=96, components=12, seed=91)
        Q = inputs.gaussian_mixture(n=180, d=96, components=6, seed=92)
    out = []
    for b in ("1", "0"):
        monkeypatch.setenv("KNN_STREAM_BOUND", b)
        si, sd = kb.knn_search_streamed(dev(Q), np.ascontiguousarray(C), 20, chunk_rows=3001)
        out.append((si.cpu().numpy(), sd.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    rows = inputs.sample_rows(len(Q), 30, seed=93)
    ref_idx, ref_dist = oracle.knn(Q, C, 20, rows=rows)
    if data == "ties":
        assert np.array_equal(out[0][0][rows], ref_idx)
