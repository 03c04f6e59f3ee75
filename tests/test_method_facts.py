"""Facts the GPU paths rely on, checked on the CPU against the FP64 oracle and plain numpy.

- Out-of-core search: the k smallest of the union of every chunk's k smallest (by distance,
  then index) are the k smallest of the whole corpus.
- Similarity certificate: for unit rows rounded to FP32 from FP64 means and norms,
  |d2(u_i, u_j) - (2 - 2 s_ij)| <= eta(d) = 9 2^-24 + (4 d + 64) 2^-53, with s_ij the FP64
  similarity from the same means and norms.
"""
import numpy as np
import pytest

import oracle
from paper_1309_5478_gb300 import inputs


@pytest.mark.parametrize("chunk", [7, 100, 333, 1000])
def test_merging_chunk_answers_gives_the_whole_answer(chunk):
    C = inputs.integer_lattice(n=1000, d=5, lo=-2, hi=2, seed=91)  # many exact ties
    Q = inputs.integer_lattice(n=30, d=5, lo=-2, hi=2, seed=92)
    k = 12
    ref_idx, ref_dist = oracle.knn(Q, C, k)
    run = [[] for _ in range(len(Q))]
    for c0 in range(0, len(C), chunk):
        kc = min(k, len(C[c0:c0 + chunk]))
        ci, cd = oracle.knn(Q, C[c0:c0 + chunk], kc)
        for r in range(len(Q)):
            run[r] = sorted(run[r] + [(cd[r, t], c0 + ci[r, t]) for t in range(kc)])[:k]
    for r in range(len(Q)):
        assert [j for _, j in run[r]] == list(ref_idx[r])
        assert [d for d, _ in run[r]] == list(ref_dist[r])


def eta(d):
    return 9.0 * 2.0 ** -24 + (4.0 * d + 64.0) * 2.0 ** -53


def unit_rows(X, centered):
    X64 = X.astype(np.float64)
    m = X64.mean(axis=1, keepdims=True) if centered else np.zeros((len(X), 1))
    c = X64 - m
    n = np.sqrt((c * c).sum(axis=1, keepdims=True))
    return (c / n).astype(np.float32), c, n


@pytest.mark.parametrize("centered", [False, True])
@pytest.mark.parametrize("d,kind", [(3, "gauss"), (128, "gauss"), (1024, "gauss"), (256, "offset"),
                                    (64, "wide"), (768, "lattice")])
def test_similarity_certificate_bound(centered, d, kind):
    rng = np.random.default_rng(93 + d)
    if kind == "gauss":
        X = rng.standard_normal((200, d)).astype(np.float32)
    elif kind == "offset":  # a large common offset: centring cancels most of each entry
        X = (1e4 + rng.standard_normal((200, d))).astype(np.float32)
    elif kind == "wide":    # entries over many binades
        X = (rng.standard_normal((200, d)) * 10.0 ** rng.uniform(-6, 6, (200, d))).astype(np.float32)
    else:
        X = inputs.integer_lattice(n=200, d=d, lo=-3, hi=3, seed=94)
    U, c, n = unit_rows(X, centered)
    U64 = U.astype(np.float64)
    s = (c @ c.T) / (n * n.T)
    sq = (U64 * U64).sum(axis=1)
    d2 = sq[:, None] + sq[None, :] - 2.0 * (U64 @ U64.T)  # exact to ~1e-16 for these sizes
    gap = np.abs(d2 - (2.0 - 2.0 * s))
    assert gap.max() <= eta(d), (gap.max(), eta(d))
