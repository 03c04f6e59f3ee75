"""Host logic of bench.py that needs no GPU: the selection-sweep shapes cover the paper's
three selection experiments, and the sampled oracle check accepts a correct answer and
rejects planted mistakes."""
import os
import sys

import numpy as np

import oracle
from paper_1309_5478_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_select_sweep_shapes_follow_the_paper():
    shapes = bench.select_sweep_shapes()
    fams = {}
    for fam, q, n, k in shapes:
        fams.setdefault(fam, []).append((q, n, k))
    # n = 2^20, Q from 2^3 to 2^8 (time per query against Q)
    assert sorted({q for q, n, k in fams["n=2^20"]}) == [8, 16, 32, 64, 128, 256]
    assert all(n == 1 << 20 for q, n, k in fams["n=2^20"])
    # n Q = 2^27 with log2(n / Q) from -3 to 19
    ratios = sorted({int(np.log2(n / q)) for q, n, k in fams["nQ=2^27"]})
    assert ratios == list(range(-3, 20, 2))
    assert all(q * n == 1 << 27 for q, n, k in fams["nQ=2^27"])
    # Q = 256 with n from 2^16 to 2^20
    assert sorted({n for q, n, k in fams["Q=256"]}) == [1 << 16, 1 << 18, 1 << 20]
    assert all(1 <= k <= min(1024, n) for _, q, n, k in shapes)


def test_oracle_check_accepts_the_answer_and_rejects_mistakes():
    X = inputs.gaussian_mixture(n=600, d=12, components=5, seed=90)
    rows = np.array([0, 7, 123, 599])
    k = 8
    ref_idx, ref_dist = oracle.knng(X, k, rows=rows)
    good = bench.oracle_check(X, rows, ref_idx.astype(np.int32), ref_dist.astype(np.float32), ref_idx, ref_dist)
    assert good["rows_identical_indices"] == len(rows) and good["rows_pass_acceptance"] == len(rows)
    bad_idx = ref_idx.astype(np.int32).copy()
    bad_idx[1, 0] = rows[1]  # the row reports itself
    bad_dist = ref_dist.astype(np.float32).copy()
    bad_dist[2, 3] *= 1.01   # a distance 1% off
    bad = bench.oracle_check(X, rows, bad_idx, bad_dist, ref_idx, ref_dist)
    assert bad["rows_pass_acceptance"] == len(rows) - 2
    assert bad["max_rel_dist_err"] > 1e-3
