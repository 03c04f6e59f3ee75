"""Parity rules between the engine and the FP64 oracle.

- integer-valued inputs (FP32 arithmetic exact): index lists and distances identical;
- float inputs: every reported distance within 1e-5 relative of the FP64 distance of
  the same pair; every oracle neighbour whose distance is below tau (1 - 1e-5) is
  reported (tau = the oracle's k-th distance); every reported neighbour's FP64
  distance is at most tau (1 + 1e-5); rows ascending; self never reported.
"""
from __future__ import annotations

import numpy as np

import oracle

REL = 1e-5


def check_exact(idx, dist, ref_idx, ref_dist):
    idx = np.asarray(idx)
    dist = np.asarray(dist)
    assert np.array_equal(idx.astype(np.int64), ref_idx), _first_diff(idx, ref_idx)
    assert np.array_equal(dist.astype(np.float64), ref_dist), _first_diff(dist, ref_dist)


def _first_diff(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    bad = np.argwhere(a.astype(np.float64) != b.astype(np.float64))
    if len(bad) == 0:
        return "equal"
    r = bad[0][0]
    return f"row {r}: got {a[r][:12]} expected {b[r][:12]}"


def check_float(Q, C, rows, idx, dist, ref_idx, ref_dist, exclude_self: bool):
    """idx/dist: engine output for the query rows `rows` (same order as ref_idx)."""
    idx = np.asarray(idx).astype(np.int64)
    dist = np.asarray(dist).astype(np.float64)
    k = ref_idx.shape[1]
    for r, i in enumerate(rows):
        gi, gd = idx[r], dist[r]
        assert np.all(np.diff(gd) >= 0), f"row {i} not ascending: {gd}"
        assert len(set(gi.tolist())) == k, f"row {i} repeats an index"
        if exclude_self:
            assert i not in gi, f"row {i} reports itself"
        # reported distances against FP64 of the same pair
        exact = np.array([oracle.sqdist(Q[i], C[j]) for j in gi])
        assert np.all(np.abs(gd - exact) <= REL * exact + 1e-30), \
            f"row {i}: distance error {np.max(np.abs(gd - exact) / np.maximum(exact, 1e-30))}"
        tau = ref_dist[r, -1]
        must = ref_idx[r][ref_dist[r] < tau * (1 - REL)]
        assert set(must.tolist()) <= set(gi.tolist()), f"row {i}: missing {set(must.tolist()) - set(gi.tolist())}"
        assert np.all(exact <= tau * (1 + REL) + 1e-30), f"row {i}: reported a point beyond the k-th distance"
