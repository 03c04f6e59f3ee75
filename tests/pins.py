"""Pins for the FP64 oracle: facts fixed by the problem's definition, not by the oracle.

Each ``pin_*`` takes a loaded oracle library and raises AssertionError when the
oracle disagrees with the pinned fact. The tests run them against the real
oracle and against deliberately broken copies of it (each broken copy must fail
at least one pin).
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import oracle
from paper_1309_5478_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    """Parse a hand-worked fixture (format described in its header)."""
    out = {"queries": None}
    section = None
    rows: dict[str, list] = {"points": [], "queries": [], "expect": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            head = line.split()[0]
            if head in ("kind", "d", "k"):
                out[head] = line.split()[1]
                continue
            if head in ("points", "queries", "expect"):
                section = head
                continue
            rows[section].append(line)
    d = int(out["d"])
    pts = np.array([[float(v) for v in r.split()] for r in rows["points"]], dtype=np.float32).reshape(-1, d)
    q = (np.array([[float(v) for v in r.split()] for r in rows["queries"]], dtype=np.float32).reshape(-1, d)
         if rows["queries"] else None)
    exp_idx, exp_dist = [], []
    for r in rows["expect"]:
        _, body = r.split(":")
        a, b = body.split("|")
        exp_idx.append([int(v) for v in a.split()])
        exp_dist.append([float(v) for v in b.split()])
    return {"kind": out["kind"], "d": d, "k": int(out["k"]), "points": pts, "queries": q,
            "idx": np.array(exp_idx), "dist": np.array(exp_dist)}


GOLDEN_FILES = ("hand_knng_1d.txt", "hand_knng_duplicates.txt", "hand_search_ties.txt")


def pin_hand_examples(lib):
    for name in GOLDEN_FILES:
        g = read_golden(name)
        if g["kind"] == "knng":
            idx, dist = oracle.knng(g["points"], g["k"], lib=lib)
        else:
            idx, dist = oracle.knn(g["queries"], g["points"], g["k"], lib=lib)
        assert np.array_equal(idx, g["idx"]), (name, idx, g["idx"])
        assert np.array_equal(dist, g["dist"]), (name, dist, g["dist"])


def lattice_expected(n: int, i: int, k: int) -> list[int]:
    """Closed form for points x_j = j * e_1: neighbours of i by |i - j|, then by index."""
    out = []
    delta = 1
    while len(out) < k:
        if i - delta >= 0:
            out.append(i - delta)
        if len(out) < k and i + delta < n:
            out.append(i + delta)
        delta += 1
    return out[:k]


def pin_lattice(lib, n: int = 300, d: int = 7, k: int = 9):
    X = np.zeros((n, d), dtype=np.float32)
    X[:, 0] = np.arange(n)
    idx, dist = oracle.knng(X, k, lib=lib)
    for i in range(n):
        e = lattice_expected(n, i, k)
        assert list(idx[i]) == e, (i, list(idx[i]), e)
        assert list(dist[i]) == [float((i - j) ** 2) for j in e], i


def exact_bruteforce(Q: np.ndarray, C: np.ndarray, k: int, exclude_self: bool):
    """All-pairs enumeration with exact Python integers (integer-valued inputs only)."""
    Qi = [[int(v) for v in row] for row in Q]
    Ci = [[int(v) for v in row] for row in C]
    res_i, res_d = [], []
    for i, q in enumerate(Qi):
        cand = []
        for j, c in enumerate(Ci):
            if exclude_self and i == j:
                continue
            cand.append((sum((a - b) * (a - b) for a, b in zip(q, c)), j))
        cand.sort()
        res_i.append([j for _, j in cand[:k]])
        res_d.append([float(s) for s, _ in cand[:k]])
    return np.array(res_i), np.array(res_d)


def pin_bruteforce(lib):
    rng_cases = [(12, 3, 1), (17, 4, 5), (23, 5, 22), (31, 2, 7), (9, 6, 8)]
    for case, (n, d, k) in enumerate(rng_cases):
        X = inputs.integer_lattice(n=n, d=d, lo=-3, hi=3, seed=1000 + case)
        idx, dist = oracle.knng(X, k, lib=lib)
        ei, ed = exact_bruteforce(X, X, k, True)
        assert np.array_equal(idx, ei), (case, idx, ei)
        assert np.array_equal(dist, ed), case
        # search form: separate query set, nothing excluded
        Q = inputs.integer_lattice(n=5, d=d, lo=-3, hi=3, seed=2000 + case)
        idx, dist = oracle.knn(Q, X, min(k, n), lib=lib)
        ei, ed = exact_bruteforce(Q, X, min(k, n), False)
        assert np.array_equal(idx, ei), case
        assert np.array_equal(dist, ed), case


def pin_row_subset(lib):
    """Answering a subset of rows (in any order) gives those rows of the full answer."""
    X = inputs.integer_lattice(n=40, d=5, lo=-4, hi=4, seed=77)
    rows = np.array([7, 3, 39, 0, 21], dtype=np.int64)
    idx, dist = oracle.knng(X, 6, rows=rows, lib=lib)
    ei, ed = exact_bruteforce(X, X, 6, True)
    assert np.array_equal(idx, ei[rows]) and np.array_equal(dist, ed[rows])


def pin_library_cdist(lib):
    """Float inputs: scipy's cdist ('sqeuclidean') plus a lexicographic sort."""
    from scipy.spatial.distance import cdist
    X = inputs.gaussian_mixture(n=257, d=19, components=4, seed=31)
    k = 11
    idx, dist = oracle.knng(X, k, lib=lib)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for i in range(X.shape[0]):
        j = np.arange(X.shape[0])
        keep = j != i
        order = np.lexsort((j[keep], D[i, keep]))[:k]
        ref_idx = j[keep][order]
        ref_d = D[i, keep][order]
        assert np.allclose(dist[i], ref_d, rtol=1e-13, atol=0), i
        # index lists agree wherever the distances are not within rounding of each other
        gaps = np.diff(np.sort(D[i, keep])[:k + 1])
        if np.all(gaps > 1e-9 * ref_d.max()):
            assert np.array_equal(idx[i], ref_idx), i


def pin_invariants(lib):
    X, targets, sources = inputs.unit_directions_with_duplicates(n=600, d=24, dup_fraction=0.05, seed=5)
    k = 8
    idx, dist = oracle.knng(X, k, lib=lib)
    n = X.shape[0]
    for i in range(n):
        assert i not in idx[i]
        assert len(set(idx[i])) == k
        assert np.all(np.diff(dist[i]) >= 0)
        # ascending (distance, index)
        for a in range(k - 1):
            assert dist[i, a] < dist[i, a + 1] or idx[i, a] < idx[i, a + 1]
    # the k-th distance is <= every excluded distance, checked with the distance alone
    for i in (0, 17, 333, n - 1):
        kth = dist[i, -1]
        for j in range(n):
            if j != i and j not in idx[i]:
                assert oracle.sqdist(X[i], X[j]) >= kth
    # symmetry of the metric, and exact duplicates at distance 0 as first neighbours
    for t, s in zip(targets, sources):
        assert dist[t, 0] == 0.0 and idx[t, 0] == s
        assert dist[s, 0] == 0.0 and idx[s, 0] == t
    for i, j in ((1, 2), (10, 500)):
        assert oracle.sqdist(X[i], X[j]) == oracle.sqdist(X[j], X[i])


def pin_full_sort(lib):
    """k = N - 1 gives each point's whole row sorted; the distances are a permutation of the row."""
    X = inputs.integer_lattice(n=16, d=3, lo=-2, hi=2, seed=9)
    n = X.shape[0]
    idx, dist = oracle.knng(X, n - 1, lib=lib)
    ei, ed = exact_bruteforce(X, X, n - 1, True)
    assert np.array_equal(idx, ei) and np.array_equal(dist, ed)
    for i in range(n):
        assert sorted(idx[i]) == [j for j in range(n) if j != i]


def pin_pythagorean(lib):
    """Closed-form distances: a query at the origin and corpus points on integer 3-4-5 / 5-12-13 shells."""
    C = np.array([[3, 4, 0], [5, 12, 0], [0, 0, 1], [8, 15, 0], [-4, 3, 0], [12, 0, 5]], dtype=np.float32)
    Q = np.zeros((1, 3), dtype=np.float32)
    idx, dist = oracle.knn(Q, C, 6, lib=lib)
    assert list(idx[0]) == [2, 0, 4, 1, 5, 3]
    assert list(dist[0]) == [1.0, 25.0, 25.0, 169.0, 169.0, 289.0]


ALL_PINS = (pin_hand_examples, pin_lattice, pin_bruteforce, pin_row_subset, pin_library_cdist,
            pin_invariants, pin_full_sort, pin_pythagorean)


def failing_pins(lib) -> list[str]:
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError, IndexError):
            failed.append(pin.__name__)
    return failed
