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


SIM_GOLDEN = (("hand_cosine_search.txt", "cosine"), ("hand_pearson_search.txt", "pearson"))


def pin_sim_hand_examples(lib):
    """Hand-worked cosine and Pearson searches: exact order, similarities to 1e-15."""
    for name, metric in SIM_GOLDEN:
        g = read_golden(name)
        idx, sim = oracle.knn_sim(g["queries"], g["points"], g["k"], metric, lib=lib)
        assert np.array_equal(idx, g["idx"]), (name, idx, g["idx"])
        assert np.allclose(sim, g["dist"], rtol=0, atol=1e-15), (name, sim, g["dist"])


def _rational_key(q, c, centered):
    """Exact order key of the cosine (centred: Pearson) of two integer vectors:
    sign(dot) dot^2 / (|q|^2 |c|^2) as a Fraction (monotone in the similarity)."""
    from fractions import Fraction
    d = len(q)
    if centered:
        mq, mc = Fraction(sum(q), d), Fraction(sum(c), d)
        q = [Fraction(v) - mq for v in q]
        c = [Fraction(v) - mc for v in c]
    dot = sum(Fraction(a) * b for a, b in zip(q, c))
    nq = sum(Fraction(a) * a for a in q)
    nc = sum(Fraction(b) * b for b in c)
    return (1 if dot >= 0 else -1) * dot * dot / (nq * nc)


def pin_sim_rational_bruteforce(lib):
    """Integer inputs: the order of exact rational similarities. Where exact values tie, any
    order of the tied points is right, so the pin checks the set of points above the k-th
    value, that every reported point is at least the k-th value, and the similarity values."""
    cases = [(14, 3, 5, 0), (19, 4, 7, 1), (25, 2, 9, 0), (11, 5, 10, 1), (30, 3, 12, 1)]
    for case, (n, d, k, centered) in enumerate(cases):
        X = inputs.integer_lattice(n=n, d=d, lo=-3, hi=4, seed=3000 + case)
        metric = "pearson" if centered else "cosine"
        Xi = [[int(v) for v in row] for row in X]
        ok = [i for i in range(n) if (len(set(Xi[i])) > 1 if centered else any(Xi[i]))]
        Xs = X[ok]
        Xi = [Xi[i] for i in ok]
        idx, sim = oracle.knng_sim(Xs, k, metric, lib=lib)
        for i in range(len(Xi)):
            keys = {j: _rational_key(Xi[i], Xi[j], centered) for j in range(len(Xi)) if j != i}
            kth = sorted(keys.values(), reverse=True)[k - 1]
            above = {j for j, v in keys.items() if v > kth}
            got = set(idx[i].tolist())
            assert i not in got, (case, i)
            assert above <= got, (case, i, above - got)
            assert all(keys[j] >= kth for j in got), (case, i)
            for t, j in enumerate(idx[i]):
                v = float(np.dot(np.array(Xi[i], float) - (np.mean(Xi[i]) if centered else 0),
                                 np.array(Xi[j], float) - (np.mean(Xi[j]) if centered else 0)))
                v /= (np.linalg.norm(np.array(Xi[i], float) - (np.mean(Xi[i]) if centered else 0)) *
                      np.linalg.norm(np.array(Xi[j], float) - (np.mean(Xi[j]) if centered else 0)))
                assert abs(sim[i, t] - v) <= 1e-14, (case, i, t, sim[i, t], v)
            assert np.all(np.diff(sim[i]) <= 0)


def pin_sim_library(lib):
    """Float inputs: scipy's cdist with 'cosine' and 'correlation' (1 - similarity)."""
    from scipy.spatial.distance import cdist
    X = inputs.gaussian_mixture(n=203, d=17, components=5, seed=41)
    Q = inputs.gaussian_mixture(n=9, d=17, components=3, seed=42)
    k = 13
    for metric, sp in (("cosine", "cosine"), ("pearson", "correlation")):
        idx, sim = oracle.knn_sim(Q, X, k, metric, lib=lib)
        S = 1.0 - cdist(Q.astype(np.float64), X.astype(np.float64), sp)
        for i in range(Q.shape[0]):
            order = np.lexsort((np.arange(X.shape[0]), -S[i]))[:k]
            assert np.allclose(sim[i], S[i, order], rtol=0, atol=1e-12), (metric, i)
            gaps = -np.diff(np.sort(S[i])[::-1][:k + 1])
            if np.all(gaps > 1e-10):
                assert np.array_equal(idx[i], order), (metric, i)


def pin_sim_invariants(lib):
    """Scaling a corpus row by a power of two changes no similarity (cosine and Pearson);
    adding an integer to every entry of an integer row changes no Pearson similarity (d = 8,
    where the row mean is exact);
    negating the corpus negates every cosine; the graph never reports a point itself."""
    X = inputs.integer_lattice(n=60, d=6, lo=-5, hi=5, seed=51).astype(np.float32)
    X = X[[len(set(r.tolist())) > 1 for r in X]]
    Q = X[:7]
    n = X.shape[0]
    for metric in ("cosine", "pearson"):
        base_i, base_s = oracle.knn_sim(Q, X, n, metric, lib=lib)
        Xs = X * np.where(np.arange(n) % 3 == 0, 4.0, 0.5).astype(np.float32)[:, None]
        i2, s2 = oracle.knn_sim(Q, Xs, n, metric, lib=lib)
        assert np.array_equal(i2, base_i) and np.array_equal(s2, base_s), metric
        gi, gs = oracle.knng_sim(X, 5, metric, lib=lib)
        for i in range(n):
            assert i not in gi[i]
            assert np.all(np.diff(gs[i]) <= 0)
            for a in range(4):
                assert gs[i, a] > gs[i, a + 1] or gi[i, a] < gi[i, a + 1]
    # d = 8: the mean of an integer row is exact, so the shifted rows centre to the same values
    X8 = inputs.integer_lattice(n=50, d=8, lo=-5, hi=5, seed=52).astype(np.float32)
    X8 = X8[[len(set(r.tolist())) > 1 for r in X8]]
    i3, s3 = oracle.knn_sim(X8[:6], X8 + np.float32(7), X8.shape[0], "pearson", lib=lib)
    pi, ps = oracle.knn_sim(X8[:6], X8, X8.shape[0], "pearson", lib=lib)
    assert np.array_equal(i3, pi) and np.array_equal(s3, ps)
    ci, cs = oracle.knn_sim(Q, X, n, "cosine", lib=lib)
    ni, ns = oracle.knn_sim(Q, -X, n, "cosine", lib=lib)
    for i in range(Q.shape[0]):
        assert np.array_equal(np.sort(ns[i]), np.sort(-cs[i]))
        a = {int(j): v for j, v in zip(ci[i], cs[i])}
        b = {int(j): v for j, v in zip(ni[i], ns[i])}
        assert all(b[j] == -a[j] for j in a)
    try:
        oracle.knn_sim(Q, np.zeros((3, X.shape[1]), np.float32), 2, "cosine", lib=lib)
    except ValueError:
        pass
    else:
        raise AssertionError("a zero-norm corpus row was accepted")


ALL_PINS = (pin_hand_examples, pin_lattice, pin_bruteforce, pin_row_subset, pin_library_cdist,
            pin_invariants, pin_full_sort, pin_pythagorean, pin_sim_hand_examples, pin_sim_rational_bruteforce,
            pin_sim_library, pin_sim_invariants)


def failing_pins(lib) -> list[str]:
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError, LookupError):
            failed.append(pin.__name__)
    return failed
