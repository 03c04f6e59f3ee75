"""Facts the GPU paths rely on, checked on the CPU against the FP64 oracle and plain numpy.

- Out-of-core search: the k smallest of the union of every chunk's k smallest (by distance,
  then index) are the k smallest of the whole corpus.
- Out-of-core running bound: with each chunk's search restricted to the points at or below the
  running k-th distance (and every chunk's answer merged as before), the answer is unchanged.
- The bound's conversion to the approximate values' scale (`bound_kernel`): with |q|^2 summed
  in FP32 as the prep pass sums it, t - exact |q|^2 <= the converted bound - E for every t.
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


@pytest.mark.parametrize("chunk", [7, 100, 333])
def test_running_bound_keeps_the_answer(chunk):
    # a later chunk only contributes points strictly below the running k-th distance (one at
    # the same distance has a higher index and loses the tie), so searching it among the points
    # at or below that distance (fewer than k of them allowed) changes nothing
    C = inputs.integer_lattice(n=1000, d=5, lo=-2, hi=2, seed=93)  # many exact ties
    Q = inputs.integer_lattice(n=30, d=5, lo=-2, hi=2, seed=94)
    k = 12
    ref_idx, ref_dist = oracle.knn(Q, C, k)
    run = [[] for _ in range(len(Q))]
    for c0 in range(0, len(C), chunk):
        Cc = C[c0:c0 + chunk]
        D = ((Q[:, None, :].astype(np.float64) - Cc[None, :, :]) ** 2).sum(-1)
        for r in range(len(Q)):
            bound = run[r][-1][0] if len(run[r]) == k else np.inf
            within = [(D[r, j], c0 + j) for j in range(len(Cc)) if D[r, j] <= bound]
            run[r] = sorted(run[r] + sorted(within)[:k])[:k]
    for r in range(len(Q)):
        assert [j for _, j in run[r]] == list(ref_idx[r])
        assert [d for d, _ in run[r]] == list(ref_dist[r])


def _prep_norm2(x):
    # |x|^2 as the prep pass forms it: each of 32 lanes an FP32 FMA chain over its stride, then
    # a five-level tree
    f32 = np.float32
    lanes = []
    for l in range(32):
        s = f32(0.0)
        for t in range(l, len(x), 32):
            s = f32(np.float64(x[t]) * np.float64(x[t]) + np.float64(s))
        lanes.append(s)
    o = 16
    while o:
        lanes = [f32(lanes[i] + lanes[i ^ o]) for i in range(32)]
        o //= 2
    return lanes[0]


def _bound_to_dprime(t, qn2, e, d):
    # the conversion of bound_kernel: FP64, then rounded up to FP32
    g = (d / 32.0 + 8.0) * 2.0 ** -24
    v = float(t) * (1.0 + 2.0 ** -40) - float(qn2) * (1.0 - g) + float(e) * (1.0 + 2.0 ** -10)
    f = np.float32(v)
    if float(f) < v:
        f = np.nextafter(f, np.float32(np.inf))
    return float(f)


@pytest.mark.parametrize("d", [3, 64, 256, 1024, 4096])
def test_bound_conversion_covers_the_exact_norm(d):
    rng = np.random.default_rng(95 + d)
    for scale in (1e-3, 1.0, 37.0):
        for _ in range(20):
            q = (rng.standard_normal(d) * scale).astype(np.float32)
            exact = float(np.sum(q.astype(np.float64) ** 2))
            qn2 = _prep_norm2(q)
            t = np.float32(exact * rng.uniform(0.5, 3.0))
            e = np.float32(rng.uniform(0.0, 1e-3) * exact)
            assert _bound_to_dprime(t, qn2, e, d) - float(e) >= float(t) - exact


# ---------------------------------------------------------------------------------------
# The similarity re-rank's dot product, replayed with the kernel's operation order and FP32
# roundings: entries centred into FP32 pairs (centre_pair), products of pairs made exact up
# to the dropped al bl (DotPairSum.add), TwoSum accumulation folded into an FP64 sum every 8
# terms per lane, lanes (element t on lane t mod 32) added by an xor-shuffle tree. The stated
# bound is 2^-38 sum_t |a_t b_t| against the exact dot product of the centred rows.

_f32 = np.float32


def _two_sum(a, b):
    s = _f32(a + b)
    bb = _f32(s - a)
    return s, _f32(_f32(a - _f32(s - bb)) + _f32(b - bb))


def _fma(a, b, c):
    # the FP32 product is exact in FP64; one rounding of the sum to FP32 (at worst a double
    # rounding, far inside the bound checked)
    return _f32(np.float64(a) * np.float64(b) + np.float64(c))


def _centre(a, mh, ml):
    s, e = _two_sum(a, _f32(-mh))
    e2, r2 = _two_sum(e, _f32(-ml))
    h, l = _two_sum(s, e2)
    return h, _f32(l + r2)


def replay_pair_dot(x, y, mx, my, centered, drop=""):
    mxh = _f32(mx)
    mxl = _f32(mx - np.float64(mxh))
    myh = _f32(my)
    myl = _f32(my - np.float64(myh))
    lanes = []
    for lane in range(32):
        acc, S, E, n = np.float64(0.0), _f32(0.0), _f32(0.0), 0
        for t in range(lane, len(x), 32):
            ah, al = _centre(x[t], mxh, mxl) if centered else (x[t], _f32(0.0))
            bh, bl = _centre(y[t], myh, myl) if centered else (y[t], _f32(0.0))
            if drop == "lo":
                al = bl = _f32(0.0)
            pr = _f32(ah * bh)
            pe = _fma(ah, bh, _f32(-pr)) if drop != "pe" else _f32(0.0)
            pe = _fma(ah, bl, _fma(al, bh, pe))
            S, e2 = _two_sum(S, pr)
            E = _f32(E + _f32(e2 + pe))
            n += 1
            if n == 8:
                acc = np.float64(acc + (np.float64(S) + np.float64(E)))
                S, E, n = _f32(0.0), _f32(0.0), 0
        lanes.append(np.float64(acc + (np.float64(S) + np.float64(E))))
    o = 16
    while o > 0:
        lanes = [np.float64(lanes[i] + lanes[i ^ o]) for i in range(32)]
        o //= 2
    return float(lanes[0])


def _pair_dot_worst(drop, pairs):
    from fractions import Fraction
    worst = 0.0
    for d, kind, centered in ((3, "gauss", False), (64, "gauss", True), (256, "offset", True),
                              (1024, "gauss", False), (1024, "offset", True), (128, "wide", True),
                              (768, "lattice", True), (300, "lattice", False)):
        rng = np.random.default_rng(95 + d)
        for _ in range(pairs):
            if kind == "gauss":
                X = rng.standard_normal((2, d))
            elif kind == "offset":  # centring cancels most of each entry
                X = 1e4 + rng.standard_normal((2, d))
            elif kind == "wide":
                X = rng.standard_normal((2, d)) * 10.0 ** rng.uniform(-6, 6, (2, d))
            else:
                X = rng.integers(-3, 4, (2, d))
            x, y = X.astype(np.float32)
            mx = float(x.astype(np.float64).mean()) if centered else 0.0
            my = float(y.astype(np.float64).mean()) if centered else 0.0
            a = [Fraction(float(v)) - Fraction(mx) for v in x]
            b = [Fraction(float(v)) - Fraction(my) for v in y]
            exact = sum(p * q for p, q in zip(a, b))
            scale = sum(abs(p * q) for p, q in zip(a, b))
            got = Fraction(replay_pair_dot(x, y, mx, my, centered, drop))
            if scale == 0:
                continue
            worst = max(worst, float(abs(got - exact) / scale))
    return worst


def test_similarity_dot_within_2_pow_minus_38():
    worst = _pair_dot_worst("", 2)
    assert worst <= 2.0 ** -38, worst
    assert worst < 2.0 ** -44, worst  # FP64-class in practice


@pytest.mark.parametrize("drop", ["pe", "lo"])
def test_similarity_dot_needs_each_correction(drop):
    # without the products' rounding errors, or without the centred pairs' low parts, the same
    # rows leave the bound far behind
    assert _pair_dot_worst(drop, 1) > 2.0 ** -30
