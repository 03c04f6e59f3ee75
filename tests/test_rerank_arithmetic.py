"""The exact re-rank's FP32 distance arithmetic, replayed on the CPU (no GPU needed).

The re-rank computes sum_t (q_t - c_t)^2 in FP32 with a fixed order: lanes of a group of
G (8, 16 or 32) take 16-byte pieces of the rows in turn, two at a time (pieces t and t + 4G);
the eight squares of a pair of pieces are summed with a multiply and seven fused
multiply-adds, those sums are accumulated per lane with TwoSum into a (sum, error) pair,
each lane rounds its pair to one float, and the lanes' floats are summed by an xor-shuffle
tree. The near-tie rule (FP32 distances within
2^-19 of each other are ordered in FP64) and the early stop need this to be within 2^-20
of the exact distance; these tests replay the same operations with FP32 rounding after
every step and check that bound against FP64 on inputs chosen to stress it.
"""
import numpy as np
import pytest

f32 = np.float32


def _fma(a, b, c):
    # a * b is exact in FP64 for FP32 operands; one rounding of the FP64 sum to FP32
    # (a double rounding at worst, well inside the bound checked below)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    err = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, err


def replay(q: np.ndarray, c: np.ndarray, G: int) -> np.float32:
    """FP32 distance with the re-rank's operation order for a group of G lanes."""
    d = q.shape[0]
    pad = (-d) % 4
    qp = np.concatenate([q, np.zeros(pad, np.float32)])
    cp = np.concatenate([c, np.zeros(pad, np.float32)])
    lane_vals = []
    for gl in range(G):
        s = f32(0.0)
        e = f32(0.0)
        for t in range(gl * 4, d, 8 * G):
            pos = [t + i for i in range(4)] + [t + 4 * G + i for i in range(4)]
            diffs = [f32(qp[p] - cp[p]) if p < len(qp) else f32(0.0) for p in pos]
            g = f32(diffs[0] * diffs[0])
            for x in diffs[1:]:
                g = _fma(x, x, g)
            s, err = _two_sum(s, g)
            e = f32(e + err)
        lane_vals.append(f32(s + e))
    v = lane_vals
    o = G // 2
    while o > 0:
        v = [f32(v[i] + v[i ^ o]) for i in range(G)]
        o //= 2
    return v[0]


def _cases(rng):
    for d in (3, 64, 130, 256, 768, 1024, 4096):
        yield d, rng.standard_normal(d).astype(np.float32), rng.standard_normal(d).astype(np.float32)
        # a large common offset: the direct difference keeps only the small part
        off = f32(1000.0)
        yield d, (off + rng.standard_normal(d)).astype(np.float32), (off + rng.standard_normal(d)).astype(np.float32)
        # entries over many binades
        sc = np.exp2(rng.integers(-20, 20, size=d)).astype(np.float32)
        yield d, (rng.standard_normal(d) * sc).astype(np.float32), (rng.standard_normal(d) * sc).astype(np.float32)
        # near neighbours: tiny differences of large values
        base = rng.standard_normal(d).astype(np.float32)
        yield d, base, (base + f32(1e-3) * rng.standard_normal(d)).astype(np.float32)
    # a constant difference: every lane adds the same piece sum again and again, so the
    # roundings of an uncompensated running sum line up (about 2e-6 at d = 4096 with this
    # value, above the bound; the TwoSum accumulation keeps them)
    for d in (1024, 4096):
        yield d, np.full(d, f32(1.5059366), np.float32), np.zeros(d, np.float32)


@pytest.mark.parametrize("G", [8, 16, 32])
def test_distance_within_2_pow_minus_20(G):
    rng = np.random.default_rng(20130910 + G)
    worst = 0.0
    for _ in range(3):
        for d, q, c in _cases(rng):
            exact = float(np.sum((q.astype(np.float64) - c.astype(np.float64)) ** 2))
            got = float(replay(q, c, G))
            if exact == 0.0:
                assert got == 0.0
                continue
            rel = abs(got - exact) / exact
            worst = max(worst, rel)
            assert rel <= 2.0 ** -20, (G, d, rel)
    # the bound is met with room: rounding errors of non-negative sums do not all align
    assert worst < 2.0 ** -21


def test_integer_inputs_are_exact():
    """Integer coordinates whose squared distance stays below 2^24 come out exact (every
    partial sum is an integer below 2^24), which the bit-exact integer parity relies on."""
    rng = np.random.default_rng(7)
    for G in (8, 16, 32):
        for d in (1, 5, 64, 128, 257):
            q = rng.integers(-8, 9, size=d).astype(np.float32)
            c = rng.integers(-8, 9, size=d).astype(np.float32)
            exact = int(np.sum((q.astype(np.int64) - c.astype(np.int64)) ** 2))
            assert float(replay(q, c, G)) == float(exact)
