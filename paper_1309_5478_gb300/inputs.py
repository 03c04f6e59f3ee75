"""Seeded synthetic inputs for the k-NN graph workloads.

This module only draws numbers: it holds none of the k-NN method's arithmetic
(no distances, norms of pairs, selection or ranking). Both the CUDA path's tests
and the FP64 oracle take their inputs from here, so a workload is defined once.

Random numbers come from a counter-based generator: splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
``key(seed, stream) + (i + 1) * golden_gamma``. Element ``i`` of stream ``s`` for
seed ``seed`` is therefore a pure function of ``(seed, s, i)`` and does not depend
on how the array is chunked, on numpy's version or on the machine.
Normals use the Box-Muller transform in FP64 and are rounded to FP32 at the end.

The paper benchmarks on uniformly random matrices (Results section); the
workloads below add the structure of the five workload families the engine is
measured on: integer lattice values, Gaussian mixtures, unit-norm directions
with exact duplicates, a batch of uneven problems, and an anisotropic mixture.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22  # elements per generation chunk (bounds temporary memory)

# stream identifiers (any distinct constants)
S_VALUES, S_COMPONENT, S_MEANS, S_SCALES, S_PERM, S_SHAPE, S_QUERY, S_SAMPLE, S_INIT = range(1, 10)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 0x2545F4914F6CDD1D + stream * 0x5851F42D4C957F2D) & (2**64 - 1)], dtype=np.uint64)
        return _mix(s + _GAMMA)[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit draws ``start .. start+count-1`` of ``(seed, stream)``."""
    k = _key(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(k + i * _GAMMA)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """FP64 uniforms in [0, 1) with 53 random bits."""
    return (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """FP64 standard normals by Box-Muller: uniforms 2p and 2p+1 give normals 2p (cosine) and 2p+1 (sine)."""
    p0 = start // 2
    p1 = (start + count + 1) // 2
    u = uniform(seed, stream, 2 * p0, 2 * (p1 - p0))
    r = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))  # 1 - u in (0, 1]
    theta = (2.0 * math.pi) * u[1::2]
    z = np.empty(2 * (p1 - p0), dtype=np.float64)
    z[0::2] = r * np.cos(theta)
    z[1::2] = r * np.sin(theta)
    off = start - 2 * p0
    return z[off:off + count]


def _rows_normal(seed: int, stream: int, n: int, d: int, row0: int = 0) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float64)
    rows_per = max(1, _CHUNK // max(d, 1))
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        out[r:r + m] = normal(seed, stream, (row0 + r) * d, m * d).reshape(m, d)
    return out


def _index_draw(seed: int, stream: int, n: int, upper: int, start: int = 0) -> np.ndarray:
    """n integers uniform in [0, upper)."""
    return np.minimum((uniform(seed, stream, start, n) * upper).astype(np.int64), upper - 1)


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """A seeded permutation of range(n): order of n distinct random 64-bit keys."""
    keys = u64(seed, stream, 0, n)
    return np.argsort(keys, kind="stable").astype(np.int64)


# ---------------------------------------------------------------------------
# workload families
# ---------------------------------------------------------------------------

SEED_BASE = 20130900


def integer_lattice(n: int = 4096, d: int = 128, lo: int = -8, hi: int = 8, seed: int = SEED_BASE + 1) -> np.ndarray:
    """Integer-valued FP32 points, each coordinate uniform in {lo..hi}."""
    span = hi - lo + 1
    out = np.empty((n, d), dtype=np.float32)
    rows_per = max(1, _CHUNK // d)
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        v = _index_draw(seed, S_VALUES, m * d, span, start=r * d) + lo
        out[r:r + m] = v.reshape(m, d).astype(np.float32)
    return out


def gaussian_mixture(n: int = 65536, d: int = 256, components: int = 64, mean_sigma: float = 2.0,
                     sigma: float = 0.5, seed: int = SEED_BASE + 2) -> np.ndarray:
    """Isotropic Gaussian mixture: means ~ N(0, mean_sigma^2 I), equal weights, per-component sigma."""
    means = _rows_normal(seed, S_MEANS, components, d) * mean_sigma
    comp = _index_draw(seed, S_COMPONENT, n, components)
    out = np.empty((n, d), dtype=np.float32)
    rows_per = max(1, _CHUNK // d)
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        z = normal(seed, S_VALUES, r * d, m * d).reshape(m, d)
        out[r:r + m] = (means[comp[r:r + m]] + sigma * z).astype(np.float32)
    return out


def unit_directions_with_duplicates(n: int = 262144, d: int = 1024, dup_fraction: float = 0.01,
                                    seed: int = SEED_BASE + 3) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Unit-norm Gaussian directions g/|g| plus exact duplicate points.

    round(dup_fraction * n) distinct target rows are overwritten with copies of
    as many distinct, non-target source rows. Returns (X, targets, sources).
    """
    out = np.empty((n, d), dtype=np.float32)
    rows_per = max(1, _CHUNK // d)
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        g = normal(seed, S_VALUES, r * d, m * d).reshape(m, d)
        g /= np.sqrt((g * g).sum(axis=1, keepdims=True))
        out[r:r + m] = g.astype(np.float32)
    n_dup = int(round(dup_fraction * n))
    perm = permutation(seed, S_PERM, n)
    targets = np.sort(perm[:n_dup])
    sources = perm[n_dup:2 * n_dup]
    out[targets] = out[sources]
    return out, targets, sources


def anisotropic_mixture(n: int = 524288, d: int = 768, components: int = 256, mean_sigma: float = 2.0,
                        scale_lo: float = 0.1, scale_hi: float = 2.0, seed: int = SEED_BASE + 5) -> np.ndarray:
    """Gaussian mixture with per-component diagonal scales log-uniform in [scale_lo, scale_hi]."""
    means = _rows_normal(seed, S_MEANS, components, d) * mean_sigma
    lu = uniform(seed, S_SCALES, 0, components * d).reshape(components, d)
    scales = np.exp(math.log(scale_lo) + lu * (math.log(scale_hi) - math.log(scale_lo)))
    comp = _index_draw(seed, S_COMPONENT, n, components)
    out = np.empty((n, d), dtype=np.float32)
    rows_per = max(1, _CHUNK // d)
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        z = normal(seed, S_VALUES, r * d, m * d).reshape(m, d)
        c = comp[r:r + m]
        out[r:r + m] = (means[c] + scales[c] * z).astype(np.float32)
    return out


def tight_groups(n: int = 262144, d: int = 1024, group: int = 128, spread: float = 0.01,
                 seed: int = SEED_BASE + 9) -> np.ndarray:
    """Groups of near-duplicate points: n / group unit-norm Gaussian centres g / |g|, each with
    `group` members c + spread * z / sqrt(d) (z standard normal), rows in a seeded order
    (members of a group are not adjacent). Within a group squared distances are about
    2 spread^2; between groups about 2."""
    groups = n // group
    centres = _rows_normal(seed, S_MEANS, groups, d)
    centres /= np.sqrt((centres * centres).sum(axis=1, keepdims=True))
    owner = permutation(seed, S_PERM, n) % groups
    out = np.empty((n, d), dtype=np.float32)
    rows_per = max(1, _CHUNK // d)
    scale = spread / math.sqrt(d)
    for r in range(0, n, rows_per):
        m = min(rows_per, n - r)
        z = normal(seed, S_VALUES, r * d, m * d).reshape(m, d)
        out[r:r + m] = (centres[owner[r:r + m]] + scale * z).astype(np.float32)
    return out


STRESS_KINDS = ("offset", "binades_bf16", "binades_fp8", "parallel")


def accumulation_stress(kind: str, n: int, d: int, seed: int = SEED_BASE + 8) -> np.ndarray:
    """Points chosen to stress the reduced-precision distance product (FP32 values).

    offset:       100 + N(0, 1) per coordinate (a large common offset: |c|^2 and 2 q.c cancel);
    binades_bf16: +-m 2^(e - 7), m uniform in {128..255}, e uniform in {-12..0}: every value is
                  exactly a BF16 number, spread over 13 binades (the rounding residual is zero, so
                  only the accumulation of the products is inexact);
    binades_fp8:  +-m 2^(e - 3), m uniform in {8..15}, e uniform in {-6..0}: exactly e4m3
                  numbers (up to a power-of-two row scale) over 7 binades;
    parallel:     unit rows (b + 0.01 g) / |b + 0.01 g| around one random unit direction b, with g
                  standard normal scaled by 1/sqrt(d): near-parallel directions.
    """
    count = n * d
    if kind == "offset":
        x = 100.0 + normal(seed, S_VALUES, 0, count)
    elif kind in ("binades_bf16", "binades_fp8"):
        bits, e_lo = (7, -12) if kind == "binades_bf16" else (3, -6)
        m = (1 << bits) + _index_draw(seed, S_VALUES, count, 1 << bits)
        e = e_lo + _index_draw(seed, S_SCALES, count, 1 - e_lo)
        sign = np.where(_index_draw(seed, S_COMPONENT, count, 2) == 0, -1.0, 1.0)
        x = sign * np.ldexp(m.astype(np.float64), (e - bits).astype(np.int64))
    elif kind == "parallel":
        b = normal(seed, S_MEANS, 0, d)
        b /= np.sqrt((b * b).sum())
        g = normal(seed, S_VALUES, 0, count).reshape(n, d) / math.sqrt(d)
        y = b[None, :] + 0.01 * g
        y /= np.sqrt((y * y).sum(axis=1, keepdims=True))
        return y.astype(np.float32)
    else:
        raise ValueError(f"unknown stress kind {kind!r}")
    return x.reshape(n, d).astype(np.float32)


def uniform_matrix(rows: int, cols: int, seed: int = SEED_BASE + 6) -> np.ndarray:
    """Uniformly random FP32 values in [0, 1): the paper's selection test matrices."""
    out = np.empty((rows, cols), dtype=np.float32)
    rows_per = max(1, _CHUNK // cols)
    for r in range(0, rows, rows_per):
        m = min(rows_per, rows - r)
        out[r:r + m] = uniform(seed, S_VALUES, r * cols, m * cols).reshape(m, cols).astype(np.float32)
    return out


@dataclass
class Problem:
    """One independent k-NN search problem of a batch."""
    M: int
    N: int
    d: int
    k: int
    seed: int

    def queries(self) -> np.ndarray:
        return _rows_normal(self.seed, S_QUERY, self.M, self.d).astype(np.float32)

    def corpus(self) -> np.ndarray:
        return _rows_normal(self.seed, S_VALUES, self.N, self.d).astype(np.float32)


BATCH_D = (64, 128, 256, 768)
BATCH_K = (1, 8, 32, 128, 512)


def batch_problems(count: int = 512, m_range=(256, 16384), n_range=(1024, 65536), d_choices=BATCH_D,
                   k_choices=BATCH_K, seed: int = SEED_BASE + 4) -> list[Problem]:
    """Shapes of a batch of independent problems; problem p draws its data from seed + 1 + p."""
    m = m_range[0] + _index_draw(seed, S_SHAPE, count, m_range[1] - m_range[0] + 1, start=0)
    n = n_range[0] + _index_draw(seed, S_SHAPE, count, n_range[1] - n_range[0] + 1, start=count)
    d = _index_draw(seed, S_SHAPE, count, len(d_choices), start=2 * count)
    k = _index_draw(seed, S_SHAPE, count, len(k_choices), start=3 * count)
    return [Problem(int(m[p]), int(n[p]), int(d_choices[d[p]]), min(int(k_choices[k[p]]), int(n[p])), seed + 1 + p)
            for p in range(count)]


def sample_rows(n: int, count: int, seed: int, stream: int = S_SAMPLE) -> np.ndarray:
    """``count`` distinct row indices of range(n), sorted (a seeded sample)."""
    count = min(count, n)
    return np.sort(permutation(seed, stream, n)[:count])
