"""Seeded input generators: determinism, chunking invariance and the workload recipes."""
import numpy as np

from paper_1309_5478_gb300 import inputs


def test_counter_based_streams_are_position_pure():
    a = inputs.u64(7, 3, 0, 1000)
    b = np.concatenate([inputs.u64(7, 3, 0, 10), inputs.u64(7, 3, 10, 990)])
    assert np.array_equal(a, b)
    assert not np.array_equal(inputs.u64(7, 3, 0, 100), inputs.u64(7, 4, 0, 100))
    z = inputs.normal(11, 1, 0, 1001)
    z2 = np.concatenate([inputs.normal(11, 1, 0, 1), inputs.normal(11, 1, 1, 1000)])
    assert np.array_equal(z, z2)


def test_splitmix64_reference_value():
    # splitmix64 seeded with 0: first output 0xE220A8397B1DCDAF (Steele et al. reference sequence)
    z = np.array([0x9E3779B97F4A7C15], dtype=np.uint64)
    assert int(inputs._mix(z)[0]) == 0xE220A8397B1DCDAF


def test_uniform_and_normal_moments():
    u = inputs.uniform(1, 1, 0, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = inputs.normal(1, 2, 0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_integer_lattice_recipe():
    X = inputs.integer_lattice(n=512, d=128)
    assert X.dtype == np.float32 and X.shape == (512, 128)
    assert X.min() == -8 and X.max() == 8 and np.array_equal(X, np.round(X))
    assert len(np.unique(X)) == 17
    assert np.array_equal(X, inputs.integer_lattice(n=512, d=128))


def test_unit_directions_duplicates():
    X, t, s = inputs.unit_directions_with_duplicates(n=5000, d=64, dup_fraction=0.01)
    assert len(t) == 50 and len(set(t) | set(s)) == 100
    assert np.array_equal(X[t], X[s])
    assert np.allclose((X.astype(np.float64) ** 2).sum(1), 1.0, atol=1e-6)


def test_mixtures_and_batch():
    X = inputs.gaussian_mixture(n=2048, d=32, components=4)
    assert X.shape == (2048, 32) and X.dtype == np.float32
    Y = inputs.anisotropic_mixture(n=1024, d=16, components=8)
    assert Y.shape == (1024, 16)
    ps = inputs.batch_problems(count=64)
    assert all(256 <= p.M <= 16384 and 1024 <= p.N <= 65536 for p in ps)
    assert {p.d for p in ps} <= set(inputs.BATCH_D) and {p.k for p in ps} <= set(inputs.BATCH_K)
    assert ps[0].queries().shape == (ps[0].M, ps[0].d)


def test_sample_rows():
    r = inputs.sample_rows(1000, 50, seed=3)
    assert len(r) == 50 and len(set(r)) == 50 and np.all(np.diff(r) > 0)
