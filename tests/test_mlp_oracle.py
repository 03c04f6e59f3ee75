"""The FP64 reference of the learned-threshold network against facts fixed without it:
a forward pass worked by hand on a sparse network, central finite differences of the
loss, the loss of a constant network, brute-force features on a tiny case and the
standardisation identity. Planted mistakes in copies of the reference must each fail
at least one of these pins."""
import math
import types

import numpy as np
import pytest

from oracle import mlp_oracle

F, H = mlp_oracle.F, mlp_oracle.H


def _params(rng, scale=0.1):
    p = np.zeros(mlp_oracle.N_PARAMS)
    p[:mlp_oracle.N_TRAIN] = rng.standard_normal(mlp_oracle.N_TRAIN) * scale
    o = mlp_oracle.N_TRAIN
    p[o:o + F] = rng.standard_normal(F) * 0.3          # mu
    p[o + F:o + 2 * F] = 0.5 + rng.random(F)           # sigma
    return p


def _index(name, *ij):
    """Position of a parameter in the flat layout W1[H][F] | b1 | W2 | b2 | mu | sigma | margin."""
    if name == "W1":
        return ij[0] * F + ij[1]
    base = {"b1": H * F, "W2": H * F + H, "b2": H * F + 2 * H, "mu": H * F + 2 * H + 1,
            "sigma": H * F + 2 * H + 1 + F}[name]
    return base + (ij[0] if ij else 0)


def pin_forward_by_hand(m):
    # two active hidden units reading features 1 and 3 (unit 0) and feature 2 (unit 5)
    p = np.zeros(m.N_PARAMS)
    p[_index("sigma", 0):_index("sigma", 0) + F] = 1.0
    p[_index("W1", 0, 1)] = 2.0
    p[_index("W1", 0, 3)] = -1.0
    p[_index("b1", 0)] = 0.5
    p[_index("W1", 5, 2)] = 1.0
    p[_index("b1", 5)] = -1.0
    p[_index("W2", 0)] = 3.0
    p[_index("W2", 5)] = -2.0
    p[_index("b2")] = 0.25
    X = np.zeros((3, F))
    X[0, 1], X[0, 3], X[0, 2] = 1.0, 0.5, 4.0   # unit0: 2 - 0.5 + 0.5 = 2 ; unit5: 3
    X[1, 1], X[1, 3], X[1, 2] = -1.0, 0.0, 0.5  # unit0: -1.5 -> 0 ; unit5: -0.5 -> 0
    X[2, 1], X[2, 3], X[2, 2] = 0.0, -2.0, 1.5  # unit0: 2.5 ; unit5: 0.5
    want = [0.25 + 3 * 2.0 - 2 * 3.0, 0.25, 0.25 + 3 * 2.5 - 2 * 0.5]
    assert np.allclose(m.forward(p, X), want, rtol=0, atol=1e-12)


def pin_standardisation(m):
    rng = np.random.default_rng(7)
    p = _params(rng)
    X = rng.standard_normal((5, F))
    mu = p[_index("mu"):_index("mu") + F].copy()
    sg = p[_index("sigma"):_index("sigma") + F].copy()
    q = p.copy()
    q[_index("mu"):_index("mu") + F] = 0.0
    q[_index("sigma"):_index("sigma") + F] = 1.0
    Z = np.array([[(X[r, f] - mu[f]) / sg[f] for f in range(F)] for r in range(5)])
    assert np.allclose(m.forward(p, X), m.forward(q, Z), rtol=1e-12, atol=1e-12)


def pin_constant_network_loss(m):
    # W2 = 0: y = b2 for every row, loss = mean (b2 - t)^2, d/db2 = 2 mean (b2 - t)
    rng = np.random.default_rng(3)
    p = _params(rng)
    p[_index("W2", 0):_index("W2", 0) + H] = 0.0
    p[_index("b2")] = 1.5
    T = [0.5, 2.0, -1.0, 1.5]
    X = rng.standard_normal((4, F))
    loss, g = m.loss_grad(p, X, T)
    want = sum((1.5 - t) ** 2 for t in T) / 4
    assert abs(loss - want) < 1e-12
    assert abs(g[_index("b2")] - 2 * sum(1.5 - t for t in T) / 4) < 1e-12
    assert np.all(g[:H * F] == 0) and np.all(g[H * F:H * F + H] == 0)  # no signal reaches layer 1


def pin_gradcheck(m):
    rng = np.random.default_rng(11)
    p = _params(rng, scale=0.2)
    X = rng.standard_normal((24, F)) * 1.5 + p[_index("mu"):_index("mu") + F]
    T = rng.standard_normal(24)
    loss, g = m.loss_grad(p, X, T)
    assert abs(loss - float(np.mean((m.forward(p, X) - T) ** 2))) < 1e-12
    picks = list(rng.choice(H * F, 24, replace=False)) + [_index("b1", i) for i in (0, 7, 100)] + \
        [_index("W2", i) for i in (1, 64, 127)] + [_index("b2")]
    h = 1e-6
    for i in picks:
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd = (m.loss_grad(a, X, T)[0] - m.loss_grad(b, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def pin_features_brute_force(m):
    rng = np.random.default_rng(5)
    d = 3
    Q = rng.standard_normal((2, d))
    S = rng.standard_normal((F - 1, d))
    S[17] = Q[1]  # a sample equal to the query: zero distance, floored log
    got = m.features(Q, S)
    for r in range(2):
        assert abs(got[r, 0] - math.log(sum(Q[r, t] ** 2 for t in range(d)))) < 1e-12
        dist = sorted(sum((Q[r, t] - S[j, t]) ** 2 for t in range(d)) for j in range(F - 1))
        for j in range(F - 1):
            want = math.log(dist[j]) if dist[j] > 0 else m.LOG_FLOOR
            assert abs(got[r, 1 + j] - max(want, m.LOG_FLOOR)) < 1e-9
    assert got[1, 1] == m.LOG_FLOOR


PINS = [pin_forward_by_hand, pin_standardisation, pin_constant_network_loss, pin_gradcheck,
        pin_features_brute_force]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(mlp_oracle)


MUTANTS = [
    ("ReLU dropped in the forward pass", "return np.maximum(A, 0.0) @ W2 + b2", "return A @ W2 + b2"),
    ("ReLU mask dropped in the backward pass", "dA = np.outer(dy, W2) * (A > 0)", "dA = np.outer(dy, W2)"),
    ("layer-1 gradient on raw features", "dW1 = dA.T @ Xn", "dW1 = dA.T @ np.asarray(X, dtype=np.float64)"),
    ("factor 2 of the squared error dropped", "dy = 2.0 * e / n", "dy = e / n"),
    ("residual sign flipped", "e = y - T", "e = T - y"),
    ("standardisation multiplies by sigma", "- mu) / sigma", "- mu) * sigma"),
    ("W1 read transposed", "p[o:o + H * F].reshape(H, F)", "p[o:o + H * F].reshape(F, H).T"),
    ("W2 and b1 swapped", "b1 = p[o:o + H]; o += H\n    W2 = p[o:o + H]; o += H",
     "W2 = p[o:o + H]; o += H\n    b1 = p[o:o + H]; o += H"),
    ("distance features unsorted", "np.log(np.sort(d2, axis=1))", "np.log(d2)"),
    ("distances not squared", "np.log(np.sort(d2, axis=1))", "np.log(np.sort(np.sqrt(d2), axis=1))"),
    ("mean over rows dropped", "loss = float(np.mean(e * e))", "loss = float(np.sum(e * e))"),
]


def _failing_pins(module):
    failed = []
    for pin in PINS:
        try:
            pin(module)
        except Exception:  # noqa: BLE001 -- any failure (assert or crash) catches the mistake
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(desc, old, new):
    src = open(mlp_oracle.__file__).read()
    assert old in src, f"mutation anchor missing: {old!r}"
    mod = types.ModuleType("mlp_mutant")
    exec(compile(src.replace(old, new), "mlp_mutant", "exec"), mod.__dict__)
    assert _failing_pins(mod), f"no pin caught the planted mistake: {desc}"


def test_unmutated_reference_passes_all_pins():
    assert _failing_pins(mlp_oracle) == []
