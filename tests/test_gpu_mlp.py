"""GPU parity of the learned-threshold network (features, forward, loss and gradient,
training, thresholds) against its FP64 reference, and exactness of k-NN graphs built
with the proposed per-row thresholds, through the C ABI."""
import numpy as np
import pytest

import oracle
from acceptance import check_float
from oracle import mlp_oracle
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

F = kb.MLP_FEATURES


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def random_params(seed, scale=0.05):
    rng = np.random.default_rng(seed)
    p = np.zeros(kb.mlp_param_count(), dtype=np.float32)
    p[:kb.MLP_TRAINED] = rng.standard_normal(kb.MLP_TRAINED) * scale
    o = kb.MLP_TRAINED
    p[o:o + F] = rng.standard_normal(F) * 0.5
    p[o + F:o + 2 * F] = 0.5 + rng.random(F)
    return p


def test_features_match_reference():
    X = inputs.anisotropic_mixture(n=700, d=96, components=8, seed=41)
    Q, S = X[:300], X[300:556]
    S = S.copy()
    S[5] = Q[7]  # a sample equal to a query: zero distance, floored log
    got = kb.mlp_features(dev(Q), dev(S)).cpu().numpy().astype(np.float64)
    want = mlp_oracle.features(Q, S)
    q2 = (Q.astype(np.float64) ** 2).sum(1)
    s2max = (S.astype(np.float64) ** 2).sum(1).max()
    assert np.allclose(got[:, 0], want[:, 0], rtol=0, atol=1e-5)
    # sorted squared distances from the FP32 expanded form: error below (d + 4) 2^-23 (|q| + |s|)^2
    tol = (96 + 4) * 2.0 ** -23 * 2 * (q2[:, None] + s2max) * 2
    assert np.all(np.abs(np.exp(got[:, 1:]) - np.exp(want[:, 1:])) <= tol)
    assert np.all(np.diff(got[:, 1:], axis=1) >= 0)
    assert got[7, 1] == mlp_oracle.LOG_FLOOR or np.exp(got[7, 1]) <= tol[7, 0]


@pytest.mark.parametrize("n", [1, 1000, 4133])
def test_loss_and_gradient_match_reference(n):
    rng = np.random.default_rng(n)
    p = random_params(n)
    X = (rng.standard_normal((n, F)) * 2 + 1).astype(np.float32)
    T = rng.standard_normal(n).astype(np.float32)
    loss, g = kb.mlp_loss_grad(dev(X), dev(T), dev(p))
    g = g.cpu().numpy().astype(np.float64)
    want_loss, want_g = mlp_oracle.loss_grad(p, X, T)
    assert abs(loss - want_loss) <= 1e-5 * want_loss
    assert np.linalg.norm(g - want_g) <= 1e-4 * np.linalg.norm(want_g)
    assert np.max(np.abs(g - want_g)) <= 1e-4 * np.max(np.abs(want_g))


def test_training_reduces_loss_and_predictions_match_reference():
    rng = np.random.default_rng(2)
    n = 6000
    X = rng.standard_normal((n, F)).astype(np.float32) * 3 + 2
    w = rng.standard_normal(F) / np.sqrt(F)
    T = (np.tanh((X - 2) @ w / 3) * 2 + 0.1 * rng.standard_normal(n)).astype(np.float32)
    p = np.zeros(kb.mlp_param_count(), dtype=np.float32)
    p[:kb.MLP_TRAINED] = rng.standard_normal(kb.MLP_TRAINED) * 0.02
    pd = dev(p)
    hist = kb.mlp_train(dev(X), dev(T), pd, epochs=25, batch=512, lr=2e-3, holdout=0.2, margin_quantile=0.95)
    assert hist[-1] < 0.25 * hist[0], hist
    pt = pd.cpu().numpy()
    n_train = n - round(n * 0.2)
    mu = pt[kb.MLP_TRAINED:kb.MLP_TRAINED + F]
    assert np.allclose(mu, X[:n_train].astype(np.float64).mean(0), rtol=1e-4, atol=1e-4)
    y, thr = kb.mlp_predict(dev(X), pd)
    y = y.cpu().numpy()
    want_y = mlp_oracle.forward(pt, X)
    assert np.allclose(y, want_y, rtol=1e-4, atol=1e-4)
    res = np.sort(T[n_train:] - want_y[n_train:])
    q = min(len(res) - 1, int(0.95 * (len(res) - 1) + 0.5))
    margin = float(pt[-1])
    assert margin >= 0 and abs(margin - max(0.0, res[q])) <= 1e-3
    assert np.allclose(thr.cpu().numpy(), np.exp(want_y + margin), rtol=1e-4)


def test_parameter_file_round_trip_on_device(tmp_path):
    p = dev(random_params(9))
    kb.mlp_save(tmp_path / "p.bin", p)
    q = torch.zeros_like(p)
    kb.mlp_load(tmp_path / "p.bin", q)
    assert torch.equal(p, q)


def _learned_thresholds(X, k, n_train, seed):
    """Thresholds for every row from a network trained on n_train rows whose targets
    (the exact k-th squared distance without the row itself) come from the engine."""
    Xd = dev(X)
    rows = inputs.sample_rows(len(X), n_train, seed=seed)
    S = X[inputs.sample_rows(len(X), F - 1, seed=seed + 1)]
    feats = kb.mlp_features(Xd, dev(S))
    _, dist = kb.knn_search(dev(X[rows]), Xd, k + 1)
    targets = torch.log(dist[:, k].contiguous())
    params = torch.zeros(kb.mlp_param_count(), dtype=torch.float32, device="cuda")
    g = torch.Generator().manual_seed(seed)
    params[:kb.MLP_TRAINED] = (torch.randn(kb.MLP_TRAINED, generator=g) * 0.02).cuda()
    ridx = torch.from_numpy(rows).cuda()
    kb.mlp_train(feats[ridx].contiguous(), targets, params, epochs=30, batch=256, lr=2e-3, holdout=0.1,
                 margin_quantile=0.99)
    _, thr = kb.mlp_predict(feats, params)
    return thr


@pytest.mark.parametrize("precision", ["auto", "fp32"])
def test_learned_threshold_keeps_graph_exact(precision):
    X = inputs.anisotropic_mixture(n=12000, d=128, components=16, seed=43)
    k = 50
    thr = _learned_thresholds(X, k, 3000, seed=44)
    Xd = dev(X)
    i0, d0, s0 = kb.knng_build(Xd, k, precision=precision, return_stats=True)
    i1, d1, s1 = kb.knng_build(Xd, k, precision=precision, row_threshold=thr, return_stats=True)
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    # most rows keep the proposal (the network is trained on the same distribution)
    assert s1["threshold_misses"] <= 0.05 * len(X)
    rows = inputs.sample_rows(len(X), 150, seed=45)
    ref_idx, ref_dist = oracle.knng(X, k, rows=rows)
    check_float(X, X, rows, i1.cpu().numpy()[rows], d1.cpu().numpy()[rows], ref_idx, ref_dist, exclude_self=True)


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_threshold_below_the_answer_falls_back_exactly(precision):
    X = inputs.anisotropic_mixture(n=5000, d=64, components=8, seed=47)
    k = 20
    Xd = dev(X)
    i0, d0 = kb.knng_build(Xd, k, precision=precision)
    # proposals: a quarter of the k-th distance on even rows (cuts the answer), generous on odd rows,
    # no threshold (NaN / inf / negative) on every 7th row
    thr = d0[:, k - 1].clone()
    thr[0::2] *= 0.25
    thr[1::2] *= 4.0
    thr[0::7] = float("nan")
    thr[3::7] = float("inf")
    thr[5::7] = -1.0
    i1, d1, s1 = kb.knng_build(Xd, k, precision=precision, row_threshold=thr.contiguous(), return_stats=True)
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    assert s1["threshold_misses"] > 0


def test_learned_threshold_cuts_the_select_work(monkeypatch):
    # what the trained network gains over the method without it: with the plain running
    # threshold (no speculation), the keys the fused sweep lets into candidate lists, with and
    # without the learned per-row thresholds, on the same clustered points; answers identical
    monkeypatch.setenv("KNN_SPECULATE", "0")
    X = inputs.anisotropic_mixture(n=20000, d=128, components=16, seed=48)
    k = 50
    thr = _learned_thresholds(X, k, 4000, seed=49)
    Xd = dev(X)
    i0, d0, s0 = kb.knng_build(Xd, k, precision="bf16", fused=1, return_stats=True)
    i1, d1, s1 = kb.knng_build(Xd, k, precision="bf16", fused=1, row_threshold=thr, return_stats=True)
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    assert s0["candidates_inserted"] > 0
    assert s1["candidates_inserted"] < 0.6 * s0["candidates_inserted"], (s0["candidates_inserted"],
                                                                         s1["candidates_inserted"])
