"""GPU parity of the batched form (one CUDA graph: persistent fused launch over the
work items of many problems + the plain form for the rest) against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle
from acceptance import check_exact, check_float
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (M, N, d, k, graph)
SHAPES = [(300, 300, 64, 8, True), (257, 5000, 96, 1, False), (1000, 3000, 128, 32, False),
          (129, 129, 37, 16, True), (640, 2100, 768, 64, False), (77, 1500, 64, 128, False),
          (200, 2000, 256, 512, False), (1500, 1500, 128, 20, True)]


def make_problems(shapes, seed0=300, integer=True, device="cuda"):
    probs, refs = [], []
    for i, (M, N, d, k, graph) in enumerate(shapes):
        gen = (lambda n, s: inputs.integer_lattice(n=n, d=d, lo=-6, hi=6, seed=s)) if integer else \
              (lambda n, s: inputs.gaussian_mixture(n=n, d=d, components=4, seed=s))
        C = gen(N, seed0 + 2 * i)
        Q = None if graph else gen(M, seed0 + 2 * i + 1)
        Ct = torch.from_numpy(C).to(device)
        Qt = None if graph else torch.from_numpy(Q).to(device)
        oi = torch.empty((M, k), dtype=torch.int32, device=device)
        od = torch.empty((M, k), dtype=torch.float32, device=device)
        probs.append({"Q": Qt, "C": Ct, "k": k, "out_idx": oi, "out_dist": od})
        refs.append((Q, C, k, graph))
    return probs, refs


def check_all(probs, refs, exact=True):
    for p, (Q, C, k, graph) in zip(probs, refs):
        idx, dist = p["out_idx"].cpu().numpy(), p["out_dist"].cpu().numpy()
        if exact:
            ref = oracle.knng(C, k) if graph else oracle.knn(Q, C, k)
            check_exact(idx, dist, *ref)
        else:
            QQ = C if graph else Q
            rows = inputs.sample_rows(QQ.shape[0], 24, seed=k)
            ri, rd = oracle.knn(QQ, C, k, rows=rows, exclude_self=graph)
            check_float(QQ, C, rows, idx[rows], dist[rows], ri, rd, graph)


@pytest.fixture(autouse=True)
def no_autotune(monkeypatch, tmp_path):
    monkeypatch.setenv("KNN_AUTOTUNE", "0")
    monkeypatch.setenv("KNN_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))


def test_mixed_batch_bit_exact():
    probs, refs = make_problems(SHAPES)
    st = kb.knn_search_batched(probs)
    assert st == [0] * len(probs)
    torch.cuda.synchronize()
    check_all(probs, refs)


@pytest.mark.parametrize("integer", [True, False])
def test_128_column_tiles(monkeypatch, integer):
    # every problem whose lists hold at most 512 keys on 128 x 128 tiles (two CTAs an SM), the
    # others (k = 512) on 128 x 256 tiles in the same batch
    monkeypatch.setenv("KNN_BATCH_TILE", "128")
    probs, refs = make_problems(SHAPES, seed0=460, integer=integer)
    st = kb.knn_search_batched(probs)
    assert st == [0] * len(probs)
    torch.cuda.synchronize()
    check_all(probs, refs, exact=integer)


def test_graph_replay_gives_the_same_answer():
    probs, refs = make_problems(SHAPES[:5], seed0=400)
    kb.knn_search_batched(probs)
    first = [(p["out_idx"].clone(), p["out_dist"].clone()) for p in probs]
    for p in probs:
        p["out_idx"].fill_(-7)
        p["out_dist"].fill_(-7.0)
    kb.knn_search_batched(probs)  # same signature: the cached graph is replayed
    for p, (i0, d0) in zip(probs, first):
        assert torch.equal(p["out_idx"], i0) and torch.equal(p["out_dist"], d0)
    check_all(probs, refs)


def test_alternating_batches_keep_their_own_descriptors():
    # two batches share the batch workspace; each keeps its graph and layout, and the descriptors
    # the workspace holds are uploaded again whenever the other batch ran in between
    pa, ra = make_problems(SHAPES[:4], seed0=420)
    pb, rb = make_problems(SHAPES[4:], seed0=440)
    runs = []
    for probs in (pa, pb, pa, pb, pa):
        for p in probs:
            p["out_idx"].fill_(-7)
            p["out_dist"].fill_(-7.0)
        assert kb.knn_search_batched(probs) == [0] * len(probs)
        runs.append([(p["out_idx"].clone(), p["out_dist"].clone()) for p in probs])
    for a, b in ((0, 2), (2, 4), (1, 3)):
        for (i0, d0), (i1, d1) in zip(runs[a], runs[b]):
            assert torch.equal(i0, i1) and torch.equal(d0, d1)
    check_all(pa, ra)
    check_all(pb, rb)


def test_batch_recipe_float_data():
    ps = inputs.batch_problems(count=16, m_range=(256, 1024), n_range=(1024, 6000))
    probs, refs = [], []
    for pr in ps:
        Q, C = pr.queries(), pr.corpus()
        probs.append({"Q": torch.from_numpy(Q).cuda(), "C": torch.from_numpy(C).cuda(), "k": pr.k,
                      "out_idx": torch.empty((pr.M, pr.k), dtype=torch.int32, device="cuda"),
                      "out_dist": torch.empty((pr.M, pr.k), dtype=torch.float32, device="cuda")})
        refs.append((Q, C, pr.k, False))
    assert kb.knn_search_batched(probs) == [0] * len(probs)
    torch.cuda.synchronize()
    check_all(probs, refs, exact=False)


def test_host_and_device_problems_mix():
    probs, refs = make_problems(SHAPES[:3], seed0=500)
    hp, hrefs = make_problems(SHAPES[3:4], seed0=600, device="cpu")
    st = kb.knn_search_batched(probs + hp)
    assert st == [0] * 4
    check_all(probs + hp, refs + hrefs)


def test_bad_problem_reports_its_status():
    probs, refs = make_problems(SHAPES[:2], seed0=700)
    bad = dict(probs[1])
    bad["k"] = 10 ** 6
    with pytest.raises(kb.KnnError):
        kb.knn_search_batched([probs[0], bad])


TUNE_SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs
C = torch.from_numpy(inputs.integer_lattice(n=4000, d=128, lo=-6, hi=6, seed=801)).cuda()
Q = torch.from_numpy(inputs.integer_lattice(n=500, d=128, lo=-6, hi=6, seed=802)).cuda()
probs = [{"Q": Q, "C": C, "k": 16, "out_idx": torch.empty((500, 16), dtype=torch.int32, device="cuda"),
          "out_dist": torch.empty((500, 16), dtype=torch.float32, device="cuda")}]
st, stats = kb.knn_search_batched(probs, return_stats=True)
print(json.dumps({"status": st, "fused_used": stats["fused_used"]}))
"""


def run_tuned_batch(cache):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, KNN_AUTOTUNE="1", KNN_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", TUNE_SCRIPT, root], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_autotuner_cache_is_written_keyed_and_reused(tmp_path):
    # each run is a fresh process: the cache file, not memory, carries the choices
    import json
    cache = tmp_path / "tune.json"
    first = run_tuned_batch(cache)
    assert first["status"] == [0]
    data = json.loads(cache.read_text())
    tag = data.pop("_device")
    assert " sm" in tag and tag.endswith(" v4"), tag
    assert data and all(v in (1, 2, 3, 4, 5) for v in data.values()), data  # measured: plain or a fused variant
    # a second process follows the file: every bucket forced to the plain form
    cache.write_text(json.dumps({"_device": tag, **{b: 1 for b in data}}))
    second = run_tuned_batch(cache)
    assert second["status"] == [0] and second["fused_used"] == 0
    # entries of another device are ignored: the bucket is measured again and the file rewritten
    cache.write_text(json.dumps({"_device": "another GPU sm1 v4", **{b: 1 for b in data}}))
    third = run_tuned_batch(cache)
    assert third["status"] == [0]
    again = json.loads(cache.read_text())
    assert again.pop("_device") == tag and set(again) == set(data)


def test_uncertified_rows_of_a_batch_are_recomputed():
    # a crowded problem (points close together far from the origin: the reduced-precision
    # bound dwarfs the distances, lists overflow and rows stay uncertified) next to an
    # ordinary one; only the crowded problem's rows go through the fallback, and both are exact
    rng = np.random.default_rng(81)
    base = rng.standard_normal(64).astype(np.float32) * 30
    C1 = (base + 0.05 * rng.standard_normal((3000, 64))).astype(np.float32)
    Q1 = (base + 0.05 * rng.standard_normal((200, 64))).astype(np.float32)
    C2 = inputs.gaussian_mixture(n=2500, d=64, components=4, seed=82)
    Q2 = inputs.gaussian_mixture(n=150, d=64, components=4, seed=83)
    probs, refs = [], []
    for Q, C, k in ((Q1, C1, 10), (Q2, C2, 12)):
        probs.append({"Q": torch.from_numpy(Q).cuda(), "C": torch.from_numpy(C).cuda(), "k": k,
                      "out_idx": torch.empty((Q.shape[0], k), dtype=torch.int32, device="cuda"),
                      "out_dist": torch.empty((Q.shape[0], k), dtype=torch.float32, device="cuda")})
        refs.append((Q, C, k, False))
    st, stats = kb.knn_search_batched(probs, precision="bf16", return_stats=True)
    assert st == [0, 0]
    assert 0 < stats["rows_fallback"] <= Q1.shape[0]
    check_all(probs, refs, exact=False)
