"""Failure paths of the engine, exercised without a GPU fault: a device-side wait that
runs out (the kernel records KNN_ETIMEOUT, drains its own copies and MMAs, and the
context stays usable), and a workspace cap that the call cannot fit (KNN_ENOMEM from
the host before any device work of that call)."""
import numpy as np
import pytest

import oracle
from acceptance import check_exact
from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_bounded_wait_gives_up_with_a_status_and_the_device_stays_usable(monkeypatch):
    # 313 row blocks, so the re-rank warps wait for whole row-block sweeps: with one poll
    # allowed per wait the kernel gives up, and the call reports it
    X = inputs.integer_lattice(n=40000, d=128, seed=91)
    monkeypatch.setenv("KNN_SYMMETRIC", "0")  # the full sweep, whose re-rank warps wait on the epilogue
    monkeypatch.setenv("KNN_WAIT_LIMIT", "1")
    with pytest.raises(kb.KnnError) as err:
        kb.knng_build(dev(X), 16, precision="bf16", fused=1)
    torch.cuda.synchronize()
    assert err.value.status == kb.KNN_ETIMEOUT
    monkeypatch.delenv("KNN_WAIT_LIMIT")
    idx, dist = kb.knng_build(dev(X), 16, precision="bf16", fused=1)
    rows = inputs.sample_rows(len(X), 64, seed=92)
    check_exact(idx.cpu().numpy()[rows], dist.cpu().numpy()[rows], *oracle.knng(X, 16, rows=rows))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_workspace_cap_below_the_need_is_enomem(precision):
    X = inputs.integer_lattice(n=3000, d=64, seed=93)
    with pytest.raises(kb.KnnError) as err:
        kb.knng_build(dev(X), 8, precision=precision, max_workspace_bytes=4096)
    assert err.value.status == kb.KNN_ENOMEM
    assert "max_workspace_bytes" in str(err.value)
    idx, dist = kb.knng_build(dev(X), 8, precision=precision)
    check_exact(idx.cpu().numpy(), dist.cpu().numpy(), *oracle.knng(X, 8))
