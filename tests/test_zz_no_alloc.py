"""knn_select_noalloc (the allocation-free select, for callers that cannot let the
library allocate device memory) matches knn_select, on two calls in a row that share
its fixed scratch array. Collected last so a failure here leaves every other test run."""
import numpy as np
import pytest

from paper_1309_5478_gb300 import binding as kb
from paper_1309_5478_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_select_matches_select_on_two_calls():
    # the second and third shapes take the block-per-row select (k >= 128, and few rows)
    for call, (rows, cols, k, seed) in enumerate([(777, 5003, 64, 5), (300, 20000, 300, 6), (12, 70000, 17, 7)]):
        D = torch.from_numpy(inputs.uniform_matrix(rows, cols, seed=seed)).cuda()
        ref_i, ref_v = kb.knn_select(D, k)
        oi = torch.empty((rows, k), dtype=torch.int32, device="cuda")
        ov = torch.empty((rows, k), dtype=torch.float32, device="cuda")
        kb.knn_select_noalloc(D, k, oi, ov)
        torch.cuda.synchronize()
        assert torch.equal(oi, ref_i), f"call {call}: indices differ"
        assert torch.equal(ov, ref_v), f"call {call}: values differ"


def test_noalloc_select_rejects_what_it_cannot_do():
    D = torch.zeros((4, 16), device="cuda")
    oi = torch.empty((4, 2), dtype=torch.int32, device="cuda")
    ov = torch.empty((4, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(kb.KnnError):  # host arrays would need staging
        kb.knn_select_noalloc(D.cpu(), 2, oi, ov)
    D[2, 5] = float("nan")
    with pytest.raises(kb.KnnError):
        kb.knn_select_noalloc(D, 2, oi, ov)
    D[2, 5] = 0.0
    kb.knn_select_noalloc(D, 2, oi, ov)  # the error word is cleared per call


def test_noalloc_select_on_a_column_slice():
    # ldd > N: the first 3001 columns of a 5000-column matrix; every row's status word
    # must still be covered by the fixed array
    D = torch.from_numpy(inputs.uniform_matrix(901, 5000, seed=8)).cuda()
    ref_i, ref_v = kb.knn_select(D, 40, n=3001)
    oi = torch.empty((901, 40), dtype=torch.int32, device="cuda")
    ov = torch.empty((901, 40), dtype=torch.float32, device="cuda")
    kb.knn_select_noalloc(D, 40, oi, ov, n=3001)
    torch.cuda.synchronize()
    assert torch.equal(oi, ref_i) and torch.equal(ov, ref_v)
    assert int(oi.max()) < 3001
