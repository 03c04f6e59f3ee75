"""The C-ABI library loads on a machine without a GPU and exports every entry point
that include/knn.h declares; host-only calls (status strings, argument checks)
work without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(knn\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_5478_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("knng_build", "knng_build_ex", "knn_search", "knn_select", "knn_search_batched",
                     "knn_status_string", "knn_last_error", "knn_shutdown"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1309_5478_gb300 import binding
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTS) <= set(names)


def test_host_only_calls(lib):
    assert lib.knn_status_string(-1) == b"KNN_EINVAL"
    assert lib.knn_status_string(0) == b"KNN_OK"
    assert lib.knn_version().decode().count(".") == 2


def test_argument_checks_need_no_device(lib):
    from paper_1309_5478_gb300 import binding
    X = np.zeros((10, 4), dtype=np.float32)
    oi = np.zeros((10, 3), dtype=np.int32)
    od = np.zeros((10, 3), dtype=np.float32)
    p = X.ctypes.data
    assert lib.knng_build(p, 10, 4, 0, oi.ctypes.data, od.ctypes.data) == binding.KNN_EINVAL
    assert b"k must be" in lib.knn_last_error()
    assert lib.knng_build(p, 10, 4, 10, oi.ctypes.data, od.ctypes.data) == binding.KNN_EINVAL
    assert lib.knng_build(p, 10, 0, 3, oi.ctypes.data, od.ctypes.data) == binding.KNN_EINVAL
    assert lib.knng_build(None, 10, 4, 3, oi.ctypes.data, od.ctypes.data) == binding.KNN_EINVAL
    opt = binding.KnnOptions()
    lib.knn_options_init(ctypes.byref(opt))
    assert opt.rerank_extra == 32 and opt.precision == binding.KNN_AUTO and opt.fused == -1
    assert lib.knn_search(p, 10, p, 10, 4, 11, oi.ctypes.data, od.ctypes.data, ctypes.byref(opt)) == binding.KNN_EINVAL
    # similarity metrics and the streamed corpus check their arguments before any device work
    assert lib.knn_search_metric(p, 10, p, 10, 4, 3, 7, oi.ctypes.data, od.ctypes.data,
                                 ctypes.byref(opt)) == binding.KNN_EINVAL
    assert b"unknown metric" in lib.knn_last_error()
    assert lib.knng_build_metric(p, 10, 4, 10, binding.METRICS["cosine"], oi.ctypes.data, od.ctypes.data,
                                 ctypes.byref(opt)) == binding.KNN_EINVAL
    thr = np.ones(10, dtype=np.float32)
    opt_t = binding.make_options(row_threshold=thr)
    assert lib.knn_search_metric(p, 10, p, 10, 4, 3, binding.METRICS["pearson"], oi.ctypes.data, od.ctypes.data,
                                 ctypes.byref(opt_t)) == binding.KNN_EINVAL
    assert b"row_threshold" in lib.knn_last_error()
    assert lib.knn_search_streamed(p, 10, p, 10, 4, 3, -1, oi.ctypes.data, od.ctypes.data,
                                   ctypes.byref(opt)) == binding.KNN_EINVAL
    assert lib.knn_search_streamed(p, 10, p, 10, 4, 0, 5, oi.ctypes.data, od.ctypes.data,
                                   ctypes.byref(opt)) == binding.KNN_EINVAL


def test_library_is_built_for_sm_103a():
    from paper_1309_5478_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)


def test_mlp_parameter_file_round_trip_on_host(lib, tmp_path):
    from paper_1309_5478_gb300 import binding
    n = lib.knn_mlp_param_count()
    assert n == binding.MLP_TRAINED + 2 * binding.MLP_FEATURES + 1
    p = (np.arange(n, dtype=np.float32) * 0.001 - 3.0).astype(np.float32)
    path = tmp_path / "net.bin"
    binding.mlp_save(path, p)
    assert path.stat().st_size == 8 + 12 + 4 * n
    q = np.zeros(n, dtype=np.float32)
    binding.mlp_load(path, q)
    assert np.array_equal(p, q)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(path.read_bytes()[:100])
    with pytest.raises(binding.KnnError):
        binding.mlp_load(bad, q)
    raw = bytearray(path.read_bytes())
    raw[12:16] = (64).to_bytes(4, "little")  # another hidden width
    bad.write_bytes(bytes(raw))
    with pytest.raises(binding.KnnError):
        binding.mlp_load(bad, q)
    with pytest.raises(binding.KnnError):
        binding.mlp_load(tmp_path / "missing.bin", q)


def test_noalloc_select_row_limit_is_checked_before_any_device_work(lib):
    from paper_1309_5478_gb300 import binding
    buf = np.zeros(16, dtype=np.float32)
    oi = np.zeros(16, dtype=np.int32)
    p = buf.ctypes.data
    # 2^20 + 1 rows: rejected by the argument checks, before the pointers are looked at
    assert lib.knn_select_noalloc(p, (1 << 20) + 1, 4, 4, 2, oi.ctypes.data, p, None) == binding.KNN_EINVAL
    assert b"at most 1048576 rows" in lib.knn_last_error()
    assert lib.knn_select_noalloc(p, 4, 4, 3, 2, oi.ctypes.data, p, None) == binding.KNN_EINVAL  # ldd < N
    assert b"ldd" in lib.knn_last_error()
