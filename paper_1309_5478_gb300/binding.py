"""Python binding of the C ABI declared in ``include/knn.h`` (argument marshalling only).

Every computation runs inside ``libknn.so``. Arrays may be torch tensors (CUDA or
CPU) or numpy arrays; CPU arrays are handed to the library as host pointers,
which it stages to the device itself. There is no fallback: if the library is
missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libknn.so")

KNN_OK, KNN_EINVAL, KNN_ENOMEM, KNN_ECUDA, KNN_ETIMEOUT, KNN_EINTERNAL, KNN_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
KNN_FP32, KNN_BF16, KNN_FP8_E4M3, KNN_AUTO = 0, 1, 2, -1
KNN_FLAG_TIMING, KNN_FLAG_NO_FALLBACK, KNN_FLAG_CHECK_FINITE = 1, 2, 4
PRECISIONS = {"fp32": KNN_FP32, "bf16": KNN_BF16, "fp8": KNN_FP8_E4M3, "auto": KNN_AUTO}


class KnnStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("candidates", ctypes.c_int64), ("rows_truncated", ctypes.c_int64),
                ("rows_uncertified", ctypes.c_int64), ("rows_fallback", ctypes.c_int64),
                ("rows_fp64_ties", ctypes.c_int64), ("threshold_misses", ctypes.c_int64),
                ("max_error_bound", ctypes.c_float), ("ms_total", ctypes.c_float), ("ms_prep", ctypes.c_float),
                ("ms_select", ctypes.c_float), ("ms_rerank", ctypes.c_float), ("ms_fallback", ctypes.c_float),
                ("ms_gemm", ctypes.c_float), ("gemm_launches", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("gemm_flops", ctypes.c_double),
                ("precision_used", ctypes.c_int32), ("fused_used", ctypes.c_int32),
                ("exact_arithmetic", ctypes.c_int32), ("list_capacity", ctypes.c_int32),
                ("candidates_inserted", ctypes.c_int64), ("max_error_ratio", ctypes.c_float),
                ("rows_reranked_in_sweep", ctypes.c_int64), ("symmetric", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KnnOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rerank_extra", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p), ("row_threshold", ctypes.c_void_p),
                ("stats", ctypes.POINTER(KnnStats)), ("max_workspace_bytes", ctypes.c_int64)]


class KnnProblem(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_void_p), ("C", ctypes.c_void_p), ("M", ctypes.c_int64), ("N", ctypes.c_int64),
                ("d", ctypes.c_int32), ("k", ctypes.c_int32), ("exclude_self", ctypes.c_int32),
                ("status", ctypes.c_int32), ("out_idx", ctypes.c_void_p), ("out_dist", ctypes.c_void_p)]


# Every symbol include/knn.h declares (checked by the tests).
EXPORTS = ("knn_options_init", "knng_build", "knng_build_ex", "knn_search", "knn_select", "knn_distances",
           "knn_search_batched", "knn_status_string", "knn_last_error", "knn_shutdown", "knn_version",
           "knn_select_noalloc", "knn_mlp_param_count", "knn_mlp_features", "knn_mlp_loss_grad", "knn_mlp_train",
           "knn_mlp_predict", "knn_mlp_save", "knn_mlp_load", "knn_search_metric", "knng_build_metric",
           "knn_search_streamed")
MLP_FEATURES, MLP_HIDDEN = 257, 128
MLP_TRAINED = MLP_HIDDEN * MLP_FEATURES + 2 * MLP_HIDDEN + 1

_lock = threading.Lock()
_lib = None


class KnnError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def load(path: str | None = None):
    """Load ``libknn.so`` (raises when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA engine library not built: {p} (run __graft_entry__.build())")
        try:
            import torch  # noqa: F401  (loads the CUDA runtime the library links against)
        except ImportError:
            pass
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        opt_p = ctypes.POINTER(KnnOptions)
        lib.knn_options_init.argtypes = [opt_p]
        lib.knn_options_init.restype = None
        lib.knng_build.argtypes = [vp, i64, i32, i32, vp, vp]
        lib.knng_build_ex.argtypes = [vp, i64, i32, i32, vp, vp, opt_p]
        lib.knn_search.argtypes = [vp, i64, vp, i64, i32, i32, vp, vp, opt_p]
        lib.knn_search_metric.argtypes = [vp, i64, vp, i64, i32, i32, i32, vp, vp, opt_p]
        lib.knng_build_metric.argtypes = [vp, i64, i32, i32, i32, vp, vp, opt_p]
        lib.knn_search_streamed.argtypes = [vp, i64, vp, i64, i32, i32, i64, vp, vp, opt_p]
        lib.knn_select.argtypes = [vp, i64, i64, i64, i32, vp, vp, opt_p]
        lib.knn_distances.argtypes = [vp, i64, vp, i64, i32, vp, i64, i32, opt_p]
        lib.knn_search_batched.argtypes = [ctypes.POINTER(KnnProblem), i32, opt_p]
        lib.knn_select_noalloc.argtypes = [vp, i64, i64, i64, i32, vp, vp, vp]
        lib.knn_select_noalloc.restype = ctypes.c_int
        lib.knn_mlp_param_count.restype = ctypes.c_int32
        lib.knn_mlp_features.argtypes = [vp, i64, vp, i32, vp, opt_p]
        lib.knn_mlp_loss_grad.argtypes = [vp, vp, i64, vp, ctypes.POINTER(ctypes.c_double), vp, opt_p]
        lib.knn_mlp_train.argtypes = [vp, vp, i64, vp, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      vp, opt_p]
        lib.knn_mlp_predict.argtypes = [vp, i64, vp, vp, vp, opt_p]
        lib.knn_mlp_save.argtypes = [ctypes.c_char_p, vp]
        lib.knn_mlp_load.argtypes = [ctypes.c_char_p, vp]
        for f in ("knn_mlp_save", "knn_mlp_load", "knn_mlp_features", "knn_mlp_loss_grad", "knn_mlp_train", "knn_mlp_predict"):
            getattr(lib, f).restype = ctypes.c_int
        for f in ("knng_build", "knng_build_ex", "knn_search", "knn_select", "knn_distances", "knn_search_batched"):
            getattr(lib, f).restype = ctypes.c_int
        lib.knn_status_string.argtypes = [ctypes.c_int]
        lib.knn_status_string.restype = ctypes.c_char_p
        lib.knn_last_error.restype = ctypes.c_char_p
        lib.knn_version.restype = ctypes.c_char_p
        lib.knn_shutdown.restype = None
        if path is None:
            _lib = lib
        return lib


def _check(lib, status: int):
    if status != KNN_OK:
        msg = lib.knn_last_error().decode() or lib.knn_status_string(status).decode()
        raise KnnError(status, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int:
    if x is None:
        return 0
    if _is_torch(x):
        assert x.is_contiguous(), "arrays must be contiguous"
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags.c_contiguous, "arrays must be contiguous numpy or torch arrays"
    return x.ctypes.data


def _as_f32(x):
    if _is_torch(x):
        import torch
        return x.to(torch.float32).contiguous() if x.dtype != torch.float32 or not x.is_contiguous() else x
    return np.ascontiguousarray(x, dtype=np.float32)


def _empty_like_out(ref, shape, kind: str):
    if _is_torch(ref):
        import torch
        dt = torch.int32 if kind == "i" else torch.float32
        pin = ref.device.type == "cpu" and ref.is_pinned()
        return torch.empty(shape, dtype=dt, device=ref.device, pin_memory=pin)
    return np.empty(shape, dtype=np.int32 if kind == "i" else np.float32)


def _stream_of(ref, stream) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if _is_torch(ref) and ref.device.type == "cuda":
        import torch
        return int(torch.cuda.current_stream(ref.device).cuda_stream)
    return 0


def make_options(precision="auto", rerank_extra: int = 32, fused: int = -1, flags: int = KNN_FLAG_CHECK_FINITE,
                 stream: int = 0, row_threshold=None, stats: KnnStats | None = None, max_workspace_bytes: int = 0):
    o = KnnOptions()
    load().knn_options_init(ctypes.byref(o))
    o.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    o.rerank_extra = int(rerank_extra)
    o.fused = int(fused)
    o.flags = int(flags)
    o.stream = stream or None
    o.row_threshold = _ptr(row_threshold) or None
    o.stats = ctypes.pointer(stats) if stats is not None else ctypes.POINTER(KnnStats)()
    o.max_workspace_bytes = int(max_workspace_bytes)
    return o


def knng_build(X, k: int, out_idx=None, out_dist=None, precision="auto", rerank_extra: int = 32, fused: int = -1,
               flags: int = KNN_FLAG_CHECK_FINITE, stream=None, row_threshold=None, return_stats: bool = False,
               max_workspace_bytes: int = 0):
    """k-NN graph of the rows of X (N x d): (idx int32 N x k, squared dist float32 N x k)."""
    lib = load()
    X = _as_f32(X)
    N, d = X.shape
    oi = out_idx if out_idx is not None else _empty_like_out(X, (N, k), "i")
    od = out_dist if out_dist is not None else _empty_like_out(X, (N, k), "f")
    st = KnnStats()
    opt = make_options(precision, rerank_extra, fused, flags, _stream_of(X, stream), row_threshold, st,
                       max_workspace_bytes)
    _check(lib, lib.knng_build_ex(_ptr(X), N, d, k, _ptr(oi), _ptr(od), ctypes.byref(opt)))
    return (oi, od, st.as_dict()) if return_stats else (oi, od)


def knn_search(Q, C, k: int, out_idx=None, out_dist=None, precision="auto", rerank_extra: int = 32, fused: int = -1,
               flags: int = KNN_FLAG_CHECK_FINITE, stream=None, row_threshold=None, return_stats: bool = False,
               max_workspace_bytes: int = 0):
    """k nearest rows of C for every row of Q: (idx int32 M x k, squared dist float32 M x k)."""
    lib = load()
    Q = _as_f32(Q)
    C = _as_f32(C)
    M, d = Q.shape
    N = C.shape[0]
    assert C.shape[1] == d
    oi = out_idx if out_idx is not None else _empty_like_out(Q, (M, k), "i")
    od = out_dist if out_dist is not None else _empty_like_out(Q, (M, k), "f")
    st = KnnStats()
    opt = make_options(precision, rerank_extra, fused, flags, _stream_of(Q, stream), row_threshold, st,
                       max_workspace_bytes)
    _check(lib, lib.knn_search(_ptr(Q), M, _ptr(C), N, d, k, _ptr(oi), _ptr(od), ctypes.byref(opt)))
    return (oi, od, st.as_dict()) if return_stats else (oi, od)


METRICS = {"euclidean": 0, "cosine": 1, "pearson": 2}


def knn_search_metric(Q, C, k: int, metric: str, out_idx=None, out_val=None, precision="auto",
                      rerank_extra: int = 32, flags: int = KNN_FLAG_CHECK_FINITE, stream=None,
                      return_stats: bool = False):
    """k most similar rows of C for every row of Q by 'cosine' or 'pearson' similarity
    (descending; 'euclidean' gives knn_search): (idx int32 M x k, value float32 M x k)."""
    lib = load()
    Q = _as_f32(Q)
    C = _as_f32(C)
    M, d = Q.shape
    N = C.shape[0]
    oi = out_idx if out_idx is not None else _empty_like_out(Q, (M, k), "i")
    ov = out_val if out_val is not None else _empty_like_out(Q, (M, k), "f")
    st = KnnStats()
    opt = make_options(precision, rerank_extra, -1, flags, _stream_of(Q, stream), None, st)
    _check(lib, lib.knn_search_metric(_ptr(Q), M, _ptr(C), N, d, k, METRICS[metric], _ptr(oi), _ptr(ov),
                                      ctypes.byref(opt)))
    return (oi, ov, st.as_dict()) if return_stats else (oi, ov)


def knn_search_streamed(Q, C, k: int, chunk_rows: int = 0, out_idx=None, out_dist=None, precision="auto",
                        rerank_extra: int = 32, flags: int = KNN_FLAG_CHECK_FINITE, stream=None,
                        return_stats: bool = False):
    """knn_search with the corpus C read in chunks of chunk_rows rows (C may stay in host memory)."""
    lib = load()
    Q = _as_f32(Q)
    C = _as_f32(C)
    M, d = Q.shape
    N = C.shape[0]
    oi = out_idx if out_idx is not None else _empty_like_out(Q, (M, k), "i")
    od = out_dist if out_dist is not None else _empty_like_out(Q, (M, k), "f")
    st = KnnStats()
    opt = make_options(precision, rerank_extra, -1, flags, _stream_of(Q, stream), None, st)
    _check(lib, lib.knn_search_streamed(_ptr(Q), M, _ptr(C), N, d, k, int(chunk_rows), _ptr(oi), _ptr(od),
                                        ctypes.byref(opt)))
    return (oi, od, st.as_dict()) if return_stats else (oi, od)


def knng_build_metric(X, k: int, metric: str, out_idx=None, out_val=None, precision="auto", rerank_extra: int = 32,
                      flags: int = KNN_FLAG_CHECK_FINITE, stream=None, return_stats: bool = False):
    """Similarity graph of the rows of X by 'cosine' or 'pearson' ('euclidean': knng_build)."""
    lib = load()
    X = _as_f32(X)
    N, d = X.shape
    oi = out_idx if out_idx is not None else _empty_like_out(X, (N, k), "i")
    ov = out_val if out_val is not None else _empty_like_out(X, (N, k), "f")
    st = KnnStats()
    opt = make_options(precision, rerank_extra, -1, flags, _stream_of(X, stream), None, st)
    _check(lib, lib.knng_build_metric(_ptr(X), N, d, k, METRICS[metric], _ptr(oi), _ptr(ov), ctypes.byref(opt)))
    return (oi, ov, st.as_dict()) if return_stats else (oi, ov)


def knn_select(D, k: int, n: int | None = None, out_idx=None, out_val=None, stream=None,
               return_stats: bool = False, timing: bool = False):
    """The k smallest entries of every row of D (M x ldd; the first n columns): (idx, values)
    (and the call's statistics with return_stats; timing fills ms_select and ms_total)."""
    lib = load()
    D = _as_f32(D)
    M, ldd = D.shape
    n = ldd if n is None else n
    oi = out_idx if out_idx is not None else _empty_like_out(D, (M, k), "i")
    ov = out_val if out_val is not None else _empty_like_out(D, (M, k), "f")
    st = KnnStats() if return_stats else None
    opt = make_options(flags=KNN_FLAG_TIMING if timing else 0, stream=_stream_of(D, stream), stats=st)
    _check(lib, lib.knn_select(_ptr(D), M, n, ldd, k, _ptr(oi), _ptr(ov), ctypes.byref(opt)))
    return (oi, ov, st.as_dict()) if return_stats else (oi, ov)


def knn_select_noalloc(D, k: int, out_idx, out_val, n: int | None = None, stream=None):
    """knn_select into caller-provided device outputs, with no allocation inside the library."""
    lib = load()
    M, ldd = D.shape
    n = ldd if n is None else n
    _check(lib, lib.knn_select_noalloc(_ptr(D), M, n, ldd, k, _ptr(out_idx), _ptr(out_val),
                                       _stream_of(D, stream) or None))
    return out_idx, out_val


def knn_distances(Q, C, full: bool = False, out=None, stream=None):
    """FP32 distance matrix: |c|^2 - 2 q.c (full=False) or the squared distance (full=True)."""
    lib = load()
    Q = _as_f32(Q)
    C = _as_f32(C)
    M, d = Q.shape
    N = C.shape[0]
    o = out if out is not None else _empty_like_out(Q, (M, N), "f")
    opt = make_options(stream=_stream_of(Q, stream))
    _check(lib, lib.knn_distances(_ptr(Q), M, _ptr(C), N, d, _ptr(o), N, 1 if full else 0, ctypes.byref(opt)))
    return o


def knn_search_batched(problems, precision="auto", rerank_extra: int = 32, flags: int = KNN_FLAG_CHECK_FINITE,
                       stream=None, return_stats: bool = False):
    """problems: list of dicts with keys Q (or None for a graph), C, k, out_idx, out_dist."""
    lib = load()
    arr = (KnnProblem * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        C = _as_f32(p["C"])
        Q = C if p.get("Q") is None else _as_f32(p["Q"])
        keep += [C, Q]
        arr[i].Q = _ptr(Q)
        arr[i].C = _ptr(C)
        arr[i].M = Q.shape[0]
        arr[i].N = C.shape[0]
        arr[i].d = C.shape[1]
        arr[i].k = int(p["k"])
        arr[i].exclude_self = 1 if p.get("Q") is None else 0
        arr[i].out_idx = _ptr(p["out_idx"])
        arr[i].out_dist = _ptr(p["out_dist"])
    ref = next((x for x in keep if _is_torch(x) and x.device.type == "cuda"), None)
    st = KnnStats()
    opt = make_options(precision, rerank_extra, -1, flags, _stream_of(ref, stream), stats=st)
    status = lib.knn_search_batched(arr, len(problems), ctypes.byref(opt))
    statuses = [arr[i].status for i in range(len(problems))]
    _check(lib, status)
    return (statuses, st.as_dict()) if return_stats else statuses


def mlp_param_count() -> int:
    return int(load().knn_mlp_param_count())


def mlp_features(Q, S, out=None, stream=None):
    """Features (M x 257) of the query rows Q against the 256 corpus samples S (device tensors)."""
    lib = load()
    Q = _as_f32(Q)
    S = _as_f32(S)
    M, d = Q.shape
    assert S.shape == (MLP_FEATURES - 1, d)
    o = out if out is not None else _empty_like_out(Q, (M, MLP_FEATURES), "f")
    opt = make_options(stream=_stream_of(Q, stream))
    _check(lib, lib.knn_mlp_features(_ptr(Q), M, _ptr(S), d, _ptr(o), ctypes.byref(opt)))
    return o


def mlp_loss_grad(features, targets, params, stream=None):
    """(loss, gradient of the trained parameters) of the network on (features, targets)."""
    import torch
    lib = load()
    g = torch.empty(MLP_TRAINED, dtype=torch.float32, device=features.device)
    loss = ctypes.c_double()
    opt = make_options(stream=_stream_of(features, stream))
    _check(lib, lib.knn_mlp_loss_grad(_ptr(features), _ptr(targets), features.shape[0], _ptr(params),
                                      ctypes.byref(loss), _ptr(g), ctypes.byref(opt)))
    return loss.value, g


def mlp_train(features, targets, params, epochs: int = 40, batch: int = 1024, lr: float = 1e-3,
              holdout: float = 0.1, margin_quantile: float = 0.99, stream=None):
    """Trains params in place on the GPU; returns the per-epoch mean training loss."""
    lib = load()
    hist = (ctypes.c_float * epochs)()
    opt = make_options(stream=_stream_of(features, stream))
    _check(lib, lib.knn_mlp_train(_ptr(features), _ptr(targets), features.shape[0], _ptr(params), epochs, batch,
                                  lr, holdout, margin_quantile, hist, ctypes.byref(opt)))
    return list(hist)


def mlp_predict(features, params, stream=None):
    """(predicted log k-th squared distance, squared-distance threshold) per row."""
    import torch
    lib = load()
    n = features.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=features.device)
    t = torch.empty(n, dtype=torch.float32, device=features.device)
    opt = make_options(stream=_stream_of(features, stream))
    _check(lib, lib.knn_mlp_predict(_ptr(features), n, _ptr(params), _ptr(y), _ptr(t), ctypes.byref(opt)))
    return y, t


def mlp_save(path: str, params) -> None:
    """Writes the parameter array (host numpy or device tensor) to a parameter file."""
    lib = load()
    _check(lib, lib.knn_mlp_save(str(path).encode(), _ptr(params)))


def mlp_load(path: str, params) -> None:
    """Reads a parameter file into params (host numpy float32 or device tensor)."""
    lib = load()
    _check(lib, lib.knn_mlp_load(str(path).encode(), _ptr(params)))


def version() -> str:
    return load().knn_version().decode()


def shutdown() -> None:
    load().knn_shutdown()
