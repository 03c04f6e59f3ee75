"""FP64 CPU oracle for exact k-NN search and k-NN graphs (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use this package. The GPU engine never imports it and it imports nothing from
the engine. The arithmetic lives in ``knn_oracle.c`` (plain C, OpenMP over rows,
FP64 direct-difference distances, full sort of each row by (distance, index));
``mlp_oracle.py`` holds the FP64 reference of the learned-threshold network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add contraction, so x86 and Arm give the
# same FP64 sums.
CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle with gcc into ``out`` (rebuilt when the source is newer)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library and declare its signatures."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build())
        f = lib.oracle_knn_rows
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                      ctypes.c_void_p]
        g = lib.oracle_knn_sim_rows
        g.restype = ctypes.c_int
        g.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                      ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                      ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_similarity.restype = ctypes.c_double
        lib.oracle_similarity.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_sqdist.restype = ctypes.c_double
        lib.oracle_sqdist.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        if path is None:
            _lib = lib
        return lib


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(load().oracle_threads())


def knn(Q: np.ndarray, C: np.ndarray, k: int, rows=None, exclude_self: bool = False, lib=None):
    """k nearest rows of ``C`` for the query rows ``rows`` of ``Q`` (all rows when None).

    Returns ``(idx, dist)``: int64 and float64 arrays of shape (len(rows), k),
    ascending by (squared distance, index); -1 / inf pad rows with fewer than k
    candidates.
    """
    lib = lib or load()
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    assert Q.ndim == 2 and C.ndim == 2 and Q.shape[1] == C.shape[1]
    M, d = Q.shape
    N = C.shape[0]
    if rows is None:
        rows = np.arange(M, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    idx = np.empty((len(rows), k), dtype=np.int64)
    dist = np.empty((len(rows), k), dtype=np.float64)
    rc = lib.oracle_knn_rows(Q.ctypes.data, M, C.ctypes.data, N, d, k, rows.ctypes.data, len(rows),
                             1 if exclude_self else 0, idx.ctypes.data, dist.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_knn_rows rejected its arguments")
    return idx, dist


def knng(X: np.ndarray, k: int, rows=None, lib=None):
    """k-NN graph rows: ``knn(X, X, k, rows, exclude_self=True)``."""
    return knn(X, X, k, rows=rows, exclude_self=True, lib=lib)


def sqdist(x: np.ndarray, y: np.ndarray) -> float:
    """FP64 squared distance of two FP32 vectors (direct difference)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return float(load().oracle_sqdist(x.ctypes.data, y.ctypes.data, x.shape[0]))


METRICS = {"cosine": 0, "pearson": 1}


def knn_sim(Q: np.ndarray, C: np.ndarray, k: int, metric: str, rows=None, exclude_self: bool = False, lib=None):
    """k most similar rows of ``C`` by cosine or Pearson similarity, for the query rows ``rows``.

    Returns ``(idx, sim)``: int64 and float64 arrays of shape (len(rows), k), descending by
    similarity, ties to the lower index. Raises ValueError on a zero-norm (centred) row.
    """
    lib = lib or load()
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    assert Q.ndim == 2 and C.ndim == 2 and Q.shape[1] == C.shape[1]
    M, d = Q.shape
    N = C.shape[0]
    if rows is None:
        rows = np.arange(M, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    idx = np.empty((len(rows), k), dtype=np.int64)
    sim = np.empty((len(rows), k), dtype=np.float64)
    rc = lib.oracle_knn_sim_rows(Q.ctypes.data, M, C.ctypes.data, N, d, k, METRICS[metric], rows.ctypes.data,
                                 len(rows), 1 if exclude_self else 0, idx.ctypes.data, sim.ctypes.data)
    if rc == -2:
        raise ValueError("a row has zero norm (after centring): the similarity is undefined")
    if rc != 0:
        raise ValueError("oracle_knn_sim_rows rejected its arguments")
    return idx, sim


def knng_sim(X: np.ndarray, k: int, metric: str, rows=None, lib=None):
    """Similarity graph rows: ``knn_sim(X, X, k, metric, rows, exclude_self=True)``."""
    return knn_sim(X, X, k, metric, rows=rows, exclude_self=True, lib=lib)


def similarity(x: np.ndarray, y: np.ndarray, metric: str) -> float:
    """FP64 cosine or Pearson similarity of two FP32 vectors (NaN for a zero norm)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return float(load().oracle_similarity(x.ctypes.data, y.ctypes.data, x.shape[0], METRICS[metric]))
