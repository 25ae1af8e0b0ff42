"""FP64 CPU oracle for balanced k-means partitioning -- TEST INFRASTRUCTURE ONLY.

Python view of ``gk_oracle.c``: a plain, slow restatement of the method of
"Balanced k-means for Parallel Geometric Partitioning" (Sections 4.1-4.5,
Algorithms 1 and 2, Eq. 1-3).  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never calls it.

Every function takes and returns numpy arrays.  Points are ``(n, d)`` arrays
(FP64, or FP32 where noted), weights ``(n,)`` FP64 or ``None``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_OK = 0
OR_INVALID = 1
OR_NOT_BALANCED = 4


class Options(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("max_balance_iter", ctypes.c_int32),
        ("final_balance_iter", ctypes.c_int32),
        ("erosion", ctypes.c_int32),
        ("delta_threshold", ctypes.c_double),
        ("threads", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("balance_passes", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("balanced", ctypes.c_int32),
        ("max_imbalance", ctypes.c_double),
        ("max_delta", ctypes.c_double),
        ("delta_threshold", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile gk_oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
                and _loads(_LIB_PATH)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _loads(path: str) -> bool:
    try:
        ctypes.CDLL(path)
        return True
    except OSError:
        return False


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.or_version.restype = i64
        L.or_bbox.argtypes = [P, i64, i32, P, P]
        L.or_hilbert_index.argtypes = [P, i32, i32]
        L.or_hilbert_index.restype = ctypes.c_uint64
        L.or_hilbert_keys_f64.argtypes = [P, i64, i32, P, P]
        L.or_hilbert_keys_f32.argtypes = [P, i64, i32, P, P]
        L.or_sort_keys.argtypes = [P, i64, P]
        L.or_sfc_centers.argtypes = [P, i64, i32, i32, P]
        L.or_assign.argtypes = [P, i64, i32, P, P, i32, P, P, P, i32]
        L.or_block_weights.argtypes = [P, P, i64, i32, P]
        L.or_block_weights.restype = dbl
        L.or_balance_bound.argtypes = [dbl, i32, dbl]
        L.or_balance_bound.restype = dbl
        L.or_balance_update.argtypes = [P, dbl, i32, i32, dbl, P, P]
        L.or_balance_update.restype = i32
        L.or_move_centers.argtypes = [P, P, P, i64, i32, i32, P, P, P, P]
        L.or_erosion.argtypes = [P, dbl, i32, P]
        L.or_default_options.argtypes = [P]
        L.or_balanced_kmeans.argtypes = [P, P, i64, i32, i32, dbl, P, P, P, P, P, P, P]
        L.or_balanced_kmeans.restype = i32
        L.or_partition.argtypes = [P, i32, P, i64, i32, i32, dbl, P, P, P, P, P]
        L.or_partition.restype = i32
        L.or_sample_first.argtypes = [i64, i32, i64]
        L.or_sample_first.restype = i64
        L.or_sample_rounds.argtypes = [i64, i64, i32]
        L.or_sample_rounds.restype = i32
        L.or_partition_sampled.argtypes = [P, i32, P, i64, i32, i32, dbl, P, i64, P, P, P, P, P]
        L.or_partition_sampled.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_options(**overrides) -> Options:
    o = Options()
    lib().or_default_options(ctypes.byref(o))
    for key, val in overrides.items():
        setattr(o, key, val)
    return o


def bbox(x):
    x = _f64(x)
    n, d = x.shape
    lo, hi = np.empty(d), np.empty(d)
    lib().or_bbox(_ptr(x), n, d, _ptr(lo), _ptr(hi))
    return lo, hi


def hilbert_index(q, b: int) -> int:
    q = np.ascontiguousarray(q, dtype=np.uint32)
    return int(lib().or_hilbert_index(_ptr(q), q.shape[0], b))


def hilbert_keys(x, return_cells: bool = False):
    """Keys of every point (FP32 or FP64 points; quantisation in that precision)."""
    if x.dtype == np.float32:
        x = np.ascontiguousarray(x)
        fn = lib().or_hilbert_keys_f32
    else:
        x = _f64(x)
        fn = lib().or_hilbert_keys_f64
    n, d = x.shape
    keys = np.empty(n, dtype=np.uint64)
    cells = np.empty((n, d), dtype=np.uint32) if return_cells else None
    fn(_ptr(x), n, d, _ptr(keys), _ptr(cells))
    return (keys, cells) if return_cells else keys


def sort_keys(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.empty(keys.shape[0], dtype=np.int64)
    lib().or_sort_keys(_ptr(keys), keys.shape[0], _ptr(perm))
    return perm


def sfc_centers(x_sorted, k: int):
    x_sorted = _f64(x_sorted)
    n, d = x_sorted.shape
    C = np.empty((k, d))
    lib().or_sfc_centers(_ptr(x_sorted), n, d, k, _ptr(C))
    return C


def assign(x, C, I, threads: int = 1):
    """Returns (A, best, second): argmin of dist/I and the two smallest values."""
    x, C, I = _f64(x), _f64(C), _f64(I)
    n, d = x.shape
    k = C.shape[0]
    A = np.empty(n, dtype=np.int32)
    best, second = np.empty(n), np.empty(n)
    lib().or_assign(_ptr(x), n, d, _ptr(C), _ptr(I), k, _ptr(A), _ptr(best), _ptr(second),
                    threads)
    return A, best, second


def block_weights(A, w, k: int):
    A = np.ascontiguousarray(A, dtype=np.int32)
    w = None if w is None else _f64(w)
    S = np.empty(k)
    W = lib().or_block_weights(_ptr(A), _ptr(w), A.shape[0], k, _ptr(S))
    return S, W


def balance_bound(W: float, k: int, eps: float) -> float:
    return float(lib().or_balance_bound(W, k, eps))


def balance_update(S, W: float, k: int, d: int, eps: float, I):
    """Returns (balanced, new_I, imbalance); I is not modified in place."""
    S = _f64(S)
    I2 = _f64(I).copy()
    imb = ctypes.c_double()
    bal = lib().or_balance_update(_ptr(S), W, k, d, eps, _ptr(I2), ctypes.byref(imb))
    return bool(bal), I2, imb.value


def move_centers(x, w, A, C):
    x, C = _f64(x), _f64(C)
    A = np.ascontiguousarray(A, dtype=np.int32)
    w = None if w is None else _f64(w)
    n, d = x.shape
    k = C.shape[0]
    C_new, delta = np.empty((k, d)), np.empty(k)
    beta = ctypes.c_double()
    lib().or_move_centers(_ptr(x), _ptr(w), _ptr(A), n, d, k, _ptr(C), _ptr(C_new),
                          _ptr(delta), ctypes.byref(beta))
    return C_new, delta, beta.value


def erosion(delta, beta: float, I):
    delta = _f64(delta)
    I2 = _f64(I).copy()
    lib().or_erosion(_ptr(delta), beta, I2.shape[0], _ptr(I2))
    return I2


def balanced_kmeans(x, w, k: int, eps: float, C0, I0, options: Options | None = None):
    """Algorithm 2 on points in processing order.  Returns a dict with A, C (centers A
    was computed with), I_used, I (state after the last update), C_moved, result."""
    x = _f64(x)
    n, d = x.shape
    w = None if w is None else _f64(w)
    C = _f64(C0).copy()
    I = _f64(I0).copy()
    I_used = np.empty(k)
    C_moved = np.empty((k, d))
    A = np.empty(n, dtype=np.int32)
    res = Result()
    opt = options if options is not None else default_options()
    lib().or_balanced_kmeans(_ptr(x), _ptr(w), n, d, k, eps, ctypes.byref(opt), _ptr(C),
                             _ptr(I), _ptr(I_used), _ptr(C_moved), _ptr(A), ctypes.byref(res))
    return {"A": A, "C": C, "I_used": I_used, "I": I, "C_moved": C_moved,
            "result": res.as_dict()}


def partition(x, w, k: int, eps: float, options: Options | None = None):
    """Whole partitioner; returns dict with A (input order), C, I (I_used), result."""
    is_f32 = 1 if x.dtype == np.float32 else 0
    x = np.ascontiguousarray(x) if is_f32 else _f64(x)
    n, d = x.shape
    w = None if w is None else _f64(w)
    A = np.empty(n, dtype=np.int32)
    C = np.empty((k, d))
    I = np.empty(k)
    res = Result()
    opt = options if options is not None else default_options()
    lib().or_partition(_ptr(x), is_f32, _ptr(w), n, d, k, eps, ctypes.byref(opt), _ptr(A),
                       _ptr(C), _ptr(I), ctypes.byref(res))
    return {"A": A, "C": C, "I": I, "result": res.as_dict()}


def sample_first(n: int, k: int, sample0: int = 0) -> int:
    """Size of the first sample of the random initialization (Section 4.5)."""
    return int(lib().or_sample_first(n, k, sample0))


def sample_rounds(n: int, m0: int, max_iter: int = 50) -> int:
    """Number of sample rounds of the random initialization (Section 4.5)."""
    return int(lib().or_sample_rounds(n, m0, max_iter))


def partition_sampled(x, w, k: int, eps: float, order, sample0: int = 0,
                      options: Options | None = None):
    """Whole partitioner with the random initialization of Section 4.5; order is a
    permutation of the input indices (the random order of the points), sample0 the
    first sample size (0: 100 k).  Returns a dict with A (input order), C, I
    (I_used), result."""
    is_f32 = 1 if x.dtype == np.float32 else 0
    x = np.ascontiguousarray(x) if is_f32 else _f64(x)
    n, d = x.shape
    w = None if w is None else _f64(w)
    order = np.ascontiguousarray(order, dtype=np.int64)
    A = np.empty(n, dtype=np.int32)
    C = np.empty((k, d))
    I = np.empty(k)
    res = Result()
    opt = options if options is not None else default_options()
    lib().or_partition_sampled(_ptr(x), is_f32, _ptr(w), n, d, k, eps, _ptr(order), sample0,
                               ctypes.byref(opt), _ptr(A), _ptr(C), _ptr(I), ctypes.byref(res))
    return {"A": A, "C": C, "I": I, "result": res.as_dict()}
