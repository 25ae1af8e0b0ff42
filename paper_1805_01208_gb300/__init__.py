"""GB300 (sm_103a) balanced k-means geometric partitioner.

Thin Python binding of the C ABI in ``include/gk.h`` (``libgk.so``).  Every step of
the computation runs in the library's CUDA kernels; this module only marshals
arguments: it passes data pointers of torch tensors (device or host) or numpy arrays
(host) and the current CUDA stream, and allocates outputs.  There is no CPU fallback:
without the built library every call raises.

Functions (same names as the C entry points, without the ``gk_`` prefix):
``hilbert_keys``, ``sfc_init``, ``assign``, ``move_centers``, ``balanced_kmeans``,
``partition``, ``release``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgk.so")

GK_OK = 0
GK_ERR_INVALID_ARG = 1
GK_ERR_CUDA = 2
GK_ERR_OOM = 3
GK_ERR_NOT_BALANCED = 4
GK_ERR_TIMEOUT = 5
GK_F32 = 0
GK_F64 = 1


class GKError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} ({status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("max_balance_iter", ctypes.c_int32),
        ("final_balance_iter", ctypes.c_int32),
        ("erosion", ctypes.c_int32),
        ("delta_threshold", ctypes.c_double),
        ("assign_dtype", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("bounds", ctypes.c_int32),
        ("supertile_tiles", ctypes.c_int32),
        ("assign_ctas_per_sm", ctypes.c_int32),
        ("hypertiles", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("balance_passes", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("balanced", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("max_imbalance", ctypes.c_double),
        ("max_delta", ctypes.c_double),
        ("delta_threshold", ctypes.c_double),
        ("avg_candidates", ctypes.c_double),
        ("rechecked_points", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("time_bootstrap_ms", ctypes.c_double),
        ("time_kmeans_ms", ctypes.c_double),
        ("time_total_ms", ctypes.c_double),
        ("time_filter_ms", ctypes.c_double),
        ("time_assign_ms", ctypes.c_double),
        ("time_balance_ms", ctypes.c_double),
        ("time_move_ms", ctypes.c_double),
        ("filter_launches", ctypes.c_int64),
        ("assign_launches", ctypes.c_int64),
        ("balance_launches", ctypes.c_int64),
        ("move_launches", ctypes.c_int64),
        ("assign_live_ms", ctypes.c_double),
        ("assign_live_launches", ctypes.c_int64),
        ("evaluated_points", ctypes.c_int64),
        ("supertile_tiles", ctypes.c_int32),
        ("assign_ctas_per_sm", ctypes.c_int32),
        ("hypertiles", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
        ("tune_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_
                if name not in ("reserved0", "reserved1")}


class Instance(ctypes.Structure):
    """gk_instance: one problem of gk_partition_batched (device pointers)."""
    _fields_ = [
        ("coords", ctypes.c_void_p),
        ("weights", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("eps", ctypes.c_double),
        ("block_out", ctypes.c_void_p),
        ("centers_out", ctypes.c_void_p),
        ("influence_out", ctypes.c_void_p),
    ]


class Quality(ctypes.Structure):
    """gk_quality (include/gk.h)."""
    _fields_ = [
        ("edge_cut", ctypes.c_int64),
        ("total_comm_volume", ctypes.c_int64),
        ("max_comm_volume", ctypes.c_int64),
        ("max_ext", ctypes.c_int64),
        ("boundary_vertices", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Diameter(ctypes.Structure):
    """gk_diameter (include/gk.h)."""
    _fields_ = [
        ("max_diameter", ctypes.c_int64),
        ("disconnected_blocks", ctypes.c_int64),
        ("bfs_levels", ctypes.c_int64),
        ("harmonic_mean", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                              ctypes.c_int32, ctypes.c_void_p)
GK_REDUCE_SUM, GK_REDUCE_MIN, GK_REDUCE_MAX = 0, 1, 2
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_alloc_refs: dict = {}  # the registered callbacks, kept alive while the library may call them

_lib = None


def lib():
    """The loaded libgk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_1805_01208_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.gk_default_options.argtypes = [P]
        L.gk_status_string.argtypes = [i32]
        L.gk_status_string.restype = ctypes.c_char_p
        L.gk_abi_version.restype = i32
        L.gk_check_wait_timeout.argtypes = [i64, P, P]
        L.gk_check_wait_timeout.restype = i32
        L.gk_hilbert_keys.argtypes = [P, i32, i64, i32, P, P]
        L.gk_sfc_init.argtypes = [P, i32, i64, i32, i32, P, P, P]
        L.gk_assign.argtypes = [P, i32, P, i64, i32, i32, P, P, i32, P, P, P]
        L.gk_move_centers.argtypes = [P, i32, P, i64, i32, i32, P, P, P, P, P, P]
        L.gk_balanced_kmeans.argtypes = [P, i32, P, i64, i32, i32, dbl, P, P, P, P, P, P]
        L.gk_partition.argtypes = [P, i32, P, i64, i32, i32, dbl, P, P, P, P, P, P]
        L.gk_partition_sampled.argtypes = [P, i32, P, i64, i32, i32, dbl, P, i64, P, P, P, P,
                                           P, P]
        L.gk_partition_quality.argtypes = [P, P, i64, i64, P, i32, P, P, P, P]
        L.gk_partition_quality.restype = i32
        L.gk_block_diameter.argtypes = [P, P, i64, i64, P, i32, i32, P, P, P]
        L.gk_block_diameter.restype = i32
        for name in ("gk_hilbert_keys", "gk_sfc_init", "gk_assign", "gk_move_centers",
                     "gk_balanced_kmeans", "gk_partition", "gk_partition_sampled"):
            getattr(L, name).restype = i32
        L.gk_move_centers_noalloc.argtypes = [P, i32, P, i64, i32, i32, P, P, P, P, P, P]
        L.gk_move_centers_noalloc.restype = i32
        L.gk_partition_batched.argtypes = [P, i32, P, P, P]
        L.gk_partition_batched.restype = i32
        L.gk_bounding_box.argtypes = [P, i32, i64, i32, P, P, P]
        L.gk_hilbert_keys_in_box.argtypes = [P, i32, i64, i32, P, P, P, P]
        L.gk_sort_keys.argtypes = [P, i64, i32, P, P]
        L.gk_balanced_kmeans_sharded.argtypes = [P, i32, P, i64, i64, i32, i32, dbl, P, P, P, P, P,
                                                 ctypes.c_void_p, P, P]
        for name in ("gk_bounding_box", "gk_hilbert_keys_in_box", "gk_sort_keys",
                     "gk_balanced_kmeans_sharded"):
            getattr(L, name).restype = i32
        L.gk_release.argtypes = []
        L.gk_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.gk_set_allocator.restype = i32
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().gk_status_string(status).decode()


def default_options(**overrides) -> Options:
    o = Options()
    lib().gk_default_options(ctypes.byref(o))
    for key, val in overrides.items():
        if key == "assign_dtype" and isinstance(val, str):
            val = GK_F64 if val == "f64" else GK_F32
        setattr(o, key, val)
    return o


# ------------------------------------------------------------------------------------
# argument marshalling
# ------------------------------------------------------------------------------------
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _dtype_code(a) -> int:
    if _is_torch(a):
        import torch
        if a.dtype == torch.float64:
            return GK_F64
        if a.dtype == torch.float32:
            return GK_F32
    else:
        if a.dtype == np.float64:
            return GK_F64
        if a.dtype == np.float32:
            return GK_F32
    raise TypeError(f"coordinates must be float32 or float64, got {a.dtype}")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(a, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if _is_torch(a) and a.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return ctypes.c_void_p(0)


def _empty(like, shape, kind):
    """Output buffer on the same side as `like` (torch device/host tensor or numpy)."""
    if _is_torch(like):
        import torch
        dt = {"i32": torch.int32, "i64": torch.int64, "f64": torch.float64, "u64": torch.int64}[kind]
        return torch.empty(shape, dtype=dt, device=like.device)
    dt = {"i32": np.int32, "i64": np.int64, "f64": np.float64, "u64": np.uint64}[kind]
    return np.empty(shape, dtype=dt)


def _check(status, where, allow=()):
    if status != GK_OK and status not in allow:
        raise GKError(status, where)
    return status


def _shape(coords):
    if len(coords.shape) != 2:
        raise ValueError("coords must be (n, d)")
    return int(coords.shape[0]), int(coords.shape[1])


def _same_dtype(coords, weights):
    if weights is not None and _dtype_code(weights) != _dtype_code(coords):
        raise TypeError("weights must have the dtype of the coordinates")


# ------------------------------------------------------------------------------------
# entry points
# ------------------------------------------------------------------------------------
def hilbert_keys(coords, stream=None):
    """uint64 Hilbert keys (returned as int64 tensors for torch inputs) in input order."""
    n, d = _shape(coords)
    keys = _empty(coords, (n,), "u64")
    st = lib().gk_hilbert_keys(_ptr(coords), _dtype_code(coords), n, d, _ptr(keys),
                               _stream(coords, stream))
    _check(st, "gk_hilbert_keys")
    return keys


def sfc_init(coords, k: int, stream=None):
    """(perm, centers): curve order (sorted position -> input index) and initial centers."""
    n, d = _shape(coords)
    perm = _empty(coords, (n,), "i64")
    centers = _empty(coords, (k, d), "f64")
    st = lib().gk_sfc_init(_ptr(coords), _dtype_code(coords), n, d, k, _ptr(perm), _ptr(centers),
                           _stream(coords, stream))
    _check(st, "gk_sfc_init")
    return perm, centers


def assign(coords, centers, influence, weights=None, assign_dtype: str = "f64", stream=None):
    """One assignment pass: (block ids, block weights)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    k = int(centers.shape[0])
    block = _empty(coords, (n,), "i32")
    bw = _empty(coords, (k,), "f64")
    st = lib().gk_assign(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k, _ptr(centers),
                         _ptr(influence), GK_F64 if assign_dtype == "f64" else GK_F32,
                         _ptr(block), _ptr(bw), _stream(coords, stream))
    _check(st, "gk_assign")
    return block, bw


def move_centers(coords, block, centers, weights=None, stream=None):
    """Weighted means of the blocks: (new centers, movement per center, beta)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    k = int(centers.shape[0])
    out = _empty(coords, (k, d), "f64")
    delta = _empty(coords, (k,), "f64")
    beta = ctypes.c_double()
    st = lib().gk_move_centers(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k,
                               _ptr(block), _ptr(centers), _ptr(out), _ptr(delta),
                               ctypes.byref(beta), _stream(coords, stream))
    _check(st, "gk_move_centers")
    return out, delta, beta.value


def move_centers_noalloc(coords, block, centers, weights=None, out=None, delta=None, stream=None):
    """move_centers with no allocation inside the library (device tensors only, k <= 4096).
    `out` / `delta` may be preallocated device tensors."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    k = int(centers.shape[0])
    out = _empty(coords, (k, d), "f64") if out is None else out
    delta = _empty(coords, (k,), "f64") if delta is None else delta
    beta = ctypes.c_double()
    st = lib().gk_move_centers_noalloc(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k,
                                       _ptr(block), _ptr(centers), _ptr(out), _ptr(delta),
                                       ctypes.byref(beta), _stream(coords, stream))
    _check(st, "gk_move_centers_noalloc")
    return out, delta, beta.value


def bounding_box(coords, stream=None):
    """(lo, hi): the points' bounding box, two numpy arrays of d FP64."""
    n, d = _shape(coords)
    lo, hi = np.empty(d), np.empty(d)
    st = lib().gk_bounding_box(_ptr(coords), _dtype_code(coords), n, d, _ptr(lo), _ptr(hi),
                               _stream(coords, stream))
    _check(st, "gk_bounding_box")
    return lo, hi


def hilbert_keys_in_box(coords, lo, hi, stream=None):
    """Hilbert keys of the points on the given bounding box (lo, hi: d values each)."""
    n, d = _shape(coords)
    keys = _empty(coords, (n,), "u64")
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    st = lib().gk_hilbert_keys_in_box(_ptr(coords), _dtype_code(coords), n, d, _ptr(lo), _ptr(hi),
                                      _ptr(keys), _stream(coords, stream))
    _check(st, "gk_hilbert_keys_in_box")
    return keys


def sort_keys(keys, d: int, stream=None):
    """Stable sort of Hilbert keys: int64 permutation (position -> index of the key)."""
    n = int(keys.shape[0])
    perm = _empty(keys, (n,), "i64")
    st = lib().gk_sort_keys(_ptr(keys), n, d, _ptr(perm), _stream(keys, stream))
    _check(st, "gk_sort_keys")
    return perm


def balanced_kmeans_sharded(coords, n_global: int, k: int, eps: float, centers, influence, reduce,
                            weights=None, options: Options | None = None, stream=None):
    """gk_balanced_kmeans on one shard (this process's contiguous range of the curve-sorted
    points of a problem of n_global points).  reduce(buf, op) replaces the int64 numpy
    array buf in place by its sum (op 0), minimum (1) or maximum (2) over all shards.
    centers / influence are updated in place.  Returns (block, result dict)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    block = _empty(coords, (n,), "i32")
    res = Result()
    opt = options if options is not None else default_options()
    failed = []

    def cb(buf, count, op, ctx):
        try:
            reduce(np.ctypeslib.as_array(buf, shape=(int(count),)), int(op))
            return 0
        except Exception as e:  # reported as a failed call (the library stops)
            failed.append(e)
            return 1

    fn = _REDUCE_FN(cb)
    st = lib().gk_balanced_kmeans_sharded(_ptr(coords), _dtype_code(coords), _ptr(weights), n,
                                          int(n_global), d, k, eps, _ptr(centers), _ptr(influence),
                                          _ptr(block), ctypes.byref(opt), ctypes.byref(res),
                                          ctypes.cast(fn, ctypes.c_void_p), None,
                                          _stream(coords, stream))
    if failed:
        raise failed[0]
    _check(st, "gk_balanced_kmeans_sharded", allow=(GK_ERR_NOT_BALANCED,))
    return block, res.as_dict()


def balanced_kmeans(coords, k: int, eps: float, centers, influence, weights=None,
                    options: Options | None = None, stream=None):
    """Balanced k-means from given centers/influence (updated in place to the state the
    returned assignment was computed with).  Returns (block, result dict)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    block = _empty(coords, (n,), "i32")
    res = Result()
    opt = options if options is not None else default_options()
    st = lib().gk_balanced_kmeans(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k, eps,
                                  _ptr(centers), _ptr(influence), _ptr(block), ctypes.byref(opt),
                                  ctypes.byref(res), _stream(coords, stream))
    _check(st, "gk_balanced_kmeans", allow=(GK_ERR_NOT_BALANCED,))
    return block, res.as_dict()


def partition(coords, k: int, eps: float, weights=None, options: Options | None = None,
              stream=None, want_state: bool = True):
    """The whole partitioner.  Returns (block, centers, influence, result dict)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    block = _empty(coords, (n,), "i32")
    centers = _empty(coords, (k, d), "f64") if want_state else None
    infl = _empty(coords, (k,), "f64") if want_state else None
    res = Result()
    opt = options if options is not None else default_options()
    st = lib().gk_partition(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k, eps,
                            ctypes.byref(opt), _ptr(block), _ptr(centers), _ptr(infl),
                            ctypes.byref(res), _stream(coords, stream))
    _check(st, "gk_partition", allow=(GK_ERR_NOT_BALANCED,))
    return block, centers, infl, res.as_dict()


def partition_sampled(coords, k: int, eps: float, order, sample0: int = 0, weights=None,
                      options: Options | None = None, stream=None, want_state: bool = True):
    """The whole partitioner with the random initialization of Section 4.5.  order: n
    int64, a permutation of [0, n) (the random order of the points; host or device);
    sample0: first sample size (0: 100 k).  Returns (block, centers, influence, result)."""
    n, d = _shape(coords)
    _same_dtype(coords, weights)
    if _is_torch(order):
        import torch
        if order.dtype != torch.int64:
            raise TypeError("order must be int64")
    elif np.asarray(order).dtype != np.int64:
        raise TypeError("order must be int64")
    if int(order.shape[0]) != n or len(order.shape) != 1:
        raise ValueError("order must have one entry per point")
    block = _empty(coords, (n,), "i32")
    centers = _empty(coords, (k, d), "f64") if want_state else None
    infl = _empty(coords, (k,), "f64") if want_state else None
    res = Result()
    opt = options if options is not None else default_options()
    st = lib().gk_partition_sampled(_ptr(coords), _dtype_code(coords), _ptr(weights), n, d, k,
                                    eps, _ptr(order), int(sample0), ctypes.byref(opt), _ptr(block),
                                    _ptr(centers), _ptr(infl), ctypes.byref(res),
                                    _stream(coords, stream))
    _check(st, "gk_partition_sampled", allow=(GK_ERR_NOT_BALANCED,))
    return block, centers, infl, res.as_dict()


def partition_quality(row_ptr, col, block, k: int, stream=None):
    """Edge cut and communication volume (Section 5) of a partition of a graph given as
    a symmetric CSR adjacency (row_ptr int64 n+1, col int32).  Returns (dict, ext, comm)
    with the per-block ext and comm as int64 arrays on the side of `block`."""
    n = int(block.shape[0])
    nnz = int(col.shape[0])
    ext = _empty(block, (k,), "i64")
    comm = _empty(block, (k,), "i64")
    q = Quality()
    st = lib().gk_partition_quality(_ptr(row_ptr), _ptr(col), n, nnz, _ptr(block), k, _ptr(ext),
                                    _ptr(comm), ctypes.byref(q), _stream(block, stream))
    _check(st, "gk_partition_quality")
    return q.as_dict(), ext, comm


def block_diameter(row_ptr, col, block, k: int, sweeps: int = 3, stream=None):
    """Lower bounds of the block diameters (Section 5) from `sweeps` breadth-first sweeps
    inside every block.  Returns (dict, diam) with diam the per-block bounds as int32 on
    the side of `block` (-1: block not connected, 0: empty block)."""
    n = int(block.shape[0])
    nnz = int(col.shape[0])
    diam = _empty(block, (k,), "i32")
    q = Diameter()
    st = lib().gk_block_diameter(_ptr(row_ptr), _ptr(col), n, nnz, _ptr(block), k, sweeps,
                                 _ptr(diam), ctypes.byref(q), _stream(block, stream))
    _check(st, "gk_block_diameter")
    return q.as_dict(), diam


def set_allocator(alloc=None, free=None):
    """Device memory for the library's workspace from the caller: alloc(nbytes) returns a
    device pointer (int, 256-byte aligned; 0 on failure), free(ptr, nbytes) takes it back.
    set_allocator() returns to cudaMalloc.  The current workspace is released first."""
    L = lib()
    if alloc is None and free is None:
        st = L.gk_set_allocator(None, None, None)
        _alloc_refs.clear()
        _check(st, "gk_set_allocator")
        return
    if alloc is None or free is None:
        raise ValueError("give both alloc and free, or neither")
    a = _ALLOC_FN(lambda nbytes, ctx: alloc(int(nbytes)) or None)
    f = _FREE_FN(lambda ptr, nbytes, ctx: free(int(ptr), int(nbytes)))
    st = L.gk_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None)
    _check(st, "gk_set_allocator")
    _alloc_refs.clear()
    _alloc_refs.update(alloc=a, free=f)


def use_torch_allocator():
    """Route the workspace through PyTorch's caching allocator (current device).  Returns
    the dict of live blocks (device pointer -> tensor), for inspection."""
    import torch
    blocks: dict = {}

    def alloc(nbytes):
        try:
            t = torch.empty(nbytes + 255, dtype=torch.uint8, device="cuda")
        except RuntimeError:
            return 0
        ptr = (t.data_ptr() + 255) & ~255
        blocks[ptr] = t
        return ptr

    def free(ptr, nbytes):
        blocks.pop(ptr, None)

    set_allocator(alloc, free)
    return blocks


def partition_batched(problems, options: Options | None = None, stream=None):
    """gk_partition_batched over a list of (coords, k, eps, weights-or-None) with CUDA
    tensors.  Returns (list of (block, centers, influence, result dict), status)."""
    import torch
    m = len(problems)
    inst = (Instance * m)()
    outs = []
    for i, (coords, k, eps, weights) in enumerate(problems):
        n, d = _shape(coords)
        _same_dtype(coords, weights)
        if not (_is_torch(coords) and coords.is_cuda):
            raise ValueError("batched problems take CUDA tensors")
        block = torch.empty(n, dtype=torch.int32, device=coords.device)
        centers = torch.empty((k, d), dtype=torch.float64, device=coords.device)
        infl = torch.empty(k, dtype=torch.float64, device=coords.device)
        inst[i] = Instance(_ptr(coords), _ptr(weights), n, d, _dtype_code(coords), k, 0, eps,
                           _ptr(block), _ptr(centers), _ptr(infl))
        outs.append((block, centers, infl))
    res = (Result * m)()
    opt = options if options is not None else default_options()
    st = lib().gk_partition_batched(ctypes.cast(inst, ctypes.c_void_p), m, ctypes.byref(opt),
                                    ctypes.cast(res, ctypes.c_void_p),
                                    _stream(problems[0][0], stream))
    _check(st, "gk_partition_batched", allow=(GK_ERR_NOT_BALANCED,))
    return [(b, c, i_, res[j].as_dict()) for j, (b, c, i_) in enumerate(outs)], st


def check_wait_timeout(limit_us=2000, stream=None):
    """Runs one bounded device-side wait that nothing completes (gk_check_wait_timeout);
    returns (status, device microseconds the wait took).  GK_ERR_TIMEOUT is expected."""
    waited = ctypes.c_int64(0)
    st = lib().gk_check_wait_timeout(int(limit_us), ctypes.byref(waited),
                                     ctypes.c_void_p(int(stream) if stream is not None else 0))
    return int(st), int(waited.value)


def release():
    lib().gk_release()


def build(force: bool = False) -> str:
    from .nvcc_build import build as _build
    return _build(force=force)
