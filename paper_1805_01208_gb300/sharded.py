"""Balanced k-means on points split over several processes, one GPU each.

The paper's distributed design (Section 4.1; Algorithm 2): every process computes the
Hilbert keys of its points on the bounding box of all points, a global sort by key
(sortGlobal) and a redistribution give each process a contiguous range of the
curve-sorted points of equal size, the initial centers are the sorted points at
positions i n/k + n/(2k), and the k-means loop then runs on every process with the
centers and influence replicated, its only exchanges being the sum of the block
weights per assignment pass (Algorithm 1, globalSumVector) and the weighted means per
movement (Algorithm 2, globalWeightedMeanVector).

This module moves the points between the processes (a sample sort with regular
sampling on the keys: one all-gather of samples, one all-to-all of the points, then a
second all-to-all into equal ranges; the block ids go back to their input owners the
same way) and hands the reductions of the loop to the process group.  Every step of
the method runs in the CUDA library: keys on the common box (gk_hilbert_keys_in_box),
the local stable sorts (gk_sort_keys), the loop (gk_balanced_kmeans_sharded).  The
library's reductions are exact integers, so the partition does not depend on how the
points are split; with the FP64 assignment it is that of gk_partition on all points.

Ties of equal keys keep the input order across processes: process r holds input points
[off_r, off_r+1) in input order, equal keys all go to one process, and every process
concatenates what it receives in sender order before its own stable sort.

The step functions are taken from a backend object (the CUDA library by default), so
that the data movement can be run with another implementation of the steps.
"""
from __future__ import annotations

import numpy as np

_OPS = None


def _ops():
    global _OPS
    if _OPS is None:
        import torch.distributed as dist
        _OPS = {0: dist.ReduceOp.SUM, 1: dist.ReduceOp.MIN, 2: dist.ReduceOp.MAX}
    return _OPS


def make_reduce(group=None):
    """The exchange of the sharded loop over a torch.distributed process group: reduce(buf,
    op) replaces the int64 numpy array buf in place by its sum / minimum / maximum over
    the group's processes (a device copy for NCCL groups)."""
    import torch
    import torch.distributed as dist

    nccl = dist.get_backend(group) == "nccl"

    def reduce(buf, op):
        t = torch.from_numpy(buf)  # shares the memory of buf
        if nccl:
            td = t.cuda()
            dist.all_reduce(td, op=_ops()[op], group=group)
            t.copy_(td.cpu())
        else:
            dist.all_reduce(t, op=_ops()[op], group=group)

    return reduce


def _device(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def _all_gather_np(arr, group):
    """Concatenation, in process order, of every process's 1-D numpy array."""
    import torch
    import torch.distributed as dist
    if arr.dtype == np.uint64:  # carried as int64 bit patterns
        out, ns = _all_gather_np(arr.view(np.int64), group)
        return out.view(np.uint64), ns
    R = dist.get_world_size(group)
    dev = _device(group)
    n = torch.tensor([arr.shape[0]], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(R)]
    dist.all_gather(ns, n, group=group)
    ns = [int(v.item()) for v in ns]
    m = max(ns) if ns else 0
    buf = torch.zeros(m, dtype=torch.from_numpy(arr[:0]).dtype, device=dev)
    buf[: arr.shape[0]] = torch.from_numpy(arr).to(dev)
    outs = [torch.zeros_like(buf) for _ in range(R)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([o[:c].cpu().numpy() for o, c in zip(outs, ns)]), ns


def _all_to_all_np(arr, send_counts, group):
    """All-to-all of the rows of a numpy array: rows [sum(send_counts[:q]) ...) go to process
    q; returns what every process sent here, concatenated in sender order."""
    import torch
    import torch.distributed as dist
    if arr.dtype == np.uint64:  # carried as int64 bit patterns
        return _all_to_all_np(arr.view(np.int64), send_counts, group).view(np.uint64)
    R = dist.get_world_size(group)
    dev = _device(group)
    sc = torch.tensor(send_counts, dtype=torch.int64, device=dev)
    rc = torch.empty(R, dtype=torch.int64, device=dev)
    dist.all_to_all_single(rc, sc, group=group)
    rc = [int(v) for v in rc.cpu().tolist()]
    row = int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1
    src = torch.from_numpy(np.ascontiguousarray(arr).reshape(-1)).to(dev)
    out = torch.empty(sum(rc) * row, dtype=src.dtype, device=dev)
    dist.all_to_all_single(out, src, [c * row for c in rc], [c * row for c in send_counts], group=group)
    return out.cpu().numpy().reshape((sum(rc),) + arr.shape[1:])


class LibraryBackend:
    """The steps of the method as calls of the CUDA library on the current device."""

    def __init__(self):
        import paper_1805_01208_gb300 as gk
        self.gk = gk

    def bounding_box(self, x):
        import torch
        return self.gk.bounding_box(torch.from_numpy(x).cuda())

    def keys_in_box(self, x, lo, hi, gidx):
        import torch
        keys = self.gk.hilbert_keys_in_box(torch.from_numpy(x).cuda(), lo, hi)
        return keys.cpu().numpy().view(np.uint64)

    def sort(self, keys, d):
        import torch
        perm = self.gk.sort_keys(torch.from_numpy(keys.view(np.int64)).cuda(), d)
        return perm.cpu().numpy()

    def kmeans(self, x, w, n_global, k, eps, C, I, reduce, options):
        import torch
        xt = torch.from_numpy(x).cuda()
        wt = None if w is None else torch.from_numpy(w).cuda()
        Ct = torch.from_numpy(C).cuda()
        It = torch.from_numpy(I).cuda()
        block, res = self.gk.balanced_kmeans_sharded(xt, n_global, k, eps, Ct, It, reduce,
                                                     weights=wt, options=options)
        return block.cpu().numpy(), Ct.cpu().numpy(), It.cpu().numpy(), res


def sample_sort(keys, payload, d, backend, group=None):
    """Global stable sort by key of the points of all processes (sortGlobal): returns this
    process's part (keys, payload arrays) of the sorted sequence; the parts are contiguous
    and in process order.  Regular sampling: every process contributes R samples of its
    sorted keys, the R - 1 splitters are every R-th of the sorted samples; a key below the
    first splitter goes to process 0, a key in [s_(q-1), s_q) to process q."""
    import torch.distributed as dist
    R = dist.get_world_size(group)
    perm = backend.sort(keys, d) if keys.shape[0] > 0 else np.zeros(0, dtype=np.int64)
    keys = keys[perm]
    payload = [a[perm] for a in payload]
    n = keys.shape[0]
    samp = keys[(np.arange(R, dtype=np.int64) * n) // R] if n > 0 else keys[:0]
    all_s, _ = _all_gather_np(samp, group)
    all_s = np.sort(all_s, kind="stable")
    splitters = all_s[np.arange(1, R, dtype=np.int64) * (all_s.shape[0] // R)] if all_s.shape[0] >= R \
        else np.full(R - 1, np.iinfo(np.uint64).max, dtype=np.uint64)
    bounds = np.searchsorted(keys, splitters, side="left")
    edges = np.concatenate([[0], bounds, [n]]).astype(np.int64)
    counts = np.diff(edges).tolist()
    keys_r = _all_to_all_np(keys, counts, group)
    pay_r = [_all_to_all_np(a, counts, group) for a in payload]
    perm = backend.sort(keys_r, d) if keys_r.shape[0] > 0 else np.zeros(0, dtype=np.int64)
    return keys_r[perm], [a[perm] for a in pay_r]


def redistribute(arrays, n_global, group=None):
    """The sorted sequence into equal contiguous ranges: process r gets the global positions
    [r n / R, (r + 1) n / R) (integer division).  arrays hold this process's part of the
    sequence, the parts contiguous and in process order."""
    import torch.distributed as dist
    R, r = dist.get_world_size(group), dist.get_rank(group)
    c = arrays[0].shape[0]
    _, counts = _all_gather_np(np.zeros(c, dtype=np.int8), group)
    start = int(sum(counts[:r]))
    targets = [(q * n_global) // R for q in range(R + 1)]
    send = []
    for q in range(R):
        lo, hi = max(start, targets[q]), min(start + c, targets[q + 1])
        send.append(max(0, hi - lo))
    return [_all_to_all_np(a, send, group) for a in arrays], targets[r]


def initial_centers(x_sorted, offset, n_global, k, group=None):
    """C[i] = the sorted point at global position i n/k + n/(2k) (Algorithm 2), from the
    process holding it (a sum over the processes with zeros elsewhere: exact)."""
    import torch
    import torch.distributed as dist
    d = x_sorted.shape[1]
    pos = np.arange(k, dtype=np.int64) * n_global // k + n_global // (2 * k)
    mine = (pos >= offset) & (pos < offset + x_sorted.shape[0])
    C = np.zeros((k, d), dtype=np.float64)
    C[mine] = x_sorted[pos[mine] - offset].astype(np.float64)
    t = torch.from_numpy(C).to(_device(group))
    dist.all_reduce(t, group=group)
    return t.cpu().numpy()


def partition_sharded(x, k, eps, weights=None, options=None, group=None, backend=None):
    """Algorithm 2 over the processes of `group`.  x: this process's input points, numpy (n_r,
    d) FP32 or FP64 (process r holds input points [off_r, off_r+1) of the whole input, in
    input order); weights: (n_r,) or None.  Returns (block ids of this process's input
    points, centers, influence, result dict of the loop).  Every process needs at least one
    input point."""
    import torch.distributed as dist
    backend = backend or LibraryBackend()
    R, r = dist.get_world_size(group), dist.get_rank(group)
    n_r, d = x.shape
    if n_r < 1:
        raise ValueError("every process needs at least one input point")
    _, in_counts = _all_gather_np(np.zeros(n_r, dtype=np.int8), group)
    off = int(sum(in_counts[:r]))
    n_global = int(sum(in_counts))
    reduce = make_reduce(group)
    # bounding box of all points, keys on it
    lo, hi = backend.bounding_box(x)
    lo64 = np.ascontiguousarray(lo, dtype=np.float64)
    hi64 = np.ascontiguousarray(hi, dtype=np.float64)
    _reduce_float(lo64, 1, reduce)
    _reduce_float(hi64, 2, reduce)
    gidx = np.arange(off, off + n_r, dtype=np.int64)
    keys = backend.keys_in_box(x, lo64, hi64, gidx)
    payload = [x, gidx] + ([weights] if weights is not None else [])
    keys_s, pay_s = sample_sort(keys, payload, d, backend, group)
    arrays, start = redistribute([keys_s] + pay_s, n_global, group)
    xs, gs = arrays[1], arrays[2]
    ws = arrays[3] if weights is not None else None
    C = initial_centers(xs, start, n_global, k, group)
    I = np.ones(k)
    block_s, C, I, res = backend.kmeans(np.ascontiguousarray(xs), None if ws is None else np.ascontiguousarray(ws),
                                        n_global, k, eps, C, I, reduce, options)
    res = dict(res, shard_offset=start, shard_points=int(xs.shape[0]))
    # block ids back to the owners of the input points
    owner = np.searchsorted(np.cumsum(in_counts), gs, side="right")
    order = np.argsort(owner, kind="stable")
    send = np.bincount(owner, minlength=R).tolist()
    g_back = _all_to_all_np(gs[order], send, group)
    b_back = _all_to_all_np(block_s[order].astype(np.int32), send, group)
    out = np.empty(n_r, dtype=np.int32)
    out[g_back - off] = b_back
    return out, C, I, res


def _reduce_float(v, op, reduce):
    """Minimum (op 1) or maximum (2) of FP64 values over the processes, through the int64
    reduction on their ordered keys."""
    b = v.view(np.int64).copy()
    keys = np.where(b >= 0, b, b ^ np.int64(0x7FFFFFFFFFFFFFFF))  # order of the values
    reduce(keys, op)
    v[:] = np.where(keys >= 0, keys, keys ^ np.int64(0x7FFFFFFFFFFFFFFF)).view(np.float64)
