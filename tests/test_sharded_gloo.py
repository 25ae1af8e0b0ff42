"""The sharded partitioner (paper_1805_01208_gb300/sharded.py) with 2 and 3 gloo ranks on
the CPU: the distributed bootstrap (keys on the common box, sample sort, redistribution
into equal curve ranges, initial centers) and the loop's exchanges, with the steps taken
from the FP64 oracle, must give exactly the oracle's partition of all points.

The points have dyadic coordinates (multiples of 2^-12) and dyadic weights, so that every
sum is exact in any order: the sharded loop then follows the single-process trajectory
bit for bit, and any slip in the data movement (a point lost or duplicated, ties of
equal keys reordered, a wrong redistribution offset or center position) shows.  The
loop below is Algorithm 2 with Algorithm 1 as the oracle runs it, every sum over the
points replaced by a local sum and an all-reduce (Algorithm 1 globalSumVector,
Algorithm 2 globalWeightedMeanVector)."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _points(n, d, seed, weighted, dup):
    rng = np.random.default_rng(seed)
    x = np.floor((rng.random((n, d)) ** 2) * 4096.0) / 4096.0  # graded, dyadic
    if dup:  # a run of identical points: equal keys spread over the ranks' inputs
        x[n // 3: n // 3 + n // 10] = x[n // 3]
    w = np.floor(rng.uniform(8.0, 80.0, n)) / 8.0 if weighted else None
    return x, w


class OracleBackend:
    """The steps of the method from the FP64 oracle (test infrastructure)."""

    def __init__(self, keys_all):
        self.keys_all = keys_all  # the oracle's keys of all points, by input index

    def bounding_box(self, x):
        return x.min(0), x.max(0)

    def keys_in_box(self, x, lo, hi, gidx):
        return self.keys_all[gidx]

    def sort(self, keys, d):
        import oracle
        return oracle.sort_keys(keys)

    def kmeans(self, x, w, n_global, k, eps, C, I, reduce, options):
        import oracle
        import torch
        import torch.distributed as dist

        def allsum(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        def allmin(a, op):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t, op=op)
            return t.numpy()

        o = options
        d = x.shape[1]
        lo = allmin(x.min(0), dist.ReduceOp.MIN)
        hi = allmin(x.max(0), dist.ReduceOp.MAX)
        ext = float((hi - lo).max())
        thr = o["delta_threshold"] if o["delta_threshold"] >= 0 else 1e-4 * ext
        res = dict(iterations=0, balance_passes=0, converged=0, balanced=0)
        C = C.copy()
        I = I.copy()
        I_used = I.copy()
        balanced = False

        def one_pass(I):
            A, _, _ = oracle.assign(x, C, I)
            S, W = oracle.block_weights(A, w, k)
            S, W = allsum(S), float(allsum(np.array([W]))[0])
            bal, I_new, imb = oracle.balance_update(S, W, k, d, eps, I)
            return A, bal, I_new

        for it in range(o["max_iter"]):
            for _ in range(o["max_balance_iter"]):
                I_used = I.copy()
                A, balanced, I = one_pass(I)
                res["balance_passes"] += 1
                if balanced:
                    break
            # movement: local sums and boxes, reduced, then the weighted means
            wv = np.ones(len(x)) if w is None else w
            sw = allsum(np.bincount(A, weights=wv, minlength=k))
            sx = allsum(np.stack([np.bincount(A, weights=wv * x[:, j], minlength=k) for j in range(d)], 1))
            blo = np.full((k, d), np.inf)
            bhi = np.full((k, d), -np.inf)
            np.minimum.at(blo, A, x)
            np.maximum.at(bhi, A, x)
            blo, bhi = allmin(blo, dist.ReduceOp.MIN), allmin(bhi, dist.ReduceOp.MAX)
            C_new = C.copy()
            delta = np.zeros(k)
            dsum, nonempty = 0.0, 0
            for c in range(k):
                if sw[c] == 0.0:
                    continue
                dd, diag = 0.0, 0.0
                for j in range(d):
                    C_new[c, j] = sx[c, j] / sw[c]
                    dd += (C_new[c, j] - C[c, j]) ** 2
                    diag += (bhi[c, j] - blo[c, j]) ** 2
                delta[c] = math.sqrt(dd)
                dsum += math.sqrt(diag)
                nonempty += 1
            beta = dsum / nonempty if nonempty else 0.0
            res["iterations"] += 1
            if delta.max() < thr:
                res["converged"] = 1
                break
            if it == o["max_iter"] - 1:
                break
            C = C_new
            if o["erosion"]:
                I = oracle.erosion(delta, beta, I)
        if not balanced:
            for _ in range(o["final_balance_iter"]):
                I_used = I.copy()
                A, balanced, I = one_pass(I)
                res["balance_passes"] += 1
                if balanced:
                    break
        res["balanced"] = int(balanced)
        return A.astype(np.int32), C, I_used, res


OPTS = dict(max_iter=8, max_balance_iter=20, final_balance_iter=50, erosion=1, delta_threshold=-1.0)


def _rank(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_1805_01208_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, d, k, seed, weighted, dup = case
        x, w = _points(n, d, seed, weighted, dup)
        keys_all = oracle.hilbert_keys(x)
        # uneven input split: rank r holds a contiguous range of the input
        cuts = [0] + [int(n * (r + 1) * (r + 2) / ((world) * (world + 1))) for r in range(world - 1)] + [n]
        lo, hi = cuts[rank], cuts[rank + 1]
        A, C, I, res = sharded.partition_sharded(
            x[lo:hi], k, 0.03, weights=None if w is None else w[lo:hi], options=OPTS,
            backend=OracleBackend(keys_all))
        q.put((rank, lo, A, C, I, res))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [
    (2, (3000, 2, 12, 5, False, False)),
    (3, (2500, 3, 9, 6, True, False)),
    (2, (2000, 2, 7, 7, False, True)),
])
def test_sharded_partition_equals_the_oracle(world, case):
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    outs.sort(key=lambda t: t[0])
    n, d, k, seed, weighted, dup = case
    x, w = _points(n, d, seed, weighted, dup)
    A = np.concatenate([o[2] for o in outs])
    ref = oracle.partition(x, w, k, 0.03, oracle.default_options(**OPTS))
    assert np.array_equal(A, ref["A"])
    for r, o in enumerate(outs):  # equal contiguous ranges of the curve-sorted points
        assert o[5]["shard_offset"] == r * n // world
        assert o[5]["shard_points"] == (r + 1) * n // world - r * n // world
    for o in outs:  # replicated state, the same on every rank
        assert np.array_equal(o[3], ref["C"]) and np.array_equal(o[4], ref["I"])
        assert o[5]["balance_passes"] == ref["result"]["balance_passes"]
        assert o[5]["iterations"] == ref["result"]["iterations"]
        assert o[5]["balanced"] == ref["result"]["balanced"]


def test_float_min_max_through_int64_keys():
    """The driver's box reduction: minimum and maximum of FP64 values through the int64
    reduction of their ordered keys, here with a second process's values stood in by a
    reduction that combines with them."""
    sys.path.insert(0, ROOT)
    from paper_1805_01208_gb300.sharded import _reduce_float
    a = np.array([-3.5, -0.0, 1e-300, -1e300, 2.0, 7.25])
    b = np.array([-4.0, 0.5, -1e-300, 1e300, np.nextafter(2.0, 3.0), 7.25])

    def with_other(other):
        ob = other.view(np.int64)
        ok = np.where(ob >= 0, ob, ob ^ np.int64(0x7FFFFFFFFFFFFFFF))

        def red(buf, op):
            buf[:] = np.minimum(buf, ok) if op == 1 else np.maximum(buf, ok)
        return red

    lo, hi = a.copy(), a.copy()
    _reduce_float(lo, 1, with_other(b))
    _reduce_float(hi, 2, with_other(b))
    assert np.array_equal(lo, np.minimum(a, b)) and np.array_equal(hi, np.maximum(a, b))
