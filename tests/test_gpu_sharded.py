"""Sharded runs on the GPU: the entry points a sharded run is built from (bounding box,
keys on a given box, the stable key sort) against the oracle, and the sharded
partitioner with 1 and 2 processes (both on cuda:0, exchanging through a gloo process
group on the host: no kernel waits on another process) against gk_partition on all
points and against the oracle's free-running trajectory.  With the FP64 assignment and
exact integer sums, the block ids, centers, influence and pass counts must be those of
the single call bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1805_01208_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def gk():
    import torch
    import paper_1805_01208_gb300 as gk
    gk.build()
    torch.cuda.set_device(0)
    return gk


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape,d,dtype,n", [("gmm", 3, "f64", 30_011), ("spots", 2, "f32", 40_000)])
def test_box_keys_and_sort_match_the_oracle(gk, shape, d, dtype, n):
    x = synth.make_points(shape, n, d, 17, dtype)
    lo, hi = gk.bounding_box(_dev(x))
    assert np.array_equal(lo, x.min(0).astype(np.float64)) and np.array_equal(hi, x.max(0).astype(np.float64))
    keys_all = oracle.hilbert_keys(x)
    # own box: the keys of gk_hilbert_keys; a subset on the box of all points: the
    # oracle's keys of those points within the whole set
    k_own = gk.hilbert_keys_in_box(_dev(x), lo, hi).cpu().numpy().view(np.uint64)
    assert np.array_equal(k_own, keys_all)
    sub = np.arange(n // 3, n // 3 + n // 4)
    k_sub = gk.hilbert_keys_in_box(_dev(x[sub]), lo, hi).cpu().numpy().view(np.uint64)
    assert np.array_equal(k_sub, keys_all[sub])
    # points outside the given box are rejected
    with pytest.raises(gk.GKError):
        gk.hilbert_keys_in_box(_dev(x), lo + 1e-3, hi)
    # the stable sort, with many equal keys
    keys = keys_all.copy()
    keys[::7] = keys[3]
    perm = gk.sort_keys(_dev(keys.view(np.int64)), d).cpu().numpy()
    assert np.array_equal(perm, oracle.sort_keys(keys))
    perm_h = gk.sort_keys(keys, d)  # host buffers
    assert np.array_equal(perm_h, oracle.sort_keys(keys))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_1805_01208_gb300 as gk
    from paper_1805_01208_gb300 import sharded, synth as sy
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        shape, n, d, k, dtype, weighted, seed = case
        x = sy.make_points(shape, n, d, seed, dtype)
        w = sy.uniform_weights(n, seed, dtype=x.dtype) if weighted else None
        cuts = [0] + [(n * (r + 1)) // world + (r * 37) % 101 for r in range(world - 1)] + [n]
        lo, hi = cuts[rank], cuts[rank + 1]
        A, C, I, res = sharded.partition_sharded(
            x[lo:hi], k, 0.03, weights=None if w is None else w[lo:hi],
            options=gk.default_options(assign_dtype="f64"))
        q.put((rank, A, C, I, res))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e), None, None, None))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [
    (1, ("gmm", 30_011, 3, 37, "f64", False, 31)),
    (2, ("gmm", 30_011, 3, 37, "f64", False, 31)),
    (2, ("radial", 20_000, 2, 20, "f64", True, 32)),
    (2, ("spots", 60_000, 2, 96, "f32", False, 33)),
])
def test_sharded_partition_equals_gk_partition_and_the_oracle(gk, world, case):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = sorted([q.get(timeout=600) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
    for o in outs:
        assert not isinstance(o[1], str), o[1]
    assert all(p.exitcode == 0 for p in procs)
    shape, n, d, k, dtype, weighted, seed = case
    x = synth.make_points(shape, n, d, seed, dtype)
    w = synth.uniform_weights(n, seed, dtype=x.dtype) if weighted else None
    A = np.concatenate([o[1] for o in outs])
    block, C, I, res = gk.partition(_dev(x), k, 0.03, weights=None if w is None else _dev(w),
                                    options=gk.default_options(assign_dtype="f64"))
    assert np.array_equal(A, block.cpu().numpy())
    for o in outs:
        assert np.array_equal(o[2], C.cpu().numpy()) and np.array_equal(o[3], I.cpu().numpy())
        assert o[4]["balance_passes"] == res["balance_passes"] and o[4]["iterations"] == res["iterations"]
        assert o[4]["status"] == res["status"]
    ref = oracle.partition(x, None if w is None else w.astype(np.float64), k, 0.03,
                           oracle.default_options(threads=THREADS))
    assert np.array_equal(A, ref["A"])
    ext = float((x.max(0) - x.min(0)).max())
    assert np.abs(outs[0][2] - ref["C"]).max() <= 1e-10 * ext
    assert np.allclose(outs[0][3], ref["I"], rtol=1e-12, atol=0)
