"""bench.py --gpus N runs N independent replicas (the method shards by points, but every
call uses one GPU): rank r times its own instance, and the JSON line takes the slowest
rank's time and the sum of the ranks' work.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1e6 * (rank + 1), dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, w))


def test_two_gloo_ranks_reduce_time_by_max_and_work_by_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 150.0, 3e6), (1, 150.0, 3e6)]


def test_replicas_are_independent_instances():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    spec = dict(shape="gmm", n=5000, d=3, seed=2, dtype="f64")
    x0, x1 = bench.replica_points(spec, 0), bench.replica_points(spec, 1)
    assert x0.shape == x1.shape == (5000, 3)
    assert not np.array_equal(x0, x1)
    from paper_1805_01208_gb300 import synth
    assert np.array_equal(x0, synth.make_points("gmm", 5000, 3, 2, "f64"))
