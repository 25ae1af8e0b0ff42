"""gk_partition_batched: many problems of mixed n, d, dtype, k and weights in one call.
Every instance must give exactly what gk_partition gives for it alone (same kernels,
exact order-independent sums), and agree with the FP64 oracle where the oracle runs."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_01208_gb300 import synth

pytestmark = pytest.mark.gpu

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


def _np(t):
    return t.cpu().numpy()


def _problems(specs):
    out = []
    for spec in specs:
        x, w = synth.instance_data(spec)
        out.append((x, w, spec))
    return out


def _run(gk, data, **opt):
    probs = [(_dev(x), spec["k"], spec["eps"], None if w is None else _dev(w)) for x, w, spec in data]
    outs, st = gk.partition_batched(probs, options=gk.default_options(**opt))
    return [(_np(b), _np(c), _np(i), r) for b, c, i, r in outs], st


MIXED = [dict(n=20_000, d=2, k=16, eps=0.03, shape="uniform", seed=71, dtype="f32", weighted=True),
         dict(n=3_001, d=3, k=9, eps=0.03, shape="gmm", seed=72, dtype="f64", weighted=False),
         dict(n=50_000, d=3, k=100, eps=0.03, shape="radial", seed=73, dtype="f32", weighted=True),
         dict(n=777, d=2, k=777, eps=0.0, shape="uniform", seed=74, dtype="f64", weighted=False),
         dict(n=120_000, d=2, k=300, eps=0.03, shape="gmm", seed=75, dtype="f32", weighted=False),
         dict(n=10_000, d=3, k=1, eps=0.03, shape="uniform", seed=76, dtype="f64", weighted=True)]


@pytest.mark.parametrize("assign_dtype", ["f32", "f64"])
def test_batched_equals_single_calls(gk, assign_dtype):
    data = _problems(MIXED)
    outs, st = _run(gk, data, assign_dtype=assign_dtype)
    for (x, w, spec), (A, C, I, r) in zip(data, outs):
        b1, C1, I1, r1 = gk.partition(_dev(x), spec["k"], spec["eps"],
                                      weights=None if w is None else _dev(w),
                                      options=gk.default_options(assign_dtype=assign_dtype))
        assert np.array_equal(A, _np(b1)), spec
        assert np.array_equal(C, _np(C1)) and np.array_equal(I, _np(I1)), spec
        assert r["balance_passes"] == r1["balance_passes"] and r["status"] == r1["status"]
        assert r["iterations"] == r1["iterations"]


def test_batched_matches_oracle(gk):
    data = _problems(MIXED[:2] + MIXED[3:4])
    outs, st = _run(gk, data)
    for (x, w, spec), (A, C, I, r) in zip(data, outs):
        wd = None if w is None else w.astype(np.float64)
        ref = oracle.partition(x.astype(np.float64), wd, spec["k"], spec["eps"],
                               oracle.default_options(threads=THREADS))
        assert r["status"] == ref["result"]["status"]
        assert np.array_equal(A, ref["A"])
        ext = float((x.max(0) - x.min(0)).max())
        assert np.abs(C - ref["C"]).max() <= 1e-10 * ext
        S, W = oracle.block_weights(A, wd, spec["k"])
        if r["balanced"]:
            assert S.max() <= (1 + spec["eps"]) * math.ceil(W / spec["k"]) * (1 + 1e-15)


def test_batched_repeated_call_reuses_the_graph(gk):
    data = _problems(MIXED[:3])
    a, _ = _run(gk, data, assign_dtype="f32")
    b, _ = _run(gk, data, assign_dtype="f32")
    for (A1, C1, I1, r1), (A2, C2, I2, r2) in zip(a, b):
        assert np.array_equal(A1, A2) and np.array_equal(C1, C2) and np.array_equal(I1, I2)


def test_batched_rejects_host_coordinates(gk):
    import ctypes
    x = np.random.default_rng(0).random((100, 2))
    inst = (gk.Instance * 1)()
    block = _dev(np.zeros(100, np.int32))
    inst[0] = gk.Instance(x.ctypes.data_as(ctypes.c_void_p), None, 100, 2, gk.GK_F64, 4, 0, 0.03,
                          ctypes.c_void_p(block.data_ptr()), None, None)
    st = gk.lib().gk_partition_batched(ctypes.cast(inst, ctypes.c_void_p), 1, None, None, None)
    assert st == gk.GK_ERR_INVALID_ARG


FP32_FORM_MAX_DISAGREEMENT = 1e-4  # FP32 form: fraction assigned differently from the FP64 argmin


@pytest.mark.slow
def test_batched_workload_64_instances(gk):
    """The 64-instance workload in the FP32 form: for every instance the balance bound
    (exactly, on the host, whenever the instance reports balance) and at most 1e-4 of the
    points assigned differently from the FP64 argmin under the returned state -- every
    point of instances up to 1e5 points, a uniform sample of 5e4 points of the others."""
    specs = synth.batched_instances(64, seed=4)
    data = _problems(specs)
    outs, st = _run(gk, data, assign_dtype="f32")
    rng = np.random.default_rng(1)
    for (x, w, spec), (A, C, I, r) in zip(data, outs):
        wd = None if w is None else w.astype(np.float64)
        S, W = oracle.block_weights(A, wd, spec["k"])
        if r["balanced"]:
            assert S.max() <= (1 + spec["eps"]) * math.ceil(W / spec["k"]) * (1 + 1e-15)
        n = len(x)
        idx = np.arange(n) if n <= 100_000 else rng.choice(n, 50_000, replace=False)
        A_ref, _, _ = oracle.assign(x[idx].astype(np.float64), C, I, threads=THREADS)
        frac = (A[idx] != A_ref).mean()
        assert frac <= FP32_FORM_MAX_DISAGREEMENT, (spec, frac)


def test_batched_with_bounds_equals_without(gk):
    """Every instance of a batch with bounds (FP64 argmin): the oracle's free-running
    trajectory exactly, and bit for bit the batch without bounds."""
    data = _problems(MIXED)
    with_b, st1 = _run(gk, data, bounds=1)
    without, st0 = _run(gk, data, bounds=0)
    assert st1 == st0
    for (x, w, spec), (A1, C1, I1, r1) in zip(data, with_b):
        wd = None if w is None else w.astype(np.float64)
        ref = oracle.partition(x, wd, spec["k"], spec["eps"], oracle.default_options(threads=THREADS))
        rr = ref["result"]
        assert r1["status"] == rr["status"] and np.array_equal(A1, ref["A"]), spec
        assert r1["balance_passes"] == rr["balance_passes"] and r1["iterations"] == rr["iterations"]
        ext = float((x.max(0) - x.min(0)).max())
        assert np.abs(C1 - ref["C"]).max() <= 1e-10 * ext
        assert np.allclose(I1, ref["I"], rtol=1e-12, atol=0)
    for (A1, C1, I1, r1), (A0, C0, I0, r0) in zip(with_b, without):
        assert np.array_equal(A1, A0) and np.array_equal(C1, C0) and np.array_equal(I1, I0)
        assert r1["balance_passes"] == r0["balance_passes"]
