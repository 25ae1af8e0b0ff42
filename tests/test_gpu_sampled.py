"""Random initialization (Section 4.5) on the GPU against the FP64 oracle: the sample
rounds on doubling samples of a given random order, then Algorithm 2 on all points
(gk_partition_sampled)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_01208_gb300 import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
TIE = 1e-12


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
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _rel_center_err(C, Cref, x):
    ext = float((x.max(0) - x.min(0)).max())
    return float(np.abs(np.asarray(C) - Cref).max() / ext)


def _assert_effective_argmin(A, x, C, I, max_frac=0.0):
    A_ref, best, second = oracle.assign(x, C, I, threads=THREADS)
    ties = (second - best) <= TIE * np.maximum(best, 1e-300)
    bad = (A != A_ref) & ~ties
    assert bad.sum() <= max_frac * len(x), f"{bad.sum()} points differ from the FP64 argmin"


def _run_both(gk, x, w, k, eps, order, sample0, **opt):
    o = gk.default_options(**opt)
    block, C, I, res = gk.partition_sampled(_dev(x), k, eps, _dev(order), sample0,
                                            weights=None if w is None else _dev(w), options=o)
    oo = oracle.default_options(threads=THREADS)
    for key in ("max_iter", "max_balance_iter", "final_balance_iter", "erosion"):
        if key in opt:
            setattr(oo, key, opt[key])
    ref = oracle.partition_sampled(x, None if w is None else w.astype(np.float64), k, eps, order,
                                   sample0, oo)
    return _np(block), _np(C), _np(I), res, ref


def _check_same_run(x, w, k, eps, A, C, I, res, ref):
    xd = x.astype(np.float64)
    rr = ref["result"]
    assert res["status"] == rr["status"] and res["balanced"] == rr["balanced"], (res, rr)
    assert res["iterations"] == rr["iterations"] and res["balance_passes"] == rr["balance_passes"]
    S, W = oracle.block_weights(A, None if w is None else w.astype(np.float64), k)
    if rr["balanced"]:
        assert S.max() <= (1 + eps) * math.ceil(W / k) * (1 + 1e-15)
    _assert_effective_argmin(A, xd, C, I)
    same = (A == ref["A"]).mean()
    assert same == 1.0, f"assignment differs from the oracle on {1 - same:.3e} of the points"
    assert _rel_center_err(C, ref["C"], xd) < 1e-10
    assert np.allclose(I, ref["I"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("shape,d,n,k,weighted,sample0", [("gmm", 3, 30_011, 37, False, 0),
                                                          ("radial", 2, 20_000, 20, True, 0),
                                                          ("uniform", 3, 4_099, 7, True, 0),
                                                          ("gmm", 2, 50_000, 16, False, 1000)])
def test_sampled_matches_oracle(gk, shape, d, n, k, weighted, sample0):
    x = synth.make_points(shape, n, d, 61, "f64")
    w = synth.uniform_weights(n, 61) if weighted else None
    order = synth.random_order(n, 61)
    m0 = oracle.sample_first(n, k, sample0)
    assert oracle.sample_rounds(n, m0) >= 3  # several rounds, samples with ragged tiles
    A, C, I, res, ref = _run_both(gk, x, w, k, 0.03, order, sample0)
    _check_same_run(x, w, k, 0.03, A, C, I, res, ref)


def test_sampled_fp32_input(gk):
    x = synth.make_points("gmm", 40_000, 3, 67, "f32")
    order = synth.random_order(len(x), 67)
    A, C, I, res, ref = _run_both(gk, x, None, 24, 0.03, order, 0)
    _check_same_run(x, None, 24, 0.03, A, C, I, res, ref)


def test_sampled_without_rounds_equals_partition(gk):
    x = synth.make_points("gmm", 25_000, 3, 71, "f64")
    order = synth.random_order(len(x), 71)
    b1, C1, I1, r1 = gk.partition_sampled(_dev(x), 50, 0.03, _dev(order), 10**6)
    b2, C2, I2, r2 = gk.partition(_dev(x), 50, 0.03)
    assert np.array_equal(_np(b1), _np(b2)) and np.array_equal(_np(C1), _np(C2))
    assert np.array_equal(_np(I1), _np(I2))
    assert r1["iterations"] == r2["iterations"] and r1["balance_passes"] == r2["balance_passes"]


def test_sampled_graph_and_host_loop_agree(gk):
    x = synth.make_points("gmm", 60_000, 2, 73, "f64")
    order = synth.random_order(len(x), 73)
    out = []
    for g in (1, 0):
        block, C, I, res = gk.partition_sampled(_dev(x), 40, 0.03, _dev(order), 0,
                                                options=gk.default_options(use_graph=g))
        out.append((_np(block), _np(C), _np(I), res))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert out[0][3]["balance_passes"] == out[1][3]["balance_passes"]
    assert out[0][3]["iterations"] == out[1][3]["iterations"]


def test_sampled_host_buffers_agree(gk):
    x = synth.make_points("radial", 30_000, 2, 79, "f64")
    order = synth.random_order(len(x), 79)
    b1, C1, I1, r1 = gk.partition_sampled(_dev(x), 24, 0.03, _dev(order))
    b2, C2, I2, r2 = gk.partition_sampled(x, 24, 0.03, order)  # host pointers, staged
    assert np.array_equal(_np(b1), b2) and np.array_equal(_np(C1), C2)


def test_sampled_repeated_calls_reuse_the_graph(gk):
    x = synth.make_points("gmm", 45_000, 3, 83, "f64")
    order = synth.random_order(len(x), 83)
    xt, ot = _dev(x), _dev(order)
    first = gk.partition_sampled(xt, 30, 0.03, ot)
    for _ in range(2):
        again = gk.partition_sampled(xt, 30, 0.03, ot)
        assert np.array_equal(_np(first[0]), _np(again[0]))
        assert np.array_equal(_np(first[1]), _np(again[1]))
    # another problem in between, then the first again
    gk.partition_sampled(_dev(x[:20_000]), 12, 0.03, _dev(synth.random_order(20_000, 1)))
    again = gk.partition_sampled(xt, 30, 0.03, ot)
    assert np.array_equal(_np(first[0]), _np(again[0]))


def test_sampled_many_centers_with_supergroups(gk):
    """k = 2500 (group records of 32 centers, supergroups of 32 groups) and four rounds:
    the result is the FP64 argmin under its returned state and meets the bound."""
    n, k = 200_000, 2500
    x = synth.make_points("gmm", n, 3, 89, "f64")
    order = synth.random_order(n, 89)
    block, C, I, res = gk.partition_sampled(_dev(x), k, 0.03, _dev(order), 12_500)
    A, C, I = _np(block), _np(C), _np(I)
    assert res["iterations"] >= 4
    S, W = oracle.block_weights(A, None, k)
    if res["balanced"]:
        assert S.max() <= 1.03 * math.ceil(W / k)
    idx = np.random.default_rng(0).choice(n, 20_000, replace=False)
    _assert_effective_argmin(A[idx], x[idx], C, I)


def test_sampled_edge_k_equals_n_and_tiny(gk):
    x = synth.make_points("uniform", 300, 2, 97, "f64")
    order = synth.random_order(300, 97)
    A, C, I, res, ref = _run_both(gk, x, None, 300, 0.0, order, 0)
    assert np.array_equal(A, ref["A"])
    xs = synth.make_points("uniform", 5, 3, 98, "f64")
    A, C, I, res, ref = _run_both(gk, xs, None, 2, 0.03, synth.random_order(5, 98), 1)
    assert np.array_equal(A, ref["A"]) and res["iterations"] == ref["result"]["iterations"]


def test_sampled_rejects_an_order_that_is_not_a_permutation(gk):
    x = _dev(synth.make_points("uniform", 2_000, 2, 101, "f64"))
    order = np.arange(2_000, dtype=np.int64)
    order[5] = 6  # duplicate: index 5 never named
    with pytest.raises(gk.GKError) as e:
        gk.partition_sampled(x, 8, 0.03, _dev(order))
    assert e.value.status == gk.GK_ERR_INVALID_ARG
    order[5] = 2_000  # out of range
    with pytest.raises(gk.GKError) as e:
        gk.partition_sampled(x, 8, 0.03, _dev(order))
    assert e.value.status == gk.GK_ERR_INVALID_ARG
    order[5] = -1
    with pytest.raises(gk.GKError):
        gk.partition_sampled(x, 8, 0.03, order)
    order[5] = 5  # the context stays usable
    block, C, I, res = gk.partition_sampled(x, 8, 0.03, _dev(order))
    assert res["balanced"] == 1


@pytest.mark.slow
def test_full_size_sampled_gmm3d_1e7_k1024(gk):
    """The benchmark workload (3D Gaussian mixture, n = 1e7, k = 1024, FP64) with the
    random initialization, checked on sampled outputs."""
    import torch
    x, w, spec = synth.workload("gmm3d_1e7_k1024_f64")
    k, eps = spec["k"], spec["eps"]
    order = synth.random_order(len(x), spec["seed"])
    xt = _dev(x)
    block, C, I, res = gk.partition_sampled(xt, k, eps, _dev(order))
    torch.cuda.synchronize()
    A, C, I = _np(block), _np(C), _np(I)
    assert res["balanced"] == 1
    assert res["iterations"] > oracle.sample_rounds(len(x), oracle.sample_first(len(x), k))
    S = np.bincount(A, minlength=k)
    assert S.max() <= (1 + eps) * math.ceil(len(x) / k)
    idx = np.random.default_rng(0).choice(len(x), 20_000, replace=False)
    _assert_effective_argmin(A[idx], x[idx], C, I)
    Cn, delta, beta = gk.move_centers(xt, _dev(A), _dev(C))
    Cr, dr, br = oracle.move_centers(x, None, A, C)
    assert _rel_center_err(_np(Cn), Cr, x) < 1e-10


def test_sampled_with_bounds_is_identical(gk):
    """Random initialization with bounds: the oracle's trajectory exactly, and bit for
    bit the run without bounds."""
    x = synth.make_points("gmm", 80_000, 3, 103, "f64")
    order = synth.random_order(len(x), 103)
    out = []
    for bounds in (1, 0):
        block, C, I, res = gk.partition_sampled(_dev(x), 40, 0.03, _dev(order), 2000,
                                                options=gk.default_options(bounds=bounds))
        out.append((_np(block), _np(C), _np(I), res))
    ref = oracle.partition_sampled(x, None, 40, 0.03, order, 2000,
                                   oracle.default_options(threads=THREADS))
    b1, C1, I1, r1 = out[0]
    rr = ref["result"]
    assert r1["status"] == rr["status"] and r1["balanced"] == rr["balanced"]
    assert np.array_equal(b1, ref["A"])
    assert r1["iterations"] == rr["iterations"] and r1["balance_passes"] == rr["balance_passes"]
    ext = float((x.max(0) - x.min(0)).max())
    assert np.abs(C1 - ref["C"]).max() <= 1e-10 * ext
    assert np.allclose(I1, ref["I"], rtol=1e-12, atol=0)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    assert out[0][3]["balance_passes"] == out[1][3]["balance_passes"]
