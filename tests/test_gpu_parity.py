"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bars: Hilbert keys, sort permutation and initial centers bit-exact; FP64 assignment
equal to the oracle's except at points whose two best effective distances are within
1e-12 relative of each other; block weights exact (unit weights) or within 1e-12
relative; centers within 1e-10 relative (of the bounding-box extent); the balance
bound met exactly."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_01208_gb300 import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
TIE = 1e-12
FP32_FORM_MAX_DISAGREEMENT = 1e-4  # FP32 form: fraction assigned differently from the FP64 argmin


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


def _points(shape, n, d, seed, dtype):
    return synth.make_points(shape, n, d, seed, dtype)


def _near_ties(x, C, I):
    """Mask of points whose two smallest effective distances are within TIE relative."""
    A, best, second = oracle.assign(x, C, I, threads=THREADS)
    return A, (second - best) <= TIE * np.maximum(best, 1e-300)


def _assert_same_assignment(A_gpu, x, C, I, max_frac=0.0):
    A_ref, ties = _near_ties(x, C, I)
    bad = (A_gpu != A_ref) & ~ties
    assert bad.sum() <= max_frac * len(x), (
        f"{bad.sum()} points differ from the FP64 argmin (ties allowed: {ties.sum()})")
    return A_ref


def _rel_center_err(C, Cref, x):
    ext = float((x.max(0) - x.min(0)).max())
    return float(np.abs(np.asarray(C) - Cref).max() / ext)


# ----------------------------------------------------------------------------------------
# Hilbert keys, sort, initial centers (bit-exact)
# ----------------------------------------------------------------------------------------
CASES = [("uniform", 2, "f64", 10_007), ("gmm", 3, "f64", 30_011), ("radial", 2, "f32", 5_003),
         ("gmm", 3, "f32", 70_001), ("spots", 2, "f32", 40_000), ("uniform", 3, "f64", 257)]


@pytest.mark.parametrize("shape,d,dtype,n", CASES)
def test_hilbert_keys_bit_exact(gk, shape, d, dtype, n):
    x = _points(shape, n, d, 7, dtype)
    keys = gk.hilbert_keys(_dev(x))
    ref = oracle.hilbert_keys(x)
    assert np.array_equal(_np(keys).view(np.uint64), ref)


def test_hilbert_keys_offset_box_and_duplicates(gk):
    rng = np.random.default_rng(3)
    x = 1000.0 + rng.random((5000, 3)) * 1e-3
    x[::5] = x[0]  # duplicates
    x[7] = x.min(0)
    keys = gk.hilbert_keys(_dev(x))
    assert np.array_equal(_np(keys).view(np.uint64), oracle.hilbert_keys(x))
    xf = x.astype(np.float32)
    keys = gk.hilbert_keys(_dev(xf))
    assert np.array_equal(_np(keys).view(np.uint64), oracle.hilbert_keys(xf))


def test_hilbert_keys_host_buffers(gk):
    x = _points("uniform", 3000, 2, 5, "f64")
    keys = gk.hilbert_keys(x)  # numpy in, numpy out: staged through the workspace
    assert np.array_equal(keys, oracle.hilbert_keys(x))


@pytest.mark.parametrize("shape,d,dtype,n", CASES)
def test_sfc_init_bit_exact(gk, shape, d, dtype, n):
    x = _points(shape, n, d, 11, dtype)
    k = min(37, n)
    perm, C = gk.sfc_init(_dev(x), k)
    ref_perm = oracle.sort_keys(oracle.hilbert_keys(x))
    assert np.array_equal(_np(perm), ref_perm)
    ref_C = oracle.sfc_centers(x.astype(np.float64)[ref_perm], k)
    assert np.array_equal(_np(C), ref_C)


def test_sort_is_stable_on_equal_keys(gk):
    x = np.zeros((10_000, 2))
    x[:, 0] = np.repeat(np.arange(10.0), 1000)  # ten distinct cells, 1000 points each
    perm, _ = gk.sfc_init(_dev(x), 3)
    ref = oracle.sort_keys(oracle.hilbert_keys(x))
    assert np.array_equal(_np(perm), ref)


# ----------------------------------------------------------------------------------------
# One assignment pass (teacher-forced: the same C, I on both sides)
# ----------------------------------------------------------------------------------------
def _sorted(x):
    return np.ascontiguousarray(x[oracle.sort_keys(oracle.hilbert_keys(x))])


@pytest.mark.parametrize("shape,d,dtype,n,k", [("uniform", 2, "f64", 50_000, 64),
                                                ("gmm", 3, "f64", 60_013, 300),
                                                ("radial", 2, "f32", 40_000, 500),
                                                ("gmm", 3, "f32", 20_000, 17)])
def test_assign_fp64_matches_oracle(gk, shape, d, dtype, n, k):
    x = _sorted(_points(shape, n, d, 13, dtype))
    rng = np.random.default_rng(k)
    C = x[rng.choice(n, k, replace=False)].astype(np.float64) + 1e-3 * rng.standard_normal((k, d))
    I = rng.uniform(0.6, 1.6, k)
    block, S = gk.assign(_dev(x), _dev(C), _dev(I), assign_dtype="f64")
    A = _np(block)
    A_ref = _assert_same_assignment(A, x.astype(np.float64), C, I)
    S_ref, _ = oracle.block_weights(A, None, k)
    assert np.array_equal(_np(S), S_ref)
    assert (A == A_ref).mean() > 0.9999


def test_assign_unsorted_points_and_many_centers(gk):
    """Points in random order make every tile span the domain: candidate lists overflow
    and the kernel scans all centers."""
    x = synth.uniform_box(20_000, 2, seed=17)
    rng = np.random.default_rng(1)
    k = 2000
    C = rng.random((k, 2))
    I = rng.uniform(0.8, 1.25, k)
    block, _ = gk.assign(_dev(x), _dev(C), _dev(I), assign_dtype="f64")
    _assert_same_assignment(_np(block), x, C, I)


@pytest.mark.parametrize("coherent", [True, False])
def test_assign_with_supergroups(gk, coherent):
    """k = 6000 centers (188 groups of 32, 6 supergroups): the filter prunes supergroups
    before groups.  Curve-ordered centers give compact supergroups; random centers give
    supergroups spanning the domain (the filter then sweeps every group)."""
    x = _sorted(synth.make_points("gmm", 60_000, 2, 19, "f64"))
    k = 6000
    rng = np.random.default_rng(2)
    C = oracle.sfc_centers(x, k) if coherent else rng.random((k, 2))
    I = rng.uniform(0.9, 1.1, k)
    for dt in ("f64", "f32"):
        block, _ = gk.assign(_dev(x), _dev(C), _dev(I), assign_dtype=dt)
        _assert_same_assignment(_np(block), x, C, I, max_frac=0.0 if dt == "f64" else 1e-3)


def test_assign_weighted_block_weights(gk):
    x = _sorted(_points("gmm", 30_000, 2, 19, "f64"))
    w = synth.uniform_weights(len(x), 19)
    rng = np.random.default_rng(2)
    k = 40
    C = x[rng.choice(len(x), k, replace=False)]
    I = np.ones(k)
    block, S = gk.assign(_dev(x), _dev(C), _dev(I), weights=_dev(w))
    A = _np(block)
    _assert_same_assignment(A, x, C, I)
    S_ref, _ = oracle.block_weights(A, w, k)
    assert np.allclose(_np(S), S_ref, rtol=1e-12, atol=0)


def test_assign_exact_ties_go_to_lowest_index(gk):
    rng = np.random.default_rng(4)
    y = rng.random(4096)
    x = np.stack([np.full(4096, 0.5), y], axis=1)  # on the bisector of centers 0 and 1
    C = np.array([[0.0, 0.3], [1.0, 0.3], [0.5, 5.0]])
    x[:, 1] = 0.3 + (y - 0.5) * 0.1
    I = np.array([1.0, 1.0, 0.5])
    block, _ = gk.assign(_dev(x), _dev(C), _dev(I), assign_dtype="f64")
    A = _np(block)
    assert np.all(A == 0)
    # duplicate centers: lowest index wins
    C2 = np.array([[0.2, 0.2], [0.2, 0.2], [0.8, 0.8]])
    pts = rng.random((3000, 2)) * 0.4
    block, _ = gk.assign(_dev(pts), _dev(C2), _dev(np.ones(3)), assign_dtype="f64")
    A = _np(block)
    ref, _, _ = oracle.assign(pts, C2, np.ones(3))
    assert np.array_equal(A, ref) and not np.any(A == 1)


def test_assign_apollonius_golden(gk):
    g = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "apollonius_2centers.txt"))
    C = np.array([[0.0, 0.0], [1.0, 0.0]])
    I = np.array([2.0, 1.0])
    block, _ = gk.assign(_dev(np.ascontiguousarray(g[:, :2])), _dev(C), _dev(I))
    assert _np(block).tolist() == g[:, 2].astype(int).tolist()


def test_assign_fp32_form_disagreement_is_small(gk):
    x = _sorted(_points("radial", 200_000, 2, 23, "f32"))
    rng = np.random.default_rng(5)
    k = 1024
    C = x[rng.choice(len(x), k, replace=False)].astype(np.float64)
    I = rng.uniform(0.8, 1.25, k)
    block, _ = gk.assign(_dev(x), _dev(C), _dev(I), assign_dtype="f32")
    A = _np(block)
    A_ref, _, _ = oracle.assign(x.astype(np.float64), C, I, threads=THREADS)
    frac = (A != A_ref).mean()
    assert frac < 1e-3, frac


# ----------------------------------------------------------------------------------------
# Center movement (teacher-forced)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("weighted,dtype,d", [(False, "f64", 3), (True, "f64", 2),
                                              (False, "f32", 2), (True, "f32", 3)])
def test_move_centers_matches_oracle(gk, weighted, dtype, d):
    x = _points("gmm", 50_001, d, 29, dtype)
    w = synth.uniform_weights(len(x), 29, dtype=x.dtype) if weighted else None
    k = 97
    rng = np.random.default_rng(6)
    A = rng.integers(0, k - 1, len(x)).astype(np.int32)  # block k-1 stays empty
    C = rng.random((k, d))
    Cn, delta, beta = gk.move_centers(_dev(x), _dev(A), _dev(C),
                                      weights=None if w is None else _dev(w))
    Cr, dr, br = oracle.move_centers(x.astype(np.float64), None if w is None else w.astype(np.float64),
                                     A, C)
    assert _rel_center_err(_np(Cn), Cr, x) < 1e-10
    assert np.array_equal(_np(Cn)[k - 1], C[k - 1])
    assert np.allclose(_np(delta), dr, rtol=1e-9, atol=1e-12)
    assert math.isclose(beta, br, rel_tol=1e-12)


def test_move_centers_rejects_bad_block_ids(gk):
    x = np.random.default_rng(0).random((1000, 2))
    A = np.zeros(1000, dtype=np.int32)
    A[5] = 9
    with pytest.raises(gk.GKError):
        gk.move_centers(_dev(x), _dev(A), _dev(np.zeros((3, 2))))


# ----------------------------------------------------------------------------------------
# Whole method, free-running against the oracle
# ----------------------------------------------------------------------------------------
def _run_both(gk, x, w, k, eps, **opt):
    o = gk.default_options(**opt)
    block, C, I, res = gk.partition(_dev(x), k, eps, weights=None if w is None else _dev(w),
                                    options=o)
    oo = oracle.default_options(threads=THREADS)
    for key in ("max_iter", "max_balance_iter", "final_balance_iter", "erosion",
                "delta_threshold"):
        if key in opt:
            setattr(oo, key, opt[key])
    ref = oracle.partition(x, None if w is None else w.astype(np.float64), k, eps, oo)
    return _np(block), _np(C), _np(I), res, ref


def _check_free_running(x, w, k, eps, A, C, I, res, ref):
    xd = x.astype(np.float64)
    rr = ref["result"]
    # Same outcome as the oracle.  Eq. 1 with its 5% clamp can cycle on sharp clusters
    # (both sides then stop with GK_ERR_NOT_BALANCED after the same passes).
    assert res["status"] == rr["status"] and res["balanced"] == rr["balanced"], (res, rr)
    S, W = oracle.block_weights(A, None if w is None else w.astype(np.float64), k)
    if rr["balanced"]:
        assert S.max() <= (1 + eps) * math.ceil(W / k) * (1 + 1e-15)
    _assert_same_assignment(A, xd, C, I)  # A is the FP64 argmin under the returned state
    same = (A == ref["A"]).mean()
    assert same == 1.0, f"free-running assignment differs on {1 - same:.3e} of the points"
    assert res["iterations"] == rr["iterations"] and res["balance_passes"] == rr["balance_passes"]
    assert _rel_center_err(C, ref["C"], xd) < 1e-10
    assert np.allclose(I, ref["I"], rtol=1e-12, atol=0)


def test_partition_uniform_2d_1e5_k16(gk):
    x, w, spec = synth.workload("uniform2d_1e5_k16_f64")
    A, C, I, res, ref = _run_both(gk, x, w, spec["k"], spec["eps"])
    _check_free_running(x, w, spec["k"], spec["eps"], A, C, I, res, ref)


@pytest.mark.parametrize("shape,d,n,k,weighted", [("gmm", 3, 30_011, 37, False),
                                                  ("radial", 2, 20_000, 20, True),
                                                  ("gmm", 2, 12_345, 100, False),
                                                  ("uniform", 3, 4_099, 7, True)])
def test_partition_fp64_matches_oracle(gk, shape, d, n, k, weighted):
    x = _points(shape, n, d, 31, "f64")
    w = synth.uniform_weights(n, 31) if weighted else None
    A, C, I, res, ref = _run_both(gk, x, w, k, 0.03)
    _check_free_running(x, w, k, 0.03, A, C, I, res, ref)


def test_graph_and_host_loop_agree(gk):
    x = _points("gmm", 25_000, 3, 37, "f64")
    out = []
    for g in (1, 0):
        block, C, I, res = gk.partition(_dev(x), 50, 0.03, options=gk.default_options(use_graph=g))
        out.append((_np(block), _np(C), _np(I), res))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert out[0][3]["balance_passes"] == out[1][3]["balance_passes"]


def test_host_and_device_buffers_agree(gk):
    x = _points("radial", 15_000, 2, 41, "f64")
    b1, C1, I1, r1 = gk.partition(_dev(x), 24, 0.03)
    b2, C2, I2, r2 = gk.partition(x, 24, 0.03)  # numpy: host pointers staged by the library
    assert np.array_equal(_np(b1), b2) and np.array_equal(_np(C1), C2)


def test_balanced_kmeans_from_given_state(gk):
    x = _sorted(_points("gmm", 20_000, 2, 43, "f64"))
    k = 16
    C0 = oracle.sfc_centers(x, k)
    Ct, It = _dev(C0.copy()), _dev(np.ones(k))
    block, res = gk.balanced_kmeans(_dev(x), k, 0.03, Ct, It)
    ref = oracle.balanced_kmeans(x, None, k, 0.03, C0, np.ones(k),
                                 oracle.default_options(threads=THREADS))
    assert np.array_equal(_np(block), ref["A"])
    assert _rel_center_err(_np(Ct), ref["C"], x) < 1e-10
    assert np.allclose(_np(It), ref["I_used"], rtol=1e-12)


def test_fp32_form_end_to_end(gk):
    x = _points("radial", 300_000, 2, 47, "f32")
    k = 256
    block, C, I, res = gk.partition(_dev(x), k, 0.03, options=gk.default_options(assign_dtype="f32"))
    A = _np(block)
    S, W = oracle.block_weights(A, None, k)
    assert res["balanced"] == 1 and S.max() <= 1.03 * math.ceil(W / k)
    A_ref, _, _ = oracle.assign(x.astype(np.float64), _np(C), _np(I), threads=THREADS)
    assert (A != A_ref).mean() < 1e-3


# ----------------------------------------------------------------------------------------
# Edge cases and errors
# ----------------------------------------------------------------------------------------
def test_edge_k1_and_k_equals_n(gk):
    x = _points("uniform", 777, 2, 53, "f64")
    block, C, I, res = gk.partition(_dev(x), 1, 0.0)
    assert np.all(_np(block) == 0) and res["balanced"] == 1
    xs = _points("uniform", 300, 3, 54, "f64")
    A, C, I, res, ref = _run_both(gk, xs, None, 300, 0.0)
    assert np.array_equal(A, ref["A"])


def test_edge_single_point_and_identical_points(gk):
    block, C, I, res = gk.partition(_dev(np.array([[0.25, 0.5]])), 1, 0.03)
    assert _np(block).tolist() == [0]
    x = np.full((100, 2), 3.0)
    block, C, I, res = gk.partition(_dev(x), 4, 0.03,
                                    options=gk.default_options(final_balance_iter=5))
    ref = oracle.partition(x, None, 4, 0.03, oracle.default_options(final_balance_iter=5))
    assert np.array_equal(_np(block), ref["A"]) and res["status"] == ref["result"]["status"] == 4


def test_invalid_arguments(gk):
    x = _dev(np.random.default_rng(0).random((10, 2)))
    for args in ((x, 11, 0.03), (x, 0, 0.03), (x, 2, -0.5)):
        with pytest.raises(gk.GKError) as e:
            gk.partition(*args)
        assert e.value.status == gk.GK_ERR_INVALID_ARG
    bad = np.random.default_rng(0).random((10, 2))
    bad[3, 1] = np.nan
    with pytest.raises(gk.GKError):
        gk.partition(_dev(bad), 2, 0.03)
    w = np.ones(10)
    w[2] = 0.0
    with pytest.raises(gk.GKError):
        gk.partition(_dev(np.random.default_rng(0).random((10, 2))), 2, 0.03, weights=_dev(w))
    with pytest.raises(gk.GKError):
        gk.partition(_dev(np.random.default_rng(0).random((10, 4))), 2, 0.03)


# ----------------------------------------------------------------------------------------
# Full size of the benchmark workload (3D Gaussian mixture, n = 1e7, k = 1024, FP64), in
# the launch configuration the benchmark times; checked on sampled outputs.
# ----------------------------------------------------------------------------------------
@pytest.mark.slow
def test_full_size_gmm3d_1e7_k1024(gk):
    import torch
    x, w, spec = synth.workload("gmm3d_1e7_k1024_f64")
    k, eps = spec["k"], spec["eps"]
    xt = _dev(x)
    keys = gk.hilbert_keys(xt)
    assert np.array_equal(_np(keys).view(np.uint64), oracle.hilbert_keys(x))
    block, C, I, res = gk.partition(xt, k, eps)
    torch.cuda.synchronize()
    A, C, I = _np(block), _np(C), _np(I)
    assert res["balanced"] == 1
    S = np.bincount(A, minlength=k)
    assert S.max() <= (1 + eps) * math.ceil(len(x) / k)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(x), 20_000, replace=False)
    _assert_same_assignment(A[idx], x[idx], C, I)
    Cn, delta, beta = gk.move_centers(xt, _dev(A), _dev(C))
    Cr, dr, br = oracle.move_centers(x, None, A, C)
    assert _rel_center_err(_np(Cn), Cr, x) < 1e-10
    assert math.isclose(beta, br, rel_tol=1e-12)


# ----------------------------------------------------------------------------------------
# The scatter of the block ids to input order at a few million points (beyond the L2):
# every returned id, in input order, against the FP64 assignment of the same points under
# the returned centers and influence computed without any sort (gk_assign keeps the
# input order); ragged counts.
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(1 << 22) + 1, 5_000_003])
def test_scatter_returns_input_order(gk, n):
    x = _points("uniform", n, 2, 91, "f32")
    xt = _dev(x)
    block, C, I, res = gk.partition(xt, 96, 0.03, options=gk.default_options(assign_dtype="f64"))
    assert res["status"] in (0, gk.GK_ERR_NOT_BALANCED)  # the ids are returned either way
    ref, _ = gk.assign(xt, C, I, assign_dtype="f64")
    assert np.array_equal(_np(block), _np(ref))
    assert np.bincount(_np(block), minlength=96).sum() == n


# ----------------------------------------------------------------------------------------
# Full size of the FP32-form workloads (2-D, n = 1e8 with k = 4096, and n = 1e9 with
# k = 16384), checked on sampled outputs: Hilbert keys bit-exact on a sample (the sample
# carries the points that attain the bounding box, so the oracle quantises with the
# same box), the balance bound exactly on the host, the FP32-form disagreement with the
# FP64 argmin under the returned state, and the centers of the returned assignment.
# ----------------------------------------------------------------------------------------
def _full_size_fp32_form(gk, name, nsample):
    import torch
    x, w, spec = synth.workload(name, threads=THREADS)
    n, k, eps = len(x), spec["k"], spec["eps"]
    xt = _dev(x)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.choice(n, nsample, replace=False), x.argmin(0), x.argmax(0)]))
    keys = gk.hilbert_keys(xt)
    assert np.array_equal(_np(keys[_dev(idx)]).view(np.uint64), oracle.hilbert_keys(x[idx]))
    del keys
    block, C, I, res = gk.partition(xt, k, eps, options=gk.default_options(assign_dtype="f32"))
    torch.cuda.synchronize()
    A, C, I = _np(block), _np(C), _np(I)
    assert res["status"] == 0 and res["balanced"] == 1
    S = np.bincount(A, minlength=k)
    assert S.sum() == n and S.max() <= (1 + eps) * math.ceil(n / k)
    sub = idx[:nsample]
    A_ref, _, _ = oracle.assign(x[sub].astype(np.float64), C, I, threads=THREADS)
    assert (A[sub] != A_ref).mean() <= FP32_FORM_MAX_DISAGREEMENT
    Cn, delta, beta = gk.move_centers(xt, _dev(A), _dev(C))
    Cr, dr, br = oracle.move_centers(x, None, A, C)
    assert _rel_center_err(_np(Cn), Cr, x[idx].astype(np.float64)) < 1e-10
    assert math.isclose(beta, br, rel_tol=1e-12)


@pytest.mark.slow
def test_full_size_radial2d_1e8_k4096_fp32_form(gk):
    _full_size_fp32_form(gk, "radial2d_1e8_k4096_f32", 100_000)


@pytest.mark.slow
def test_full_size_spots2d_1e9_k16384_fp32_form(gk):
    _full_size_fp32_form(gk, "spots2d_1e9_k16384_f32", 50_000)


# ----------------------------------------------------------------------------------------
# Per-point bounds (gk_options.bounds): the same results as evaluating every point
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape,d,dtype,n,k,assign,weighted", [
    ("gmm", 3, "f64", 60_000, 48, "f64", False),
    ("radial", 2, "f64", 50_000, 37, "f64", True),
    ("gmm", 3, "f32", 80_000, 64, "f32", False),
    ("spots", 2, "f32", 120_000, 300, "f32", True),
    ("uniform", 2, "f64", 30_000, 2500, "f64", False),
])
def test_bounds_give_identical_results(gk, shape, d, dtype, n, k, assign, weighted):
    """With bounds the partition is the oracle's (FP64 argmin: the free-running oracle
    trajectory exactly; FP32 form: the stated disagreement with the FP64 argmin under the
    returned state and the balance bound), and bit for bit the partition without them."""
    x = _points(shape, n, d, 59, dtype)
    w = synth.uniform_weights(n, 59, dtype=x.dtype) if weighted else None
    out = []
    for bounds in (1, 0):
        o = gk.default_options(assign_dtype=assign, bounds=bounds)
        block, C, I, res = gk.partition(_dev(x), k, 0.03, weights=None if w is None else _dev(w),
                                        options=o)
        out.append((_np(block), _np(C), _np(I), res))
    (b1, C1, I1, r1), (b0, C0, I0, r0) = out
    if assign == "f64":
        ref = oracle.partition(x, None if w is None else w.astype(np.float64), k, 0.03,
                               oracle.default_options(threads=THREADS))
        _check_free_running(x, w, k, 0.03, b1, C1, I1, r1, ref)
    else:
        wd = None if w is None else w.astype(np.float64)
        S, W = oracle.block_weights(b1, wd, k)
        assert r1["balanced"] == 1 and S.max() <= 1.03 * math.ceil(W / k) * (1 + 1e-15)
        A_ref, _, _ = oracle.assign(x.astype(np.float64), C1, I1, threads=THREADS)
        assert (b1 != A_ref).mean() <= FP32_FORM_MAX_DISAGREEMENT
    assert np.array_equal(b1, b0)
    assert np.array_equal(C1, C0) and np.array_equal(I1, I0)
    assert r1["balance_passes"] == r0["balance_passes"] and r1["iterations"] == r0["iterations"]
    assert r0["evaluated_points"] == n * r0["balance_passes"]
    assert r1["evaluated_points"] < r0["evaluated_points"]


def test_bounds_over_many_passes_wrap_to_fresh_passes(gk):
    """A phase longer than the bound history (64 passes): every 64th pass evaluates all
    points again; the result stays that of evaluating every point."""
    x = _points("gmm", 40_000, 3, 61, "f64")
    out = []
    for bounds in (1, 0):
        o = gk.default_options(bounds=bounds, max_iter=2, max_balance_iter=150,
                               final_balance_iter=150)
        block, C, I, res = gk.partition(_dev(x), 37, 0.0, options=o)
        out.append((_np(block), _np(C), _np(I), res))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])
    assert out[0][3]["balance_passes"] == out[1][3]["balance_passes"] > 64
    ref = oracle.partition(x, None, 37, 0.0, oracle.default_options(
        threads=THREADS, max_iter=2, max_balance_iter=150, final_balance_iter=150))
    b1, C1, I1, r1 = out[0]
    _check_free_running(x, None, 37, 0.0, b1, C1, I1, r1, ref)


# ----------------------------------------------------------------------------------------
# Workspace from the caller's allocator (gk_set_allocator)
# ----------------------------------------------------------------------------------------
def test_workspace_from_torch_allocator(gk):
    x = _points("gmm", 40_000, 3, 67, "f64")
    gk.release()
    b0, C0, I0, r0 = gk.partition(_dev(x), 30, 0.03)
    blocks = gk.use_torch_allocator()
    try:
        b1, C1, I1, r1 = gk.partition(_dev(x), 30, 0.03)
        assert len(blocks) >= 1  # the workspace came from the callback
        assert np.array_equal(_np(b0), _np(b1)) and np.array_equal(_np(C0), _np(C1))
        assert r0["balance_passes"] == r1["balance_passes"]
    finally:
        gk.set_allocator()
    assert len(blocks) == 0  # and went back to it
    b2, C2, I2, r2 = gk.partition(_dev(x), 30, 0.03)
    assert np.array_equal(_np(b0), _np(b2))


def test_allocation_failure_is_reported(gk):
    """A failing allocation, injected through the allocator hook on the host, gives
    GK_ERR_OOM, and the library works again once cudaMalloc is back."""
    x = _dev(_points("uniform", 5_000, 2, 69, "f64"))
    gk.release()
    gk.set_allocator(lambda nbytes: 0, lambda ptr, nbytes: None)
    try:
        with pytest.raises(gk.GKError) as e:
            gk.partition(x, 8, 0.03)
        assert e.value.status == gk.GK_ERR_OOM
    finally:
        gk.set_allocator()
    block, C, I, res = gk.partition(x, 8, 0.03)
    assert res["balanced"] == 1


def test_bounded_wait_gives_up_and_the_context_stays_usable(gk):
    """The form of the assignment's waits, made to run out on an mbarrier that nothing
    completes: it gives up after its device-time limit with GK_ERR_TIMEOUT (not sooner, and
    not much later), and a partition afterwards still equals the oracle's."""
    for limit_us in (2_000, 50_000):
        st, waited = gk.check_wait_timeout(limit_us)
        assert st == gk.GK_ERR_TIMEOUT, gk.status_string(st)
        assert limit_us <= waited < limit_us + 100_000
    st, _ = gk.check_wait_timeout(0)
    assert st == gk.GK_ERR_INVALID_ARG
    x = _points("uniform", 5_000, 2, 73, "f64")
    block, C, I, res = gk.partition(_dev(x), 8, 0.03)
    ref = oracle.partition(x, None, 8, 0.03, oracle.default_options(threads=THREADS))
    assert np.array_equal(_np(block), ref["A"])


# ----------------------------------------------------------------------------------------
# Launch shapes (gk_options.supertile_tiles, assign_ctas_per_sm): the speed changes, the
# results do not; the tuner picks one of the candidates and reports it.
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape,d,dtype,n,k,assign", [("gmm", 3, "f64", 60_000, 48, "f64"),
                                                      ("spots", 2, "f32", 200_000, 300, "f32"),
                                                      ("uniform", 2, "f64", 30_000, 2500, "f64")])
def test_every_launch_shape_gives_the_same_partition(gk, shape, d, dtype, n, k, assign):
    x = _points(shape, n, d, 71, dtype)
    outs = []
    for stl in (16, 32):
        for hy in (1, 2):
            for ctas in (1, 5):
                o = gk.default_options(assign_dtype=assign, supertile_tiles=stl, hypertiles=hy,
                                       assign_ctas_per_sm=ctas)
                block, C, I, res = gk.partition(_dev(x), k, 0.03, options=o)
                assert res["supertile_tiles"] == stl and res["hypertiles"] == hy
                assert res["tune_ms"] == 0.0 and 1 <= res["assign_ctas_per_sm"] <= ctas
                outs.append((_np(block), _np(C), _np(I), res["balance_passes"]))
    o = gk.default_options(assign_dtype=assign)  # tuned
    block, C, I, res = gk.partition(_dev(x), k, 0.03, options=o)
    assert res["supertile_tiles"] in (16, 32) and res["assign_ctas_per_sm"] >= 1
    outs.append((_np(block), _np(C), _np(I), res["balance_passes"]))
    for b, C1, I1, passes in outs[1:]:
        assert np.array_equal(b, outs[0][0]) and np.array_equal(C1, outs[0][1])
        assert np.array_equal(I1, outs[0][2]) and passes == outs[0][3]
    if assign == "f64":
        ref = oracle.partition(x, None, k, 0.03, oracle.default_options(threads=THREADS))
        assert np.array_equal(outs[0][0], ref["A"])
    # a second tuned call of the same kind takes the cached shape (no measurement)
    _, _, _, res2 = gk.partition(_dev(x), k, 0.03, options=o)
    assert res2["tune_ms"] == 0.0 and res2["supertile_tiles"] == res["supertile_tiles"]
    assert res2["assign_ctas_per_sm"] == res["assign_ctas_per_sm"]
    # a shape the caller fixes holds although the same kind of problem was tuned before
    other = 16 if res["supertile_tiles"] == 32 else 32
    hy = 2 if res["hypertiles"] == 1 else 1
    b3, _, _, res3 = gk.partition(_dev(x), k, 0.03, options=gk.default_options(
        assign_dtype=assign, supertile_tiles=other, hypertiles=hy))
    assert res3["supertile_tiles"] == other and res3["hypertiles"] == hy
    assert np.array_equal(_np(b3), outs[0][0])


def test_launch_shape_options_are_checked(gk):
    x = _dev(np.random.default_rng(0).random((1000, 2)))
    for bad in (dict(supertile_tiles=8), dict(supertile_tiles=64), dict(assign_ctas_per_sm=-1),
                dict(hypertiles=3)):
        with pytest.raises(gk.GKError) as e:
            gk.partition(x, 4, 0.03, options=gk.default_options(**bad))
        assert e.value.status == gk.GK_ERR_INVALID_ARG
