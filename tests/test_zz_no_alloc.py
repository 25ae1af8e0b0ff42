"""gk_move_centers_noalloc, the center-movement step for callers that must not allocate
device memory while they run (their device memory belongs to their own pool or
allocator, or their loop cannot take the device synchronisation that a cudaMalloc or
cudaFree may cause), against gk_move_centers and against the FP64 oracle.

Collected last on purpose: it runs the variant twice in a row (the second call must not
see the first call's leftovers in the shared scratch array) and passes both alone in a
fresh process and after the other tests."""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_01208_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-10  # center tolerance of the parity tests (relative to the box extent)


@pytest.fixture(scope="module")
def gk():
    import torch
    import paper_1805_01208_gb300 as gk
    gk.build()
    torch.cuda.set_device(0)
    return gk


def _call_noalloc(gk, xt, wt, bt, ct, k, beta_dev=None):
    """One call through the C ABI.  beta goes to a host double, or to beta_dev (a CUDA
    tensor of one FP64) when given."""
    import torch
    n, d = xt.shape
    out = torch.empty((k, d), dtype=torch.float64, device=xt.device)
    delta = torch.empty(k, dtype=torch.float64, device=xt.device)
    beta = ctypes.c_double(-1.0)
    bptr = ctypes.byref(beta) if beta_dev is None else ctypes.c_void_p(beta_dev.data_ptr())
    code = gk.GK_F64 if xt.dtype == torch.float64 else gk.GK_F32
    st = gk.lib().gk_move_centers_noalloc(
        ctypes.c_void_p(xt.data_ptr()), code,
        None if wt is None else ctypes.c_void_p(wt.data_ptr()), n, d, k,
        ctypes.c_void_p(bt.data_ptr()), ctypes.c_void_p(ct.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(delta.data_ptr()), bptr,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    b = beta.value if beta_dev is None else float(beta_dev.cpu()[0])
    return st, out.cpu().numpy(), delta.cpu().numpy(), b


@pytest.mark.parametrize("shape,d,dtype,n,k,weighted", [("gmm", 3, "f64", 200_003, 1000, False),
                                                        ("radial", 2, "f32", 150_000, 4096, True)])
def test_noalloc_move_centers_matches_allocating_path_and_oracle(gk, shape, d, dtype, n, k, weighted):
    import torch
    rng = np.random.default_rng(n)
    for call in range(2):  # two calls in a row share the scratch array
        x = synth.make_points(shape, n, d, 100 + call, dtype)
        w = synth.uniform_weights(n, 100 + call, dtype=x.dtype) if weighted else None
        A = rng.integers(0, k - 1, n).astype(np.int32)  # block k-1 empty
        C = rng.random((k, d))
        xt, bt, ct = (torch.from_numpy(a).cuda() for a in (x, A, C))
        wt = None if w is None else torch.from_numpy(w).cuda()
        # beta to host memory on the first call, to device memory on the second
        bdev = None if call == 0 else torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st, Cn, dn, beta = _call_noalloc(gk, xt, wt, bt, ct, k, beta_dev=bdev)
        assert st == gk.GK_OK, gk.status_string(st)
        ext = float((x.max(0) - x.min(0)).max())
        # the FP64 oracle (weighted means of the points, bounding-box diagonals)
        Co, do, bo = oracle.move_centers(x.astype(np.float64),
                                         None if w is None else w.astype(np.float64), A, C)
        assert np.abs(Cn - Co).max() <= RTOL * ext
        assert np.allclose(dn, do, rtol=RTOL, atol=RTOL * ext)
        assert math.isclose(beta, bo, rel_tol=RTOL)
        # the allocating entry point
        Cr, dr, br = gk.move_centers(xt, bt, ct, weights=wt)
        Cr, dr = Cr.cpu().numpy(), dr.cpu().numpy()
        assert np.abs(Cn - Cr).max() <= RTOL * ext
        assert np.allclose(dn, dr, rtol=RTOL, atol=RTOL * ext)
        assert math.isclose(beta, br, rel_tol=RTOL)
        assert np.array_equal(Cn[k - 1], C[k - 1])


def test_noalloc_allocates_nothing(gk):
    """The property the entry point exists for: no call of the library's workspace
    allocator, no growth of PyTorch's pool and no change of the device's free memory
    across a call (after a first call, which may load the kernels)."""
    import torch
    n, d, k = 100_000, 2, 512
    x = synth.make_points("uniform", n, d, 5, "f64")
    A = np.random.default_rng(5).integers(0, k, n).astype(np.int32)
    C = np.random.default_rng(6).random((k, d))
    xt, bt, ct = (torch.from_numpy(a).cuda() for a in (x, A, C))
    calls = {"alloc": 0, "free": 0}
    blocks = {}

    def alloc(nbytes):
        calls["alloc"] += 1
        t = torch.empty(nbytes + 255, dtype=torch.uint8, device="cuda")
        ptr = (t.data_ptr() + 255) & ~255
        blocks[ptr] = t
        return ptr

    def free(ptr, nbytes):
        calls["free"] += 1
        blocks.pop(ptr, None)

    gk.set_allocator(alloc, free)
    try:
        st, C1, _, b1 = _call_noalloc(gk, xt, None, bt, ct, k)  # first call: set-up
        assert st == gk.GK_OK
        out = torch.empty((k, d), dtype=torch.float64, device="cuda")
        delta = torch.empty(k, dtype=torch.float64, device="cuda")
        beta = ctypes.c_double(0.0)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        torch_bytes0 = torch.cuda.memory_reserved()
        calls0 = dict(calls)
        st = gk.lib().gk_move_centers_noalloc(
            ctypes.c_void_p(xt.data_ptr()), gk.GK_F64, None, n, d, k,
            ctypes.c_void_p(bt.data_ptr()), ctypes.c_void_p(ct.data_ptr()),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(delta.data_ptr()),
            ctypes.byref(beta), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert st == gk.GK_OK
        assert calls == calls0 == {"alloc": 0, "free": 0}
        assert torch.cuda.memory_reserved() == torch_bytes0
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        assert np.array_equal(out.cpu().numpy(), C1) and beta.value == b1
    finally:
        gk.set_allocator()


def test_noalloc_rejects_k_beyond_its_scratch(gk):
    import torch
    x = torch.rand((1000, 2), dtype=torch.float64, device="cuda")
    k = 4097
    A = torch.zeros(1000, dtype=torch.int32, device="cuda")
    C = torch.zeros((k, 2), dtype=torch.float64, device="cuda")
    st, _, _, _ = _call_noalloc(gk, x, None, A, C, k)
    assert st == gk.GK_ERR_INVALID_ARG


def test_noalloc_rejects_bad_input_and_stays_usable(gk):
    """Block ids outside [0, k), a NaN coordinate and a negative weight are found on the
    device and reported; a good call right after still gives the right result."""
    import torch
    n, d, k = 5000, 2, 64
    rng = np.random.default_rng(9)
    x = rng.random((n, d))
    w = rng.uniform(1, 10, n)
    A = rng.integers(0, k, n).astype(np.int32)
    C = rng.random((k, d))

    def run(xa, wa, Aa):
        xt, bt, ct = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (xa, Aa, C))
        wt = None if wa is None else torch.from_numpy(wa).cuda()
        return _call_noalloc(gk, xt, wt, bt, ct, k)

    bad_id = A.copy()
    bad_id[n // 2] = k
    assert run(x, w, bad_id)[0] == gk.GK_ERR_INVALID_ARG
    neg_id = A.copy()
    neg_id[7] = -1
    assert run(x, None, neg_id)[0] == gk.GK_ERR_INVALID_ARG
    nan_x = x.copy()
    nan_x[123, 1] = np.nan
    assert run(nan_x, w, A)[0] == gk.GK_ERR_INVALID_ARG
    neg_w = w.copy()
    neg_w[4321] = -2.0
    assert run(x, neg_w, A)[0] == gk.GK_ERR_INVALID_ARG
    st, Cn, _, beta = run(x, w, A)
    assert st == gk.GK_OK
    Co, _, bo = oracle.move_centers(x, w, A, C)
    assert np.abs(Cn - Co).max() <= RTOL and math.isclose(beta, bo, rel_tol=RTOL)
