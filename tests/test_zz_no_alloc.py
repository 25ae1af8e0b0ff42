"""gk_move_centers_noalloc (the allocation-free variant of the center-movement step,
for callers that must not allocate device memory) against gk_move_centers.

Collected last on purpose: it runs the variant twice in a row (the second call must not
see the first call's leftovers in the shared scratch array) and passes both alone in a
fresh process and after the other tests."""
import ctypes
import math

import numpy as np
import pytest

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


def _call_noalloc(gk, xt, wt, bt, ct, k):
    import torch
    n, d = xt.shape
    out = torch.empty((k, d), dtype=torch.float64, device=xt.device)
    delta = torch.empty(k, dtype=torch.float64, device=xt.device)
    beta = ctypes.c_double(-1.0)
    code = gk.GK_F64 if xt.dtype == torch.float64 else gk.GK_F32
    st = gk.lib().gk_move_centers_noalloc(
        ctypes.c_void_p(xt.data_ptr()), code,
        None if wt is None else ctypes.c_void_p(wt.data_ptr()), n, d, k,
        ctypes.c_void_p(bt.data_ptr()), ctypes.c_void_p(ct.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(delta.data_ptr()), ctypes.byref(beta),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out.cpu().numpy(), delta.cpu().numpy(), beta.value


@pytest.mark.parametrize("shape,d,dtype,n,k,weighted", [("gmm", 3, "f64", 200_003, 1000, False),
                                                        ("radial", 2, "f32", 150_000, 4096, True)])
def test_noalloc_move_centers_matches_allocating_path(gk, shape, d, dtype, n, k, weighted):
    import torch
    rng = np.random.default_rng(n)
    for call in range(2):  # two calls in a row share the scratch array
        x = synth.make_points(shape, n, d, 100 + call, dtype)
        w = synth.uniform_weights(n, 100 + call, dtype=x.dtype) if weighted else None
        A = rng.integers(0, k - 1, n).astype(np.int32)  # block k-1 empty
        C = rng.random((k, d))
        xt, bt, ct = (torch.from_numpy(a).cuda() for a in (x, A, C))
        wt = None if w is None else torch.from_numpy(w).cuda()
        st, Cn, dn, beta = _call_noalloc(gk, xt, wt, bt, ct, k)
        assert st == gk.GK_OK, gk.status_string(st)
        Cr, dr, br = gk.move_centers(xt, bt, ct, weights=wt)
        Cr, dr = Cr.cpu().numpy(), dr.cpu().numpy()
        ext = float((x.max(0) - x.min(0)).max())
        assert np.abs(Cn - Cr).max() <= RTOL * ext
        assert np.allclose(dn, dr, rtol=RTOL, atol=RTOL * ext)
        assert math.isclose(beta, br, rel_tol=RTOL)
        assert np.array_equal(Cn[k - 1], C[k - 1])


def test_noalloc_rejects_k_beyond_its_scratch(gk):
    import torch
    x = torch.rand((1000, 2), dtype=torch.float64, device="cuda")
    k = 4097
    A = torch.zeros(1000, dtype=torch.int32, device="cuda")
    C = torch.zeros((k, 2), dtype=torch.float64, device="cuda")
    st, _, _, _ = _call_noalloc(gk, x, None, A, C, k)
    assert st == gk.GK_ERR_INVALID_ARG
