"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/gk.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgk():
    from paper_1805_01208_gb300.nvcc_build import build
    path = build()
    return ctypes.CDLL(path)


def _declared():
    text = open(os.path.join(ROOT, "include", "gk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gk_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("gk_hilbert_keys", "gk_sfc_init", "gk_balanced_kmeans", "gk_partition",
                 "gk_assign", "gk_move_centers", "gk_release", "gk_default_options",
                 "gk_status_string", "gk_abi_version", "gk_partition_batched",
                 "gk_partition_sampled", "gk_partition_quality", "gk_block_diameter",
                 "gk_set_allocator", "gk_check_wait_timeout"):
        assert want in names


def test_every_declared_symbol_is_exported(libgk):
    missing = [name for name in _declared() if not hasattr(libgk, name)]
    assert not missing, missing


def test_host_only_helpers(libgk):
    import paper_1805_01208_gb300 as gk
    assert gk.lib().gk_abi_version() == 3
    o = gk.default_options()
    assert (o.max_iter, o.max_balance_iter, o.final_balance_iter, o.erosion) == (50, 50, 500, 1)
    assert o.delta_threshold < 0 and o.assign_dtype == gk.GK_F64 and o.use_graph == 1
    assert o.bounds == 0 and o.supertile_tiles == 0 and o.assign_ctas_per_sm == 0
    assert o.hypertiles == 0
    assert gk.status_string(gk.GK_ERR_NOT_BALANCED) == "GK_ERR_NOT_BALANCED"
    assert gk.status_string(99) == "GK_UNKNOWN_STATUS"
    for bad in (0, -5, 10_000_001):  # the wait limit is checked before any launch
        assert gk.check_wait_timeout(bad)[0] == gk.GK_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    import paper_1805_01208_gb300 as gk
    # gk_options: 4 int32, double, 4 int32, 3 int32 shapes, 1 int32 reserved
    assert ctypes.sizeof(gk.Options) == 4 * 4 + 8 + 4 * 4 + 3 * 4 + 1 * 4
    assert ctypes.sizeof(gk.Result) == (6 * 4 + 4 * 8 + 2 * 8 + 3 * 8 + 4 * 8 + 4 * 8 + 8 + 8 + 8
                                        + 4 * 4 + 8)
    # gk_instance: 2 pointers, int64, 4 int32, double, 3 pointers
    assert ctypes.sizeof(gk.Instance) == 2 * 8 + 8 + 4 * 4 + 8 + 3 * 8


def test_batched_rejects_empty_batch_before_any_launch(libgk):
    import paper_1805_01208_gb300 as gk
    L = gk.lib()
    assert L.gk_partition_batched(None, 0, None, None, None) == gk.GK_ERR_INVALID_ARG
    inst = (gk.Instance * 1)()
    assert L.gk_partition_batched(ctypes.cast(inst, ctypes.c_void_p), 0, None, None, None) == \
        gk.GK_ERR_INVALID_ARG


def test_sampled_rejects_missing_order_before_any_launch(libgk):
    import paper_1805_01208_gb300 as gk
    L = gk.lib()
    x = np.zeros((4, 2))
    blk = np.zeros(4, dtype=np.int32)
    st = L.gk_partition_sampled(x.ctypes.data_as(ctypes.c_void_p), gk.GK_F64, None, 4, 2, 2, 0.03,
                                None, 0, None, blk.ctypes.data_as(ctypes.c_void_p), None, None,
                                None, None)
    assert st == gk.GK_ERR_INVALID_ARG


def test_quality_rejects_bad_arguments_before_any_launch(libgk):
    import paper_1805_01208_gb300 as gk
    L = gk.lib()
    assert ctypes.sizeof(gk.Quality) == 40
    rp = np.zeros(3, dtype=np.int64)
    blk = np.zeros(2, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.gk_partition_quality(None, None, 2, 0, P(blk), 1, None, None, None, None) == \
        gk.GK_ERR_INVALID_ARG
    assert L.gk_partition_quality(P(rp), None, 2, 0, P(blk), 0, None, None, None, None) == \
        gk.GK_ERR_INVALID_ARG
    assert L.gk_partition_quality(P(rp), None, 2, 4, P(blk), 1, None, None, None, None) == \
        gk.GK_ERR_INVALID_ARG


def test_diameter_rejects_bad_arguments_before_any_launch(libgk):
    import paper_1805_01208_gb300 as gk
    L = gk.lib()
    assert ctypes.sizeof(gk.Diameter) == 32
    rp = np.zeros(3, dtype=np.int64)
    blk = np.zeros(2, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for args in ((None, None, 2, 0, P(blk), 1, 3), (P(rp), None, 2, 0, P(blk), 0, 3),
                 (P(rp), None, 2, 4, P(blk), 1, 3), (P(rp), None, 2, 0, P(blk), 1, 0),
                 (P(rp), None, 2, 0, P(blk), 1, 65), (P(rp), None, 0, 0, P(blk), 1, 3)):
        assert L.gk_block_diameter(*args, None, None, None) == gk.GK_ERR_INVALID_ARG


def test_set_allocator_needs_both_callbacks(libgk):
    import paper_1805_01208_gb300 as gk
    L = gk.lib()
    alloc = gk._ALLOC_FN(lambda nbytes, ctx: None)
    assert L.gk_set_allocator(ctypes.cast(alloc, ctypes.c_void_p), None, None) == gk.GK_ERR_INVALID_ARG
    assert L.gk_set_allocator(None, None, None) == gk.GK_OK
    with pytest.raises(ValueError):
        gk.set_allocator(alloc=lambda n: 0)


def test_library_is_built_for_sm103a(libgk):
    from paper_1805_01208_gb300.nvcc_build import ARCH
    assert "arch=compute_103a,code=sm_103a" in ARCH


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1805_01208_gb300 as gk
    monkeypatch.setattr(gk, "_lib", None)
    monkeypatch.setattr(gk, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gk.lib()
