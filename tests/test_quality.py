"""Partition quality measures of Section 5 (edge cut, communication volume): the numpy
oracle pinned by hand-counted graphs, closed forms on lattice meshes and brute force
(CPU), and gk_partition_quality against it (GPU)."""
import math

import numpy as np
import pytest

from oracle import quality as oq
from paper_1805_01208_gb300 import synth


def _csr(n, edges):
    """Symmetric CSR of an undirected edge list."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in adj])
    col = np.array([u for r in adj for u in r], dtype=np.int32)
    return row_ptr, col


# ----------------------------------------------------------------------------------------
# Oracle pins (CPU)
# ----------------------------------------------------------------------------------------
def test_path_graph_by_hand():
    rp, col = _csr(4, [(0, 1), (1, 2), (2, 3)])
    q = oq.quality(rp, col, np.array([0, 0, 1, 1]), 2)
    assert q["edge_cut"] == 1 and list(q["ext"]) == [1, 1] and list(q["comm"]) == [1, 1]
    assert q["total_comm_volume"] == 2 and q["max_comm_volume"] == 1


def test_star_graph_by_hand():
    # center 0 in block 0; leaves in blocks 1, 2, 2, 3
    rp, col = _csr(5, [(0, 1), (0, 2), (0, 3), (0, 4)])
    q = oq.quality(rp, col, np.array([0, 1, 2, 2, 3]), 4)
    assert q["edge_cut"] == 4
    assert list(q["ext"]) == [4, 1, 2, 1]
    assert list(q["comm"]) == [3, 1, 2, 1]  # the center sees three other blocks
    assert q["total_comm_volume"] == 7 and q["max_comm_volume"] == 3


def test_self_loops_and_one_block():
    rp, col = _csr(3, [(0, 0), (0, 1), (1, 2)])
    q = oq.quality(rp, col, np.array([0, 0, 0]), 1)
    assert q["edge_cut"] == 0 and q["total_comm_volume"] == 0


def _slabs(x, axis_cells, k, grading=2.0):
    """Block = slab of the lattice index along axis 0 (recovered from the graded, jittered
    coordinate: the jitter keeps every vertex inside (i + 1/4, i + 3/4) / nx)."""
    u = x[:, 0] ** (1.0 / grading) * axis_cells
    i = np.floor(u).astype(np.int64)
    return (i * k // axis_cells).astype(np.int32)


def test_lattice_slab_closed_forms_3d():
    nx, ny, nz, k = 12, 5, 4, 3  # slabs of 4 layers
    x, rp, col = synth.lattice_mesh((nx, ny, nz), 3)
    block = _slabs(x, nx, k)
    assert np.bincount(block).tolist() == [4 * ny * nz] * 3
    q = oq.quality(rp, col, block, k)
    assert q["edge_cut"] == (k - 1) * ny * nz
    assert list(q["comm"]) == [ny * nz, 2 * ny * nz, ny * nz]
    assert q["total_comm_volume"] == 2 * (k - 1) * ny * nz
    assert rp[-1] == 2 * (3 * nx * ny * nz - ny * nz - nx * nz - nx * ny)  # 6-neighbour lattice


def test_lattice_half_closed_forms_2d():
    nx, ny = 10, 7
    x, rp, col = synth.lattice_mesh((nx, ny), 4)
    block = _slabs(x, nx, 2)
    q = oq.quality(rp, col, block, 2)
    assert q["edge_cut"] == 2 * ny - 1  # ny lattice edges and ny - 1 diagonals cross
    assert list(q["comm"]) == [ny, ny]
    edges = (nx - 1) * ny + nx * (ny - 1) + (nx - 1) * (ny - 1)
    assert rp[-1] == 2 * edges


def test_random_graph_against_brute_force():
    rng = np.random.default_rng(7)
    n, k = 60, 5
    edges = {tuple(sorted(e)) for e in rng.integers(0, n, (150, 2)).tolist() if e[0] != e[1]}
    rp, col = _csr(n, sorted(edges))
    block = rng.integers(0, k, n)
    q = oq.quality(rp, col, block, k)
    ext = [0] * k
    comm = [0] * k
    for v in range(n):
        nb = [u for a, u in edges if a == v] + [a for a, u in edges if u == v]
        ext[block[v]] += sum(1 for u in nb if block[u] != block[v])
        comm[block[v]] += len({block[u] for u in nb} - {block[v]})
    assert list(q["ext"]) == ext and list(q["comm"]) == comm
    assert q["edge_cut"] == sum(1 for a, b in edges if block[a] != block[b])


# ----------------------------------------------------------------------------------------
# GPU against the oracle
# ----------------------------------------------------------------------------------------
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


def _check(gk, rp, col, block, k, on_device=True):
    args = (_dev(rp), _dev(col), _dev(block)) if on_device else (rp, col, block)
    q, ext, comm = gk.partition_quality(*args, k)
    ref = oq.quality(rp, col, block, k)
    assert np.array_equal(_np(ext), ref["ext"]) and np.array_equal(_np(comm), ref["comm"])
    for key in ("edge_cut", "total_comm_volume", "max_comm_volume", "max_ext"):
        assert q[key] == ref[key], key
    v = np.repeat(np.arange(len(block)), np.diff(rp))
    assert q["boundary_vertices"] == len(np.unique(v[(block[v] != block[col]) & (v != col)]))
    return q


@pytest.mark.gpu
@pytest.mark.parametrize("on_device", [True, False])
def test_gpu_quality_hand_graphs(gk, on_device):
    rp, col = _csr(5, [(0, 1), (0, 2), (0, 3), (0, 4)])
    _check(gk, rp, col, np.array([0, 1, 2, 2, 3], dtype=np.int32), 4, on_device)
    rp, col = _csr(3, [(0, 0), (0, 1), (1, 2)])
    _check(gk, rp, col, np.zeros(3, dtype=np.int32), 1, on_device)


@pytest.mark.gpu
@pytest.mark.parametrize("dims,k", [((40, 30, 20), 64), ((300, 200), 37)])
def test_gpu_quality_of_a_partition_on_lattice_meshes(gk, dims, k):
    x, rp, col = synth.lattice_mesh(dims, 5)
    block, C, I, res = gk.partition(_dev(x), k, 0.03)
    _check(gk, rp, col, _np(block).astype(np.int32), k)


@pytest.mark.gpu
def test_gpu_quality_random_graph_and_random_blocks(gk):
    rng = np.random.default_rng(9)
    n, k = 5000, 77
    e = rng.integers(0, n, (40_000, 2))
    rp, col = _csr(n, [tuple(r) for r in e.tolist()])  # parallel edges and self-loops too
    _check(gk, rp, col, rng.integers(0, k, n).astype(np.int32), k)


@pytest.mark.gpu
def test_gpu_quality_rejects_malformed_input(gk):
    rp, col = _csr(4, [(0, 1), (1, 2), (2, 3)])
    for bad_block in ([0, 0, 2, 1], [0, -1, 1, 1]):
        with pytest.raises(gk.GKError):
            gk.partition_quality(_dev(rp), _dev(col), _dev(np.array(bad_block, dtype=np.int32)), 2)
    bad_col = col.copy()
    bad_col[2] = 9
    with pytest.raises(gk.GKError):
        gk.partition_quality(_dev(rp), _dev(bad_col), _dev(np.zeros(4, dtype=np.int32)), 1)
    bad_rp = rp.copy()
    bad_rp[2] = 100
    with pytest.raises(gk.GKError):
        gk.partition_quality(_dev(bad_rp), _dev(col), _dev(np.zeros(4, dtype=np.int32)), 1)
    q = _check(gk, rp, col, np.array([0, 0, 1, 1], dtype=np.int32), 2)  # still usable
    assert q["edge_cut"] == 1


@pytest.mark.gpu
@pytest.mark.slow
def test_gpu_quality_full_size_mesh(gk):
    """A 3-D graded mesh of 8e6 vertices partitioned into 1024 blocks: the GPU measures
    equal the oracle's, and balanced k-means cuts fewer edges than the curve split."""
    x, rp, col = synth.lattice_mesh((200, 200, 200), 6)
    k = 1024
    block, C, I, res = gk.partition(_dev(x), k, 0.03)
    q = _check(gk, rp, col, _np(block).astype(np.int32), k)
    perm, _ = gk.sfc_init(_dev(x), k)
    n = len(x)
    sfc = np.empty(n, dtype=np.int32)
    sfc[_np(perm)] = (np.arange(n, dtype=np.int64) * k // n).astype(np.int32)
    qs = _check(gk, rp, col, sfc, k)
    assert q["edge_cut"] < qs["edge_cut"]
