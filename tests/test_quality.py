"""Partition quality measures of Section 5 (edge cut, communication volume, block
diameter): the numpy oracle pinned by hand-counted graphs, closed forms on lattice meshes,
trees and brute force (CPU), and the GPU entry points against it (GPU)."""
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


def _tree(n, rng):
    """A random tree on n vertices (vertex i > 0 hangs below a random earlier vertex)."""
    return [(int(rng.integers(0, i)), i) for i in range(1, n)]


def test_diameter_hand_graphs():
    # cycle of 8: block 0 is the path 0-1-2-3-4-5 (its own diameter 5 although 5 and 0
    # are 3 apart through block 1), block 1 = {6, 7}, block 2 empty
    rp, col = _csr(8, [(i, (i + 1) % 8) for i in range(8)])
    block = np.array([0, 0, 0, 0, 0, 0, 1, 1])
    for f in (oq.block_diameter_exact, oq.block_diameter_sweeps):
        assert f(rp, col, block, 3).tolist() == [5, 1, 0]
    # star: diameter 2; a block of two separate vertices: not connected
    rp, col = _csr(6, [(0, 1), (0, 2), (0, 3), (4, 4)])
    block = np.array([0, 0, 0, 0, 1, 1])
    for f in (oq.block_diameter_exact, oq.block_diameter_sweeps):
        assert f(rp, col, block, 2).tolist() == [2, -1]
    s = oq.diameter_summary([2, -1], [4, 2])
    assert s == {"max_diameter": 2, "disconnected_blocks": 1, "harmonic_mean": 2 / 0.5}
    assert oq.diameter_summary([0, 3, 6], [1, 4, 7])["harmonic_mean"] == 2 / (1 / 3 + 1 / 6)
    assert oq.diameter_summary([-1], [2])["harmonic_mean"] == math.inf
    assert oq.diameter_summary([0, 0], [1, 0])["harmonic_mean"] == 0.0


def test_diameter_sweep_starts_follow_the_reading():
    """The first sweep starts at the block's smallest vertex index, a later one at the
    smallest index among the vertices the previous sweep reached last."""
    # path 1-0-2-3-4: from vertex 0 the eccentricity is 3 (from vertex 4 it would be 4)
    rp, col = _csr(5, [(1, 0), (0, 2), (2, 3), (3, 4)])
    assert oq.block_diameter_sweeps(rp, col, np.zeros(5, dtype=np.int64), 1, 1).tolist() == [3]
    # edges 0-1, 0-3, 1-2, 1-4, 2-3: the sweep from 0 reaches {2, 4} last (distance 2); the
    # sweep from 2 has eccentricity 2 and reaches {0, 4} last, the one from 0 again 2.  (From
    # 4 the second sweep would find 3, the exact diameter, via 4-1-0-3.)
    rp, col = _csr(5, [(0, 1), (0, 3), (1, 2), (1, 4), (2, 3)])
    block = np.zeros(5, dtype=np.int64)
    for sweeps in (2, 3):
        assert oq.block_diameter_sweeps(rp, col, block, 1, sweeps).tolist() == [2]
    assert oq.block_diameter_exact(rp, col, block, 1).tolist() == [3]


def test_diameter_sweeps_exact_on_trees():
    """On a tree a sweep from any vertex ends at an end of a longest path, so the second
    sweep already gives the exact diameter."""
    rng = np.random.default_rng(12)
    for n in (2, 7, 40, 300):
        rp, col = _csr(n, _tree(n, rng))
        block = np.zeros(n, dtype=np.int64)
        exact = oq.block_diameter_exact(rp, col, block, 1)
        assert oq.block_diameter_sweeps(rp, col, block, 1, sweeps=2).tolist() == exact.tolist()
        assert oq.block_diameter_sweeps(rp, col, block, 1).tolist() == exact.tolist()
    # a forest, one tree per block, vertices shuffled
    sizes = [5, 30, 1, 12]
    edges, off = [], 0
    for m in sizes:
        edges += [(a + off, b + off) for a, b in _tree(m, rng)]
        off += m
    perm = rng.permutation(off)
    rp, col = _csr(off, [(int(perm[a]), int(perm[b])) for a, b in edges])
    block = np.empty(off, dtype=np.int64)
    block[perm] = np.repeat(np.arange(len(sizes)), sizes)
    assert oq.block_diameter_sweeps(rp, col, block, 4).tolist() == \
        oq.block_diameter_exact(rp, col, block, 4).tolist()


def test_diameter_sweeps_within_factor_two():
    rng = np.random.default_rng(13)
    for trial in range(6):
        n, k = 80, 4
        e = {tuple(sorted(p)) for p in rng.integers(0, n, (140, 2)).tolist() if p[0] != p[1]}
        rp, col = _csr(n, sorted(e))
        block = rng.integers(0, k, n)
        exact = oq.block_diameter_exact(rp, col, block, k)
        lb1 = oq.block_diameter_sweeps(rp, col, block, k, sweeps=1)
        lb = oq.block_diameter_sweeps(rp, col, block, k)
        assert np.array_equal(exact < 0, lb < 0) and np.array_equal(lb1 < 0, lb < 0)
        c = exact >= 0
        assert np.all(lb[c] <= exact[c]) and np.all(2 * lb[c] >= exact[c])
        assert np.all(lb1[c] <= lb[c])


def test_diameter_lattice_closed_forms():
    # 3-D, 6 neighbours: a box block of a x b x c vertices has diameter
    # (a - 1) + (b - 1) + (c - 1); two sweeps reach it (the first ends at a corner)
    nx, ny, nz, k = 12, 5, 4, 3
    x, rp, col = synth.lattice_mesh((nx, ny, nz), 3)
    block = _slabs(x, nx, k)
    want = [3 + (ny - 1) + (nz - 1)] * k
    assert oq.block_diameter_exact(rp, col, block, k).tolist() == want
    assert oq.block_diameter_sweeps(rp, col, block, k).tolist() == want
    # 2-D triangulated grid ((+1, +1) diagonals): a box of a x b vertices has diameter
    # (a - 1) + (b - 1), between the corners that no diagonal shortens
    nx, ny = 10, 7
    x, rp, col = synth.lattice_mesh((nx, ny), 4)
    block = _slabs(x, nx, 2)
    assert oq.block_diameter_exact(rp, col, block, 2).tolist() == [4 + ny - 1] * 2
    lb = oq.block_diameter_sweeps(rp, col, block, 2)
    assert np.all(lb <= 4 + ny - 1) and np.all(2 * lb >= 4 + ny - 1)


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


def _check_diam(gk, rp, col, block, k, sweeps=3, on_device=True):
    args = (_dev(rp), _dev(col), _dev(block)) if on_device else (rp, col, block)
    q, diam = gk.block_diameter(*args, k, sweeps)
    ref = oq.block_diameter_sweeps(rp, col, block, k, sweeps)
    assert np.array_equal(_np(diam), ref)
    s = oq.diameter_summary(ref, np.bincount(block, minlength=k))
    assert q["max_diameter"] == s["max_diameter"]
    assert q["disconnected_blocks"] == s["disconnected_blocks"]
    hm = s["harmonic_mean"]
    if hm in (0.0, math.inf):
        assert q["harmonic_mean"] == hm
    else:  # a sum of k reciprocals in another order
        assert math.isclose(q["harmonic_mean"], hm, rel_tol=1e-12)
    assert q["bfs_levels"] >= sweeps * max(s["max_diameter"], 0) // 2
    return q, _np(diam)


@pytest.mark.gpu
@pytest.mark.parametrize("on_device", [True, False])
def test_gpu_diameter_hand_graphs(gk, on_device):
    rp, col = _csr(8, [(i, (i + 1) % 8) for i in range(8)])
    q, d = _check_diam(gk, rp, col, np.array([0, 0, 0, 0, 0, 0, 1, 1], dtype=np.int32), 3,
                       on_device=on_device)
    assert d.tolist() == [5, 1, 0]
    rp, col = _csr(6, [(0, 1), (0, 2), (0, 3), (4, 4)])
    q, d = _check_diam(gk, rp, col, np.array([0, 0, 0, 0, 1, 1], dtype=np.int32), 2,
                       on_device=on_device)
    assert d.tolist() == [2, -1] and q["disconnected_blocks"] == 1
    q, d = _check_diam(gk, rp, col, np.zeros(6, dtype=np.int32), 1, sweeps=1, on_device=on_device)
    assert d.tolist() == [-1] and q["harmonic_mean"] == math.inf


@pytest.mark.gpu
def test_gpu_diameter_exact_on_a_forest(gk):
    rng = np.random.default_rng(21)
    sizes = [1, 2, 50, 700, 3000, 9]
    edges, off = [], 0
    for m in sizes:
        edges += [(a + off, b + off) for a, b in _tree(m, rng)]
        off += m
    perm = rng.permutation(off)
    rp, col = _csr(off, [(int(perm[a]), int(perm[b])) for a, b in edges])
    block = np.empty(off, dtype=np.int32)
    block[perm] = np.repeat(np.arange(len(sizes)), sizes)
    q, d = _check_diam(gk, rp, col, block, len(sizes), sweeps=2)
    assert d.tolist() == oq.block_diameter_exact(rp, col, block, len(sizes)).tolist()


@pytest.mark.gpu
@pytest.mark.parametrize("dims,k", [((40, 30, 20), 64), ((300, 200), 37)])
@pytest.mark.parametrize("sweeps", [1, 3])
def test_gpu_diameter_of_a_partition_on_lattice_meshes(gk, dims, k, sweeps):
    x, rp, col = synth.lattice_mesh(dims, 5)
    block, C, I, res = gk.partition(_dev(x), k, 0.03)
    _check_diam(gk, rp, col, _np(block).astype(np.int32), k, sweeps)


@pytest.mark.gpu
def test_gpu_diameter_lattice_slabs_closed_form(gk):
    nx, ny, nz, k = 24, 9, 7, 6
    x, rp, col = synth.lattice_mesh((nx, ny, nz), 8)
    block = _slabs(x, nx, k)
    q, d = _check_diam(gk, rp, col, block, k)
    assert d.tolist() == [3 + (ny - 1) + (nz - 1)] * k


@pytest.mark.gpu
def test_gpu_diameter_random_graph_and_random_blocks(gk):
    rng = np.random.default_rng(10)
    n, k = 5000, 40
    e = rng.integers(0, n, (12_000, 2))
    rp, col = _csr(n, [tuple(r) for r in e.tolist()])  # parallel edges and self-loops too
    block = rng.integers(0, k, n).astype(np.int32)
    q, d = _check_diam(gk, rp, col, block, k + 3)  # three empty blocks
    assert q["disconnected_blocks"] > 0 and d[-3:].tolist() == [0, 0, 0]


@pytest.mark.gpu
def test_gpu_diameter_hubs_overflow_the_level_buffer(gk):
    """Two trees whose hubs reach 20,000 and 3,000 leaves in one level: one CTA round finds
    more new vertices than its shared buffer holds, so the rest are appended one by one.
    On trees two sweeps give the exact diameter: 12 (leaf, hub, leaf 1 and a path of ten
    hanging from it) and 2 (a star)."""
    rng = np.random.default_rng(3)
    leaves = 20_000
    edges = [(0, i) for i in range(1, leaves + 1)]
    prev = 1
    for v in range(leaves + 1, leaves + 11):
        edges.append((prev, v))
        prev = v
    h = leaves + 11
    edges += [(h, h + i) for i in range(1, 3001)] + [(0, h)]  # the hub-hub edge is cut
    n = h + 3001
    perm = rng.permutation(n)
    rp, col = _csr(n, [(int(perm[a]), int(perm[b])) for a, b in edges])
    blk = np.zeros(n, dtype=np.int32)
    blk[h:] = 1
    block = np.empty(n, dtype=np.int32)
    block[perm] = blk
    q, d = _check_diam(gk, rp, col, block, 2, sweeps=2)
    assert d.tolist() == [12, 2]


@pytest.mark.gpu
def test_gpu_diameter_rejects_malformed_input(gk):
    rp, col = _csr(4, [(0, 1), (1, 2), (2, 3)])
    with pytest.raises(gk.GKError):
        gk.block_diameter(_dev(rp), _dev(col), _dev(np.array([0, 0, 2, 1], dtype=np.int32)), 2)
    bad_col = col.copy()
    bad_col[2] = -3
    with pytest.raises(gk.GKError):
        gk.block_diameter(_dev(rp), _dev(bad_col), _dev(np.zeros(4, dtype=np.int32)), 1)
    bad_rp = rp.copy()
    bad_rp[1] = -1
    with pytest.raises(gk.GKError):
        gk.block_diameter(_dev(bad_rp), _dev(col), _dev(np.zeros(4, dtype=np.int32)), 1)
    q, d = _check_diam(gk, rp, col, np.zeros(4, dtype=np.int32), 1)  # still usable
    assert d.tolist() == [3]


@pytest.mark.gpu
@pytest.mark.slow
def test_gpu_quality_full_size_mesh(gk):
    """A 3-D graded mesh of 8e6 vertices partitioned into 1024 blocks: the GPU measures
    (edge cut, communication volume, diameter bounds) equal the oracle's, and balanced
    k-means cuts fewer edges than the curve split."""
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
    _check_diam(gk, rp, col, _np(block).astype(np.int32), k)
    _check_diam(gk, rp, col, sfc, k)
