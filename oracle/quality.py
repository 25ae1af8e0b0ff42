"""Partition quality measures of Section 5 -- TEST INFRASTRUCTURE ONLY (FP64/int64
numpy restatement; only ``tests/`` and the CPU legs of ``bench.py`` may use it).

For a graph G = (V, E) given as a symmetric adjacency list (CSR: ``row_ptr`` of n + 1
offsets, ``col`` the neighbours, every undirected edge stored in both rows) and a
partition Pi = (V_0 .. V_{k-1}) given by block ids:

  ext(V_i)  = number of edges {u, v} with u in V_i and v outside V_i;
  edge cut  = (sum_i ext(V_i)) / 2  (every cut edge is external to both its blocks);
  comm(V_i) = sum over v in V_i of the number of blocks other than V_i that hold a
              neighbour of v (the communication volume; reading: the printed set does
              not exclude V_i itself, which would add one for every vertex with a
              neighbour in its own block and so measure block sizes, not communication);
  maximum / total communication volume = max_i / sum_i comm(V_i).

Self-loops are ignored.  Everything here is a direct count over the stored pairs.
"""
from __future__ import annotations

import numpy as np


def _pairs(row_ptr, col):
    """(v, u) for every stored adjacency entry, self-loops removed."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    v = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    keep = v != col
    return v[keep], col[keep]


def block_ext_comm(row_ptr, col, block, k: int):
    """ext(V_i) and comm(V_i) for every block i (int64 arrays of length k)."""
    block = np.asarray(block, dtype=np.int64)
    v, u = _pairs(row_ptr, col)
    bv, bu = block[v], block[u]
    foreign = bv != bu
    ext = np.bincount(bv[foreign], minlength=k).astype(np.int64)
    # distinct (vertex, foreign block) pairs, counted for the vertex's block
    pairs = np.unique(np.stack([v[foreign], bu[foreign]], axis=1), axis=0)
    comm = np.bincount(block[pairs[:, 0]], minlength=k).astype(np.int64) if len(pairs) else \
        np.zeros(k, dtype=np.int64)
    return ext, comm


def quality(row_ptr, col, block, k: int):
    """Edge cut, total and maximum communication volume, largest ext."""
    ext, comm = block_ext_comm(row_ptr, col, block, k)
    return {"edge_cut": int(ext.sum() // 2), "total_comm_volume": int(comm.sum()),
            "max_comm_volume": int(comm.max()), "max_ext": int(ext.max()), "ext": ext,
            "comm": comm}


# ----------------------------------------------------------------------------------------
# Block diameter (Section 5): diam(V_i) = max over u, v in V_i of dist(u, v), dist taken
# in the subgraph induced by V_i (so a block that is not connected has an infinite
# diameter, as the paper's evaluation notes).  The paper evaluates a lower bound from
# the first rounds of iFUB instead of the exact value; reading: a lower bound from
# `sweeps` breadth-first sweeps per block, the first from the block's smallest vertex
# index, each later one from the vertex the previous sweep reached last (the smallest
# index among those at the largest distance).  Every sweep's eccentricity lies in
# [diam / 2, diam], so the bound is a 2-approximation like the paper's; on trees two
# sweeps are already exact.
#
# Per block the result is the bound (>= 0), -1 for a block that is not connected, and 0
# for an empty block.
# ----------------------------------------------------------------------------------------
def _adjacency(row_ptr, col):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    return row_ptr, col


def block_diameter_exact(row_ptr, col, block, k: int):
    """Exact diameters by a breadth-first search from every vertex of every block
    (pure Python; small graphs only)."""
    row_ptr, col = _adjacency(row_ptr, col)
    block = np.asarray(block, dtype=np.int64)
    n = len(row_ptr) - 1
    members = [[] for _ in range(k)]
    for v in range(n):
        members[block[v]].append(v)
    out = np.zeros(k, dtype=np.int64)
    for b in range(k):
        for s in members[b]:
            dist = {s: 0}
            queue = [s]
            for v in queue:
                for u in col[row_ptr[v]:row_ptr[v + 1]].tolist():
                    if block[u] == b and u not in dist:
                        dist[u] = dist[v] + 1
                        queue.append(u)
            if len(dist) < len(members[b]):
                out[b] = -1
                break
            out[b] = max(out[b], max(dist.values()))
    return out


def _bfs_within_blocks(row_ptr, col, block, sources):
    """Distances from one source per block inside each block's induced subgraph, all
    blocks at once (level by level; -1 = not reached)."""
    n = len(row_ptr) - 1
    dist = np.full(n, -1, dtype=np.int64)
    front = np.asarray(sources, dtype=np.int64)
    dist[front] = 0
    level = 0
    while len(front):
        deg = row_ptr[front + 1] - row_ptr[front]
        tail = np.repeat(front, deg)
        first = np.repeat(row_ptr[front] - (np.cumsum(deg) - deg), deg)
        u = col[first + np.arange(int(deg.sum()), dtype=np.int64)]
        fresh = (block[u] == block[tail]) & (dist[u] < 0)
        front = np.unique(u[fresh])
        level += 1
        dist[front] = level
    return dist


def block_diameter_sweeps(row_ptr, col, block, k: int, sweeps: int = 3):
    """Per-block diameter lower bounds from breadth-first sweeps (the reading above)."""
    row_ptr, col = _adjacency(row_ptr, col)
    block = np.asarray(block, dtype=np.int64)
    n = len(row_ptr) - 1
    ids = np.arange(n, dtype=np.int64)
    size = np.bincount(block, minlength=k)
    nonempty = size > 0
    start = np.full(k, n, dtype=np.int64)
    np.minimum.at(start, block, ids)
    bound = np.zeros(k, dtype=np.int64)
    connected = np.ones(k, dtype=bool)
    for s in range(sweeps):
        dist = _bfs_within_blocks(row_ptr, col, block, start[nonempty])
        if s == 0:
            connected = np.bincount(block[dist >= 0], minlength=k) == size
        ecc = np.full(k, -1, dtype=np.int64)
        np.maximum.at(ecc, block, dist)
        bound = np.maximum(bound, ecc)
        last = np.nonzero(dist == ecc[block])[0]
        start = np.full(k, n, dtype=np.int64)
        np.minimum.at(start, block[last], last)
    return np.where(nonempty, np.where(connected, bound, -1), 0)


def diameter_summary(diam, size):
    """Largest bound over connected blocks, the number of blocks that are not connected,
    and the harmonic mean over the blocks of at least two vertices (a block that is not
    connected adds 1/inf = 0 to the sum of reciprocals, as in the paper's aggregation;
    +inf when every such block is disconnected, 0 when there is none)."""
    diam = np.asarray(diam, dtype=np.int64)
    size = np.asarray(size)
    big = size >= 2
    conn = diam >= 0
    recip = np.zeros(len(diam), dtype=np.float64)
    pos = big & conn
    recip[pos] = 1.0 / diam[pos]
    m = int(big.sum())
    s = float(recip.sum())
    hm = 0.0 if m == 0 else (np.inf if s == 0.0 else m / s)
    return {"max_diameter": int(diam[conn].max()) if conn.any() else 0,
            "disconnected_blocks": int((~conn).sum()), "harmonic_mean": hm}
