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
