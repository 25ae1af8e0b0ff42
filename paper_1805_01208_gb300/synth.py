"""Seeded synthetic point clouds shaped like the meshes balanced k-means partitions.

The paper partitions the vertex sets of 2D/3D simulation meshes (DIMACS, climate,
Alya and Delaunay meshes; Section 5.2).  None of those files are available, so
these generators stand in for them with the same scales and the same kinds of
structure: uniform point sets (Delaunay meshes of random points), strongly
varying density (adaptively refined meshes) and optional node weights
(2.5D climate meshes).

This module only draws random numbers (numpy PCG64, chunked with one
independent stream per chunk of 2^22 points so that any n is reproducible and
can be generated in parallel).  It holds none of the method's arithmetic; the
CUDA library and the FP64 oracle both take its output as input.
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 22


def _chunks(n: int):
    for start in range(0, n, CHUNK):
        yield start // CHUNK, start, min(n, start + CHUNK)


def _rng(seed: int, tag: int, chunk: int) -> np.random.Generator:
    return np.random.default_rng([seed, tag, chunk])


def _fill(n: int, d: int, dtype, seed: int, tag: int, fn, threads: int | None = None):
    out = np.empty((n, d), dtype=dtype)

    def work(args):
        ci, s, e = args
        out[s:e] = fn(_rng(seed, tag, ci), e - s, s)

    jobs = list(_chunks(n))
    if len(jobs) > 1:
        with ThreadPoolExecutor(max_workers=threads or min(16, len(jobs))) as ex:
            list(ex.map(work, jobs))
    else:
        for j in jobs:
            work(j)
    return out


def uniform_box(n: int, d: int, seed: int, dtype=np.float64, threads=None) -> np.ndarray:
    """Uniform in the unit square / cube (Delaunay meshes of random points)."""
    return _fill(n, d, dtype, seed, 11, lambda r, m, s: r.random((m, d)), threads)


def radial_disk(n: int, d: int, seed: int, dtype=np.float32, threads=None) -> np.ndarray:
    """Radially graded density in the unit disk / ball: radius uniform in [0, 1) and a
    uniform direction, i.e. pdf proportional to 1/r in 2D (1/r^2 in 3D)."""

    def fn(r, m, s):
        rad = r.random(m)
        if d == 2:
            th = r.random(m) * (2.0 * math.pi)
            return np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
        v = r.standard_normal((m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * rad[:, None]

    return _fill(n, d, dtype, seed, 12, fn, threads)


def gaussian_mixture(n: int, d: int, seed: int, components: int = 32, dtype=np.float64,
                     threads=None) -> np.ndarray:
    """Mixture of anisotropic Gaussians (locally refined meshes): means uniform in the
    unit cube, per-axis sigma log-uniform in [0.005, 0.05], a uniformly random rotation
    per component, component weights proportional to 10^U(0,2) (about 100x density
    variation)."""
    g = np.random.default_rng([seed, 13])
    mu = g.random((components, d))
    sig = np.exp(g.uniform(math.log(0.005), math.log(0.05), (components, d)))
    rot = np.empty((components, d, d))
    for c in range(components):
        qm, rm = np.linalg.qr(g.standard_normal((d, d)))
        rot[c] = qm * np.sign(np.diag(rm))
    wts = 10.0 ** g.uniform(0.0, 2.0, components)
    wts /= wts.sum()

    def fn(r, m, s):
        comp = r.choice(components, size=m, p=wts)
        z = r.standard_normal((m, d)) * sig[comp]
        return mu[comp] + np.einsum("mij,mj->mi", rot[comp], z)

    return _fill(n, d, dtype, seed, 14, fn, threads)


def spots_background(n: int, seed: int, spots: int = 256, dtype=np.float32,
                     threads=None) -> np.ndarray:
    """2D: half the points uniform in the unit square, half in isotropic Gaussian
    refinement spots with centers uniform in the square and sigma log-uniform in
    [1e-3, 1e-2]."""
    g = np.random.default_rng([seed, 15])
    mu = g.random((spots, 2))
    sig = np.exp(g.uniform(math.log(1e-3), math.log(1e-2), spots))

    def fn(r, m, s):
        out = r.random((m, 2))
        in_spot = r.random(m) < 0.5
        cnt = int(in_spot.sum())
        comp = r.integers(0, spots, cnt)
        out[in_spot] = mu[comp] + r.standard_normal((cnt, 2)) * sig[comp, None]
        return out

    return _fill(n, 2, dtype, seed, 16, fn, threads)


def uniform_weights(n: int, seed: int, lo: float = 1.0, hi: float = 10.0,
                    dtype=np.float64) -> np.ndarray:
    """Node weights uniform in [lo, hi] (weighted 2.5D meshes)."""
    out = np.empty(n, dtype=dtype)
    for ci, s, e in _chunks(n):
        out[s:e] = _rng(seed, 17, ci).uniform(lo, hi, e - s)
    return out


def random_order(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of [0, n) as int64: the random order of the points
    that the random initialization of Section 4.5 takes its samples from."""
    return np.random.default_rng([seed, 19]).permutation(n).astype(np.int64)


def lattice_mesh(dims, seed: int, grading: float = 2.0, jitter: float = 0.5, dtype=np.float64):
    """A graded, jittered lattice mesh standing in for the paper's simulation meshes in
    the quality measures of Section 5.  dims = (nx, ny) or (nx, ny, nz) vertices per axis.
    Vertex (i, j[, l]) sits at ((i + 0.5 + jitter U(-1/2, 1/2)) / nx) ** grading per axis
    (grading > 1 refines the mesh towards the origin, as adaptive refinement does); edges
    join lattice neighbours along each axis and, in 2-D, along the (+1, +1) diagonal (a
    triangulated grid, degree 6 inside).  The vertices are returned in a random order.
    Returns (points (n, d), row_ptr (n + 1,) int64, col int32) with every edge stored in
    both of its rows."""
    dims = tuple(int(v) for v in dims)
    d = len(dims)
    n = int(np.prod(dims))
    rng = np.random.default_rng([seed, 20])
    idx = np.indices(dims).reshape(d, -1)  # lattice coordinates of lattice vertex L
    u = (idx + 0.5 + jitter * (rng.random((d, n)) - 0.5)) / np.array(dims)[:, None]
    pts_lattice = (u ** grading).T
    # stencil of lattice neighbours (both directions of every edge direction)
    steps = [tuple(1 if a == b else 0 for b in range(d)) for a in range(d)]
    if d == 2:
        steps.append((1, 1))
    steps = steps + [tuple(-c for c in st) for st in steps]
    strides = np.array([int(np.prod(dims[a + 1:])) for a in range(d)], dtype=np.int64)
    L = np.arange(n, dtype=np.int64)
    nbr = np.empty((n, len(steps)), dtype=np.int64)
    valid = np.ones((n, len(steps)), dtype=bool)
    for q, st in enumerate(steps):
        for a in range(d):
            c = idx[a] + st[a]
            valid[:, q] &= (c >= 0) & (c < dims[a])
        nbr[:, q] = L + int(np.dot(st, strides))
    cnt_lat = valid.sum(1)
    rp_lat = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_lat, out=rp_lat[1:])
    col_lat = nbr[valid]  # row-major: the rows stay grouped
    # random vertex order: input position p holds lattice vertex order[p]
    order = rng.permutation(n)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n, dtype=np.int64)
    cnt = cnt_lat[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    src_start = np.repeat(rp_lat[order] - row_ptr[:-1], cnt)
    b = pos[col_lat[src_start + np.arange(row_ptr[-1], dtype=np.int64)]]
    return pts_lattice[order].astype(dtype), row_ptr, b.astype(np.int32)


# --------------------------------------------------------------------------------
# Named workloads.  Sizes and shapes of the partitioning benchmarks this library is
# measured on; seeds fixed so that every run sees the same points.
# --------------------------------------------------------------------------------
WORKLOADS = {
    "uniform2d_1e5_k16_f64": dict(n=100_000, d=2, k=16, eps=0.03, dtype="f64", shape="uniform",
                                  seed=1, assign="f64", weighted=False),
    "gmm3d_1e7_k1024_f64": dict(n=10_000_000, d=3, k=1024, eps=0.03, dtype="f64", shape="gmm",
                                seed=2, assign="f64", weighted=False),
    "radial2d_1e8_k4096_f32": dict(n=100_000_000, d=2, k=4096, eps=0.03, dtype="f32",
                                   shape="radial", seed=3, assign="f32", weighted=False),
    "spots2d_1e9_k16384_f32": dict(n=1_000_000_000, d=2, k=16384, eps=0.03, dtype="f32",
                                   shape="spots", seed=5, assign="f32", weighted=False),
}


def make_points(shape: str, n: int, d: int, seed: int, dtype: str = "f64", threads=None):
    dt = np.float64 if dtype == "f64" else np.float32
    if shape == "uniform":
        return uniform_box(n, d, seed, dt, threads)
    if shape == "gmm":
        return gaussian_mixture(n, d, seed, dtype=dt, threads=threads)
    if shape == "radial":
        return radial_disk(n, d, seed, dt, threads)
    if shape == "spots":
        assert d == 2
        return spots_background(n, seed, dtype=dt, threads=threads)
    raise ValueError(shape)


def workload(name: str, n: int | None = None, threads=None):
    """Points (and weights or None) of a named workload, optionally with fewer points."""
    spec = dict(WORKLOADS[name])
    if n is not None:
        spec["n"] = n
    x = make_points(spec["shape"], spec["n"], spec["d"], spec["seed"], spec["dtype"], threads)
    w = None
    if spec["weighted"]:
        w = uniform_weights(spec["n"], spec["seed"], dtype=x.dtype)
    return x, w, spec


def batched_instances(count: int = 64, seed: int = 4, max_n: int | None = None):
    """Instance descriptions for batched runs: n log-uniform in [1e4, 1e7], d in {2, 3},
    k = round(2^U(3,9)) clamped to [8, 512], weights uniform in [1, 10], FP32 points;
    shapes cycle uniform / Gaussian mixture / radial.  max_n caps n (smaller tests)."""
    shapes = ["uniform", "gmm", "radial"]
    out = []
    for i in range(count):
        g = np.random.default_rng([seed * 1000 + i, 18])
        n = int(10.0 ** g.uniform(4.0, 7.0))
        if max_n is not None:
            n = min(n, max_n)
        d = 2 if g.random() < 0.5 else 3
        k = int(min(512, max(8, round(2.0 ** g.uniform(3.0, 9.0)))))
        k = min(k, n)
        out.append(dict(n=n, d=d, k=k, eps=0.03, shape=shapes[i % 3], seed=seed * 1000 + i,
                        dtype="f32", weighted=True))
    return out


def instance_data(spec: dict, threads=None):
    x = make_points(spec["shape"], spec["n"], spec["d"], spec["seed"], spec["dtype"], threads)
    w = uniform_weights(spec["n"], spec["seed"], dtype=x.dtype) if spec.get("weighted") else None
    return x, w
