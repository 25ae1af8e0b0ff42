"""The seeded input generators (CPU): deterministic, and the structure the tests and the
benchmark rely on (a permutation for the random order; a symmetric adjacency without
self-loops and the lattice degrees for the meshes)."""
import numpy as np
import pytest

from paper_1805_01208_gb300 import synth


def test_random_order_is_a_seeded_permutation():
    a = synth.random_order(10_000, 3)
    assert a.dtype == np.int64 and np.array_equal(np.sort(a), np.arange(10_000))
    assert np.array_equal(a, synth.random_order(10_000, 3))
    assert not np.array_equal(a, synth.random_order(10_000, 4))


@pytest.mark.parametrize("dims", [(7, 5), (6, 4, 3), (1, 9), (2, 2, 2)])
def test_lattice_mesh_adjacency(dims):
    x, rp, col = synth.lattice_mesh(dims, 11)
    n = int(np.prod(dims))
    d = len(dims)
    assert x.shape == (n, d) and rp.shape == (n + 1,) and rp[0] == 0 and rp[-1] == len(col)
    v = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(v != col)  # no self-loops
    pairs = set(zip(v.tolist(), col.tolist()))
    assert len(pairs) == len(col)  # no repeated entries
    assert all((b, a) in pairs for a, b in pairs)  # symmetric
    deg = np.diff(rp)
    assert deg.max() <= (6 if d == 2 else 2 * d)
    assert np.all((x > 0) & (x < 1))
    x2, rp2, col2 = synth.lattice_mesh(dims, 11)
    assert np.array_equal(x, x2) and np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_workload_points_are_seeded():
    a, _, spec = synth.workload("uniform2d_1e5_k16_f64", n=5000)
    b, _, _ = synth.workload("uniform2d_1e5_k16_f64", n=5000)
    assert a.shape == (5000, 2) and np.array_equal(a, b)
