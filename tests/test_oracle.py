"""Pins for the FP64 oracle: each test checks it against something other than itself --
values fixed by the paper or by mathematics, textbook/library routines, closed forms and
brute force on tiny inputs (CPU only)."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# ----------------------------------------------------------------------------------------
# Hilbert curve (Section 3.1, Algorithm 2 "sfcIndex"): the oracle's level descent.
# ----------------------------------------------------------------------------------------

def _cells(d, b):
    return list(itertools.product(range(1 << b), repeat=d))


def _curve(d, b):
    cells = _cells(d, b)
    keys = [oracle.hilbert_index(np.array(c), b) for c in cells]
    order = np.argsort(keys)
    return [cells[i] for i in order], sorted(keys)


def test_hilbert_2d_order2_matches_hilberts_figure():
    want = [tuple(int(v) for v in r) for r in _golden("hilbert2d_order2.txt")]
    got, _ = _curve(2, 2)
    assert got == want


def test_hilbert_3d_order1_is_gray_code_order():
    want = [tuple(int(v) for v in r) for r in _golden("hilbert3d_order1.txt")]
    got, _ = _curve(3, 1)
    assert got == want


def test_hilbert_2d_order1_orientation():
    got, _ = _curve(2, 1)
    assert got == [(0, 0), (0, 1), (1, 1), (1, 0)]


@pytest.mark.parametrize("d,b", [(2, 1), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_hilbert_is_bijection(d, b):
    _, keys = _curve(d, b)
    assert keys == list(range(1 << (d * b)))


@pytest.mark.parametrize("d,b", [(2, 5), (3, 4)])
def test_hilbert_consecutive_cells_are_adjacent(d, b):
    cells, _ = _curve(d, b)
    steps = np.abs(np.diff(np.array(cells), axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    assert cells[0] == (0,) * d


@pytest.mark.parametrize("d,b", [(2, 4), (3, 3)])
def test_hilbert_prefixes_are_aligned_subcubes(d, b):
    cells, _ = _curve(d, b)
    arr = np.array(cells)
    for level in range(1, b + 1):
        side = 1 << (b - level)
        block = side ** d
        for s in range(0, len(cells), block):
            chunk = arr[s:s + block]
            lo = chunk.min(axis=0)
            assert np.all(chunk.max(axis=0) - lo == side - 1)
            assert np.all(lo % side == 0)


def _skilling_key(q, b):
    """J. Skilling, 'Programming the Hilbert curve' (2004): axes -> transposed index,
    then the transposed bits read out most significant level first, axis 0 first.
    Written independently of the oracle (different algorithm: in-place bit transforms)."""
    d = len(q)
    X = [int(v) for v in q]
    Q = 1 << (b - 1)
    while Q > 1:
        P = Q - 1
        for i in range(d):
            if X[i] & Q:
                X[0] ^= P
            else:
                t = (X[0] ^ X[i]) & P
                X[0] ^= t
                X[i] ^= t
        Q >>= 1
    for i in range(1, d):
        X[i] ^= X[i - 1]
    t = 0
    Q = 1 << (b - 1)
    while Q > 1:
        if X[d - 1] & Q:
            t ^= Q - 1
        Q >>= 1
    X = [v ^ t for v in X]
    key = 0
    for lev in range(b - 1, -1, -1):
        for i in range(d):
            key = (key << 1) | ((X[i] >> lev) & 1)
    return key


@pytest.mark.parametrize("d,b", [(2, 3), (3, 3)])
def test_hilbert_is_skillings_curve_all_cells(d, b):
    for c in _cells(d, b):
        assert oracle.hilbert_index(np.array(c), b) == _skilling_key(c, b)


@pytest.mark.parametrize("d,b", [(2, 32), (3, 21)])
def test_hilbert_is_skillings_curve_full_width(d, b):
    rng = np.random.default_rng(7)
    for _ in range(300):
        c = rng.integers(0, 1 << b, size=d, dtype=np.uint64)
        assert oracle.hilbert_index(c.astype(np.uint32), b) == _skilling_key(c, b)


def test_quantisation_closed_forms():
    # unit square: extent 1 = 2^0 -> cell = floor(x * 2^32); x = 1 clamps to 2^32 - 1
    x = np.array([[0.0, 0.0], [0.5, 0.25], [1.0, 1.0]])
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0], [1 << 31, 1 << 30], [(1 << 32) - 1, (1 << 32) - 1]]
    # box [3, 5] x [0, 0.5]: extent 2 -> side 2^1, cell = floor((x - lo) * 2^31)
    x = np.array([[3.0, 0.0], [4.0, 0.5], [5.0, 0.25]])
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0], [1 << 31, 1 << 30], [(1 << 32) - 1, 1 << 29]]
    # the largest extent on the second axis: box [0, 0.5] x [3, 5], extent 2 -> side 2^1
    x = np.array([[0.0, 3.0], [0.25, 4.0], [0.5, 5.0]])
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0], [1 << 29, 1 << 31], [1 << 30, (1 << 32) - 1]]
    # 3D, extent 3 -> side 4 = 2^2, b = 21 -> cell = floor((x - lo) * 2^19)
    x = np.array([[0.0, 0.0, 0.0], [3.0, 1.0, 2.0]])
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0, 0], [3 << 19, 1 << 19, 2 << 19]]
    # all points equal: every cell 0, every key 0
    keys, q = oracle.hilbert_keys(np.full((5, 3), 7.25), return_cells=True)
    assert np.all(q == 0) and np.all(keys == 0)
    # a cell is the floor, not the nearest integer: x = 0.75 + 0.75 * 2^-32 (exact in FP64)
    # on the unit square scales to 3 * 2^30 + 0.75, in cell 3 * 2^30
    x = np.array([[0.0, 0.0], [0.75 + 0.75 * 2.0 ** -32, 0.5], [1.0, 1.0]])
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q[1].tolist() == [3 << 30, 1 << 31]


def test_quantisation_fp32_subtracts_in_fp32():
    # lo = 1.0f, x = 1 + 2^-23 (next float): the FP32 difference is 2^-23 exactly;
    # extent is 1 -> cell = floor(2^-23 * 2^32) = 2^9.
    x = np.array([[1.0, 0.0], [1.0 + 2.0 ** -23, 1.0], [2.0, 0.5]], dtype=np.float32)
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert int(q[1, 0]) == 1 << 9
    assert int(q[2, 1]) == 1 << 31
    # lo = 2^-30, x = 1 + 2^-23: the exact difference 1 + 2^-23 - 2^-30 is not a float; FP32
    # rounds it to 1 + 2^-23.  The extent is above 1 -> side 2, cell = floor(v * 2^31):
    # 2^31 + 2^8 from the FP32 difference (2^31 + 2^8 - 2 from an FP64 one).
    x = np.array([[2.0 ** -30, 0.0], [1.0 + 2.0 ** -23, 1.0]], dtype=np.float32)
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0], [(1 << 31) + (1 << 8), 1 << 31]]
    # the extent itself is the FP64 difference of the FP32 bounds: lo = -2^-30, hi = 1 give
    # 1 + 2^-30 > 1 -> side 2 (an FP32 difference would round it to 1 -> side 1); the point
    # at hi then has v = fl32(1 + 2^-30) = 1 and cell 2^31
    x = np.array([[-(2.0 ** -30), 0.0], [1.0, 0.5]], dtype=np.float32)
    _, q = oracle.hilbert_keys(x, return_cells=True)
    assert q.tolist() == [[0, 0], [1 << 31, 1 << 30]]


def test_keys_of_points_follow_cells():
    rng = np.random.default_rng(3)
    x = rng.random((200, 2))
    keys, q = oracle.hilbert_keys(x, return_cells=True)
    for i in range(0, 200, 17):
        assert keys[i] == _skilling_key(q[i], 32)


# ----------------------------------------------------------------------------------------
# Sort and initial centers (Algorithm 2).
# ----------------------------------------------------------------------------------------

def test_sort_is_numpy_stable_argsort():
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 50, size=5000).astype(np.uint64) << np.uint64(40)
    keys[::7] = np.uint64(2 ** 64 - 1)
    perm = oracle.sort_keys(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))


def test_sfc_centers_closed_form():
    xs = np.arange(20, dtype=np.float64).reshape(10, 2)
    C = oracle.sfc_centers(xs, 3)
    # i*n/k + n/(2k) with n = 10, k = 3: 0 + 1, 3 + 1, 6 + 1
    assert np.array_equal(C, xs[[1, 4, 7]])
    C = oracle.sfc_centers(xs, 10)
    assert np.array_equal(C, xs)


# ----------------------------------------------------------------------------------------
# Assignment (Section 4.2, Algorithm 1).
# ----------------------------------------------------------------------------------------

def test_assign_apollonius_closed_form():
    g = _golden("apollonius_2centers.txt")
    C = np.array([[0.0, 0.0], [1.0, 0.0]])
    I = np.array([2.0, 1.0])
    A, _, _ = oracle.assign(g[:, :2], C, I)
    assert A.tolist() == g[:, 2].astype(int).tolist()


def test_assign_unit_influence_is_nearest_center():
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(11)
    for d in (2, 3):
        x = rng.random((3000, d))
        C = rng.random((37, d))
        A, best, second = oracle.assign(x, C, np.ones(37), threads=2)
        dist, idx = cKDTree(C).query(x)
        clear = (second - best) > 1e-12 * best
        assert np.array_equal(A[clear], idx[clear])
        assert np.allclose(best, dist, rtol=1e-14, atol=0)


def test_assign_matches_squared_brute_force():
    rng = np.random.default_rng(12)
    for d in (2, 3):
        x = rng.random((2000, d))
        C = rng.random((20, d))
        I = rng.uniform(0.5, 2.0, 20)
        A, best, second = oracle.assign(x, C, I)
        sq = ((x[:, None, :] - C[None, :, :]) ** 2).sum(-1) / I[None, :] ** 2
        ref = np.argmin(sq, axis=1)
        clear = (second - best) > 1e-12 * best
        assert clear.mean() > 0.99
        assert np.array_equal(A[clear], ref[clear])
        assert np.allclose(best, np.sqrt(sq.min(axis=1)), rtol=1e-13)
        # the runner-up is the second smallest effective distance (equal to best on a tie)
        assert np.allclose(second, np.sqrt(np.sort(sq, axis=1)[:, 1]), rtol=1e-13)


def test_assign_ties_go_to_lowest_index():
    C = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0], [2.0, 0.0]])
    I = np.array([1.0, 1.0, 1.0, 1.0])
    x = np.array([[0.0, 0.0], [1.0, 0.0]])
    A, _, _ = oracle.assign(x, C, I)
    # (0,0): centers 1 and 2 coincide -> 1.  (1,0): centers 0,1,2,3 all at distance 1 -> 0.
    assert A.tolist() == [1, 0]


# ----------------------------------------------------------------------------------------
# Block weights, balance bound and influence update (Section 2, Section 4.2, Eq. 1).
# ----------------------------------------------------------------------------------------

def test_block_weights_match_bincount():
    rng = np.random.default_rng(2)
    A = rng.integers(0, 9, 1000).astype(np.int32)
    S, W = oracle.block_weights(A, None, 10)
    assert np.array_equal(S, np.bincount(A, minlength=10).astype(float)) and W == 1000
    w = rng.uniform(1, 10, 1000)
    S, W = oracle.block_weights(A, w, 10)
    assert np.allclose(S, np.bincount(A, weights=w, minlength=10), rtol=1e-13)
    assert math.isclose(W, w.sum(), rel_tol=1e-13)


def test_balance_bound_closed_form():
    assert oracle.balance_bound(100.0, 16, 0.03) == pytest.approx(1.03 * 7, rel=1e-15)
    assert oracle.balance_bound(96.0, 16, 0.0) == 6.0
    assert oracle.balance_bound(1e5, 16, 0.03) == pytest.approx(6437.5, rel=1e-15)


def test_balance_update_closed_form():
    k, d, eps = 4, 2, 0.03
    W = 400.0  # target 100 per block, bound 103
    I = np.array([1.0, 2.0, 0.5, 1.0])
    S = np.array([102.0, 100.0, 98.0, 100.0])
    bal, I2, imb = oracle.balance_update(S, W, k, d, eps, I)
    assert bal and np.array_equal(I2, I) and imb == pytest.approx(0.02)
    S = np.array([50.0, 104.0, 246.0, 0.0])
    bal, I2, imb = oracle.balance_update(S, W, k, d, eps, I)
    assert not bal and imb == pytest.approx(1.46)
    want = np.array([1.0 * 1.05,                   # gamma 2 -> sqrt 1.41 -> clamp 1.05
                     2.0 * math.sqrt(100 / 104),   # oversized -> shrinks, inside the clamp
                     0.5 * 0.95,                   # gamma 0.41 -> clamp 0.95
                     1.0 * 1.05])                  # empty block -> largest growth
    assert np.allclose(I2, want, rtol=1e-15)
    bal, I3, _ = oracle.balance_update(np.array([50.0, 104.0, 246.0, 0.0]), W, k, 3, eps, I)
    assert I3[1] == pytest.approx(2.0 * (100 / 104) ** (1 / 3), rel=1e-15)


def test_balance_target_is_the_mean_and_imbalance_uses_the_ceiling():
    """W/k not an integer: the target of Eq. 1 is W/k = 2.5 itself, the bound and the
    imbalance use the ceiling 3 (Section 2)."""
    k, d, eps, W = 4, 2, 0.0, 10.0
    S = np.array([3.1, 2.5, 2.4, 2.0])  # 3.1 > 3: unbalanced
    I = np.array([1.0, 1.0, 2.0, 0.5])
    bal, I2, imb = oracle.balance_update(S, W, k, d, eps, I)
    assert not bal and imb == pytest.approx(3.1 / 3.0 - 1.0, rel=1e-15)
    want = I * np.array([0.95,                  # sqrt(2.5 / 3.1) = 0.898 -> clamp
                         1.0,                   # at the target: unchanged
                         math.sqrt(2.5 / 2.4),  # 1.0206, inside the clamp
                         1.05])                 # sqrt(1.25) = 1.118 -> clamp
    assert np.allclose(I2, want, rtol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_influence_update_moves_size_to_target(d):
    """Section 4.2's derivation: with uniform density and everything else fixed, scaling a
    block's influence by gamma^(1/d) scales its size by gamma.  Block 0 is a ball around
    the origin whose radius is set by a competitor so far away that its effective distance
    is nearly constant over the unit ball; k = 2, so the target is n/2."""
    rng = np.random.default_rng(21 + d)
    n = 200_000
    v = rng.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = v * rng.random(n)[:, None] ** (1.0 / d)  # uniform in the unit ball
    frac0 = 0.47
    R0 = frac0 ** (1.0 / d)
    L = 1e4
    C = np.zeros((2, d))
    C[1, 0] = L
    I = np.array([1.0, L / R0])
    A, _, _ = oracle.assign(x, C, I)
    S, W = oracle.block_weights(A, None, 2)
    assert abs(S[0] / n - frac0) < 0.005
    bal, I_new, _ = oracle.balance_update(S, W, 2, d, 0.03, I)
    assert not bal and I_new[0] > I[0]  # undersized block gains influence
    I_applied = np.array([I_new[0], I[1]])  # update block 0 only ("all else equal")
    A2, _, _ = oracle.assign(x, C, I_applied)
    S2, _ = oracle.block_weights(A2, None, 2)
    assert abs(S2[0] / (n / 2) - 1.0) < 0.01


# ----------------------------------------------------------------------------------------
# Movement and erosion (Algorithm 2, Eq. 2-3).
# ----------------------------------------------------------------------------------------

def test_move_centers_weighted_means_and_beta():
    x = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 4.0], [10.0, 10.0], [13.0, 14.0]])
    w = np.array([1.0, 1.0, 2.0, 1.0, 3.0])
    A = np.array([0, 0, 0, 2, 2], dtype=np.int32)
    C = np.array([[1.0, 1.0], [5.0, 5.0], [11.0, 11.0]])
    Cn, delta, beta = oracle.move_centers(x, w, A, C)
    assert np.allclose(Cn[0], [2.0 / 4.0, 8.0 / 4.0])
    assert np.array_equal(Cn[1], C[1]) and delta[1] == 0.0  # empty block stays
    assert np.allclose(Cn[2], [(10 + 39) / 4.0, (10 + 42) / 4.0])
    assert delta[0] == pytest.approx(math.hypot(0.5, 1.0))
    # block diagonals: block 0 box 2 x 4, block 2 box 3 x 4 -> mean of sqrt(20) and 5
    assert beta == pytest.approx((math.sqrt(20.0) + 5.0) / 2.0)


def test_move_centers_matches_numpy():
    rng = np.random.default_rng(9)
    x = rng.random((5000, 3))
    w = rng.uniform(1, 10, 5000)
    A = rng.integers(0, 7, 5000).astype(np.int32)
    C = rng.random((8, 3))
    Cn, delta, beta = oracle.move_centers(x, w, A, C)
    for c in range(7):
        m = A == c
        want = (w[m, None] * x[m]).sum(0) / w[m].sum()
        assert np.allclose(Cn[c], want, rtol=1e-13)
    assert np.array_equal(Cn[7], C[7])
    assert np.allclose(delta, np.linalg.norm(Cn - C, axis=1), rtol=1e-13)


def test_erosion_closed_forms():
    I = np.array([0.3, 1.7, 1.0, 2.5, 0.8])
    delta = np.array([0.0, 0.0, 5.0, 1e6, 0.4])
    beta = 0.8
    I2 = oracle.erosion(delta, beta, I)
    # delta = 0 -> alpha = 0 -> unchanged (exp(log(I)) within a few ulps)
    assert np.allclose(I2[:2], I[:2], rtol=4 * np.finfo(float).eps, atol=0)
    assert I2[2] == pytest.approx(1.0, abs=1e-15)          # influence 1 stays 1
    assert I2[3] == pytest.approx(1.0, abs=1e-12)          # huge move -> back to 1
    # 2/(1+exp(-t)) - 1 = tanh(t/2): alpha = tanh(delta / (2 beta))
    alpha = math.tanh(0.4 / (2 * 0.8))
    assert I2[4] == pytest.approx(0.8 ** (1 - alpha), rel=1e-14)


# ----------------------------------------------------------------------------------------
# Whole method (Algorithm 2).
# ----------------------------------------------------------------------------------------

def _effective_argmin(x, C, I):
    sq = ((x[:, None, :] - C[None, :, :]) ** 2).sum(-1) / I[None, :] ** 2
    order = np.sort(sq, axis=1)
    return np.argmin(sq, axis=1), order[:, 0], order[:, 1]


@pytest.mark.parametrize("d,k,weighted", [(2, 8, False), (3, 12, False), (2, 10, True)])
def test_partition_meets_bound_and_is_weighted_voronoi(d, k, weighted):
    rng = np.random.default_rng(100 + d + k)
    n = 3000
    x = rng.random((n, d)) ** 2  # graded density
    w = rng.uniform(1, 10, n) if weighted else None
    out = oracle.partition(x, w, k, 0.03, oracle.default_options(threads=2))
    res = out["result"]
    assert res["status"] == oracle.OR_OK and res["balanced"] == 1
    S, W = oracle.block_weights(out["A"], w, k)
    assert S.max() <= (1.03) * math.ceil(W / k)
    ref, b1, b2 = _effective_argmin(x, out["C"], out["I"])
    clear = (b2 - b1) > 1e-10 * b1
    assert np.array_equal(out["A"][clear], ref[clear])


def test_lloyd_special_case_and_monotone_objective():
    """With eps so large that every assignment is balanced and erosion off, influences
    stay 1 and Algorithm 2 is Lloyd's algorithm (Section 3.3): nearest-center assignment
    and plain means; its objective never increases."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(31)
    x = rng.random((4000, 2))
    keys = oracle.hilbert_keys(x)
    xs = x[oracle.sort_keys(keys)]
    k = 9
    C = oracle.sfc_centers(xs, k)
    last = math.inf
    for it in range(1, 6):
        opt = oracle.default_options(max_iter=it, erosion=0, delta_threshold=0.0)
        out = oracle.balanced_kmeans(xs, None, k, 1e9, C, np.ones(k), opt)
        assert np.array_equal(out["I_used"], np.ones(k))
        # textbook Lloyd from the same start, it iterations
        Cl = C.copy()
        for step in range(it):
            _, A = cKDTree(Cl).query(xs)
            if step < it - 1:
                Cl = np.array([xs[A == c].mean(0) if np.any(A == c) else Cl[c] for c in range(k)])
        assert np.array_equal(out["A"], A)
        assert np.allclose(out["C"], Cl, rtol=1e-12, atol=1e-15)
        obj = ((xs - out["C"][out["A"]]) ** 2).sum()
        assert obj <= last * (1 + 1e-12)
        last = obj


def test_balanced_kmeans_outputs_are_consistent():
    rng = np.random.default_rng(41)
    x = rng.random((2500, 3)) ** 3
    keys = oracle.hilbert_keys(x)
    xs = x[oracle.sort_keys(keys)]
    k = 16
    C0 = oracle.sfc_centers(xs, k)
    out = oracle.balanced_kmeans(xs, None, k, 0.03, C0, np.ones(k))
    ref, b1, b2 = _effective_argmin(xs, out["C"], out["I_used"])
    clear = (b2 - b1) > 1e-10 * b1
    assert np.array_equal(out["A"][clear], ref[clear])
    Cm, _, _ = oracle.move_centers(xs, None, out["A"], out["C"])
    assert np.allclose(out["C_moved"], Cm, rtol=1e-14)
    assert out["result"]["balanced"] == 1


def test_default_movement_threshold_is_a_ten_thousandth_of_the_extent():
    """Reading of the defaults: deltaThreshold = 1e-4 x the largest extent of the points'
    bounding box unless the caller gives one; the loop stops when every center moved less."""
    rng = np.random.default_rng(31)
    x = rng.random((4000, 2)) * np.array([8.0, 2.0]) + np.array([-3.0, 5.0])
    x[0], x[1] = [-3.0, 5.0], [5.0, 7.0]  # the box is [-3, 5] x [5, 7]: extent 8
    r = oracle.partition(x, None, 6, 0.03, oracle.default_options(max_iter=3))["result"]
    assert r["delta_threshold"] == 1e-4 * 8.0
    r = oracle.partition(x, None, 6, 0.03, oracle.default_options(max_iter=3,
                                                                  delta_threshold=0.25))["result"]
    assert r["delta_threshold"] == 0.25
    # a threshold above every movement stops after the first iteration, converged
    r = oracle.partition(x, None, 6, 0.03, oracle.default_options(delta_threshold=100.0))["result"]
    assert r["iterations"] == 1 and r["converged"] == 1


def test_invalid_arguments_rejected():
    x = np.zeros((3, 2))
    assert oracle.partition(x, None, 4, 0.03)["result"]["status"] == oracle.OR_INVALID
    assert oracle.partition(np.zeros((3, 4)), None, 2, 0.03)["result"]["status"] == oracle.OR_INVALID
    assert oracle.partition(x, None, 2, -0.1)["result"]["status"] == oracle.OR_INVALID


# ----------------------------------------------------------------------------------------
# Random initialization (Section 4.5): samples of the random order that double after
# every round with center movement.
# ----------------------------------------------------------------------------------------

def test_sample_sizes_and_rounds_closed_forms():
    # first sample: 100 per block (100 per process, as many processes as blocks), >= k, <= n
    assert oracle.sample_first(10**7, 1024) == 102_400
    assert oracle.sample_first(10**7, 1024, 5000) == 5000
    assert oracle.sample_first(10**7, 1024, 10) == 1024
    assert oracle.sample_first(5000, 1024) == 5000
    # rounds = ceil(log2(n / m0)), the paper's count with n_local = n / k, at most maxIter-1
    for n, m0 in [(10**7, 102_400), (2**20, 2**10), (2**20 + 1, 2**10), (3000, 1600),
                  (1600, 1600), (100, 1600), (10**9, 1_638_400)]:
        want = max(0, math.ceil(math.log2(n / m0) - 1e-12)) if n > m0 else 0
        assert oracle.sample_rounds(n, m0, 10**6) == want, (n, m0)
    assert oracle.sample_rounds(2**20, 2**10, 5) == 4


def _gmm(n, d, seed):
    rng = np.random.default_rng(seed)
    mu = rng.random((6, d))
    comp = rng.integers(0, 6, n)
    return mu[comp] + 0.05 * rng.standard_normal((n, d))


@pytest.mark.parametrize("sample0,max_iter", [(10**6, 50), (0, 1)])
def test_sampled_without_rounds_is_the_plain_partition(sample0, max_iter):
    """No sample round (first sample >= n, or maxIter 1): exactly Algorithm 2."""
    x = _gmm(3000, 2, 7)
    order = np.random.default_rng(1).permutation(len(x))
    opt = oracle.default_options(max_iter=max_iter, threads=2)
    a = oracle.partition_sampled(x, None, 8, 0.03, order, sample0, opt)
    b = oracle.partition(x, None, 8, 0.03, opt)
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["C"], b["C"])
    assert np.array_equal(a["I"], b["I"]) and a["result"] == b["result"]


@pytest.mark.parametrize("weighted", [False, True])
def test_sample_round_on_one_copy_of_doubled_points_is_a_full_iteration(weighted):
    """Every point twice (same weight), the order listing one copy of each first, and the
    first sample exactly those copies: a sample round sees the whole point set at half
    weight, which gives the same assignment, balance decisions (k divides the sample, so
    the bound scales exactly), centers, movement and erosion as a first iteration on all
    points.  So the sampled run equals the plain run up to summation order."""
    m, k = 1200, 8
    x1 = _gmm(m, 2, 11)
    x = np.concatenate([x1, x1])
    w = None
    if weighted:
        w1 = np.random.default_rng(3).uniform(1, 10, m)
        w = np.concatenate([w1, w1])
    rng = np.random.default_rng(5)
    order = np.concatenate([rng.permutation(m), m + rng.permutation(m)])
    opt = oracle.default_options(max_iter=6, threads=2)
    a = oracle.partition_sampled(x, w, k, 0.03, order, m, opt)
    b = oracle.partition(x, w, k, 0.03, opt)
    ra, rb = a["result"], b["result"]
    assert oracle.sample_rounds(2 * m, m, 6) == 1
    assert ra["iterations"] == rb["iterations"] and ra["balance_passes"] == rb["balance_passes"]
    assert ra["balanced"] == rb["balanced"] and ra["converged"] == rb["converged"]
    assert np.array_equal(a["A"], b["A"])
    assert np.allclose(a["C"], b["C"], rtol=0, atol=1e-12)
    assert np.allclose(a["I"], b["I"], rtol=1e-12, atol=0)


def test_sampled_depends_on_the_order_only_through_the_sample_sets():
    """Shuffling the order inside each round's new points keeps every sample set, and the
    samples are taken in curve order: bit-identical results.  Moving one point from the
    first sample to the second changes them."""
    n, k, m0 = 5000, 10, 1000
    x = _gmm(n, 3, 13)
    rng = np.random.default_rng(17)
    order = rng.permutation(n)
    opt = oracle.default_options(max_iter=8, threads=2)
    a = oracle.partition_sampled(x, None, k, 0.03, order, m0, opt)
    o2 = order.copy()
    for lo, hi in [(0, 1000), (1000, 2000), (2000, 4000), (4000, 5000)]:
        o2[lo:hi] = rng.permutation(o2[lo:hi])
    b = oracle.partition_sampled(x, None, k, 0.03, o2, m0, opt)
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["C"], b["C"])
    assert a["result"] == b["result"]
    o3 = order.copy()
    o3[[0, 1500]] = o3[[1500, 0]]
    c = oracle.partition_sampled(x, None, k, 0.03, o3, m0, opt)
    assert not np.array_equal(a["C"], c["C"])


def test_sampled_partition_meets_bound_and_is_weighted_voronoi():
    x = _gmm(20_000, 2, 19)
    k = 12
    order = np.random.default_rng(2).permutation(len(x))
    out = oracle.partition_sampled(x, None, k, 0.03, order, 0, oracle.default_options(threads=2))
    res = out["result"]
    assert res["balanced"] == 1
    S, W = oracle.block_weights(out["A"], None, k)
    assert S.max() <= 1.03 * math.ceil(W / k)
    ref, b1, b2 = _effective_argmin(x, out["C"], out["I"])
    clear = (b2 - b1) > 1e-10 * b1
    assert np.array_equal(out["A"][clear], ref[clear])


def test_sampled_rejects_an_order_that_is_not_a_permutation():
    x = _gmm(500, 2, 23)
    order = np.arange(500)
    order[7] = 8
    assert oracle.partition_sampled(x, None, 4, 0.03, order)["result"]["status"] == oracle.OR_INVALID
    order[7] = 500
    assert oracle.partition_sampled(x, None, 4, 0.03, order)["result"]["status"] == oracle.OR_INVALID


# ----------------------------------------------------------------------------------------
# The paper's multi-process semantics (replicated centers, summed local block sizes and
# coordinate sums; Section 4, Algorithm 1 globalSumVector): with exact reductions the
# result does not depend on how the points are cut into process shards.
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("shards", [2, 5, 16])
def test_sharded_reductions_equal_the_global_ones(shards):
    rng = np.random.default_rng(200 + shards)
    n, d, k = 6000, 3, 11
    x = rng.random((n, d)) ** 2
    C = x[rng.choice(n, k, replace=False)]
    I = rng.uniform(0.8, 1.2, k)
    A, _, _ = oracle.assign(x, C, I)
    S_glob, W = oracle.block_weights(A, None, k)
    # each shard (a contiguous range of the curve order, as after the redistribution)
    # assigns its own points against the replicated centers and sums locally
    keys = oracle.hilbert_keys(x)
    order = oracle.sort_keys(keys)
    cuts = np.linspace(0, n, shards + 1).astype(int)
    S = np.zeros(k)
    sums = np.zeros((k, d))
    for a, b in zip(cuts[:-1], cuts[1:]):
        idx = order[a:b]
        As, _, _ = oracle.assign(x[idx], C, I)
        assert np.array_equal(As, A[idx])
        S += np.bincount(As, minlength=k)
        for c in range(k):
            sums[c] += x[idx][As == c].sum(0)
    assert np.array_equal(S, S_glob) and S.sum() == W == n
    C_new, _, _ = oracle.move_centers(x, None, A, C)
    nonempty = S > 0
    assert np.allclose(sums[nonempty] / S[nonempty, None], C_new[nonempty], rtol=1e-13, atol=0)
