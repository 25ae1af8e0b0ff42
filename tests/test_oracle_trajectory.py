"""Hand-worked trajectories of balanced k-means (Algorithm 2 with Algorithm 1, Eq. 1-3)
that pin how the loop composes its steps.

Six points on the x axis, two blocks, eps = 0, unit weights:

    x = -1, 0, 1, 1.95, 4, 5;   C = (0, 0), (4, 0);   I = (1, 1).

Every quantity below is worked out by hand from the paper's definitions (no call of
the oracle's arithmetic): the balance bound is ceil(6/2) = 3 and the target size W/k
is 3; with I = (1, 1) the points -1, 0, 1, 1.95 go to block 0 (1.95 is 1.95 from
center 0 and 2.05 from center 1), so S = (4, 2): unbalanced.  Eq. 1 (oversized blocks
lose influence) gives the factors sqrt(3/4) = 0.866 and sqrt(3/2) = 1.22, clamped to
0.95 and 1.05.  Under I = (0.95, 1.05) the point 1.95 is at effective distance
1.95/0.95 = 2.053 from center 0 and 2.05/1.05 = 1.952 from center 1, so it moves and
S = (3, 3) is balanced.

The erosion of Eq. 2-3 is written here as alpha = tanh(delta / (2 beta)) and
I^(1 - alpha) (the same function as the printed 2/(1 + exp(-delta/beta)) - 1 and
exp((1 - alpha) log I) for delta >= 0), beta the mean bounding-box diagonal of the
non-empty blocks.

What the scenarios fix, each a plausible slip in the loop that the step-level pins
cannot see:
  A  a phase that ends at its pass limit unbalanced: the erosion acts on the influence
     as adapted after that last pass (not on the influence the pass used), and the next
     phase assigns with the eroded value; the last phase does not move the centers;
  B  the same, then the balance-only passes with the centers fixed, until the point
     1.95 moves (a closed form for the number of passes);
  C  a phase whose movement is below the threshold: the loop stops before the erosion,
     the returned centers are those the assignment used, and the final passes start
     from the adapted influence;
  D  a phase that becomes balanced on its second pass, a movement, the erosion and a
     second phase;
  E  (eps = 1, every assignment balanced: Lloyd's algorithm) a last phase whose
     assignment differs from the one before: its moved centers are reported but the
     returned centers are those the last assignment used.
The GPU path runs the same scenarios against the same hand-worked values."""
import math

import numpy as np
import pytest

import oracle

X = np.array([[-1.0, 0.0], [0.0, 0.0], [1.0, 0.0], [1.95, 0.0], [4.0, 0.0], [5.0, 0.0]])
C0 = np.array([[0.0, 0.0], [4.0, 0.0]])
I0 = np.ones(2)
K, EPS = 2, 0.0
CLAMP = np.array([0.95, 1.05])  # the clamped Eq. 1 factors of S = (4, 2)


def _erode(I, delta, beta):
    alpha = np.tanh(np.asarray(delta) / (2.0 * beta))
    return np.asarray(I) ** (1.0 - alpha)


def _expected(name):
    """(options, expected outputs) of scenario name, all worked out by hand."""
    A_before = np.array([0, 0, 0, 0, 1, 1])  # 1.95 with block 0
    A_after = np.array([0, 0, 0, 1, 1, 1])   # 1.95 moved to block 1
    if name in ("A", "B"):
        # phase 1, one pass with I = (1, 1): S = (4, 2), adapted I = (0.95, 1.05)
        # movement: block 0 mean (-1 + 0 + 1 + 1.95)/4 = 0.4875, block 1 mean 4.5;
        # delta = (0.4875, 0.5); diagonals 2.95 and 1, beta = 1.975
        C1 = np.array([[0.4875, 0.0], [4.5, 0.0]])
        Ie = _erode(CLAMP, [0.4875, 0.5], 1.975)
        # phase 2 (the last) assigns with C1 and Ie: 1.95 is 1.4625/Ie0 = 1.53 from
        # center 0 and 2.55/Ie1 = 2.44 from center 1, so A and S do not change; the
        # pass adapts I to Ie * (0.95, 1.05); no movement in the last phase
        if name == "A":
            opt = dict(max_iter=2, max_balance_iter=1, final_balance_iter=0, erosion=1,
                       delta_threshold=0.0)
            out = dict(A=A_before, C=C1, I_used=Ie, I=Ie * CLAMP, C_moved=C1,
                       status=oracle.OR_NOT_BALANCED, iterations=2, passes=2, converged=0,
                       balanced=0, imbalance=4.0 / 3.0 - 1.0, max_delta=0.0)
            return opt, out
        # B: final passes with C1 fixed; pass m uses Ie * (0.95^m, 1.05^m) while S stays
        # (4, 2); 1.95 moves once I1/I0 > 2.55/1.4625, then S = (3, 3)
        r_e = Ie[1] / Ie[0]
        m = math.ceil(math.log((2.55 / 1.4625) / r_e) / math.log(1.05 / 0.95))
        assert m == 5  # and far from a tie: m = 4 and m = 5 bracket the ratio widely
        Im = Ie * CLAMP ** m
        opt = dict(max_iter=2, max_balance_iter=1, final_balance_iter=50, erosion=1,
                   delta_threshold=0.0)
        out = dict(A=A_after, C=C1, I_used=Im, I=Im, C_moved=C1, status=oracle.OR_OK,
                   iterations=2, passes=2 + m, converged=0, balanced=1, imbalance=0.0,
                   max_delta=0.0)
        return opt, out
    if name == "C":
        # phase 1 as in A, movement delta = (0.4875, 0.5) below the threshold 1: stop
        # (converged) before the erosion, centers stay C0; one final pass with
        # I = (0.95, 1.05) moves 1.95: balanced
        opt = dict(max_iter=5, max_balance_iter=1, final_balance_iter=50, erosion=1,
                   delta_threshold=1.0)
        out = dict(A=A_after, C=C0, I_used=CLAMP, I=CLAMP,
                   C_moved=np.array([[0.4875, 0.0], [4.5, 0.0]]), status=oracle.OR_OK,
                   iterations=1, passes=2, converged=1, balanced=1, imbalance=0.0,
                   max_delta=0.5)
        return opt, out
    if name == "D":
        # phase 1: pass 1 unbalanced, pass 2 (I = (0.95, 1.05)) balanced; movement:
        # block 0 mean 0 (delta 0), block 1 mean (1.95 + 4 + 5)/3 = 3.65 (delta 0.35);
        # diagonals 2 and 3.05, beta = 2.525; erosion leaves I0 (delta 0) and shrinks
        # I1 towards 1; phase 2 with C = (0, 3.65): 1.95 stays in block 1 (2.05 against
        # 1.62), S = (3, 3) balanced; the last phase does not move
        C1 = np.array([[0.0, 0.0], [3.65, 0.0]])
        Ie = _erode(CLAMP, [0.0, 0.35], 2.525)
        opt = dict(max_iter=2, max_balance_iter=5, final_balance_iter=0, erosion=1,
                   delta_threshold=0.0)
        out = dict(A=A_after, C=C1, I_used=Ie, I=Ie, C_moved=C1, status=oracle.OR_OK,
                   iterations=2, passes=3, converged=0, balanced=1, imbalance=0.0,
                   max_delta=0.0)
        return opt, out
    if name == "E":
        # eps = 1: the bound 6 is always met, no influence update, erosion of I = 1 stays
        # 1 (Lloyd's algorithm).  From C = (0, 1): block 0 = {-1, 0}, block 1 = {1, 1.95,
        # 4, 5}; means -0.5 and 11.95/4 = 2.9875; phase 2 (the last): 1 is 1.5 from
        # center 0 and 1.9875 from center 1, so it changes block; the moved centers of
        # that phase, 0 and 3.65, are reported but not taken
        opt = dict(max_iter=2, max_balance_iter=5, final_balance_iter=0, erosion=1,
                   delta_threshold=0.0)
        out = dict(A=A_after, C=np.array([[-0.5, 0.0], [2.9875, 0.0]]), I_used=np.ones(2),
                   I=np.ones(2), C_moved=np.array([[0.0, 0.0], [3.65, 0.0]]),
                   status=oracle.OR_OK, iterations=2, passes=2, converged=0, balanced=1,
                   imbalance=0.0, max_delta=0.6625, eps=1.0,
                   C_start=np.array([[0.0, 0.0], [1.0, 0.0]]))
        return opt, out
    raise KeyError(name)


def _check(A, C, I_used, res, out, I=None, C_moved=None):
    assert np.array_equal(np.asarray(A), out["A"])
    assert np.allclose(C, out["C"], rtol=1e-14, atol=1e-14)
    assert np.allclose(I_used, out["I_used"], rtol=1e-13, atol=0)
    if I is not None:
        assert np.allclose(I, out["I"], rtol=1e-13, atol=0)
    if C_moved is not None:
        assert np.allclose(C_moved, out["C_moved"], rtol=1e-14, atol=1e-14)
    assert res["status"] == out["status"]
    assert res["iterations"] == out["iterations"]
    assert res["balance_passes"] == out["passes"]
    assert res["converged"] == out["converged"] and res["balanced"] == out["balanced"]
    assert math.isclose(res["max_imbalance"], out["imbalance"], rel_tol=1e-14, abs_tol=1e-15)
    assert math.isclose(res["max_delta"], out["max_delta"], rel_tol=1e-14, abs_tol=1e-15)


@pytest.mark.parametrize("name", ["A", "B", "C", "D", "E"])
def test_oracle_loop_follows_the_hand_worked_trajectory(name):
    opt, out = _expected(name)
    r = oracle.balanced_kmeans(X, None, K, out.get("eps", EPS), out.get("C_start", C0), I0,
                               oracle.default_options(**opt))
    _check(r["A"], r["C"], r["I_used"], r["result"], out, I=r["I"], C_moved=r["C_moved"])


def test_hand_worked_steps_agree_with_the_step_functions():
    """The single steps behind the scenarios, as the pinned step functions compute them
    (a check of the hand arithmetic above, not of the loop)."""
    A, _, _ = oracle.assign(X, C0, I0)
    assert np.array_equal(A, [0, 0, 0, 0, 1, 1])
    S, W = oracle.block_weights(A, None, K)
    bal, I1, imb = oracle.balance_update(S, W, K, 2, EPS, I0)
    assert not bal and np.array_equal(I1, CLAMP) and math.isclose(imb, 1.0 / 3.0)
    Cn, delta, beta = oracle.move_centers(X, None, A, C0)
    assert np.allclose(Cn, [[0.4875, 0.0], [4.5, 0.0]]) and math.isclose(beta, 1.975)
    assert np.allclose(oracle.erosion(delta, beta, CLAMP), _erode(CLAMP, delta, beta), rtol=1e-14)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["A", "B", "C", "D", "E"])
def test_gpu_loop_follows_the_hand_worked_trajectory(name):
    import torch
    import paper_1805_01208_gb300 as gk
    gk.build()
    torch.cuda.set_device(0)
    opt, out = _expected(name)
    for use_graph in (1, 0):
        o = gk.default_options(use_graph=use_graph, **opt)
        C = torch.from_numpy(out.get("C_start", C0).copy()).cuda()
        I = torch.from_numpy(I0.copy()).cuda()
        block, res = gk.balanced_kmeans(torch.from_numpy(X).cuda(), K, out.get("eps", EPS), C, I,
                                        options=o)
        _check(block.cpu().numpy(), C.cpu().numpy(), I.cpu().numpy(), res, out)
