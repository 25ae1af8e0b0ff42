"""The rule of the per-point bounds option (gk_options.bounds), checked in FP64 on the
CPU: inside a phase the centers stay fixed and only the influences change; a point whose
recorded ratio rho (smallest other effective squared distance over its own, at its last
evaluation t1) exceeds (largest growth of any center's 1/I^2 since t1) / (smallest growth)
keeps its block.  Here every pass evaluates all points anyway and the test asserts that
every point the rule would skip indeed kept its argmin, over influence trajectories drawn
like Eq. 1's clamped updates."""
import numpy as np
import pytest


@pytest.mark.parametrize("seed,d,k", [(1, 2, 12), (2, 3, 40), (3, 2, 100)])
def test_skipped_points_keep_their_block(seed, d, k):
    rng = np.random.default_rng(seed)
    n = 4000
    x = rng.random((n, d))
    C = x[rng.choice(n, k, replace=False)]
    D2 = ((x[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    I = np.ones(k)
    g_hist = []
    rho = np.zeros(n)
    t1 = np.zeros(n, dtype=int)
    skipped = 0
    for t in range(40):
        g = 1.0 / I ** 2
        g_hist.append(g.copy())
        E = D2 * g[None, :]
        A = np.argmin(E, 1)
        part = np.partition(E, 1, axis=1)
        if t > 0:
            G = np.array(g_hist)
            ratios = G[1:] / G[:-1]
            lmin = np.concatenate([[0.0], np.cumsum(np.log(ratios.min(1)))])
            lmax = np.concatenate([[0.0], np.cumsum(np.log(ratios.max(1)))])
            thr = np.exp((lmax[t] - lmax[t1]) - (lmin[t] - lmin[t1]))
            skip = rho > thr * (1 + 1e-9)
            assert np.all(A[skip] == A_prev[skip]), "a skipped point changed block"
            skipped += skip.sum()
            ev = ~skip
        else:
            ev = np.ones(n, bool)
        with np.errstate(divide="ignore"):  # a point on a center: rho = inf
            rho[ev] = part[ev, 1] / part[ev, 0]
        t1[ev] = t
        A_prev = np.where(ev, A, A_prev) if t > 0 else A.copy()
        # an Eq. 1 style update: each influence by a factor in [0.95, 1.05]
        I = I * np.clip(rng.normal(1.0, 0.03, k), 0.95, 1.05)
    assert skipped > 0  # the rule does skip points
