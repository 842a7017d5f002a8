"""Brute force on the output trajectories: K = 3, N = 2 with fixed particles.  Level 0
combines steps 0 and 1 (two iid pair draws, Algorithm 1); level 1 combines that block with
the leaf at t = 2 (Algorithm 6: step 2 passes through level 0).  The law of one output
slot's trajectory (i0, i1, i2) is summed exactly over the 16 possible level-0 outputs; the
oracle's log-weights (Eq. normalized-weights) and dense draws, composed over the two levels
as Algorithm 1 stitches them, must reproduce it."""
import itertools

import numpy as np
from scipy import stats

from oracle import core
from paper_2202_02264_gb300 import workloads as W


def _setup():
    m = W.lgssm_1d()
    K, N = 3, 2
    _, y = W.simulate(m, K, 77)
    X = np.array([[[-0.4], [0.9]], [[0.2], [-1.1]], [[1.3], [0.1]]])     # [K][N][d]
    lw = np.log(np.array([[0.3, 0.7], [0.5, 0.5], [0.5, 0.5]]))         # leaf weights
    return m, y, K, N, X, lw


def _level1(m, y, K, X, lw, tau):
    """logW of the root combination given the level-0 output trajectories tau[l] = (i0, i1):
    the left block's end states are X_1[i1], its weights uniform."""
    N = len(tau)
    xl = np.array([X[1][t[1]] for t in tau])
    return core.logw_matrix(m, y, K, 2, xl, X[2], np.full(N, -np.log(N)), lw[2])


def _exact(m, y, K, N, X, lw):
    W0 = core.logw_matrix(m, y, K, 1, X[0], X[1], lw[0], lw[1])
    P0 = np.exp(W0 - W0.max())
    P0 /= P0.sum()
    law = np.zeros((N, N, N))
    pairs = [(i, j) for i in range(N) for j in range(N)]
    for tau in itertools.product(pairs, repeat=N):
        p_tau = np.prod([P0[t] for t in tau])
        W1 = _level1(m, y, K, X, lw, tau)
        P1 = np.exp(W1 - W1.max())
        P1 /= P1.sum()
        for l in range(N):
            for r in range(N):
                law[tau[l][0], tau[l][1], r] += p_tau * P1[l, r]
    return law


def test_output_trajectory_law_by_enumeration():
    m, y, K, N, X, lw = _setup()
    law = _exact(m, y, K, N, X, lw)
    assert abs(law.sum() - 1.0) < 1e-12
    W0 = core.logw_matrix(m, y, K, 1, X[0], X[1], lw[0], lw[1])
    R = 20000
    counts = np.zeros((N, N, N))
    for rep in range(R):
        li, ri = core.dense_pairs(W0, 123, 2 * rep, 0, N)             # level 0, both slots
        tau = [(int(li[n]), int(ri[n])) for n in range(N)]
        l1, r1 = core.dense_pairs(_level1(m, y, K, X, lw, tau), 123, 2 * rep + 1, 0, 1)   # slot 0
        t = tau[int(l1[0])]
        counts[t[0], t[1], int(r1[0])] += 1
    exp = law.ravel() * R
    keep = exp > 0
    assert counts.ravel()[~keep].sum() == 0
    assert stats.chisquare(counts.ravel()[keep], exp[keep]).pvalue > 1e-3
