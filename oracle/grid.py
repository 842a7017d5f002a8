"""Grid forward-backward smoother for one-dimensional models (test infrastructure only).

The stochastic-volatility model has no closed-form smoother.  For d = 1 its smoothing
marginals can be computed to high accuracy by discretising the state on a fine uniform
grid and running the discrete forward-backward recursions (the finite-state case cited in
Section 1 of the paper, Rabiner 1989).  Plain numpy in FP64, log domain.
"""
from __future__ import annotations

import numpy as np
from scipy.special import logsumexp


def sv_grid_smoother(mu, phi, sigma, y, n_grid=2001, width=9.0):
    """Smoothing means E[x_t | y_{0:K-1}] and log p(y) for the SV model on a grid."""
    y = np.asarray(y, np.float64).reshape(-1)
    K = y.shape[0]
    s0 = sigma / np.sqrt(1.0 - phi * phi)
    g = np.linspace(mu - width * s0, mu + width * s0, n_grid)
    dx = g[1] - g[0]
    # transition log-density matrix T[i, j] = log p(g_j | g_i) + log dx
    mean = mu + phi * (g - mu)
    logT = (-0.5 * ((g[None, :] - mean[:, None]) / sigma) ** 2 - np.log(sigma)
            - 0.5 * np.log(2 * np.pi) + np.log(dx))
    logprior = -0.5 * ((g - mu) / s0) ** 2 - np.log(s0) - 0.5 * np.log(2 * np.pi) + np.log(dx)

    def logh(t):
        return -0.5 * np.log(2 * np.pi) - 0.5 * g - 0.5 * y[t] ** 2 * np.exp(-g)

    la = np.zeros((K, n_grid))
    la[0] = logprior + logh(0)
    for t in range(1, K):
        la[t] = logsumexp(la[t - 1][:, None] + logT, axis=0) + logh(t)
    loglik = float(logsumexp(la[-1]))
    lb = np.zeros((K, n_grid))
    for t in range(K - 2, -1, -1):
        lb[t] = logsumexp(logT + (logh(t + 1) + lb[t + 1])[None, :], axis=1)
    lp = la + lb
    lp -= logsumexp(lp, axis=1, keepdims=True)
    p = np.exp(lp)
    means = p @ g
    var = p @ (g * g) - means ** 2
    return means, var, loglik
