"""Grid forward-backward smoother for one-dimensional models (test infrastructure only).

The stochastic-volatility model and the models of the paper's experiments (Poisson counts,
theta-logistic, constrained random walk) have no closed-form smoother.  For d = 1 their
smoothing marginals can be computed to high accuracy by discretising the state on a fine
uniform grid and running the discrete forward-backward recursions (the finite-state case
cited in Section 1 of the paper, Rabiner 1989).  Plain numpy / scipy in FP64, log domain,
with every density written from the model's definition (not from the oracle's C code).
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


def forward_backward(g, logprior, logT, logh):
    """Smoothing means and variances on the grid g: logprior [n] and logT [n][n] include the
    cell width, logh [K][n] the potentials."""
    K = logh.shape[0]
    n = g.shape[0]
    la = np.zeros((K, n))
    la[0] = logprior + logh[0]
    for t in range(1, K):
        la[t] = logsumexp(la[t - 1][:, None] + logT, axis=0) + logh[t]
    lb = np.zeros((K, n))
    for t in range(K - 2, -1, -1):
        lb[t] = logsumexp(logT + (logh[t + 1] + lb[t + 1])[None, :], axis=1)
    lp = la + lb
    lp -= logsumexp(lp, axis=1, keepdims=True)
    p = np.exp(lp)
    means = p @ g
    return means, p @ (g * g) - means ** 2, float(logsumexp(la[-1]))


def model_grid_smoother(model, y, n_grid=2001, lo=None, hi=None):
    """Grid smoothing means / variances / log p(y) of a one-dimensional workloads.SSM
    (linear-Gaussian, SV, Poisson counts, theta-logistic, constrained random walk)."""
    from scipy import stats
    y = np.asarray(y, np.float64).reshape(-1)
    K = y.shape[0]
    kind = model.kind
    if kind == 0:
        A, Q = float(np.atleast_2d(model.A)[0, 0]), float(np.atleast_2d(model.Q)[0, 0])
        mean_fn = lambda x: A * x
        sd = np.sqrt(Q)
        prior = stats.norm(float(np.ravel(model.m0)[0]), np.sqrt(float(np.atleast_2d(model.P0)[0, 0])))
        Rsd = np.sqrt(float(np.atleast_2d(model.R)[0, 0]))
        logh_fn = lambda t, x: stats.norm(x, Rsd).logpdf(y[t])
    elif kind in (1, 2):
        lam = model.lam if kind == 2 else 1.0
        mean_fn = lambda x: model.mu + model.phi * (lam * x - model.mu)
        sd = model.sigma
        prior = stats.norm(model.mu, model.sigma / np.sqrt(1.0 - model.phi ** 2))
        if kind == 1:
            logh_fn = lambda t, x: stats.norm(0.0, np.exp(x / 2)).logpdf(y[t])
        else:
            logh_fn = lambda t, x: stats.poisson(np.exp(x)).logpmf(y[t])
    elif kind == 3:
        mean_fn = lambda x: x + model.tau0 - model.tau1 * np.exp(model.tau2 * x)
        sd = model.sigma
        prior = stats.norm(0.0, 1.0)
        logh_fn = lambda t, x: stats.norm(x, model.obs_sd).logpdf(y[t])
    elif kind == 4:
        mean_fn = lambda x: x
        sd = model.sigma
        prior = stats.norm(0.0, 1.0)
        logh_fn = lambda t, x: np.where(np.abs(x) <= model.bound, 0.0, -np.inf)
    else:
        raise ValueError(kind)
    if lo is None or hi is None:
        if kind == 4:
            lo, hi = -model.bound, model.bound
        elif kind in (1, 2):
            s0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
            c0 = model.mu if kind == 1 else model.mu * (1 - model.phi) / (1 - model.phi * model.lam)
            lo, hi = c0 - 9 * s0, c0 + 9 * s0
        else:
            lo, hi = y.min() - 6.0, y.max() + 6.0
    g = np.linspace(lo, hi, n_grid)
    dx = g[1] - g[0]
    logT = stats.norm(mean_fn(g)[:, None], sd).logpdf(g[None, :]) + np.log(dx)
    logprior = prior.logpdf(g) + np.log(dx)
    logh = np.stack([logh_fn(t, g) for t in range(K)])
    return forward_backward(g, logprior, logT, logh)
