"""The linearised Gaussian smoother of Section 4.1 (Algorithm 4), sequential FP64 (test
infrastructure only).

Algorithm 4 linearises the state-space model around Gaussian marginals q_t = N(m_t, P_t),
smooths the linearised model exactly, and takes the smoothed marginals as the next q_t; the
result serves as the proposals q_t = nu_t of Algorithm 2.  Here the smoothing is the plain
sequential Kalman filter and Rauch-Tung-Striebel smoother (the device runs the same model
through temporally parallel scans).

  * Linear-Gaussian model: the linearisation is the model itself, so one pass gives the
    Kalman/RTS marginals.
  * Stochastic volatility (y_t = exp(x_t / 2) v_t): the observation noise is not additive;
    each pass expands log h_t(y_t | x) = -x/2 - y_t^2 e^{-x} / 2 + const to second order
    around m_t, which is the Gaussian pseudo-observation z_t = m_t + g_t / lambda_t with
    variance 1 / lambda_t, where g_t = -1/2 + lambda_t and lambda_t = y_t^2 e^{-m_t} / 2 (no
    observation where lambda_t vanishes).  A fixed point of the iteration is the posterior
    mode, with the inverse negative Hessian there as covariance.
"""
from __future__ import annotations

import numpy as np

from . import kalman


def kalman_rts_affine(F, c, Q, m0, P0, z, R, obs):
    """Kalman filter and RTS smoother of x_t = F x_{t-1} + c + N(0, Q), x_0 ~ N(m0, P0),
    z_t = x_t + N(0, R_t) observed where obs[t].  Returns (means [K][d], covariances
    [K][d][d])."""
    z = np.asarray(z, np.float64)
    K, d = z.shape
    F = np.atleast_2d(F).astype(np.float64)
    Q = np.atleast_2d(Q).astype(np.float64)
    c = np.asarray(c, np.float64).reshape(d)
    mf = np.zeros((K, d))
    Pf = np.zeros((K, d, d))
    mp = np.zeros((K, d))
    Pp = np.zeros((K, d, d))
    m = np.asarray(m0, np.float64).reshape(d)
    P = np.atleast_2d(P0).astype(np.float64)
    for t in range(K):
        if t > 0:
            m = F @ m + c
            P = F @ P @ F.T + Q
        mp[t], Pp[t] = m, P
        if obs[t]:
            S = P + np.atleast_2d(R[t])
            G = P @ np.linalg.inv(S)
            m = m + G @ (z[t] - m)
            P = P - G @ S @ G.T
            P = 0.5 * (P + P.T)
        mf[t], Pf[t] = m, P
    ms, Ps = mf.copy(), Pf.copy()
    for t in range(K - 2, -1, -1):
        J = Pf[t] @ F.T @ np.linalg.inv(Pp[t + 1])
        ms[t] = mf[t] + J @ (ms[t + 1] - mp[t + 1])
        Ps[t] = Pf[t] + J @ (Ps[t + 1] - Pp[t + 1]) @ J.T
    return ms, Ps


def sv_pseudo_observations(y, m):
    """The second-order expansion of log h_t around m_t: (z, variance, observed)."""
    y = np.asarray(y, np.float64).reshape(-1)
    lam = 0.5 * y * y * np.exp(-np.asarray(m, np.float64).reshape(-1))
    obs = (lam > 1e-300) & np.isfinite(lam)
    safe = np.where(obs, lam, 1.0)
    z = np.where(obs, m.reshape(-1) + (lam - 0.5) / safe, 0.0)
    return z, 1.0 / safe, obs


def linearized_smoother(model, y, iterations=1, init_mean=None):
    """Algorithm 4's Gaussian marginals: (means [K][d], standard deviations [K][d])."""
    y = np.asarray(y, np.float64)
    if model.kind == 0:  # linear-Gaussian
        ms, Ps, _ = kalman.kalman_rts(model.A, model.Q, model.R, model.m0, model.P0, y)
        return ms, np.sqrt(np.einsum("tii->ti", Ps))
    K = y.shape[0]
    s2 = model.sigma ** 2
    m = np.full(K, model.mu) if init_mean is None else np.asarray(init_mean, np.float64).reshape(K)
    for _ in range(max(1, iterations)):
        z, r, obs = sv_pseudo_observations(y, m)
        ms, Ps = kalman_rts_affine([[model.phi]], [model.mu * (1 - model.phi)], [[s2]], [model.mu],
                                   [[s2 / (1 - model.phi ** 2)]], z[:, None], r[:, None, None], obs)
        m = ms[:, 0]
    return ms, np.sqrt(Ps[:, :, 0])
