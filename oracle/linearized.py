"""The linearised Gaussian smoother of Section 4.1 (Algorithm 4), sequential FP64 (test
infrastructure only).

Algorithm 4 linearises the state-space model around Gaussian marginals q_t = N(m_t, P_t),
smooths the linearised model exactly, and takes the smoothed marginals as the next q_t; the
result serves as the proposals q_t = nu_t of Algorithm 2.  Here the smoothing is the plain
sequential Kalman filter and Rauch-Tung-Striebel smoother (the device runs the same model
through temporally parallel scans).

  * Linear-Gaussian model: the linearisation is the model itself, so one pass gives the
    Kalman/RTS marginals.
  * Poisson counts (Section 5.1): log h_t = y_t x - e^x is expanded in the same way.
  * Theta-logistic (Section 5.2): the observation is linear-Gaussian and the transition mean
    m(x) = x + tau0 - tau1 e^{tau2 x} is linearised around the previous means (the iterated
    extended Kalman smoother the paper uses), first around y_t.
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
    """Kalman filter and RTS smoother of x_t = F_t x_{t-1} + c_t + N(0, Q), x_0 ~ N(m0, P0),
    z_t = x_t + N(0, R_t) observed where obs[t]; F, c are one matrix / vector for every step
    or per-step arrays [K][d][d] / [K][d].  Returns (means [K][d], covariances [K][d][d])."""
    z = np.asarray(z, np.float64)
    K, d = z.shape
    F = np.asarray(F, np.float64)
    c = np.asarray(c, np.float64)
    Ft = F.reshape(K, d, d) if F.size == K * d * d and F.ndim == 3 else np.broadcast_to(F.reshape(d, d), (K, d, d))
    ct = c.reshape(K, d) if c.size == K * d and c.ndim == 2 else np.broadcast_to(c.reshape(d), (K, d))
    Q = np.atleast_2d(Q).astype(np.float64)
    mf = np.zeros((K, d))
    Pf = np.zeros((K, d, d))
    mp = np.zeros((K, d))
    Pp = np.zeros((K, d, d))
    m = np.asarray(m0, np.float64).reshape(d)
    P = np.atleast_2d(P0).astype(np.float64)
    for t in range(K):
        if t > 0:
            m = Ft[t] @ m + ct[t]
            P = Ft[t] @ P @ Ft[t].T + Q
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
        J = Pf[t] @ Ft[t + 1].T @ np.linalg.inv(Pp[t + 1])
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


def cox_pseudo_observations(y, m):
    """The second-order expansion of log h_t = y_t x - e^x around m_t (Poisson counts):
    lambda_t = e^{m_t}, gradient y_t - e^{m_t}; (z, variance, observed)."""
    y = np.asarray(y, np.float64).reshape(-1)
    lam = np.exp(np.asarray(m, np.float64).reshape(-1))
    return m.reshape(-1) + (y - lam) / lam, 1.0 / lam, np.ones(y.shape[0], bool)


def theta_transitions(model, m):
    """The theta-logistic transition into step t linearised around m_{t-1}:
    F_t = 1 - tau1 tau2 e^{tau2 m}, c_t = m + tau0 - tau1 e^{tau2 m} - F_t m."""
    m = np.asarray(m, np.float64).reshape(-1)
    K = m.shape[0]
    F = np.ones((K, 1, 1))
    c = np.zeros((K, 1))
    e = np.exp(model.tau2 * m[:-1])
    F[1:, 0, 0] = 1.0 - model.tau1 * model.tau2 * e
    c[1:, 0] = m[:-1] + model.tau0 - model.tau1 * e - F[1:, 0, 0] * m[:-1]
    return F, c


def linearized_smoother(model, y, iterations=1, init_mean=None):
    """Algorithm 4's Gaussian marginals: (means [K][d], standard deviations [K][d])."""
    y = np.asarray(y, np.float64)
    if model.kind == 0:  # linear-Gaussian
        ms, Ps, _ = kalman.kalman_rts(model.A, model.Q, model.R, model.m0, model.P0, y)
        return ms, np.sqrt(np.einsum("tii->ti", Ps))
    K = y.shape[0]
    s2 = model.sigma ** 2
    if model.kind == 3:  # theta-logistic: linearise the transition, first around y_t
        m = y[:, 0].copy() if init_mean is None else np.asarray(init_mean, np.float64).reshape(K)
        for _ in range(max(1, iterations)):
            F, c = theta_transitions(model, m)
            ms, Ps = kalman_rts_affine(F, c, [[s2]], [0.0], [[1.0]], y, np.full((K, 1, 1), model.obs_sd ** 2),
                                       np.ones(K, bool))
            m = ms[:, 0]
        return ms, np.sqrt(Ps[:, :, 0])
    A = model.phi * (model.lam if model.kind == 2 else 1.0)
    m = np.full(K, model.mu) if init_mean is None else np.asarray(init_mean, np.float64).reshape(K)
    for _ in range(max(1, iterations)):
        z, r, obs = (cox_pseudo_observations if model.kind == 2 else sv_pseudo_observations)(y, m)
        ms, Ps = kalman_rts_affine([[A]], [model.mu * (1 - model.phi)], [[s2]], [model.mu],
                                   [[s2 / (1 - model.phi ** 2)]], z[:, None], r[:, None, None], obs)
        m = ms[:, 0]
    return ms, np.sqrt(Ps[:, :, 0])
