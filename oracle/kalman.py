"""Kalman filter and Rauch-Tung-Striebel smoother (test infrastructure only).

The linear-Gaussian model of the workloads, x_t = A x_{t-1} + N(0, Q), y_t = x_t + N(0, R),
x_0 ~ N(m0, P0), has a closed-form smoothing distribution (Kalman 1960; Rauch, Tung and
Striebel 1965, cited in Section 1 of the paper).  dSMC targets it exactly (Propositions 1
and 2), so these moments pin the oracle and the device path on linear-Gaussian inputs.
Plain textbook recursions in FP64.
"""
from __future__ import annotations

import numpy as np


def kalman_rts(A, Q, R, m0, P0, y):
    """Return (smoothed means [K][d], smoothed covariances [K][d][d], log p(y_{0:K-1}))."""
    y = np.asarray(y, np.float64)
    K, d = y.shape
    A = np.atleast_2d(A)
    mf = np.zeros((K, d))
    Pf = np.zeros((K, d, d))
    mp = np.zeros((K, d))
    Pp = np.zeros((K, d, d))
    loglik = 0.0
    m, P = np.asarray(m0, np.float64).reshape(d), np.atleast_2d(P0).astype(np.float64)
    for t in range(K):
        if t > 0:
            m = A @ m
            P = A @ P @ A.T + Q
        mp[t], Pp[t] = m, P
        S = P + R
        v = y[t] - m
        Sinv = np.linalg.inv(S)
        G = P @ Sinv
        _, logdet = np.linalg.slogdet(2.0 * np.pi * S)
        loglik += -0.5 * (logdet + v @ Sinv @ v)
        m = m + G @ v
        P = P - G @ S @ G.T
        P = 0.5 * (P + P.T)
        mf[t], Pf[t] = m, P
    ms = mf.copy()
    Ps = Pf.copy()
    for t in range(K - 2, -1, -1):
        J = Pf[t] @ A.T @ np.linalg.inv(Pp[t + 1])
        ms[t] = mf[t] + J @ (ms[t + 1] - mp[t + 1])
        Ps[t] = Pf[t] + J @ (Ps[t + 1] - Pp[t + 1]) @ J.T
    return ms, Ps, loglik


def rts_for(model, y):
    """Kalman/RTS of a workloads.SSM linear-Gaussian model."""
    return kalman_rts(model.A, model.Q, model.R, model.m0, model.P0, y)
