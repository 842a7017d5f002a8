"""Pins of the oracle's linearised Gaussian smoother (Section 4.1, Algorithm 4), CPU only.

  * The affine Kalman filter and RTS smoother with time-varying observation noise and
    missing observations equals Gaussian conditioning of the joint law of (x_{0:K-1}, z)
    written out densely.
  * For the stochastic-volatility model the iteration's fixed point is the posterior mode:
    the gradient of the log joint density (written out by hand) vanishes there, and the
    smoothed variances are the diagonal of the inverse negative Hessian at the mode.
  * The same fixed-point property for the Poisson-count model (second-order observation
    expansion) and the theta-logistic model (iterated extended smoother).
"""
import numpy as np

from oracle import linearized
from paper_2202_02264_gb300 import workloads as W


def _dense_conditioning(F, c, Q, m0, P0, z, R, obs):
    K, d = z.shape
    mu = np.zeros((K, d))
    V = np.zeros((K, d, d))
    mu[0], V[0] = m0, P0
    for t in range(1, K):
        mu[t] = F @ mu[t - 1] + c
        V[t] = F @ V[t - 1] @ F.T + Q
    S = np.zeros((K * d, K * d))
    for t in range(K):
        for s in range(t + 1):
            B = np.linalg.matrix_power(F, t - s) @ V[s]   # Cov(x_t, x_s)
            S[t * d:(t + 1) * d, s * d:(s + 1) * d] = B
            S[s * d:(s + 1) * d, t * d:(t + 1) * d] = B.T
    idx = np.concatenate([np.arange(t * d, (t + 1) * d) for t in range(K) if obs[t]])
    Rb = np.zeros((len(idx), len(idx)))
    o = 0
    for t in range(K):
        if obs[t]:
            Rb[o:o + d, o:o + d] = R[t]
            o += d
    Szz = S[np.ix_(idx, idx)] + Rb
    Sxz = S[:, idx]
    G = Sxz @ np.linalg.inv(Szz)
    mean = mu.reshape(-1) + G @ (z.reshape(-1)[idx] - mu.reshape(-1)[idx])
    cov = S - G @ Sxz.T
    return mean.reshape(K, d), np.stack([cov[t * d:(t + 1) * d, t * d:(t + 1) * d] for t in range(K)])


def test_affine_kalman_rts_equals_dense_conditioning():
    rng = np.random.default_rng(3)
    K, d = 7, 2
    F = np.array([[0.7, 0.2], [-0.1, 0.9]])
    c = np.array([0.3, -0.2])
    Q = np.array([[1.0, 0.3], [0.3, 0.5]])
    m0 = np.array([0.1, -0.4])
    P0 = np.array([[2.0, 0.4], [0.4, 1.0]])
    z = rng.standard_normal((K, d))
    R = np.stack([np.diag(rng.uniform(0.2, 2.0, d)) for _ in range(K)])
    obs = np.array([True, True, False, True, True, False, True])
    ms, Ps = linearized.kalman_rts_affine(F, c, Q, m0, P0, z, R, obs)
    md, Pd = _dense_conditioning(F, c, Q, m0, P0, z, R, obs)
    np.testing.assert_allclose(ms, md, atol=1e-11)
    np.testing.assert_allclose(Ps, Pd, atol=1e-11)


def _sv_grad_and_neg_hessian(model, y, x):
    mu, phi, s2 = model.mu, model.phi, model.sigma ** 2
    s02 = s2 / (1 - phi * phi)
    K = x.size
    g = np.zeros(K)
    h = np.zeros((K, K))
    g[0] -= (x[0] - mu) / s02
    h[0, 0] += 1 / s02
    for t in range(1, K):
        r = x[t] - mu - phi * (x[t - 1] - mu)
        g[t] -= r / s2
        g[t - 1] += phi * r / s2
        h[t, t] += 1 / s2
        h[t - 1, t - 1] += phi * phi / s2
        h[t, t - 1] -= phi / s2
        h[t - 1, t] -= phi / s2
    e = 0.5 * y * y * np.exp(-x)
    g += -0.5 + e
    h[np.diag_indices(K)] += e
    return g, h


def test_sv_iteration_converges_to_the_posterior_mode():
    K = 64
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    y = y[:, 0]
    ms, sd = linearized.linearized_smoother(m, y[:, None], iterations=60)
    g, h = _sv_grad_and_neg_hessian(m, y, ms[:, 0])
    assert np.abs(g).max() < 1e-8, np.abs(g).max()
    var = np.diag(np.linalg.inv(h))
    np.testing.assert_allclose(sd[:, 0] ** 2, var, rtol=1e-8)
    # a single pass from the stationary mean is not yet the mode
    ms1, _ = linearized.linearized_smoother(m, y[:, None], iterations=1)
    g1, _ = _sv_grad_and_neg_hessian(m, y, ms1[:, 0])
    assert np.abs(g1).max() > 1e-3


def test_sv_warm_start_is_a_continuation():
    """Starting from the result of j passes and running i more equals i + j passes."""
    K = 32
    m = W.sv(K)
    _, y = W.simulate(m, K, 11)
    a, sa = linearized.linearized_smoother(m, y, iterations=5)
    b0, _ = linearized.linearized_smoother(m, y, iterations=2)
    b, sb = linearized.linearized_smoother(m, y, iterations=3, init_mean=b0[:, 0])
    np.testing.assert_allclose(a, b, atol=1e-12)
    np.testing.assert_allclose(sa, sb, atol=1e-12)


def _theta_grad(model, y, x):
    """Gradient of the theta-logistic log joint density, written out by hand."""
    K = x.size
    s2, r2 = model.sigma ** 2, model.obs_sd ** 2
    g = np.zeros(K)
    g[0] -= x[0]
    e = np.exp(model.tau2 * x[:-1])
    res = x[1:] - (x[:-1] + model.tau0 - model.tau1 * e)
    g[1:] -= res / s2
    g[:-1] += res * (1.0 - model.tau1 * model.tau2 * e) / s2
    g += (y - x) / r2
    return g


def _cox_grad(model, y, x):
    mu, phi, lam, s2 = model.mu, model.phi, model.lam, model.sigma ** 2
    K = x.size
    g = np.zeros(K)
    g[0] -= (x[0] - mu) * (1 - phi * phi) / s2
    res = x[1:] - (mu + phi * (lam * x[:-1] - mu))
    g[1:] -= res / s2
    g[:-1] += res * phi * lam / s2
    g += y - np.exp(x)
    return g


def test_theta_logistic_iterated_extended_smoother_converges_to_the_mode():
    m = W.theta_logistic()
    K = 60
    _, y = W.simulate(m, K, 41)
    ms, _ = linearized.linearized_smoother(m, y, iterations=40)
    assert np.abs(_theta_grad(m, y[:, 0], ms[:, 0])).max() < 1e-8


def test_cox_iterated_smoother_converges_to_the_mode():
    m = W.cox(80)
    _, y = W.simulate(m, 80, 40)
    ms, _ = linearized.linearized_smoother(m, y, iterations=40)
    assert np.abs(_cox_grad(m, y[:, 0], ms[:, 0])).max() < 1e-8
