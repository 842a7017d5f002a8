"""Pins of the oracle's random numbers, model densities and closed forms (CPU only)."""
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import core, kalman
from paper_2202_02264_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox4x32-10 against its published known-answer vectors."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = core.philox(r[0:4], r[4:6])
        assert list(out) == r[6:10]


def test_philox_uniformity():
    """Words of consecutive counters are uniform and uncorrelated (chi-square on bytes)."""
    ctr = np.zeros((50000, 4), np.uint32)
    ctr[:, 0] = np.arange(50000)
    ctr[:, 1] = 7
    out = core.philox_many(ctr, [0x1234, 0x5678])
    b = out.view(np.uint8).reshape(-1)
    h = np.bincount(b, minlength=256)
    assert stats.chisquare(h).pvalue > 1e-4
    u = (out[:, 0] >> 8).astype(np.float64) / 2**24
    v = (out[:, 1] >> 8).astype(np.float64) / 2**24
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.02


def _lg(d):
    return W.lgssm_dn(d) if d > 1 else W.lgssm_1d()


@pytest.mark.parametrize("d", [1, 3])
def test_model_densities_against_scipy(d):
    m = _lg(d)
    K = 5
    _, y = W.simulate(m, K, 11)
    rng = np.random.default_rng(0)
    for t in range(K):
        xp, x = rng.standard_normal(d), rng.standard_normal(d)
        lf, lh, lnu, lq, lfmax = core.model_logdens(m, y, K, t, xp, x)
        assert lf == pytest.approx(stats.multivariate_normal(m.A @ xp, m.Q).logpdf(x), abs=1e-12)
        assert lh == pytest.approx(stats.multivariate_normal(x, m.R).logpdf(y[t]), abs=1e-12)
        assert lq == pytest.approx(stats.norm(y[t], m.prop_scale).logpdf(x).sum(), abs=1e-12)
        assert lnu == pytest.approx(lq, abs=1e-12)  # nu_t = q_t
        assert lfmax == pytest.approx(stats.multivariate_normal(np.zeros(d), m.Q).logpdf(np.zeros(d)), abs=1e-12)
    # nu_t proportional to h_t: N(x; y_t, R)
    m2 = _lg(d)
    m2.nu = W.NU_PROP_H
    x = rng.standard_normal(d)
    _, lh, lnu, _, _ = core.model_logdens(m2, y, K, 2, x, x)
    assert lnu == pytest.approx(stats.multivariate_normal(y[2], m2.R).logpdf(x), abs=1e-12)


def test_sv_densities_and_nu_normaliser():
    K = 4
    m = W.sv(K)
    _, y = W.simulate(m, K, 5)
    xp, x = np.array([-0.7]), np.array([-1.3])
    lf, lh, lnu, lq, lfmax = core.model_logdens(m, y, K, 1, xp, x)
    assert lf == pytest.approx(stats.norm(m.mu + m.phi * (xp[0] - m.mu), m.sigma).logpdf(x[0]), abs=1e-12)
    assert lh == pytest.approx(stats.norm(0, np.exp(x[0] / 2)).logpdf(y[1, 0]), abs=1e-12)
    s0 = m.sigma / np.sqrt(1 - m.phi**2)
    assert lq == pytest.approx(stats.norm(m.mu, s0).logpdf(x[0]), abs=1e-12)
    assert lfmax == pytest.approx(stats.norm(0, m.sigma).logpdf(0.0), abs=1e-12)
    # nu proportional to h: the normaliser is the integral of h_t over x, 1/|y_t|
    m.nu = W.NU_PROP_H
    _, lh, lnu, _, _ = core.model_logdens(m, y, K, 1, xp, x)
    Z, _ = integrate.quad(lambda s: stats.norm(0, np.exp(s / 2)).pdf(y[1, 0]), -40, 40, limit=400)
    assert lnu == pytest.approx(lh - np.log(Z), abs=1e-7)


def _dense_gaussian_posterior(A, Q, R, m0, P0, y):
    """Smoothing moments by conditioning the joint Gaussian of (x_{0:K-1}, y_{0:K-1})."""
    K, d = y.shape
    cov = np.zeros((K * d, K * d))
    V = [P0]
    for t in range(1, K):
        V.append(A @ V[-1] @ A.T + Q)
    for t in range(K):
        for s in range(t + 1):
            c = np.linalg.matrix_power(A, t - s) @ V[s]   # Cov(x_t, x_s)
            cov[t*d:(t+1)*d, s*d:(s+1)*d] = c
            cov[s*d:(s+1)*d, t*d:(t+1)*d] = c.T
    mu = np.concatenate([np.linalg.matrix_power(A, t) @ m0 for t in range(K)])
    Syy = cov + np.kron(np.eye(K), R)
    g = np.linalg.solve(Syy, y.reshape(-1) - mu)
    post_mean = mu + cov @ g
    post_cov = cov - cov @ np.linalg.solve(Syy, cov)
    ll = stats.multivariate_normal(mu, Syy).logpdf(y.reshape(-1))
    return post_mean.reshape(K, d), post_cov, ll


@pytest.mark.parametrize("d", [1, 3])
def test_kalman_rts_against_dense_conditioning(d):
    m = _lg(d)
    K = 7
    _, y = W.simulate(m, K, 3)
    ms, Ps, ll = kalman.rts_for(m, y)
    pm, pc, ll2 = _dense_gaussian_posterior(m.A, m.Q, m.R, m.m0, m.P0, y)
    np.testing.assert_allclose(ms, pm, atol=1e-10)
    for t in range(K):
        np.testing.assert_allclose(Ps[t], pc[t*d:(t+1)*d, t*d:(t+1)*d], atol=1e-10)
    assert ll == pytest.approx(ll2, abs=1e-9)


def test_grid_smoother_against_quadrature():
    """The grid forward-backward routine against direct quadrature of the K = 1 and K = 2
    posteriors of the stochastic-volatility model, before it serves as its reference."""
    from oracle import grid
    mu, phi, sigma = -1.0, 0.95, 0.3
    y = np.array([0.3, -0.2, 0.5])
    means, var, ll = grid.sv_grid_smoother(mu, phi, sigma, y, n_grid=4001)
    means2, var2, ll2 = grid.sv_grid_smoother(mu, phi, sigma, y, n_grid=1001)
    np.testing.assert_allclose(means, means2, atol=1e-6)   # grid-converged
    s0 = sigma / np.sqrt(1 - phi**2)
    c = 1.0 / np.sqrt(2 * np.pi)
    p0 = lambda x: c / s0 * np.exp(-0.5 * ((x - mu) / s0) ** 2)
    h = lambda t, x: c * np.exp(-0.5 * x - 0.5 * y[t] ** 2 * np.exp(-x))
    f = lambda xn, x: c / sigma * np.exp(-0.5 * ((xn - mu - phi * (x - mu)) / sigma) ** 2)
    Z, _ = integrate.quad(lambda x: p0(x) * h(0, x), -15, 10, limit=400)
    M, _ = integrate.quad(lambda x: x * p0(x) * h(0, x), -15, 10, limit=400)
    m1, _, ll1 = grid.sv_grid_smoother(mu, phi, sigma, y[:1], n_grid=4001)
    assert m1[0] == pytest.approx(M / Z, abs=1e-6)
    assert ll1 == pytest.approx(np.log(Z), abs=1e-6)
    joint = lambda x1, x0: p0(x0) * h(0, x0) * f(x1, x0) * h(1, x1)
    lo, hi = mu - 8 * s0, mu + 8 * s0
    Z2, _ = integrate.dblquad(joint, lo, hi, lo, hi, epsabs=1e-10)
    M0, _ = integrate.dblquad(lambda x1, x0: x0 * joint(x1, x0), lo, hi, lo, hi, epsabs=1e-10)
    M1, _ = integrate.dblquad(lambda x1, x0: x1 * joint(x1, x0), lo, hi, lo, hi, epsabs=1e-10)
    m2, _, ll2 = grid.sv_grid_smoother(mu, phi, sigma, y[:2], n_grid=4001)
    assert m2[0] == pytest.approx(M0 / Z2, abs=1e-5)
    assert m2[1] == pytest.approx(M1 / Z2, abs=1e-5)
    assert ll2 == pytest.approx(np.log(Z2), abs=1e-5)
