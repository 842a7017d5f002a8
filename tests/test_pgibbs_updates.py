"""The parameter steps of the particle-Gibbs sampler on the theta-logistic model (Section 3.2,
Section 5.2), CPU only: each draws from its full conditional, checked against that
conditional computed by brute force on a grid (prior times likelihood, normalised
numerically), for fixed trajectories simulated from the model."""
import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

from paper_2202_02264_gb300 import pgibbs as P, workloads as W

PRIOR = P.ThetaPrior()


def _data(K=120, seed=5):
    m = W.theta_logistic()
    x, y = W.simulate(m, K, seed)
    return m, x[:, 0], y[:, 0]


def _grid_moments(logp, g):
    w = np.exp(logp - logsumexp(logp))
    mean = (w * g).sum()
    return mean, (w * (g - mean) ** 2).sum()


def test_r2_conditional():
    m, x, y = _data()
    rng = np.random.default_rng(1)
    s = np.array([P.update_r2(rng, PRIOR, x, y) for _ in range(40000)])
    g = np.linspace(1e-3, 0.5, 20001)
    logp = stats.invgamma(PRIOR.a, scale=PRIOR.b).logpdf(g) + stats.norm(x[:, None], np.sqrt(g)[None, :]).logpdf(
        y[:, None]).sum(0)
    mean, var = _grid_moments(logp, g)
    assert abs(s.mean() - mean) < 5 * np.sqrt(var / s.size)
    assert s.var() == pytest.approx(var, rel=0.05)


def test_tau01_conditional():
    m, x, y = _data()
    rng = np.random.default_rng(2)
    tau2, q2 = m.tau2, m.sigma ** 2
    s = np.array([P.update_tau01(rng, PRIOR, x, tau2, q2) for _ in range(40000)])
    g0 = np.linspace(m.tau0 - 0.6, m.tau0 + 0.6, 301)
    g1 = np.linspace(m.tau1 - 0.6, m.tau1 + 0.6, 301)
    T0, T1 = np.meshgrid(g0, g1, indexing="ij")
    dlt = x[1:] - x[:-1]
    e = np.exp(tau2 * x[:-1])
    res = dlt[None, None, :] - T0[..., None] + T1[..., None] * e[None, None, :]
    logp = (-0.5 * (res ** 2).sum(-1) / q2 - 0.5 * (T0 ** 2 + T1 ** 2) / PRIOR.s_tau ** 2).ravel()
    w = np.exp(logp - logsumexp(logp))
    mean = np.array([(w * T0.ravel()).sum(), (w * T1.ravel()).sum()])
    for k in range(2):
        v = (w * ([T0, T1][k].ravel() - mean[k]) ** 2).sum()
        assert abs(s[:, k].mean() - mean[k]) < 5 * np.sqrt(v / s.shape[0])
        assert s[:, k].var() == pytest.approx(v, rel=0.06)


def test_q2_conditional():
    m, x, y = _data()
    rng = np.random.default_rng(3)
    s = np.array([P.update_q2(rng, PRIOR, x, m.tau0, m.tau1, m.tau2) for _ in range(40000)])
    g = np.linspace(1e-4, 0.2, 20001)
    dlt = x[1:] - x[:-1] - m.tau0 + m.tau1 * np.exp(m.tau2 * x[:-1])
    logp = stats.invgamma(PRIOR.a, scale=PRIOR.b).logpdf(g) + stats.norm(0, np.sqrt(g)[None, :]).logpdf(
        dlt[:, None]).sum(0)
    mean, var = _grid_moments(logp, g)
    assert abs(s.mean() - mean) < 5 * np.sqrt(var / s.size)


def test_tau2_metropolis_hastings_targets_its_conditional():
    m, x, y = _data()
    rng = np.random.default_rng(4)
    q2 = m.sigma ** 2
    t = m.tau2
    chain = []
    for i in range(60000):
        t = P.update_tau2(rng, PRIOR, x, m.tau0, m.tau1, t, q2)
        if i >= 2000:
            chain.append(t)
    chain = np.array(chain)
    g = np.linspace(1e-4, 3.0, 30001)
    logp = np.array([P.log_target_tau2(PRIOR, x, m.tau0, m.tau1, v, q2) for v in g])
    mean, var = _grid_moments(logp, g)
    # correlated chain: batch means for the standard error
    bm = chain[: (chain.size // 50) * 50].reshape(50, -1).mean(1)
    assert abs(chain.mean() - mean) < 5 * bm.std(ddof=1) / np.sqrt(50)
