"""Pins of the oracle on the models of the paper's experiments (CPU only): the Poisson-count
model of Section 5.1, the theta-logistic model of Section 5.2 and the constrained random walk
of Section 5.3 (with the uniform proposal on the constraint).

  * Densities: the oracle's log p, log h, log P_0 and log q against scipy.
  * The generic grid smoother reproduces Kalman/RTS on the linear-Gaussian model and the
    dedicated stochastic-volatility grid.
  * dSMC means against the grid smoother over seeds (Monte Carlo rule), every resampler.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import core, grid, kalman
from paper_2202_02264_gb300 import workloads as W

from test_oracle_smoother import _check_against, _seed_means


def test_densities_against_scipy():
    rng = np.random.default_rng(2)
    K = 6
    for m in (W.cox(K), W.theta_logistic(), W.crw()):
        _, y = W.simulate(m, K, 3)
        for _ in range(5):
            t = int(rng.integers(1, K))
            xp, x = rng.normal(0.2, 0.6, 2)
            f, h, nu, q, fmax = core.model_logdens(m, y, K, t, np.array([xp]), np.array([x]))
            if m.kind == W.COX:
                mean = m.mu + m.phi * (m.lam * xp - m.mu)
                hh = stats.poisson(np.exp(x)).logpmf(y[t, 0])
            elif m.kind == W.THETA_LOGISTIC:
                mean = xp + m.tau0 - m.tau1 * np.exp(m.tau2 * xp)
                hh = stats.norm(x, m.obs_sd).logpdf(y[t, 0])
            else:
                mean = xp
                hh = 0.0 if abs(x) <= m.bound else -np.inf
            assert f == pytest.approx(stats.norm(mean, m.sigma).logpdf(x), abs=1e-12)
            assert h == pytest.approx(hh, abs=1e-12) or (h == hh == -np.inf)
            assert fmax == pytest.approx(stats.norm(0, m.sigma).logpdf(0), abs=1e-12)
            if m.prop_kind == W.PROP_UNIFORM:
                qq = -np.log(2 * m.prop_scale) if abs(x) <= m.prop_scale else -np.inf
            elif m.prop_kind == W.PROP_GAUSS:
                qq = stats.norm(m.prop_mean[t, 0], m.prop_std[t, 0]).logpdf(x)
            else:
                qq = stats.norm(y[t, 0], m.prop_scale).logpdf(x)
            assert q == pytest.approx(qq, abs=1e-12) or (q == qq == -np.inf)


def test_generic_grid_reproduces_kalman_and_the_sv_grid():
    m = W.lgssm_1d()
    _, y = W.simulate(m, 12, 5)
    ms, Ps, ll = kalman.rts_for(m, y)
    gm, gv, gll = grid.model_grid_smoother(m, y[:, 0], n_grid=3001, lo=-12, hi=12)
    np.testing.assert_allclose(gm, ms[:, 0], atol=1e-6)
    np.testing.assert_allclose(gv, Ps[:, 0, 0], atol=1e-6)
    assert gll == pytest.approx(ll, abs=1e-6)
    sv = W.sv(16)
    _, ys = W.simulate(sv, 16, 9)
    a = grid.sv_grid_smoother(sv.mu, sv.phi, sv.sigma, ys[:, 0])
    b = grid.model_grid_smoother(sv, ys[:, 0])
    np.testing.assert_allclose(a[0], b[0], atol=1e-8)


@pytest.mark.parametrize("name", ["cox", "theta_logistic", "crw"])
@pytest.mark.parametrize("resampler", ["dense", "rsf"])
def test_dsmc_matches_grid_on_the_paper_models(name, resampler):
    wl = W.workload(name, K=24, N=256)
    gm, _, _ = grid.model_grid_smoother(wl.model, wl.y[:, 0])
    _check_against(_seed_means(wl.model, wl.y, wl.K, wl.N, 32, resampler=resampler), gm[:, None])


def test_uniform_proposal_particles_inside_the_constraint():
    wl = W.workload("crw", K=8, N=500)
    X, lw, _ = core.init(wl.model, wl.y, 8, 500, 3)
    assert (np.abs(X) <= wl.model.bound).all()
    # t >= 1, nu_t = q_t: every leaf weight is 1 / N
    np.testing.assert_allclose(lw[1:], -np.log(500), atol=1e-12)


def test_all_zero_weights_are_reported_as_degenerate():
    """Every particle outside the constraint: the combination's weights are all zero, which
    the oracle reports instead of dividing by a zero sum."""
    import dataclasses
    m = dataclasses.replace(W.crw(sigma=0.4, bound=1e-3), prop_scale=1.0)
    with pytest.raises(RuntimeError, match="degenerate"):
        core.smooth(m, np.zeros((4, 1)), 4, 16, 5)
