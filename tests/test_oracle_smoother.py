"""Pins of the oracle dSMC smoother against closed forms and invariants (CPU only).

dSMC targets the exact smoothing distribution (Propositions 1 and 2), so on
linear-Gaussian models its means converge to the Kalman/RTS means; on the
stochastic-volatility model they converge to the grid forward-backward means.
"""
import numpy as np
import pytest

from oracle import core, grid, kalman
from paper_2202_02264_gb300 import workloads as W


def _seed_means(m, y, K, N, R, **kw):
    return np.array([core.smooth(m, y, K, N, 1000 + r, **kw)["mean"] for r in range(R)])


def _check_against(means, ref, zmax=6.5, cover=0.985):
    """Seed-averaged means against a reference: z = (mean_R - ref) / (sd / sqrt(R)) is
    t-distributed with R - 1 degrees of freedom when dSMC is unbiased at this N.  The number
    of |z| > 3 must stay within a binomial bound of its expectation, no |z| may reach zmax,
    and single runs must fall within 3 sd of the reference at the normal rate."""
    from scipy import stats as _st
    R = means.shape[0]
    sd = means.std(0, ddof=1)
    z = np.abs(means.mean(0) - ref) / (sd / np.sqrt(R))
    n = z.size
    p3 = 2 * _st.t.sf(3.0, R - 1)
    allowed = n * p3 + 4 * np.sqrt(n * p3) + 1
    assert (z > 3).sum() <= allowed, ((z > 3).sum(), allowed)
    assert z.max() < zmax, z.max()
    assert (np.abs(means - ref) <= 3 * sd).mean() >= cover


@pytest.mark.parametrize("nu", [W.NU_EQ_Q, W.NU_PROP_H])
def test_dsmc_matches_rts_1d(nu):
    wl = W.workload("lgssm_1d")
    m = W.lgssm_1d(nu)
    ms, _, _ = kalman.rts_for(m, wl.y)
    _check_against(_seed_means(m, wl.y, wl.K, wl.N, 64), ms)


def test_dsmc_matches_rts_3d_non_power_of_two():
    """Non-symmetric A (a transposed A would fail) and K = 13 (pass-through blocks)."""
    m = W.lgssm_dn(3)
    K, N = 13, 128
    _, y = W.simulate(m, K, 31)
    ms, _, _ = kalman.rts_for(m, y)
    _check_against(_seed_means(m, y, K, N, 48), ms)


def test_dsmc_rejection_matches_rts():
    wl = W.workload("lgssm_1d", K=17, N=64)
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    _check_against(_seed_means(wl.model, wl.y, wl.K, wl.N, 48, resampler="rs"), ms)


@pytest.mark.parametrize("resampler", ["systematic", "rsf"])
def test_dsmc_systematic_and_factorised_match_rts(resampler):
    """Systematic positions and rejection with factorised proposals target the same smoother."""
    wl = W.workload("lgssm_1d", K=17, N=64)
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    _check_against(_seed_means(wl.model, wl.y, wl.K, wl.N, 48, resampler=resampler), ms)


def test_dsmc_factorised_sv_matches_grid():
    K, N = 24, 256
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    gm, _, _ = grid.sv_grid_smoother(m.mu, m.phi, m.sigma, y[:, 0])
    _check_against(_seed_means(m, y, K, N, 32, resampler="rsf"), gm[:, None])


def test_dsmc_metropolis_hastings_near_rts():
    """Algorithm 7 is biased for finite B; with B = 256 steps per slot its seed-averaged means
    sit within a small multiple of the dense sampler's distance from the RTS means."""
    wl = W.workload("lgssm_1d", K=17, N=64)
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    mh = _seed_means(wl.model, wl.y, wl.K, wl.N, 24, resampler="mh", rs_max_attempts=256)
    de = _seed_means(wl.model, wl.y, wl.K, wl.N, 24)
    e_mh = np.sqrt(((mh.mean(0) - ms) ** 2).mean())
    e_de = np.sqrt(((de.mean(0) - ms) ** 2).mean())
    assert e_mh < 2.0 * e_de + 0.02, (e_mh, e_de)


@pytest.mark.parametrize("resampler", ["dense", "rs", "mh", "systematic", "rsf"])
def test_output_values_are_leaf_particles(resampler):
    """Every output trajectory takes, at each time t, one of the N particles drawn at t (the
    stitching of Algorithm 1 only selects), for every sampler; K = 11 has pass-through blocks."""
    wl = W.workload("lgssm_1d", K=11, N=32)
    out = core.smooth(wl.model, wl.y, wl.K, wl.N, 9, resampler=resampler, want_traj=True,
                      rs_max_attempts=(64 if resampler == "mh" else 1 << 20))
    traj, X = out["traj"], out["X_leaf"]
    for t in range(wl.K):
        leaf = {float(v) for v in X[t, :, 0]}
        assert all(float(v) in leaf for v in traj[t, :, 0]), t


def test_dsmc_sv_matches_grid():
    K, N = 24, 256
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    gm, _, _ = grid.sv_grid_smoother(m.mu, m.phi, m.sigma, y[:, 0])
    _check_against(_seed_means(m, y, K, N, 32), gm[:, None])


def test_likelihood_estimate_unbiased():
    """E[L_hat / L] = 1 (the normalising-constant recursion of Eq. (rec-loglik))."""
    wl = W.workload("lgssm_1d", K=8, N=32)
    _, _, ll = kalman.rts_for(wl.model, wl.y)
    r = np.array([np.exp(core.smooth(wl.model, wl.y, wl.K, wl.N, 5000 + s)["logL"] - ll)
                  for s in range(600)])
    assert abs(r.mean() - 1.0) < 4 * r.std(ddof=1) / np.sqrt(len(r))


def test_error_rate_half_order():
    """Proposition 4: the L_p error decays as N^{-1/2}."""
    wl = W.workload("lgssm_1d", K=16)
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    Ns = np.array([16, 64, 256])
    rmse = []
    for N in Ns:
        e = _seed_means(wl.model, wl.y, wl.K, int(N), 32) - ms
        rmse.append(np.sqrt((e ** 2).mean()))
    slope = np.polyfit(np.log(Ns), np.log(rmse), 1)[0]
    assert -0.68 < slope < -0.32, slope


def test_pairs_resolve_to_trajectories():
    """Composing the stored pair arrays top-down over the Algorithm 6 tree reproduces the
    trajectories the explicit copies of Algorithm 1 produce (bit for bit)."""
    m = W.lgssm_dn(2)
    K, N = 11, 8
    _, y = W.simulate(m, K, 4)
    o = core.smooth(m, y, K, N, 77, want_traj=True, want_pairs=True)
    pairs, X, traj = o["pairs"], o["X_leaf"], o["traj"]
    L = core.num_levels(K)
    offs = np.cumsum([0] + [core.merges_at_level(K, l) for l in range(L)])
    for t in range(K):
        sigma = np.arange(N)
        for l in range(L - 1, -1, -1):
            size = 1 << l
            a = (t // (2 * size)) * 2 * size
            if a + size >= K:
                continue                       # passed through at this level
            g = offs[l] + a // (2 * size)
            sigma = pairs[g, 1 if t >= a + size else 0][sigma]
        np.testing.assert_array_equal(traj[t], X[t][sigma])


def test_k1_returns_weighted_leaf():
    m = W.lgssm_1d()
    _, y = W.simulate(m, 1, 3)
    N = 50
    X, lw, lL = core.init(m, y, 1, N, 12)
    o = core.smooth(m, y, 1, N, 12)
    assert o["mean"][0, 0] == pytest.approx((np.exp(lw[0]) * X[0, :, 0]).sum(), abs=1e-12)
    assert o["logL"] == pytest.approx(lL[0], abs=1e-12)


def test_n1_is_concatenation():
    m = W.lgssm_dn(2)
    K = 9
    _, y = W.simulate(m, K, 3)
    o = core.smooth(m, y, K, 1, 5, want_traj=True, want_pairs=True)
    assert (o["pairs"] == 0).all()
    np.testing.assert_array_equal(o["traj"], o["X_leaf"])
    # log L = sum of leaf terms + sum over combinations of log omega at the single pair
    X, lw, lL = core.init(m, y, K, 1, 5)
    inc = 0.0
    L = core.num_levels(K)
    for l in range(L):
        size = 1 << l
        for mm in range(core.merges_at_level(K, l)):
            c = 2 * mm * size + size
            inc += core.logw_matrix(m, y, K, c, X[c - 1], X[c], np.zeros(1), np.zeros(1))[0, 0]
    assert o["logL"] == pytest.approx(lL.sum() + inc, abs=1e-9)


def test_init_weights():
    """Algorithm 2: t = 0 weights h_0 P_0 / q_0, t >= 1 weights nu_t / q_t, normalised;
    proposals N(y_t, 1)."""
    from scipy import stats
    m = W.lgssm_1d()
    K, N = 6, 4000
    _, y = W.simulate(m, K, 8)
    X, lw, lL = core.init(m, y, K, N, 21)
    np.testing.assert_allclose(np.exp(lw).sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(lw[1:], -np.log(N), atol=1e-12)   # nu = q
    np.testing.assert_allclose(lL[1:], 0.0, atol=1e-12)
    x0 = X[0, :, 0]
    raw = (stats.norm(x0, 0.5).logpdf(y[0, 0]) + stats.norm(0, 1).logpdf(x0)
           - stats.norm(y[0, 0], 1).logpdf(x0))
    np.testing.assert_allclose(lw[0], raw - np.logaddexp.reduce(raw), atol=1e-12)
    assert lL[0] == pytest.approx(np.logaddexp.reduce(raw) - np.log(N), abs=1e-12)
    z = (X[:, :, 0] - y[:, :1]).reshape(-1)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_conditional_keeps_reference():
    """Section 3.2: slot 0 is the reference at every combination and in the output."""
    m = W.lgssm_dn(2)
    K, N = 10, 16
    _, y = W.simulate(m, K, 4)
    x_ref = np.random.default_rng(1).standard_normal((K, 2))
    o = core.smooth(m, y, K, N, 3, x_ref=x_ref, want_traj=True)
    assert (o["pairs"][:, :, 0] == 0).all()
    np.testing.assert_array_equal(o["traj"][:, 0, :], x_ref)
    # the next reference is one of the candidate trajectories: every x*_t is a particle
    for t in range(K):
        assert (np.abs(o["X_leaf"][t] - o["x_star"][t]).sum(1) == 0).any()


def test_particle_gibbs_stationary_on_rts():
    """Proposition (Conditional dSMC): the chain x* <- c-dSMC(x*) leaves the smoother
    invariant, so its time averages match the RTS means."""
    m = W.lgssm_1d()
    K, N, S = 8, 16, 1200
    _, y = W.simulate(m, K, 9)
    ms, _, _ = kalman.rts_for(m, y)
    x = np.zeros((K, 1))
    chain = []
    for s in range(S):
        x = core.smooth(m, y, K, N, 42, counter_base=s, x_ref=x)["x_star"]
        chain.append(x[:, 0].copy())
    chain = np.array(chain[100:])
    nb = 20
    bm = chain[: (len(chain) // nb) * nb].reshape(nb, -1, K).mean(1)
    se = bm.std(0, ddof=1) / np.sqrt(nb)
    z = np.abs(bm.mean(0) - ms[:, 0]) / se
    assert z.max() < 4.5, z
