"""The parallel-in-time linearised Gaussian smoother (Section 4.1, Algorithm 4) on the device,
through the C ABI, against the oracle's sequential FP64 smoother; and dSMC with its
marginals as proposals q_t = nu_t (DSMC_PROP_GAUSS): the same smoother (RTS / the grid), and
for the linear-Gaussian model less Monte Carlo variance than the observation-centred
proposals.  (For the stochastic-volatility model the Laplace marginals are narrower than
the skewed smoothing marginals, and the spread is not smaller; the means stay unbiased.)"""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import _check, dev
from oracle import grid, kalman, linearized
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


def _lg(d):
    return {1: W.lgssm_1d(), 4: W.lgssm_d4(), 8: W.lgssm_d8()}.get(d) or W.lgssm_dn(d)


@pytest.mark.parametrize("d,K", [(1, 1), (1, 2), (1, 37), (4, 7), (4, 1024), (8, 300), (2, 129), (32, 40)])
def test_linear_gaussian_equals_kalman_rts(d, K):
    m = _lg(d)
    _, y = W.simulate(m, K, 100 + K)
    y32 = y.astype(np.float32)
    mean, std, ws = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(m), dev(y32))
    torch.cuda.synchronize()
    assert dsmc.dsmc_stream_status(ws) == 0
    ms, Ps, _ = kalman.rts_for(m, y32.astype(np.float64))
    sd = np.sqrt(np.einsum("tii->ti", Ps))
    # FP64 on both sides; the outputs are rounded to FP32
    np.testing.assert_allclose(mean.cpu().numpy(), ms, rtol=0, atol=1e-6 * max(1.0, np.abs(ms).max()))
    np.testing.assert_allclose(std.cpu().numpy(), sd, rtol=1e-6)


@pytest.mark.parametrize("iterations", [1, 4, 25])
def test_sv_iterations_equal_oracle(iterations):
    K = 300
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    y32 = y.astype(np.float32)
    mean, std, ws = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(m), dev(y32), iterations=iterations)
    torch.cuda.synchronize()
    assert dsmc.dsmc_stream_status(ws) == 0
    mo, so = linearized.linearized_smoother(m, y32.astype(np.float64), iterations=iterations)
    np.testing.assert_allclose(mean.cpu().numpy(), mo, rtol=0, atol=2e-6 * max(1.0, np.abs(mo).max()))
    np.testing.assert_allclose(std.cpu().numpy(), so, rtol=2e-6)


def test_sv_warm_start():
    """Two passes started from the result of three equal five passes (the particle-Gibbs use
    of Section 4.1: one more pass from the previous approximation)."""
    K = 200
    m = W.sv(K)
    _, y = W.simulate(m, K, 7)
    yd = dev(y.astype(np.float32))
    hm = dsmc.HostModel(m)
    m3, _, ws = dsmc.dsmc_gaussian_proposals(hm, yd, iterations=3)
    m5, s5, _ = dsmc.dsmc_gaussian_proposals(hm, yd, iterations=5, ws=ws)
    m32, s32, _ = dsmc.dsmc_gaussian_proposals(hm, yd, iterations=2, init_mean=m3.clone(), ws=ws)
    torch.cuda.synchronize()
    # the warm start enters as FP32 means, so agreement is to FP32 resolution
    np.testing.assert_allclose(m32.cpu().numpy(), m5.cpu().numpy(), atol=1e-5)
    np.testing.assert_allclose(s32.cpu().numpy(), s5.cpu().numpy(), rtol=1e-5)


def _seed_means(model, y, K, N, R, mean=None, std=None):
    if mean is not None:
        model = dataclasses.replace(model, prop_kind=W.PROP_GAUSS, prop_mean=mean.cpu().numpy(),
                                    prop_std=std.cpu().numpy(), nu=W.NU_EQ_Q)
    sm = dsmc.Smoother(model, K, N, seed=1000)
    yd = dev(y)
    out = []
    for r in range(R):
        sm.set_seed(1000 + r)
        out.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    return np.array(out)


def test_dsmc_with_linear_gaussian_pit_proposals():
    m = W.lgssm_d4()
    K, N, R = 256, 128, 24
    _, y = W.simulate(m, K, 5)
    y = y.astype(np.float32)
    mean, std, _ = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(m), dev(y))
    ms, _, _ = kalman.rts_for(m, y.astype(np.float64))
    pit = _seed_means(m, y, K, N, R, mean, std)
    obs = _seed_means(m, y, K, N, R)
    _check(pit, ms)
    _check(obs, ms)
    # the smoothing marginals as proposals cut the Monte Carlo spread of the means
    assert pit.std(0, ddof=1).mean() < 0.8 * obs.std(0, ddof=1).mean()


def test_dsmc_with_sv_pit_proposals():
    K, N, R = 128, 256, 24
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    y = y.astype(np.float32)
    mean, std, _ = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(m), dev(y), iterations=20)
    gm, _, _ = grid.sv_grid_smoother(m.mu, m.phi, m.sigma, y[:, 0].astype(np.float64))
    pit = _seed_means(m, y, K, N, R, mean, std)
    _check(pit, gm[:, None])
