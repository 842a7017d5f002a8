"""Particle Gibbs with parameter updates on the theta-logistic model (Section 3.2, Section 5.2)
on the device.

  * With the parameters held fixed, the chain of reference trajectories is a Markov chain
    that leaves p(x | y, theta) invariant (conditional dSMC, Algorithm 5): its time averages
    equal the grid forward-backward smoothing means within batch-means Monte Carlo error,
    with the observation-centred proposal and with Algorithm 4's Gaussian proposals.
  * With the parameter steps on, the chain runs with every device status clear, x*_t moves
    at every t in most sweeps, and the parameters stay in the region of the values the data
    were simulated from.
"""
import numpy as np
import pytest
import torch

from oracle import grid
from paper_2202_02264_gb300 import dsmc, pgibbs as P, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


def _data(K):
    m = W.theta_logistic()
    _, y = W.simulate(m, K, 52)
    y = y[:, 0].astype(np.float32).astype(np.float64)
    return m, y


def _state(m):
    return P.ThetaState(m.tau0, m.tau1, m.tau2, m.sigma ** 2, m.obs_sd ** 2)


@pytest.mark.parametrize("pit", [False, True])
def test_fixed_parameters_chain_targets_the_smoother(pit):
    K, N, sweeps, burn = 64, 256, 1200, 100
    m, y = _data(K)
    gm, gv, _ = grid.model_grid_smoother(m, y)
    g = P.ThetaLogisticGibbs(y, N, _state(m), seed=9, pit_proposals=pit, update_theta=False)
    ch = g.run(sweeps)
    xs = np.array(ch.x[burn:])
    nb = 40
    bm = xs[: (xs.shape[0] // nb) * nb].reshape(nb, -1, K).mean(1)
    se = bm.std(0, ddof=1) / np.sqrt(nb)
    z = (xs.mean(0) - gm) / np.maximum(se, 1e-3 * np.sqrt(gv))
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    assert np.mean(np.abs(z) > 2.5) < 0.08
    assert (ch.updated / sweeps).min() > 0.3


def test_parameter_updates_run_and_stay_near_the_truth():
    K, N, sweeps = 120, 256, 400
    m, y = _data(K)
    start = P.ThetaState(0.0, 0.0, 0.5, 0.05, 0.05)
    g = P.ThetaLogisticGibbs(y, N, start, seed=3)
    ch = g.run(sweeps)
    th = ch.theta[100:]
    r = np.sqrt(np.mean([t.r2 for t in th]))
    q = np.sqrt(np.mean([t.q2 for t in th]))
    assert 0.5 * m.obs_sd < r < 2.0 * m.obs_sd
    assert q < 3.0 * m.sigma
    # the drift tau0 - tau1 exp(tau2 x) nearly vanishes at the level the series hovers around
    drift = np.mean([t.tau0 - t.tau1 * np.exp(t.tau2 * np.mean(y)) for t in th])
    assert abs(drift) < 0.1, drift
    assert (ch.updated / sweeps).mean() > 0.5
    assert ch.device_s > 0 and ch.wall_s > ch.device_s
