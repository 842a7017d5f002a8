"""The models of the paper's experiments on the device (through the C ABI): the Poisson-count
model of Section 5.1, the theta-logistic model of Section 5.2 (non-linear transition mean)
and the constrained random walk of Section 5.3 (indicator potential, uniform proposal).

  * Algorithm 2 particles and leaf weights against the oracle.
  * Combination log-weights within 1e-5 relative of the FP64 oracle on identical particles,
    indices bit-exact against the device-precision sampler (dense) and the factorised
    rejection sampler.
  * Smoothing means within Monte Carlo error of the grid forward-backward smoother.
  * Algorithm 4's Gaussian proposals for the Poisson-count and theta-logistic models against
    the oracle's sequential linearised smoother.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import _check, dev, endpoint_indices
from oracle import core, grid, linearized
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu

NAMES = ["cox", "theta_logistic", "crw"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


@pytest.mark.parametrize("name", NAMES)
def test_init_matches_oracle(name):
    K, N = 40, 300
    wl = W.workload(name, K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=77)
    sm.init(dev(wl.y))
    torch.cuda.synchronize()
    X, lw, lL = core.init(wl.model, wl.y.astype(np.float32).astype(np.float64), K, N, 77)
    np.testing.assert_allclose(sm.X.cpu().numpy().astype(np.float64), X, rtol=0, atol=2e-5 * max(1, np.abs(X).max()))
    lwg = sm.logw.cpu().numpy().astype(np.float64)
    assert (np.abs(lwg - lw) <= 5e-5 * np.maximum(1, np.abs(lw))).all()
    assert sm.status() == 0


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("level", [0, 2])
def test_logw_and_indices(name, level):
    K, N = 13, 200
    wl = W.workload(name, K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=11, fused_max_merges=-1)
    y = dev(wl.y)
    sm.init(y)
    for l in range(level + 1):
        sm.merge_level(y, l)
    torch.cuda.synchronize()
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws)
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    pairs = sm.pairs.cpu().numpy()
    a, c, iL, iR = endpoint_indices(pairs, K, N, level, M - 1)
    b = min(a + 2 * (1 << level), K) - 1
    wl_ = lw[c - 1] if level == 0 else np.full(N, -np.log(N))
    wr_ = lw[c] if b == c else np.full(N, -np.log(N))
    ref = core.logw_matrix(wl.model, wl.y.astype(np.float32).astype(np.float64), K, c, X[c - 1][iL], X[c][iR], wl_,
                           wr_)
    got = dbg["logW"].cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref)
    assert (np.isfinite(got) == fin).all()
    err = np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
    assert err.max() <= 1e-5, err.max()
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(), dbg["e"].cpu().numpy(),
                                 dbg["B"], sm.cfg.seed, dbg["gid"], 0, N)
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


@pytest.mark.parametrize("name", NAMES)
def test_factored_rejection_indices(name):
    K, N, level = 9, 160, 1
    wl = W.workload(name, K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=13, resampler=dsmc.RS_FACTORED)
    y = dev(wl.y)
    sm.init(y)
    for l in range(level + 1):
        sm.merge_level(y, l)
    torch.cuda.synchronize()
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_lazy_weights(sm.cfg, sm.hm, level, M - 1, sm.ws)
    pa, pc, acc = (dbg[k].cpu().numpy() for k in ("pa", "pc", "acc"))
    assert (acc <= 1.0 + 2.0 ** -10).all()
    li, ri, att, st = core.kp_rsf_pairs(pa, pc, acc, sm.cfg.seed, dbg["gid"], 0, N, max_attempts=1 << 26)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("resampler", [dsmc.MULTINOMIAL, dsmc.RS_FACTORED])
def test_means_vs_grid(name, resampler):
    K, N, R = 64, 512, 32
    wl = W.workload(name, K=K, N=N)
    gm, _, _ = grid.model_grid_smoother(wl.model, wl.y[:, 0].astype(np.float32).astype(np.float64))
    sm = dsmc.Smoother(wl.model, K, N, seed=1000, resampler=resampler)
    yd = dev(wl.y)
    g = []
    for r in range(R):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), gm[:, None])


@pytest.mark.parametrize("name,iterations", [("cox", 1), ("cox", 15), ("theta_logistic", 1), ("theta_logistic", 25)])
def test_gaussian_proposals_equal_oracle(name, iterations):
    K = 120
    wl = W.workload(name, K=K, N=64)
    y32 = wl.y.astype(np.float32)
    mean, std, ws = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(wl.model), dev(y32), iterations=iterations)
    torch.cuda.synchronize()
    assert dsmc.dsmc_stream_status(ws) == 0
    mo, so = linearized.linearized_smoother(wl.model, y32.astype(np.float64), iterations=iterations)
    np.testing.assert_allclose(mean.cpu().numpy(), mo, rtol=0, atol=2e-6 * max(1.0, np.abs(mo).max()))
    np.testing.assert_allclose(std.cpu().numpy(), so, rtol=2e-6)


def test_degenerate_weights_report_status_and_the_context_stays_usable():
    """A constrained walk whose proposal puts (almost surely) every particle outside the
    constraint: every pair weight is zero.  The oracle refuses it as degenerate; the device
    reports a degenerate (or non-finite) status instead of faulting, draws its fallback pairs,
    and the next smoothing on the same buffers is clean."""
    import dataclasses
    K, N = 4, 16
    m = dataclasses.replace(W.crw(sigma=0.4, bound=1e-3), prop_scale=1.0)
    y = np.zeros((K, 1))
    with pytest.raises(RuntimeError, match="degenerate"):
        core.smooth(m, y, K, N, 5)
    sm = dsmc.Smoother(m, K, N, seed=5)
    sm.smooth(dev(y))
    torch.cuda.synchronize()
    assert sm.status() in (6, 7)
    pairs = sm.pairs.cpu().numpy()
    assert ((pairs >= 0) & (pairs < N)).all()
    ok = W.crw()
    sm2 = dsmc.Smoother(ok, K, N, seed=6)
    sm2.smooth(dev(y))
    torch.cuda.synchronize()
    assert sm2.status() == 0
