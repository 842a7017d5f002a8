"""GPU pair draws against the paper's law, and the two samplers added beside Algorithm 1's
multinomial draws (through the C ABI).

  * Brute force, independent of the device-precision checkers: K = 2, N <= 4, fixed
    particles (Algorithm 2 once), then many draws of the one combination with fresh Philox
    streams (counter bases).  The exact law is the normalised weight matrix W of
    Eq. (normalized-weights), enumerated by the FP64 oracle on the GPU's own particles; the
    multinomial, rejection (uniform and factorised proposals), Metropolis-Hastings (many
    steps) and conditional draws are chi-square tested against it, the systematic draws by
    their floor / ceil counts and their mean counts.
  * The law of an output trajectory at K = 3, N = 2 (two levels), enumerated over the 16
    level-0 outputs, against GPU smoothings.
  * Systematic resampling and the factorised-proposal rejection sampler: indices bit-exact
    against the oracle's (CPU-pinned) device-precision checkers fed the device's own
    weights, smoothing means against Kalman/RTS and the grid smoother.
"""
import itertools

import numpy as np
import pytest
import torch
from scipy import stats

from exact_laws import chi2_pvalue, kp_law
from gpu_helpers import _check, dev, endpoint_indices
from oracle import core, grid, kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


# ------------------------------------------------------------------ brute force, K = 2
def _bf_smoother(name, N, resampler, cond=False, B=0):
    K = 2
    wl = W.workload(name, K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=4242, resampler=resampler, rs_max_attempts=B)
    y = dev(wl.y)
    xr = dev(np.asarray(wl.x_true, np.float32).reshape(K, -1)) if cond else None
    sm.init(y, x_ref=xr)
    torch.cuda.synchronize()
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    yo = wl.y.astype(np.float32).astype(np.float64)
    logW = core.logw_matrix(wl.model, yo, K, 1, X[0], X[1], lw[0], lw[1])
    P = np.exp(logW - logW.max())
    return sm, y, P / P.sum()


def _bf_draws(sm, y, reps, cond=False):
    out = np.empty((reps, 2, sm.N), np.int64)
    for r in range(reps):
        sm.cfg.counter_base = r
        sm.merge_level(y, 0, conditional=cond)
        out[r] = sm.pairs[0].cpu().numpy()
    assert sm.status() == 0
    return out


@pytest.mark.parametrize("name,N", [("lgssm_1d", 3), ("sv", 4)])
@pytest.mark.parametrize("resampler", ["multinomial", "rs", "rs_factored", "mh"])
def test_brute_force_draws_follow_W(name, N, resampler):
    code = {"multinomial": dsmc.MULTINOMIAL, "rs": dsmc.RS, "rs_factored": dsmc.RS_FACTORED,
            "mh": dsmc.MH}[resampler]
    sm, y, P = _bf_smoother(name, N, code, B=256 if resampler == "mh" else 0)
    d = _bf_draws(sm, y, 90_000 // N)
    assert chi2_pvalue(d[:, 0].ravel(), d[:, 1].ravel(), P) > 1e-3


def test_brute_force_conditional_draws():
    """Algorithm 5: slot 0 is (0, 0); slots 1..N-1 are independent draws from W."""
    N = 4
    sm, y, P = _bf_smoother("lgssm_1d", N, dsmc.MULTINOMIAL, cond=True)
    d = _bf_draws(sm, y, 30_000, cond=True)
    assert (d[:, :, 0] == 0).all()
    assert chi2_pvalue(d[:, 0, 1:].ravel(), d[:, 1, 1:].ravel(), P) > 1e-3


@pytest.mark.parametrize("name,N", [("lgssm_1d", 3), ("sv", 4)])
def test_brute_force_systematic_counts(name, N):
    """Systematic positions (k + U) / N: every pair's count among the N slots is the floor or
    the ceiling of N W_ij (up to FP32 rounding of the device weights), and over many U the
    mean count is N W_ij."""
    sm, y, P = _bf_smoother(name, N, dsmc.SYSTEMATIC)
    reps = 20_000
    d = _bf_draws(sm, y, reps)
    counts = np.zeros((reps, N * N))
    for r in range(reps):
        counts[r] = np.bincount(d[r, 0] * N + d[r, 1], minlength=N * N)
    target = N * P.ravel()
    assert (np.abs(counts - target) < 1 + 1e-4).all()
    z = np.abs(counts.mean(0) - target) / (0.5 / np.sqrt(reps))
    assert z.max() < 5, z.max()


# ------------------------------------------------------------------ K = 3, N = 2 trajectory law
def test_output_trajectory_law_on_gpu():
    m = W.lgssm_1d()
    K, N = 3, 2
    _, y = W.simulate(m, K, 77)
    sm = dsmc.Smoother(m, K, N, seed=9, want_traj=True)
    yd = dev(y)
    sm.init(yd)
    torch.cuda.synchronize()
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    assert len({float(v) for v in X[:, :, 0].ravel()}) == K * N   # values identify the particles
    yo = y.astype(np.float32).astype(np.float64)
    W0 = core.logw_matrix(m, yo, K, 1, X[0], X[1], lw[0], lw[1])
    P0 = np.exp(W0 - W0.max())
    P0 /= P0.sum()
    law = np.zeros((N, N, N))
    pairs = [(i, j) for i in range(N) for j in range(N)]
    for tau in itertools.product(pairs, repeat=N):
        p_tau = np.prod([P0[t] for t in tau])
        xl = np.array([X[1][t[1]] for t in tau])
        W1 = core.logw_matrix(m, yo, K, 2, xl, X[2], np.full(N, -np.log(N)), lw[2])
        P1 = np.exp(W1 - W1.max())
        P1 /= P1.sum()
        for l in range(N):
            for r in range(N):
                law[tau[l][0], tau[l][1], r] += p_tau * P1[l, r]
    R = 20_000
    counts = np.zeros((N, N, N))
    for rep in range(R):
        sm.cfg.counter_base = rep
        sm.merge_level(yd, 0)
        sm.merge_level(yd, 1)
        sm.resolve()
        tr = sm.traj[:, 0, 0].cpu().numpy().astype(np.float64)   # slot 0's trajectory
        idx = [int(np.flatnonzero(X[t, :, 0] == tr[t])[0]) for t in range(K)]
        counts[idx[0], idx[1], idx[2]] += 1
    assert sm.status() == 0
    exp = law.ravel() * R
    keep = exp > 0
    assert counts.ravel()[~keep].sum() == 0
    assert stats.chisquare(counts.ravel()[keep], exp[keep]).pvalue > 1e-3


# ------------------------------------------------------------------ systematic resampling
def _level(name, K, N, level, resampler, fused=0, compute=dsmc.FP32, seed=11):
    wl = W.workload(name, K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=seed, resampler=resampler, fused_max_merges=fused, compute=compute)
    y = dev(wl.y)
    sm.init(y)
    for l in range(level + 1):
        sm.merge_level(y, l)
    torch.cuda.synchronize()
    return wl, sm


@pytest.mark.parametrize("fused", [0, -1], ids=["fused-small-levels", "split-kernels"])
@pytest.mark.parametrize("name,K,N,level,compute", [("lgssm_d8", 16, 300, 1, dsmc.FP32),
                                                    ("lgssm_1d", 37, 1000, 2, dsmc.FP32),
                                                    ("sv", 9, 700, 0, dsmc.FP32),
                                                    ("lgssm_d4", 6, 96, 2, dsmc.FP32),
                                                    ("sv", 3, 4096, 0, dsmc.FP32),
                                                    ("lgssm_d4", 8, 2500, 1, dsmc.BF16)])
def test_systematic_indices_bit_exact(name, K, N, level, compute, fused):
    wl, sm = _level(name, K, N, level, dsmc.SYSTEMATIC, fused=fused, compute=compute)
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("r", "tiles", "e"))
    r, t, e = dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(), dbg["e"].cpu().numpy()
    li, ri = core.kp_sys_pairs(r, t, e, dbg["B"], sm.cfg.seed, dbg["gid"], 0, N)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    # the systematic property on the device's own fixed-point law
    if N <= 1000:
        P = kp_law(r, t, e, dbg["B"])
        c = np.bincount(pairs[dbg["gid"], 0].astype(np.int64) * N + pairs[dbg["gid"], 1], minlength=N * N)
        assert (np.abs(c - N * P.ravel()) < 1 + 1e-6).all()
    assert sm.status() == 0


def test_systematic_means_vs_rts():
    wl = W.workload("lgssm_1d")
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    sm = dsmc.Smoother(wl.model, wl.K, wl.N, seed=1000, resampler=dsmc.SYSTEMATIC)
    yd = dev(wl.y)
    g = []
    for r in range(64):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), ms)


def test_systematic_conditional_stays_multinomial():
    """Conditional combinations draw multinomially whatever the resampler (Algorithm 5)."""
    wl = W.workload("lgssm_1d", K=16, N=64)
    y = dev(wl.y)
    xin = dev(np.asarray(wl.x_true, np.float32).reshape(16, -1))
    out = []
    for res in (dsmc.MULTINOMIAL, dsmc.SYSTEMATIC):
        sm = dsmc.Smoother(wl.model, 16, 64, seed=5, resampler=res)
        xo = torch.empty_like(xin)
        sm.conditional(y, xin, xo)
        torch.cuda.synchronize()
        assert sm.status() == 0
        out.append((sm.pairs.clone(), xo.clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ factorised proposals
@pytest.mark.parametrize("name,K,N,level", [("sv", 8, 500, 0), ("sv", 16, 333, 2), ("lgssm_1d", 5, 64, 2),
                                            ("lgssm_d4", 6, 96, 1), ("lgssm_d8", 4, 200, 0)])
def test_factored_rejection_indices_bit_exact(name, K, N, level):
    """Device pairs equal the oracle's device-precision factorised sampler fed the device's
    own proposal weights and acceptance ratios; those ratios are at most 1 (up to rounding),
    and pa_i pc_j acc_ij is proportional to the FP64 pair weights on the same particles."""
    wl, sm = _level(name, K, N, level, dsmc.RS_FACTORED)
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_lazy_weights(sm.cfg, sm.hm, level, M - 1, sm.ws)
    pa, pc, acc = (dbg[k].cpu().numpy() for k in ("pa", "pc", "acc"))
    assert (acc <= 1.0 + 2.0 ** -10).all() and (acc >= 0).all()
    li, ri, att, st = core.kp_rsf_pairs(pa, pc, acc, sm.cfg.seed, dbg["gid"], 0, N, max_attempts=1 << 26)
    assert st == 0
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    a, c, iL, iR = endpoint_indices(pairs, K, N, level, M - 1)
    b = min(a + 2 * (1 << level), K) - 1
    wl_ = lw[c - 1] if level == 0 else np.full(N, -np.log(N))
    wr_ = lw[c] if b == c else np.full(N, -np.log(N))
    ref = core.logw_matrix(wl.model, wl.y.astype(np.float32).astype(np.float64), K, c, X[c - 1][iL], X[c][iR],
                           wl_, wr_)
    with np.errstate(divide="ignore"):
        got = np.log(pa.astype(np.float64))[:, None] + np.log(pc.astype(np.float64))[None, :] + \
            np.log(acc.astype(np.float64))
    ok = np.isfinite(got) & (ref > ref.max() - 30)
    shift = np.median((ref - got)[ok])
    assert np.abs(got[ok] + shift - ref[ok]).max() < 2e-4 * max(1.0, np.abs(ref).max())
    assert sm.status() == 0


def test_factored_means_vs_rts_and_fewer_attempts():
    wl = W.workload("lgssm_1d")
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    yd = dev(wl.y)
    g = []
    sm = dsmc.Smoother(wl.model, wl.K, wl.N, seed=1000, resampler=dsmc.RS_FACTORED)
    for r in range(48):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), ms)
    att_f = dsmc.dsmc_lazy_attempts(sm.cfg, sm.hm, sm.ws)
    su = dsmc.Smoother(wl.model, wl.K, wl.N, seed=1000 + 47, resampler=dsmc.RS)
    su.smooth(yd)
    att_u = dsmc.dsmc_lazy_attempts(su.cfg, su.hm, su.ws)
    assert att_f >= (wl.K - 1) * wl.N and att_f < att_u, (att_f, att_u)


def test_factored_sv_means_vs_grid():
    K, N = 256, 1024
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    gm, _, _ = grid.sv_grid_smoother(m.mu, m.phi, m.sigma, y[:, 0])
    sm = dsmc.Smoother(m, K, N, seed=1000, resampler=dsmc.RS_FACTORED)
    yd = dev(y)
    g = []
    for r in range(24):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), gm[:, None])


def test_factored_conditional_keeps_slot_zero():
    wl = W.workload("sv", K=33, N=128)
    y = dev(wl.y)
    xin = dev(np.asarray(wl.x_true, np.float32).reshape(33, -1))
    xo = torch.empty_like(xin)
    sm = dsmc.Smoother(wl.model, 33, 128, seed=3, resampler=dsmc.RS_FACTORED)
    sm.conditional(y, xin, xo)
    torch.cuda.synchronize()
    assert sm.status() == 0
    assert (sm.pairs[:, :, 0] == 0).all()
    X = sm.X.cpu().numpy()
    o = xo.cpu().numpy()
    for t in range(33):
        assert (np.abs(X[t] - o[t]).sum(1) == 0).any()
