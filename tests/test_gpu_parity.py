"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Rules (spec contract):
  * indices (pairs) bit-exact when both sides consume the same Philox uniforms and the
    same weight arrays (the device's own FP32 weights, exported);
  * log-weights within 1e-5 relative: |dlogW| <= 1e-5 max(1, |logW|) on identical particles;
  * smoothing means within 3 Monte Carlo standard errors of RTS / the grid reference.
"""
import numpy as np
import pytest
import torch

from oracle import core, grid, kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

from gpu_helpers import _check, _gpu_means, dev, endpoint_indices, level_offsets, levels

pytestmark = pytest.mark.gpu

LOGW_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


# ------------------------------------------------------------------------ RNG
def test_philox_bit_exact():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for seed in [0, 1, 0xDEADBEEFCAFEF00D]:
        g = dsmc.dsmc_debug_philox(dev(ctr.view(np.int32), torch.int32), seed).cpu().numpy().view(np.uint32)
        o = core.philox_many(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        np.testing.assert_array_equal(g, o)


# ------------------------------------------------------------------------ Algorithm 2
@pytest.mark.parametrize("name,K,N,nu", [("lgssm_d8", 40, 300, W.NU_EQ_Q), ("lgssm_1d", 33, 97, W.NU_PROP_H),
                                         ("sv", 50, 200, W.NU_EQ_Q), ("sv", 20, 64, W.NU_PROP_H),
                                         ("lgssm_d4", 16, 1000, W.NU_PROP_H)])
def test_init_matches_oracle(name, K, N, nu):
    wl = W.workload(name, K=K, N=N)
    m = wl.model
    m.nu = nu
    sm = dsmc.Smoother(m, K, N, seed=77)
    y = dev(wl.y)
    sm.init(y)
    torch.cuda.synchronize()
    X, lw, lL = core.init(m, wl.y.astype(np.float32).astype(np.float64), K, N, 77)
    Xg = sm.X.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Xg, X, rtol=0, atol=2e-5 * max(1.0, np.abs(X).max()))
    lwg = sm.logw.cpu().numpy().astype(np.float64)
    assert (np.abs(lwg - lw) <= LOGW_RTOL * np.maximum(1, np.abs(lw)) * 5).all()
    np.testing.assert_allclose(sm.logL.cpu().numpy(), lL, atol=1e-4)
    assert sm.status() == 0


def test_conditional_init_keeps_reference():
    wl = W.workload("lgssm_d8", K=16, N=64)
    sm = dsmc.Smoother(wl.model, 16, 64, seed=5)
    xr = dev(np.random.default_rng(0).standard_normal((16, 8)))
    sm.init(dev(wl.y), x_ref=xr)
    torch.cuda.synchronize()
    assert torch.equal(sm.X[:, 0, :], xr)


# ------------------------------------------------------------------------ one level
def _level_setup(name, K, N, level, resampler=dsmc.MULTINOMIAL, seed=11, nu=W.NU_EQ_Q,
                 conditional=False, fused=0):
    wl = W.workload(name, K=K, N=N)
    m = wl.model
    m.nu = nu
    sm = dsmc.Smoother(m, K, N, seed=seed, resampler=resampler, fused_max_merges=fused)
    y = dev(wl.y)
    xr = dev(np.zeros((K, m.d))) if conditional else None
    sm.init(y, x_ref=xr)
    for l in range(level + 1):
        sm.merge_level(y, l, conditional=conditional)
    torch.cuda.synchronize()
    return wl, m, sm


CASES = [("lgssm_d8", 64, 64, 0), ("lgssm_d8", 16, 300, 1), ("lgssm_1d", 37, 1000, 2),
         ("sv", 9, 700, 3), ("lgssm_d4", 12, 2500, 0), ("lgssm_d4", 6, 96, 2)]


@pytest.mark.parametrize("fused", [0, -1], ids=["fused-small-levels", "split-kernels"])
@pytest.mark.parametrize("name,K,N,level", CASES)
def test_logw_rows_and_indices(name, K, N, level, fused):
    """For the last combination of a level: device log-weights vs the oracle's FP64 on the
    same particles; device row weights vs the exact row sums; device pairs vs the oracle's
    device-precision sampler fed the device's own weights and the same uniforms."""
    wl, m, sm = _level_setup(name, K, N, level, fused=fused)
    M = core.merges_at_level(K, level)
    mi = M - 1
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, mi, sm.ws)
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    pairs = sm.pairs.cpu().numpy()
    a, c, iL, iR = endpoint_indices(pairs, K, N, level, mi)
    b = min(a + 2 * (1 << level), K) - 1
    wl_ = lw[c - 1] if level == 0 else np.full(N, -np.log(N))
    wr_ = lw[c] if b == c else np.full(N, -np.log(N))
    yo = wl.y.astype(np.float32).astype(np.float64)
    ref = core.logw_matrix(m, yo, K, c, X[c - 1][iL], X[c][iR], wl_, wr_)
    got = dbg["logW"].cpu().numpy().astype(np.float64)
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= LOGW_RTOL, err.max()
    # row weights: r_i proportional to sum_j exp(logW_ij)
    rs = np.exp(np.logaddexp.reduce(ref, axis=1) - np.logaddexp.reduce(ref, axis=1).max())
    r = dbg["r"].cpu().numpy().astype(np.float64)
    big = rs > 1e-6
    np.testing.assert_allclose(r[big], rs[big], rtol=2e-4)
    # indices bit-exact with the device-precision sampler
    g = dbg["gid"]
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(),
                                 dbg["e"].cpu().numpy(), dbg["B"], sm.cfg.seed, g, 0, N)
    # the row totals the device exports are the sums of its tile weights
    np.testing.assert_allclose(dbg["rowsum"].cpu().numpy(), dbg["tiles"].cpu().numpy().sum(1),
                               rtol=1e-5, atol=0)
    np.testing.assert_array_equal(pairs[g, 0], li)
    np.testing.assert_array_equal(pairs[g, 1], ri)
    assert sm.status() == 0


@pytest.mark.parametrize("name,K,N,level", [("sv", 8, 500, 0), ("sv", 16, 333, 2), ("lgssm_1d", 5, 64, 2)])
def test_rejection_indices_bit_exact(name, K, N, level):
    wl, m, sm = _level_setup(name, K, N, level, resampler=dsmc.RS)
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("logW", "ratio"))
    q = dbg["ratio"].cpu().numpy()
    assert (q <= 1.0 + 1e-6).all() and (q >= 0).all()
    li, ri, att, st = core.kp_rs_pairs(q, sm.cfg.seed, dbg["gid"], 0, N, max_attempts=1 << 20)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    # the ratio is exp(logW - log wbar): consistent with the exported log-weights
    lW = dbg["logW"].cpu().numpy().astype(np.float64)
    rq = np.exp(lW - lW.max())
    assert np.allclose(q / q.max(), rq, rtol=1e-4, atol=1e-7)
    assert sm.status() == 0


@pytest.mark.parametrize("name,K,N,level", [("sv", 8, 500, 0), ("sv", 16, 333, 2), ("lgssm_1d", 5, 64, 2),
                                            ("lgssm_d4", 6, 96, 1)])
def test_metropolis_hastings_indices_bit_exact(name, K, N, level):
    """Algorithm 7 on the device against the oracle's device-precision chain fed the same
    FP32 ratios: B = 64 steps from (n, n), u r(I, J) < r(I*, J*)."""
    wl, m, sm = _level_setup(name, K, N, level, resampler=dsmc.MH)
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("ratio",))
    q = dbg["ratio"].cpu().numpy()
    li, ri = core.kp_mh_pairs(q, sm.cfg.seed, dbg["gid"], 0, N, 64)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


def test_metropolis_hastings_conditional_keeps_slot_zero_and_smooths():
    """Conditional Algorithm 7 keeps slot 0 = (0, 0) at every level; a whole MH smoothing
    with many steps lands near the Kalman/RTS means (its bias shrinks with B)."""
    wl, m, sm = _level_setup("lgssm_1d", 16, 200, 3, resampler=dsmc.MH, conditional=True)
    pairs = sm.pairs.cpu().numpy()
    assert (pairs[:, :, 0] == 0).all()
    assert sm.status() == 0
    wl = W.workload("lgssm_1d")
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    y = dev(wl.y)
    errs = {}
    for res, B in ((dsmc.MULTINOMIAL, 0), (dsmc.MH, 256)):
        g = []
        for r in range(16):
            smr = dsmc.Smoother(wl.model, wl.K, 256, seed=3000 + r, resampler=res, rs_max_attempts=B)
            g.append(smr.smooth(y).cpu().numpy().copy())
            assert smr.status() == 0
        errs[res] = np.sqrt(((np.mean(g, 0) - ms) ** 2).mean())
    assert errs[dsmc.MH] < 2.0 * errs[dsmc.MULTINOMIAL] + 0.02, errs


def test_level0_increment_matches_oracle():
    """log L after level 0 = log L_{c-1} + log L_c + log sum_ij exp(logW_ij) (Eq. Lab)."""
    wl, m, sm = _level_setup("lgssm_d8", 16, 256, 0)
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    yo = wl.y.astype(np.float32).astype(np.float64)
    smb = dsmc.Smoother(m, 16, 256, seed=11)
    smb.init(dev(wl.y))
    torch.cuda.synchronize()
    L0 = smb.logL.cpu().numpy()
    Lg = sm.logL.cpu().numpy()
    for mi in range(8):
        a, c = 2 * mi, 2 * mi + 1
        ref = core.logw_matrix(m, yo, 16, c, X[c - 1], X[c], lw[c - 1], lw[c])
        inc = np.logaddexp.reduce(ref.reshape(-1))
        assert Lg[a] == pytest.approx(L0[a] + L0[c] + inc, abs=2e-5 * max(1, abs(inc)))


# ------------------------------------------------------------------------ resolution
@pytest.mark.parametrize("K,N", [(11, 8), (32, 64), (100, 33)])
def test_resolution_bit_exact(K, N):
    wl = W.workload("lgssm_d4", K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=3, want_traj=True)
    sm.smooth(dev(wl.y))
    torch.cuda.synchronize()
    X = sm.X.cpu().numpy()
    pairs = sm.pairs.cpu().numpy()
    traj = sm.traj.cpu().numpy()
    offs = level_offsets(K)
    L = levels(K)
    for t in range(K):
        sig = np.arange(N)
        for l in range(L - 1, -1, -1):
            sz = 1 << l
            p = (t // (2 * sz)) * 2 * sz
            if p + sz >= K:
                continue
            sig = pairs[offs[l] + p // (2 * sz), 1 if t >= p + sz else 0][sig]
        np.testing.assert_array_equal(traj[t], X[t][sig])
    mean = sm.mean.cpu().numpy()
    np.testing.assert_allclose(mean, traj.astype(np.float64).mean(1), rtol=1e-6, atol=1e-6)
    assert ((pairs >= 0) & (pairs < N)).all()


def test_conditional_keeps_slot0_and_star_is_a_particle():
    K, N = 20, 64
    wl = W.workload("lgssm_d4", K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=9, want_traj=True)
    xr = dev(np.random.default_rng(2).standard_normal((K, 4)))
    out = torch.empty_like(xr)
    sm.conditional(dev(wl.y), xr, out)
    torch.cuda.synchronize()
    assert (sm.pairs[:, :, 0] == 0).all()
    assert torch.equal(sm.traj[:, 0, :], xr)
    X = sm.X.cpu().numpy()
    o = out.cpu().numpy()
    for t in range(K):
        assert (np.abs(X[t] - o[t]).sum(1) == 0).any()


# ------------------------------------------------------------------------ statistics
@pytest.mark.parametrize("nu", [W.NU_EQ_Q, W.NU_PROP_H])
def test_means_vs_rts_1d(nu):
    wl = W.workload("lgssm_1d")
    m = W.lgssm_1d(nu)
    ms, _, _ = kalman.rts_for(m, wl.y)
    _check(_gpu_means(m, wl.y, wl.K, wl.N, 64), ms)


def test_means_vs_rts_d8_ragged():
    m = W.lgssm_d8()
    K, N = 100, 300
    _, y = W.simulate(m, K, 77)
    ms, _, _ = kalman.rts_for(m, y)
    _check(_gpu_means(m, y, K, N, 32), ms)


def test_means_rejection_vs_rts():
    wl = W.workload("lgssm_1d", K=24, N=256)
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    _check(_gpu_means(wl.model, wl.y, wl.K, wl.N, 32, resampler=dsmc.RS), ms)


def test_sv_means_vs_grid():
    K, N = 64, 512
    m = W.sv(K)
    _, y = W.simulate(m, K, 2264 + 3)
    gm, _, _ = grid.sv_grid_smoother(m.mu, m.phi, m.sigma, y[:, 0])
    _check(_gpu_means(m, y, K, N, 32), gm[:, None])


def test_logL_unbiased():
    wl = W.workload("lgssm_1d", K=8, N=32)
    _, _, ll = kalman.rts_for(wl.model, wl.y)
    sm = dsmc.Smoother(wl.model, 8, 32, seed=0)
    yd = dev(wl.y)
    r = []
    for s in range(600):
        sm.set_seed(5000 + s)
        sm.smooth(yd)
        r.append(float(sm.logL_out.item()))
    r = np.exp(np.array(r) - ll)
    assert abs(r.mean() - 1.0) < 4 * r.std(ddof=1) / np.sqrt(len(r))


def test_gpu_vs_oracle_same_seeds():
    """Same seeds, same Philox streams: the device and the oracle are two independent
    implementations of the same smoother; their seed-averaged means agree."""
    wl = W.workload("lgssm_1d", K=16, N=128)
    R = 32
    g = _gpu_means(wl.model, wl.y, wl.K, wl.N, R)
    o = np.array([core.smooth(wl.model, wl.y.astype(np.float32).astype(np.float64), wl.K, wl.N, 1000 + r)["mean"]
                  for r in range(R)])
    sd = np.sqrt((g.var(0, ddof=1) + o.var(0, ddof=1)) / 2)
    z = np.abs(g.mean(0) - o.mean(0)) / (sd * np.sqrt(2.0 / R))
    assert z.max() < 4.5


# ------------------------------------------------------------------------ edge cases
def test_k1_weighted_leaf():
    m = W.lgssm_1d()
    _, y = W.simulate(m, 1, 3)
    sm = dsmc.Smoother(m, 1, 50, seed=12)
    mean = sm.smooth(dev(y)).cpu().numpy()
    X = sm.X.cpu().numpy()[0, :, 0].astype(np.float64)
    w = np.exp(sm.logw.cpu().numpy()[0].astype(np.float64))
    assert mean[0, 0] == pytest.approx((w * X).sum(), abs=1e-5)


def test_n1_is_concatenation():
    wl = W.workload("lgssm_d4", K=9, N=1)
    sm = dsmc.Smoother(wl.model, 9, 1, seed=4, want_traj=True)
    sm.smooth(dev(wl.y))
    torch.cuda.synchronize()
    assert (sm.pairs == 0).all()
    assert torch.equal(sm.traj, sm.X)


def test_nonfinite_observation_reports_status():
    wl = W.workload("lgssm_1d", K=8, N=32)
    y = wl.y.copy()
    y[3] = np.nan
    sm = dsmc.Smoother(wl.model, 8, 32, seed=1)
    sm.smooth(dev(y))
    assert sm.status() == 6
    assert ((sm.pairs >= 0) & (sm.pairs < 32)).all()
    # the context stays usable
    sm.smooth(dev(wl.y))
    assert sm.status() == 0


@pytest.mark.parametrize("resampler", [dsmc.RS, dsmc.RS_FACTORED])
def test_rejection_cap_reports_status(resampler):
    """A slot that reaches the attempt cap keeps the pair (-1, -1), never a plausible index;
    the status reads DSMC_ERR_RS_LIMIT, every downstream read of the pair is bounds-checked,
    and the next smoothing on the same context is clean."""
    wl = W.workload("lgssm_d8", K=4, N=64)
    sm = dsmc.Smoother(wl.model, 4, 64, seed=1, resampler=resampler, rs_max_attempts=1)
    sm.smooth(dev(wl.y))
    assert sm.status() == 8
    p = sm.pairs.cpu().numpy()
    capped = (p[:, 0] == -1) & (p[:, 1] == -1)
    assert capped.any()
    assert ((p[:, 0] >= 0) & (p[:, 0] < 64) & (p[:, 1] >= 0) & (p[:, 1] < 64) | capped).all()
    ok = dsmc.Smoother(wl.model, 4, 64, seed=1, resampler=resampler)
    ok.smooth(dev(wl.y))
    assert ok.status() == 0


def test_max_dense_n():
    wl = W.workload("sv", K=2, N=16384)
    sm = dsmc.Smoother(wl.model, 2, 16384, seed=1)
    sm.smooth(dev(wl.y))
    assert sm.status() == 0
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, 0, 0, sm.ws, want=("r", "rowsum", "tiles", "e"))
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(),
                                 dbg["e"].cpu().numpy(), dbg["B"], sm.cfg.seed, dbg["gid"], 0, 16384)
    p = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(p[0, 0], li)
    np.testing.assert_array_equal(p[0, 1], ri)


def test_small_merge_chunks_same_result():
    """Splitting a level into several launch chunks does not change any draw."""
    wl = W.workload("lgssm_d4", K=40, N=96)
    a = dsmc.Smoother(wl.model, 40, 96, seed=21)
    b = dsmc.Smoother(wl.model, 40, 96, seed=21, max_merges_per_launch=3)
    y = dev(wl.y)
    a.smooth(y)
    b.smooth(y)
    torch.cuda.synchronize()
    assert torch.equal(a.pairs, b.pairs)
    assert torch.equal(a.mean, b.mean)


@pytest.mark.parametrize("name,K,N,cond", [("lgssm_d8", 45, 1000, False), ("lgssm_1d", 100, 2500, False),
                                           ("sv", 33, 96, True), ("lgssm_d4", 20, 33, False),
                                           ("lgssm_d8", 64, 64, True), ("lgssm_d4", 3, 4096, False)])
def test_fused_level_matches_split(name, K, N, cond):
    """The fused single-launch level (one cluster per combination) and the split per-level
    kernels draw the same pairs and give the same means and log-likelihood, level by level
    (every level fused against no level fused; d <= 8 so both use 512-thread reductions)."""
    wl = W.workload(name, K=K, N=N)
    y = dev(wl.y)
    out = []
    for fm in (-1, 1 << 30):
        sm = dsmc.Smoother(wl.model, K, N, seed=77, fused_max_merges=fm)
        if cond:
            xin = dev(np.asarray(wl.x_true, np.float32).reshape(K, -1))
            xout = torch.empty_like(xin)
            sm.conditional(y, xin, xout)
            extra = xout.clone()
        else:
            sm.smooth(y)
            extra = None
        torch.cuda.synchronize()
        assert sm.status() == 0
        out.append((sm.pairs.clone(), sm.mean.clone(), sm.logL_out.clone(), extra))
    (p0, m0, l0, x0), (p1, m1, l1, x1) = out
    assert torch.equal(p0, p1)
    assert torch.equal(m0, m1)
    assert torch.equal(l0, l1)
    if cond:
        assert torch.equal(x0, x1)


def test_bench_configuration_full_size():
    """The timed workload (d = 8, K = N = 1024): RTS within Monte Carlo error over seeds,
    and, on sampled combinations of the bottom and top levels, log-weights within 1e-5 and
    indices bit-exact against the oracle."""
    wl = W.workload("lgssm_d8")
    K, N = wl.K, wl.N
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    g = _gpu_means(wl.model, wl.y, K, N, 24)
    _check(g, ms)
    sm = dsmc.Smoother(wl.model, K, N, seed=31)
    y = dev(wl.y)
    sm.init(y)
    yo = wl.y.astype(np.float32).astype(np.float64)
    for level in range(levels(K)):
        sm.merge_level(y, level)
        if level not in (0, 4, levels(K) - 1):
            continue
        M = core.merges_at_level(K, level)
        mi = M - 1
        dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, mi, sm.ws)
        X = sm.X.cpu().numpy().astype(np.float64)
        lw = sm.logw.cpu().numpy().astype(np.float64)
        pairs = sm.pairs.cpu().numpy()
        a, c, iL, iR = endpoint_indices(pairs, K, N, level, mi)
        rows = np.random.default_rng(level).choice(N, 64, replace=False)
        wl_ = lw[c - 1][iL][rows] if level == 0 else np.full(64, -np.log(N))
        wr_ = lw[c] if level == 0 else np.full(N, -np.log(N))
        ref = core.logw_matrix(wl.model, yo, K, c, X[c - 1][iL][rows], X[c][iR], wl_, wr_)
        got = dbg["logW"].cpu().numpy().astype(np.float64)[rows]
        err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() <= LOGW_RTOL, (level, err.max())
        li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(),
                                     dbg["e"].cpu().numpy(), dbg["B"], sm.cfg.seed, dbg["gid"], 0, N)
        np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
        np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


# ------------------------------------------------------------------------ tensor cores
# unit roundoff of the tensor-core operand types (BF16: 8 significant bits, TF32: 11)
TC_UNIT = {dsmc.TF32: 2.0 ** -11, dsmc.BF16: 2.0 ** -8}


def _cross_term_scale(m, X, c):
    """max_ij sum_k |u_ik| |v_jk| for the level-0 combination with right time c: the scale of
    the rounding error of the cross term when u and v are rounded to the MMA type
    (u_i = log2(e) Q^-1 (A x_i + c_f - mu), v_j = x_j - mu, mu = mean of the right particles)."""
    xl, xr = X[c - 1].astype(np.float64), X[c].astype(np.float64)
    if m.kind == W.SV:
        A, cf, Qi = np.array([[m.phi]]), np.array([m.mu * (1 - m.phi)]), np.array([[1 / m.sigma ** 2]])
    else:
        A, cf, Qi = m.A, np.zeros(m.d), np.linalg.inv(m.Q)
    mu = xr.mean(0)
    u = np.log2(np.e) * (xl @ A.T + cf - mu) @ Qi.T
    v = xr - mu
    return float((np.abs(u) @ np.abs(v).T).max())


@pytest.mark.parametrize("compute", [dsmc.TF32, dsmc.BF16])
@pytest.mark.parametrize("name,K,N,level", [("lgssm_d8", 16, 1000, 0), ("lgssm_d8", 9, 300, 3),
                                            ("lgssm_d4", 8, 2500, 0), ("lgssm_d4", 8, 2500, 1),
                                            ("sv", 6, 64, 0), ("sv", 6, 64, 2),
                                            ("lgssm_1d", 5, 4096, 0), ("lgssm_d16", 4, 256, 0),
                                            ("lgssm_d32", 4, 256, 0)])
def test_tensor_core_tiles_and_indices(compute, name, K, N, level):
    """The tcgen05 cross term: tile weights within the precision's error of the FP32 path on
    identical particles, and indices bit-exact against the oracle's device-precision
    sampler fed the device's own (tensor-core) weights."""
    wl = W.workload(name, K=K, N=N)
    if compute == dsmc.TF32 and wl.model.d > 16:
        pytest.skip("TF32 cross term: dx <= 16")
    y = dev(wl.y)
    out = {}
    for cm in (dsmc.FP32, compute):
        # split kernels on every level (a fused level would use the FP32 cross term)
        sm = dsmc.Smoother(wl.model, K, N, seed=5, compute=cm, fused_max_merges=-1)
        sm.init(y)
        for l in range(level + 1):
            sm.merge_level(y, l)
        torch.cuda.synchronize()
        M = core.merges_at_level(K, level)
        out[cm] = (sm, dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws))
    if level == 0:
        # a tile weight is a positive combination of its pair weights, so its log2 error is
        # at most the largest exponent error: both operands rounded (2 u S), the two-term
        # alpha / beta splits and FP32 accumulation (0.01 covers |alpha|, |beta| < 1000)
        t32 = out[dsmc.FP32][1]["tiles"].cpu().numpy().astype(np.float64)
        ttc = out[compute][1]["tiles"].cpu().numpy().astype(np.float64)
        big = t32 > 1e-6 * t32.max()
        err = np.abs(np.log2(ttc[big]) - np.log2(t32[big]))
        X = out[compute][0].X.cpu().numpy()
        tol = 2.05 * TC_UNIT[compute] * _cross_term_scale(wl.model, X, 2 * (M - 1) + 1) + 0.01
        assert err.max() < tol, (err.max(), tol)
    sm, dbg = out[compute]
    pairs = sm.pairs.cpu().numpy()
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(),
                                 dbg["e"].cpu().numpy(), dbg["B"], sm.cfg.seed, dbg["gid"], 0, N)
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


@pytest.mark.parametrize("compute", [dsmc.TF32, dsmc.BF16])
def test_tensor_core_means_vs_rts(compute):
    m = W.lgssm_d8()
    K, N = 100, 500
    _, y = W.simulate(m, K, 77)
    ms, _, _ = kalman.rts_for(m, y)
    sm = dsmc.Smoother(m, K, N, seed=1000, compute=compute)
    yd = dev(y)
    g = []
    for r in range(32):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), ms)


@pytest.mark.parametrize("compute", [dsmc.TF32, dsmc.BF16])
def test_tensor_core_bench_configuration(compute):
    wl = W.workload("lgssm_d8")
    ms, _, _ = kalman.rts_for(wl.model, wl.y)
    sm = dsmc.Smoother(wl.model, wl.K, wl.N, seed=1000, compute=compute)
    yd = dev(wl.y)
    g = []
    for r in range(24):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), ms)


def test_particle_gibbs_chain_on_rts():
    """Conditional dSMC sweeps at fixed parameters (Section 3.2): the chain of references
    x* <- c-dSMC(x*) leaves the smoother invariant, so its time averages agree with the
    Kalman/RTS means within batch-means Monte Carlo error; every sweep keeps slot 0."""
    m = W.lgssm_1d()
    K, N, S, burn = 32, 64, 800, 100
    _, y = W.simulate(m, K, 19)
    ms, _, _ = kalman.rts_for(m, y)
    sm = dsmc.Smoother(m, K, N, seed=77)
    yd = dev(y)
    xa = torch.zeros((K, 1), dtype=torch.float32, device="cuda")
    xb = torch.empty_like(xa)
    chain = []
    for s in range(S):
        sm.set_seed(77, counter_base=s)
        sm.conditional(yd, xa, xb)
        if s == 0:
            torch.cuda.synchronize()
            assert (sm.pairs[:, :, 0] == 0).all()
        xa, xb = xb, xa
        if s >= burn:
            chain.append(xa[:, 0].clone())
    assert sm.status() == 0
    chain = torch.stack(chain).cpu().numpy()
    nb = 25
    bm = chain[: (len(chain) // nb) * nb].reshape(nb, -1, K).mean(1)
    se = bm.std(0, ddof=1) / np.sqrt(nb)
    z = np.abs(bm.mean(0) - ms[:, 0]) / se
    assert z.max() < 4.5, z.max()


def test_tensor_core_wait_runs_out_and_reports_timeout():
    """Failure detection on the device: with the test switch on, the tensor-core launch
    issues no MMA, so the epilogue's wait on its accumulator reaches its iteration limit;
    the kernel records DSMC_ERR_TIMEOUT, frees its tensor memory and returns, and the next
    smoothing on the same context runs clean."""
    wl = W.workload("lgssm_d4", K=8, N=256)
    y = dev(wl.y)
    sm = dsmc.Smoother(wl.model, 8, 256, seed=3, compute=dsmc.BF16, fused_max_merges=-1)
    sm.init(y)
    dsmc.dsmc_debug_stall_tensor_cores(True)
    try:
        sm.merge_level(y, 0)
        torch.cuda.synchronize()
    finally:
        dsmc.dsmc_debug_stall_tensor_cores(False)
    assert sm.status() == 9          # DSMC_ERR_TIMEOUT
    sm2 = dsmc.Smoother(wl.model, 8, 256, seed=3, compute=dsmc.BF16, fused_max_merges=-1)
    sm2.smooth(y)
    torch.cuda.synchronize()
    assert sm2.status() == 0
    assert torch.isfinite(sm2.mean).all()
