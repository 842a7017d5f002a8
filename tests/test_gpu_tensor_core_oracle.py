"""The tensor-core (tcgen05) cross term against the FP64 oracle, and the headline batched
configuration at full size (through the C ABI).

  * Tile weights: the device's BF16 / TF32 tile sums, scaled by its per-row shift, against
    the log-sum-exp of the oracle's FP64 log-weights (Eq. normalized-weights) over the same
    tile's columns on the same particles.  A tile weight is a positive combination of its
    pairs' weights, so its log error is at most the largest exponent error: both operands
    rounded to the MMA type (2.05 u S in base 2, S = max_ij sum_k |u_ik| |v_jk|), the
    two-term splits of the row / column terms and FP32 accumulation (0.01), plus the FP32
    path's own 1e-5 relative.
  * The batched workload's shape: full-length sequences (K about 4000) of the d = 4
    linear-Gaussian batch, N = 512, BF16 cross term, no fused small level, up to 16384
    combinations per launch: tile weights against the oracle and indices bit-exact at the
    bottom, middle and top levels; smoothing means of the batched call (split kernels and
    the fused tensor-core level kernel) within Monte Carlo error of Kalman/RTS; the batched
    call equal to each sequence alone.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import _check, dev, endpoint_indices, levels
from oracle import core, kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu

TC_UNIT = {dsmc.TF32: 2.0 ** -11, dsmc.BF16: 2.0 ** -8}
LN2 = np.log(2.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


def _transition(m):
    if m.kind == W.SV:
        return np.array([[m.phi]]), np.array([m.mu * (1 - m.phi)]), np.array([[1 / m.sigma ** 2]])
    return np.asarray(m.A), np.zeros(m.d), np.linalg.inv(m.Q)


def cross_scale(m, xl, xr):
    """max_ij sum_k |u_ik| |v_jk| with u_i = log2(e) Q^-1 (A xl_i + c - mu), v_j = xr_j - mu,
    mu the mean of the right states: the scale of the cross term's rounding error."""
    A, cf, Qi = _transition(m)
    mu = xr.mean(0)
    u = np.log2(np.e) * (xl @ A.T + cf - mu) @ Qi.T
    return float((np.abs(u) @ np.abs(xr - mu).T).max())


def check_tiles_against_oracle(wl, sm, level, m_idx, compute, rows=None):
    """Device tile weights of combination m_idx of `level` against the oracle's FP64 tile
    log-sum-exps on the same particles; returns the worst error and its bound."""
    K, N = sm.K, sm.N
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, m_idx, sm.ws, want=("tiles",))
    shift, delta = dsmc.dsmc_debug_row_shift(sm.cfg, sm.hm, level, m_idx, sm.ws)
    X = sm.X.cpu().numpy().astype(np.float64)
    lw = sm.logw.cpu().numpy().astype(np.float64)
    pairs = sm.pairs.cpu().numpy()
    a, c, iL, iR = endpoint_indices(pairs, K, N, level, m_idx)
    b = min(a + 2 * (1 << level), K) - 1
    rows = np.arange(N) if rows is None else rows
    wl_ = (lw[c - 1][iL] if level == 0 else np.full(N, -np.log(N)))[rows]
    wr_ = lw[c][iR] if b == c else np.full(N, -np.log(N))
    xl, xr = X[c - 1][iL], X[c][iR]
    ref = core.logw_matrix(wl.model, wl.y.astype(np.float32).astype(np.float64), K, c, xl[rows], xr, wl_, wr_)
    B, nT = dbg["B"], dbg["nT"]
    ref_t = np.stack([np.logaddexp.reduce(ref[:, k * B:min((k + 1) * B, N)], axis=1) for k in range(nT)], axis=1)
    t = dbg["tiles"].cpu().numpy().astype(np.float64)[rows]
    sh = shift.cpu().numpy()[rows][:, None] + delta.cpu().numpy().astype(np.float64)[rows][:, None] * LN2
    big = t > 1e-6 * t.max(axis=1, keepdims=True)
    got = sh + np.log(np.where(big, t, 1.0))
    err = np.abs(got - ref_t)[big]
    tol = LN2 * (2.05 * TC_UNIT.get(compute, 0.0) * cross_scale(wl.model, xl, xr) + 0.01) + 1e-4 * max(1.0, np.abs(ref_t).max())
    return float(err.max()), float(tol), dbg


@pytest.mark.parametrize("compute", [dsmc.TF32, dsmc.BF16])
@pytest.mark.parametrize("name,K,N,level", [("lgssm_d8", 16, 1000, 0), ("lgssm_d8", 9, 300, 3),
                                            ("lgssm_d4", 8, 2500, 1), ("sv", 6, 64, 0), ("sv", 33, 512, 2),
                                            ("lgssm_1d", 5, 4096, 0), ("lgssm_d16", 4, 256, 0),
                                            ("lgssm_d32", 4, 256, 1)])
def test_tensor_core_tiles_against_fp64_oracle(compute, name, K, N, level):
    wl = W.workload(name, K=K, N=N)
    if compute == dsmc.TF32 and wl.model.d > 16:
        pytest.skip("TF32 cross term: dx <= 16")
    sm = dsmc.Smoother(wl.model, K, N, seed=5, compute=compute, fused_max_merges=-1)
    y = dev(wl.y)
    sm.init(y)
    for l in range(level + 1):
        sm.merge_level(y, l)
    torch.cuda.synchronize()
    M = core.merges_at_level(K, level)
    rows = None if N <= 1024 else np.random.default_rng(1).choice(N, 256, replace=False)
    err, tol, _ = check_tiles_against_oracle(wl, sm, level, M - 1, compute, rows)
    assert err < tol, (err, tol)
    assert sm.status() == 0


def _headline_sequences(n=2):
    bw = W.batch_workload(256, 512)
    order = np.argsort(bw.Ks)[::-1][:n]
    return bw, [int(i) for i in order]


def test_headline_shape_levels_against_oracle():
    """Two full-length sequences of the batched d = 4 workload, N = 512, BF16, the bench's
    schedule (no fused level, up to 16384 combinations per launch): at the bottom, middle
    and top levels, the last combination's tile weights (64 sampled rows) against the FP64
    oracle and its indices bit-exact against the device-precision sampler."""
    bw, idx = _headline_sequences()
    N = bw.N
    for s in idx:
        K = int(bw.Ks[s])
        wl = W.Workload(f"batch_seq{s}", bw.model, K, N, bw.ys[s], None)
        sm = dsmc.Smoother(bw.model, K, N, seed=1000 + s, compute=dsmc.BF16, fused_max_merges=-1,
                           max_merges_per_launch=16384)
        y = dev(bw.ys[s])
        sm.init(y)
        L = levels(K)
        for level in range(L):
            sm.merge_level(y, level)
            if level not in (0, L // 2, L - 1):
                continue
            torch.cuda.synchronize()
            M = core.merges_at_level(K, level)
            rows = np.random.default_rng(level).choice(N, 64, replace=False)
            err, tol, dbg = check_tiles_against_oracle(wl, sm, level, M - 1, dsmc.BF16, rows)
            assert err < tol, (s, level, err, tol)
            full = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("r", "tiles", "e"))
            li, ri = core.kp_dense_pairs(full["r"].cpu().numpy(), full["tiles"].cpu().numpy(),
                                         full["e"].cpu().numpy(), full["B"], sm.cfg.seed, full["gid"], 0, N)
            pairs = sm.pairs.cpu().numpy()
            np.testing.assert_array_equal(pairs[full["gid"], 0], li)
            np.testing.assert_array_equal(pairs[full["gid"], 1], ri)
        assert sm.status() == 0


@pytest.mark.parametrize("tc_fused", [-1, 1])
def test_headline_shape_batched_means_and_alone(tc_fused):
    """The batched call (BF16, schedule (-1, 16384), split kernels or the fused tensor-core
    level kernel) on the two longest sequences: seed-averaged means within Monte Carlo error
    of Kalman/RTS, and the pairs of each sequence equal to its own single-sequence smoothing."""
    bw, idx = _headline_sequences()
    N = bw.N
    Ks = [int(bw.Ks[s]) for s in idx]
    ys = [dev(bw.ys[s]) for s in idx]
    R = 16
    means = [[] for _ in idx]
    b = dsmc.BatchSmoother(bw.model, Ks, N, seeds=[0] * len(idx), compute=dsmc.BF16, fused_max_merges=-1,
                           max_merges_per_launch=16384, tc_fused=tc_fused)
    b.set_inputs(ys)
    for r in range(R):
        b.seeds = [1000 + 7 * r + k for k in range(len(idx))]
        b.smooth()
        for k in range(len(idx)):
            means[k].append(b.mean[k].cpu().numpy().copy())
    assert b.status() == 0
    for k, s in enumerate(idx):
        ms, _, _ = kalman.rts_for(bw.model, bw.ys[s])
        _check(np.array(means[k]), ms)
    # the last batch equals each sequence smoothed alone with the same seed
    for k, s in enumerate(idx):
        sm = dsmc.Smoother(bw.model, Ks[k], N, seed=b.seeds[k], compute=dsmc.BF16, fused_max_merges=-1,
                           max_merges_per_launch=16384, tc_fused=tc_fused)
        sm.smooth(ys[k])
        torch.cuda.synchronize()
        assert torch.equal(sm.pairs, b.pairs[k])
        assert torch.equal(sm.mean, b.mean[k])
