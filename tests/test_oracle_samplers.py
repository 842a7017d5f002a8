"""Pins of the oracle's schedule and pair samplers against exact laws (CPU only).

The N x N pair law of Eq. (normalized-weights) is a finite categorical distribution; at
small N it is enumerated exactly and the samplers are checked by chi-square tests on many
independent slots.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import core
from paper_2202_02264_gb300 import workloads as W


def alg6_merges(K):
    """Appendix A, Algorithm 6 run literally with 1-based indices and padding flags b_t:
    returns the (level, a, c, b) of every combination in 0-based inclusive time indices."""
    L = 0
    while 2 ** L < K:
        L += 1
    b = [None] + [1] * K + [0] * (2 ** L - K)   # b[1..2^L]
    out = []
    for l in range(L):
        size = 2 ** l
        for n in range(1, 2 ** (L - l) + 1, 2):   # adjacent (odd, even) Y pairs
            if 1 + n * size <= 2 ** L and b[1 + n * size] == 1:
                a = (n - 1) * size
                c = n * size
                e = min((n + 1) * size, K) - 1
                out.append((l, a, c, e))
    return out


@pytest.mark.parametrize("K", list(range(1, 34)) + [100, 127, 128, 129, 1000, 1024])
def test_schedule_matches_algorithm6(K):
    ms = alg6_merges(K)
    assert len(ms) == K - 1
    L = core.num_levels(K)
    assert L == (0 if K == 1 else math.ceil(math.log2(K)))
    for l in range(L):
        assert core.merges_at_level(K, l) == sum(1 for m in ms if m[0] == l)
    # every merge's right block starts before K; blocks are left-aligned powers of two
    for (l, a, c, e) in ms:
        assert a % (2 ** (l + 1)) == 0 and c == a + 2 ** l and c < K and e < K


def _chi2(li, ri, P):
    N = P.shape[0]
    counts = np.bincount(li.astype(np.int64) * N + ri, minlength=N * N).astype(np.float64)
    p = P.reshape(-1)
    keep = p > 0
    assert counts[~keep].sum() == 0, "a zero-probability pair was drawn"
    exp = p[keep] / p[keep].sum() * counts.sum()
    return stats.chisquare(counts[keep], exp).pvalue


def _model_logW(N, seed):
    """Exact FP64 log-weights of one combination of a 2-D linear-Gaussian model, built from
    scipy densities (independent of the oracle's own density code)."""
    m = W.lgssm_dn(2)
    rng = np.random.default_rng(seed)
    xl = rng.standard_normal((N, 2))
    xr = rng.standard_normal((N, 2)) + 0.3
    wl = np.log(rng.dirichlet(np.ones(N)))
    wr = np.log(rng.dirichlet(np.ones(N)))
    y = np.array([[0.1, -0.2], [0.4, 0.2]])
    out = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            out[i, j] = (stats.multivariate_normal(m.A @ xl[i], m.Q).logpdf(xr[j])
                         + stats.multivariate_normal(xr[j], m.R).logpdf(y[1])
                         - stats.norm(y[1], 1.0).logpdf(xr[j]).sum() + wl[i] + wr[j])
    got = core.logw_matrix(m, y, 2, 1, xl, xr, wl, wr)
    np.testing.assert_allclose(got, out, atol=1e-11)
    return out


@pytest.mark.parametrize("N", [2, 3, 4])
def test_dense_sampler_chi_square(N):
    logW = _model_logW(N, N)
    P = np.exp(logW - logW.max())
    P /= P.sum()
    li, ri = core.dense_pairs(logW, seed=99, gid=5, n0=0, n1=200_000)
    assert _chi2(li, ri, P) > 1e-3


def test_dense_sampler_asymmetric_orientation():
    """Row index = left block (time c-1), column = right block: a matrix with all its mass
    in one off-diagonal cell exposes a transposition."""
    logW = np.full((3, 3), -50.0)
    logW[0, 2] = 0.0
    li, ri = core.dense_pairs(logW, seed=1, gid=0, n0=0, n1=1000)
    assert (li == 0).all() and (ri == 2).all()


@pytest.mark.parametrize("N", [3, 4])
def test_rejection_sampler_chi_square(N):
    logW = _model_logW(N, 10 + N)
    P = np.exp(logW - logW.max())
    P /= P.sum()
    li, ri, att, st = core.rs_pairs(logW, logW.max() + 0.3, seed=7, gid=3, n0=0, n1=100_000)
    assert st == 0
    assert _chi2(li, ri, P) > 1e-3
    # expected attempts per slot = N^2 wbar / sum(omega)
    expect = N * N * np.exp(logW.max() + 0.3) / np.exp(logW).sum()
    assert att / 100_000 == pytest.approx(expect, rel=0.03)


def test_rejection_sampler_cap():
    logW = np.full((4, 4), -30.0)
    li, ri, att, st = core.rs_pairs(logW, 0.0, seed=7, gid=3, n0=0, n1=8, max_attempts=16)
    assert st == 8 and att == 8 * 16
    assert ((0 <= li) & (li < 4)).all() and ((0 <= ri) & (ri < 4)).all()


def _q24(x, ref):
    """floor(x 2^(24 - E)) with 2^(E-2) <= ref < 2^(E-1): the fixed-point image the sampler
    uses for weights below twice their reference, from numpy's frexp (independent of the
    oracle's bit manipulation)."""
    _, e_ref = np.frexp(np.float64(ref))      # ref = m 2^e_ref, m in [0.5, 1)
    E = int(e_ref) + 1
    x = np.asarray(x, np.float64)
    out = np.minimum(np.floor(np.ldexp(x, min(24 - E, 127))), 2.0**32 - 1)
    out[(x <= 0) | (np.abs(x) < np.finfo(np.float32).tiny)] = 0
    return out


def _kp_law(r, t, e, B):
    """Exact law of the three-stage sampler: rows by the truncated 2^40 fixed-point weights,
    tiles and columns by their fixed-point images."""
    N = r.shape[0]
    nT = t.shape[1]
    Rq = np.floor(np.clip(r.astype(np.float64), 0, 1) * 2.0**40)
    P = np.zeros((N, N))
    for i in range(N):
        qt = _q24(t[i], t[i].max())
        for k in range(nT):
            j0, j1 = k * B, min((k + 1) * B, N)
            qe = _q24(e[i, j0:j1], t[i, k])
            if qe.sum() == 0 or qt.sum() == 0:
                continue
            P[i, j0:j1] = Rq[i] / Rq.sum() * qt[k] / qt.sum() * qe / qe.sum()
    return P


def test_kp_dense_sampler_chi_square():
    rng = np.random.default_rng(4)
    N, B = 7, 3            # three tiles, the last one ragged (one column)
    nT = 3
    r = rng.uniform(0.05, 1, N).astype(np.float32)
    r[2] = 0.0             # a zero row is never chosen
    r[r.argmax()] = 1.0
    e = rng.uniform(0, 1, (N, N)).astype(np.float32)
    e[:, 4] = 0.0          # a zero column is never chosen
    e[5] *= np.float32(1e-30)   # a row far below 1: the fixed point scales per row
    t = np.stack([[e[i, k * B:(k + 1) * B].sum() for k in range(nT)] for i in range(N)]).astype(np.float32)
    li, ri = core.kp_dense_pairs(r, t, e, B, seed=3, gid=11, n0=0, n1=300_000)
    P = _kp_law(r, t, e, B)
    assert (li != 2).all() and (ri != 4).all()
    assert _chi2(li, ri, P) > 1e-3
    # the fixed-point law is the plain product law of the weights to 2^-23: the same draws
    # pass against r_i / sum r * t_ik / sum_k t_ik * e_ij / sum_(j in tile k) e_ij directly
    rd, td, ed = r.astype(np.float64), t.astype(np.float64), e.astype(np.float64)
    Pw = np.zeros((N, N))
    for i in range(N):
        for k in range(nT):
            j0, j1 = k * B, min((k + 1) * B, N)
            if ed[i, j0:j1].sum() > 0:
                Pw[i, j0:j1] = rd[i] / rd.sum() * td[i, k] / td[i].sum() * ed[i, j0:j1] / ed[i, j0:j1].sum()
    assert _chi2(li, ri, Pw) > 1e-3


def test_kp_dense_sampler_zero_tail_and_single_row():
    """All mass in one row and its last (ragged) tile: every draw lands there."""
    N, B = 5, 2
    r = np.zeros(N, np.float32)
    r[3] = 1.0
    e = np.zeros((N, N), np.float32)
    e[3, 4] = 0.25
    t = np.zeros((N, 3), np.float32)
    t[3, 2] = 0.25
    li, ri = core.kp_dense_pairs(r, t, e, B, seed=3, gid=0, n0=0, n1=500)
    assert (li == 3).all() and (ri == 4).all()


def test_kp_fixed_point_image():
    """The bit-pattern quantisation equals floor(x 2^(24-E)) computed through frexp/ldexp."""
    rng = np.random.default_rng(9)
    N = B = 64                                 # one tile per row
    for scale in [1.0, 1e-20, 1e20]:
        e = (rng.uniform(0, 1, (N, N)) * scale).astype(np.float32)
        t = e.sum(1, keepdims=True).astype(np.float32)
        for i in [0, 17, 63]:
            q_ref = _q24(e[i], t[i, 0])
            rr = np.zeros(N, np.float32)
            rr[i] = 1.0                        # all row weight on row i
            li, ri = core.kp_dense_pairs(rr, t, e, B, seed=5, gid=i, n0=0, n1=20000)
            assert (li == i).all()
            p = q_ref / q_ref.sum()
            counts = np.bincount(ri, minlength=B)
            assert stats.chisquare(counts, p * counts.sum()).pvalue > 1e-3
