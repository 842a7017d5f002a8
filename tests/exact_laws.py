"""Exact finite laws of the pair samplers, written from their definitions with numpy only
(no oracle code): the targets the chi-square pins compare draws against."""
import numpy as np
from scipy import stats

U23_STEPS = 2 ** 23


def u23_grid():
    """The 2^23 values u23 can take, ((k + 0.5) 2^-23), exact in FP32."""
    return ((np.arange(U23_STEPS, dtype=np.float64) + 0.5) * 2.0 ** -23).astype(np.float32)


def accept_count(r):
    """#{u in the u23 grid : u < r} for FP32 r (elementwise): the acceptance count of
    Algorithm 8's test u < ratio out of 2^23."""
    r = np.asarray(r, np.float32).astype(np.float64)
    c = np.ceil(r * U23_STEPS - 0.5)
    return np.clip(c, 0, U23_STEPS)


def mh_accept_count(cur, prop, grid=None):
    """#{u in the u23 grid : fl32(u cur) < prop}: the FP32 move rule of Algorithm 7 on
    ratios (the product rounds once; fl32(u cur) is non-decreasing in u, so a binary
    search over the grid counts it)."""
    g = u23_grid() if grid is None else grid
    cur = np.float32(cur)
    prop = np.float32(prop)
    lo, hi = 0, U23_STEPS          # first k with fl(u_k cur) >= prop
    while lo < hi:
        mid = (lo + hi) // 2
        if np.float32(g[mid] * cur) < prop:
            lo = mid + 1
        else:
            hi = mid
    return lo


def kp_mh_transition(ratio):
    """Transition matrix over the N^2 pairs of the device-precision Algorithm 7 chain:
    uniform proposals, move iff fl32(u r(s)) < r(s') (u on the u23 grid)."""
    r = np.asarray(ratio, np.float32).ravel()
    S = r.size
    g = u23_grid()
    P = np.zeros((S, S))
    for s in range(S):
        for t in range(S):
            if t != s:
                P[s, t] = mh_accept_count(r[s], r[t], g) / U23_STEPS / S
        P[s, s] = 1.0 - P[s].sum()
    return P


def q24(x, ref):
    """floor(x 2^(24 - E)) with 2^(E-2) <= ref < 2^(E-1), from numpy's frexp: the fixed-point
    image the three-stage sampler takes of a weight x >= 0 against its reference."""
    _, e_ref = np.frexp(np.float64(ref))
    E = int(e_ref) + 1
    x = np.asarray(x, np.float64)
    out = np.minimum(np.floor(np.ldexp(x, min(24 - E, 127))), 2.0 ** 32 - 1)
    out[(x <= 0) | (np.abs(x) < np.finfo(np.float32).tiny)] = 0
    return out


def kp_law(r, t, e, B):
    """Exact law of the three-stage sampler: rows by the truncated 2^40 fixed-point weights,
    tiles and columns by their fixed-point images."""
    N = r.shape[0]
    nT = t.shape[1]
    Rq = np.floor(np.clip(r.astype(np.float64), 0, 1) * 2.0 ** 40)
    P = np.zeros((N, N))
    for i in range(N):
        qt = q24(t[i], t[i].max())
        for k in range(nT):
            j0, j1 = k * B, min((k + 1) * B, N)
            qe = q24(e[i, j0:j1], t[i, k])
            if qe.sum() == 0 or qt.sum() == 0:
                continue
            P[i, j0:j1] = Rq[i] / Rq.sum() * qt[k] / qt.sum() * qe / qe.sum()
    return P


def chi2_pvalue(li, ri, P):
    """Chi-square p-value of pair draws (li, ri) against the law P [N][N]; a draw of a
    zero-probability pair fails outright."""
    N = P.shape[0]
    counts = np.bincount(np.asarray(li, np.int64) * N + np.asarray(ri, np.int64),
                         minlength=N * N).astype(np.float64)
    p = P.reshape(-1)
    keep = p > 0
    assert counts[~keep].sum() == 0, "a zero-probability pair was drawn"
    exp = p[keep] / p[keep].sum() * counts.sum()
    return stats.chisquare(counts[keep], exp).pvalue
