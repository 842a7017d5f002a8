"""Helpers shared by the GPU tests: device tensors, the Algorithm 6 schedule, endpoint
indices of a combination by composing stored pairs, and the seed-averaged Monte Carlo check
of smoothing means against a reference."""
import numpy as np
import torch

from oracle import core
from paper_2202_02264_gb300 import dsmc


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def levels(K):
    L = 0
    while (1 << L) < K:
        L += 1
    return L


def level_offsets(K):
    L = levels(K)
    offs = [0]
    for l in range(L):
        offs.append(offs[-1] + core.merges_at_level(K, l))
    return offs


def endpoint_indices(pairs, K, N, level, m):
    """Particle indices of the left block at c-1 and the right block at c, by composing the
    stored pairs (the same walk the oracle test pins against explicit copies)."""
    offs = level_offsets(K)
    size = 1 << level
    a = 2 * m * size
    c = a + size

    def walk(t, top):
        sig = np.arange(N)
        for l in range(top - 1, -1, -1):
            sz = 1 << l
            p = (t // (2 * sz)) * 2 * sz
            if p + sz >= K:
                continue
            g = offs[l] + p // (2 * sz)
            sig = pairs[g, 1 if t >= p + sz else 0][sig]
        return sig

    return a, c, walk(c - 1, level), walk(c, level)


def _gpu_means(m, y, K, N, R, resampler=dsmc.MULTINOMIAL, seed0=1000):
    sm = dsmc.Smoother(m, K, N, seed=seed0, resampler=resampler)
    yd = dev(y)
    out = []
    for r in range(R):
        sm.set_seed(seed0 + r)
        out.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    return np.array(out)


def _check(means, ref, family_alpha=1e-3, cover=0.985):
    """Seed-averaged means against a reference: z = (mean_R - ref) / (sd / sqrt(R)) is
    t-distributed with R - 1 degrees of freedom when dSMC is unbiased at this N.  The number
    of |z| > 3 must stay within a binomial bound of its expectation; no |z| may reach the
    larger of 6.5 and the t quantile at which any of the n coordinates exceeds it with
    probability family_alpha (7.5 for R = 24 and n = 8192: with few seeds the t tails are
    heavy); single runs must fall within 3 sd of the reference at the normal rate."""
    from scipy import stats as _st
    R = means.shape[0]
    sd = means.std(0, ddof=1)
    z = np.abs(means.mean(0) - ref) / (sd / np.sqrt(R))
    n = z.size
    p3 = 2 * _st.t.sf(3.0, R - 1)
    allowed = n * p3 + 4 * np.sqrt(n * p3) + 1
    assert (z > 3).sum() <= allowed, ((z > 3).sum(), allowed)
    zmax = max(6.5, _st.t.isf(family_alpha / (2 * n), R - 1))
    assert z.max() < zmax, (z.max(), zmax)
    assert (np.abs(means - ref) <= 3 * sd).mean() >= cover
