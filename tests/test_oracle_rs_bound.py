"""The bound of Algorithm 8 (reading of the paper), brute force on random combinations:
every pair's log-weight lies below the hull bound used for one-dimensional states, which
lies below the finite-set bound; a particle planted far in the proposal's tail moves the
finite-set bound and leaves the hull bound where the pairs are."""
import numpy as np
import pytest

from oracle import core
from paper_2202_02264_gb300 import workloads as W


def _case(model, K, N, seed, c=3, outlier=None):
    rng = np.random.default_rng(seed)
    _, y = W.simulate(model, K, 500 + seed)
    xl = rng.normal(-1.0, 1.0, (N, 1))
    xr = rng.normal(-1.0, 1.0, (N, 1))
    if outlier is not None:
        xr[0, 0] = outlier
    wl = rng.normal(0.0, 0.5, N)
    wr = rng.normal(0.0, 0.5, N)
    wl -= np.log(np.exp(wl).sum())
    wr -= np.log(np.exp(wr).sum())
    return y, xl, xr, wl, wr


@pytest.mark.parametrize("name", ["sv", "lgssm_1d"])
@pytest.mark.parametrize("seed", range(6))
def test_pairs_below_hull_bound_below_finite_bound(name, seed):
    K, N = 8, 48
    model = W.sv(K) if name == "sv" else W.lgssm_1d()
    y, xl, xr, wl, wr = _case(model, K, N, seed)
    logW = core.logw_matrix(model, y, K, 3, xl, xr, wl, wr)
    fin, hull = core.rs_bounds(model, y, K, 3, xl, xr, wl, wr)
    assert logW.max() <= hull + 1e-9
    assert hull <= fin + 1e-12


def test_tail_particle_sets_the_finite_bound_not_the_hull_bound():
    K, N = 8, 48
    model = W.sv(K)
    base = _case(model, K, N, 11)
    far = _case(model, K, N, 11, outlier=4.5)         # far above every transition mean
    fin0, hull0 = core.rs_bounds(model, base[0], K, 3, *base[1:])
    fin1, hull1 = core.rs_bounds(model, far[0], K, 3, *far[1:])
    logW1 = core.logw_matrix(model, far[0], K, 3, *far[1:])
    assert fin1 > fin0 + 2.0                           # the tail particle raised it
    assert hull1 < fin1 - 2.0                          # the hull bound did not follow
    assert logW1.max() <= hull1 + 1e-9
