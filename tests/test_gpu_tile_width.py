"""The tile width of the row tile sums (`tile_cols`), which the autotuner searches (through the
C ABI): with 64-column tiles at N = 512 the draws are still bit-exact against the oracle's
device-precision sampler fed the device's own weights (the 64-column tiles go through the
two-half column stage), the tile sums are sums of their pair weights, and the smoothing
means of a batched call land on Kalman/RTS."""
import numpy as np
import pytest
import torch

from gpu_helpers import _check, dev
from oracle import core, kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


@pytest.mark.parametrize("compute", [dsmc.FP32, dsmc.BF16])
@pytest.mark.parametrize("level", [0, 2])
def test_wide_tiles_indices_bit_exact(compute, level):
    K, N = 21, 512
    wl = W.workload("lgssm_d4", K=K, N=N)
    sm = dsmc.Smoother(wl.model, K, N, seed=31, compute=compute, fused_max_merges=-1, tile_cols=64)
    y = dev(wl.y)
    sm.init(y)
    for l in range(level + 1):
        sm.merge_level(y, l)
    torch.cuda.synchronize()
    M = core.merges_at_level(K, level)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("r", "tiles", "e", "rowsum"))
    assert dbg["B"] == 64 and dbg["nT"] == 8
    tiles = dbg["tiles"].cpu().numpy()
    e = dbg["e"].cpu().numpy().astype(np.float64)   # the pair weights 2^(e_ij) the draws recompute
    if compute == dsmc.FP32:   # each tile weight is the sum of its 64 pair weights
        ref = np.stack([e[:, 64 * k:64 * (k + 1)].sum(1) for k in range(8)], axis=1)
        np.testing.assert_allclose(tiles, ref, rtol=2e-5, atol=0)
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), tiles, dbg["e"].cpu().numpy(), dbg["B"], sm.cfg.seed,
                                 dbg["gid"], 0, N)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


def test_wide_tiles_batched_means_on_rts():
    bw = W.batch_workload(6, 512)
    Ks = [int(k) for k in bw.Ks]
    R = 16
    b = dsmc.BatchSmoother(bw.model, Ks, 512, seeds=[0] * len(Ks), compute=dsmc.BF16, fused_max_merges=-1,
                           max_merges_per_launch=16384, tile_cols=64)
    b.set_inputs([dev(y) for y in bw.ys])
    means = [[] for _ in Ks]
    for r in range(R):
        b.seeds = [2000 + 11 * r + k for k in range(len(Ks))]
        b.smooth()
        for k in range(len(Ks)):
            means[k].append(b.mean[k].cpu().numpy().copy())
    assert b.status() == 0
    for k in range(len(Ks)):
        ms, _, _ = kalman.rts_for(bw.model, bw.ys[k])
        _check(np.array(means[k]), ms)
