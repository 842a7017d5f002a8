"""The fused tensor-core level kernel (tc_fused > 0: operand rows, tcgen05 cross term,
exponentials, row CDF and draws of a combination in one persistent warp-specialised kernel)
against the split kernels (through the C ABI).  The fused kernel repeats the split path's
arithmetic function for function, so pairs, means, second moments and log L are equal bit
for bit; with the inspection switch on it also stores its intermediate weights, which then
reproduce its indices through the oracle's device-precision sampler and its tile sums match
the FP64 oracle within the precision's bound."""
import numpy as np
import pytest
import torch

from oracle import core, kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

from gpu_helpers import _check, dev
from test_gpu_tensor_core_oracle import check_tiles_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build
    build.build()
    dsmc.load()


def _run(wl, K, N, compute, tc, resampler=dsmc.MULTINOMIAL, cond=False, chunk=0, seed=77):
    sm = dsmc.Smoother(wl.model, K, N, seed=seed, compute=compute, resampler=resampler, fused_max_merges=-1,
                       tc_fused=tc, max_merges_per_launch=chunk)
    sm.m2 = torch.empty_like(sm.mean)
    y = dev(wl.y)
    if cond:
        xin = dev(np.asarray(wl.x_true, np.float32).reshape(K, -1))
        xout = torch.empty_like(xin)
        sm.conditional(y, xin, xout)
        extra = xout
    else:
        sm.smooth(y)
        extra = sm.m2
    torch.cuda.synchronize()
    return sm, extra


@pytest.mark.parametrize("name,K,N,compute,resampler,cond", [
    ("lgssm_d4", 37, 512, dsmc.BF16, dsmc.MULTINOMIAL, False),
    ("lgssm_d4", 100, 500, dsmc.BF16, dsmc.MULTINOMIAL, False),
    ("lgssm_d4", 64, 256, dsmc.TF32, dsmc.MULTINOMIAL, False),
    ("lgssm_1d", 33, 97, dsmc.BF16, dsmc.MULTINOMIAL, False),
    ("sv", 129, 384, dsmc.BF16, dsmc.MULTINOMIAL, False),
    ("sv", 40, 512, dsmc.TF32, dsmc.SYSTEMATIC, False),
    ("lgssm_dn2", 20, 130, dsmc.BF16, dsmc.MULTINOMIAL, False),
    ("lgssm_d4", 45, 512, dsmc.BF16, dsmc.MULTINOMIAL, True),
    ("sv", 16, 64, dsmc.BF16, dsmc.MULTINOMIAL, True),
    ("lgssm_d4", 3, 2, dsmc.BF16, dsmc.MULTINOMIAL, False),
])
def test_fused_tc_equals_split(name, K, N, compute, resampler, cond):
    if name == "lgssm_dn2":
        m = W.lgssm_dn(2)
        _, y = W.simulate(m, K, 5)
        wl = W.Workload("lgssm_dn2", m, K, N, y, None)
    else:
        wl = W.workload(name, K=K, N=N)
    a, xa = _run(wl, K, N, compute, -1, resampler, cond)
    b, xb = _run(wl, K, N, compute, 1, resampler, cond)
    assert a.status() == 0 and b.status() == 0
    assert torch.equal(a.pairs, b.pairs)
    assert torch.equal(a.mean, b.mean)
    assert torch.equal(a.logL_out, b.logL_out)
    assert torch.equal(xa, xb)


def test_fused_tc_chunking_and_batch_equal_split():
    """A batch of uneven sequences (N = 512, BF16): the fused kernel over chunks of 64
    combinations equals the split kernels, sequence by sequence."""
    bw = W.batch_workload(12, 512, lo=40, hi=700)
    Ks = [int(k) for k in bw.Ks]
    ys = [dev(y) for y in bw.ys]
    outs = []
    for tc, chunk in ((-1, 0), (1, 64), (1, 0)):
        b = dsmc.BatchSmoother(bw.model, Ks, 512, compute=dsmc.BF16, fused_max_merges=-1,
                               max_merges_per_launch=chunk, tc_fused=tc)
        b.set_inputs(ys)
        b.smooth()
        torch.cuda.synchronize()
        assert b.status() == 0
        outs.append(([p.clone() for p in b.pairs], [m.clone() for m in b.mean], b.logL_out.clone()))
    for o in outs[1:]:
        assert all(torch.equal(x, y) for x, y in zip(outs[0][0], o[0]))
        assert all(torch.equal(x, y) for x, y in zip(outs[0][1], o[1]))
        assert torch.equal(outs[0][2], o[2])


@pytest.mark.parametrize("name,K,N,level", [("lgssm_d4", 16, 512, 0), ("lgssm_d4", 40, 300, 3), ("sv", 20, 128, 2)])
def test_fused_tc_inspection_indices_and_oracle(name, K, N, level):
    wl = W.workload(name, K=K, N=N)
    dsmc.dsmc_debug_keep_weights(True)
    try:
        sm = dsmc.Smoother(wl.model, K, N, seed=5, compute=dsmc.BF16, fused_max_merges=-1, tc_fused=1)
        y = dev(wl.y)
        sm.init(y)
        for l in range(level + 1):
            sm.merge_level(y, l)
        torch.cuda.synchronize()
    finally:
        dsmc.dsmc_debug_keep_weights(False)
    M = core.merges_at_level(K, level)
    err, tol, _ = check_tiles_against_oracle(wl, sm, level, M - 1, dsmc.BF16)
    assert err < tol, (err, tol)
    dbg = dsmc.dsmc_debug_merge_weights(sm.cfg, sm.hm, level, M - 1, sm.ws, want=("r", "tiles", "e"))
    li, ri = core.kp_dense_pairs(dbg["r"].cpu().numpy(), dbg["tiles"].cpu().numpy(), dbg["e"].cpu().numpy(),
                                 dbg["B"], sm.cfg.seed, dbg["gid"], 0, N)
    pairs = sm.pairs.cpu().numpy()
    np.testing.assert_array_equal(pairs[dbg["gid"], 0], li)
    np.testing.assert_array_equal(pairs[dbg["gid"], 1], ri)
    assert sm.status() == 0


def test_fused_tc_means_vs_rts():
    m = W.lgssm_d4()
    K, N = 200, 512
    _, y = W.simulate(m, K, 77)
    ms, _, _ = kalman.rts_for(m, y)
    sm = dsmc.Smoother(m, K, N, seed=1000, compute=dsmc.BF16, tc_fused=1)
    yd = dev(y)
    g = []
    for r in range(24):
        sm.set_seed(1000 + r)
        g.append(sm.smooth(yd).cpu().numpy().copy())
    assert sm.status() == 0
    _check(np.array(g), ms)


def test_fused_tc_wait_runs_out_and_reports_timeout():
    """With the test switch on, the fused kernel's control thread issues no MMA: the epilogue's
    bounded wait runs out, every role stops, DSMC_ERR_TIMEOUT is recorded, the tensor memory is
    freed, and the next smoothing on the same context runs clean."""
    wl = W.workload("lgssm_d4", K=8, N=256)
    y = dev(wl.y)
    sm = dsmc.Smoother(wl.model, 8, 256, seed=3, compute=dsmc.BF16, fused_max_merges=-1, tc_fused=1)
    sm.init(y)
    dsmc.dsmc_debug_stall_tensor_cores(True)
    try:
        sm.merge_level(y, 0)
        torch.cuda.synchronize()
    finally:
        dsmc.dsmc_debug_stall_tensor_cores(False)
    assert sm.status() == 9
    sm2 = dsmc.Smoother(wl.model, 8, 256, seed=3, compute=dsmc.BF16, fused_max_merges=-1, tc_fused=1)
    sm2.smooth(y)
    torch.cuda.synchronize()
    assert sm2.status() == 0
    assert torch.isfinite(sm2.mean).all()
