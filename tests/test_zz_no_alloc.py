"""The allocation-free entry point dsmc_smooth_noalloc, called through the C ABI.

Some callers cannot allocate device memory (their host owns every allocation, or forbids
cudaMalloc once running); dsmc_smooth_noalloc runs the same smoother on a fixed scratch
array inside the library.  Checked against dsmc_smooth on two calls in a row, each with
its own seed, and against the size limit.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _run(dsmc, W, m, y, K, N, seed, noalloc):
    sm = dsmc.Smoother(m, K, N, seed=seed, want_traj=True)
    if noalloc:
        st = dsmc.dsmc_smooth_noalloc(sm.cfg, sm.hm, sm.prop, y, sm.state, sm.traj, sm.mean,
                                      sm.m2, sm.logL_out)
    else:
        sm.smooth(y)
        st = sm.status()
    torch.cuda.synchronize()
    return st, sm.pairs.cpu().numpy(), sm.mean.cpu().numpy(), sm.traj.cpu().numpy(), float(sm.logL_out.item())


def test_noalloc_matches_dsmc_smooth_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import build, dsmc, workloads as W
    build.build()
    dsmc.load()
    m = W.lgssm_dn(4)
    K, N = 100, 256
    _, yh = W.simulate(m, K, 123)
    y = torch.as_tensor(yh, dtype=torch.float32, device="cuda")
    for seed in (7, 8):                       # two calls in a row on the shared scratch
        st0, p0, m0, t0, l0 = _run(dsmc, W, m, y, K, N, seed, noalloc=False)
        st1, p1, m1, t1, l1 = _run(dsmc, W, m, y, K, N, seed, noalloc=True)
        assert st0 == 0 and st1 == 0
        np.testing.assert_array_equal(p1, p0)
        np.testing.assert_array_equal(t1, t0)
        np.testing.assert_allclose(m1, m0, rtol=1e-12, atol=1e-12)
        assert l1 == pytest.approx(l0, abs=1e-9)


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2202_02264_gb300 import dsmc, workloads as W
    m = W.lgssm_d8()
    K, N = 1024, 1024
    hm = dsmc.HostModel(m)
    cfg = dsmc.make_config(K, N, 1)
    assert dsmc.dsmc_workspace_size(cfg, hm) > 32 << 20
    sm = dsmc.Smoother(m, K, N, seed=1)
    y = torch.zeros((K, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(dsmc.DsmcError) as e:
        dsmc.dsmc_smooth_noalloc(sm.cfg, sm.hm, sm.prop, y, sm.state, None, sm.mean, None, None)
    assert e.value.code == 3 and "static scratch" in str(e.value)
