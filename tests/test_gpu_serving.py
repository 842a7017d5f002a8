"""The continuous-batching server on the GPU: every request's result is the same alone and
in the mix (bit for bit), whatever joins or leaves the lanes around it and whatever the
budget lets run at once."""
import numpy as np
import pytest
import torch

from paper_2202_02264_gb300 import dsmc, serving as S, workloads as W

pytestmark = pytest.mark.gpu


def _mix(n=12, seed=3):
    rng = np.random.default_rng(seed)
    models = {"lg2": W.lgssm_dn(2), "lg8": W.lgssm_d8(), "sv": W.sv(1)}
    out = []
    for rid in range(n):
        name = ["lg2", "lg8", "sv"][rid % 3]
        N = [64, 96][rng.integers(2)]
        K = int(rng.integers(1, 300))
        m = models[name]
        _, y = W.simulate(m, K, 60000 + rid)
        x_ref = W.simulate(m, K, 61000 + rid)[0] if rid % 5 == 4 else None
        out.append(S.Request(rid, f"{name}/N{N}", m, N, y, 5000 + 17 * rid, 0.0002 * rid, x_ref, rid % 4))
    return out


def _alone(r: S.Request, compute):
    sm = dsmc.Smoother(r.model, r.K, r.N, seed=r.seed, compute=compute)
    sm.set_seed(r.seed, counter_base=r.counter_base)
    y = torch.as_tensor(np.asarray(r.y, np.float32), device="cuda")
    xo = None
    if r.x_ref is None:
        sm.smooth(y)
    else:
        xi = torch.as_tensor(np.asarray(r.x_ref, np.float32), device="cuda")
        xo = torch.empty_like(xi)
        sm.conditional(y, xi, xo)
    torch.cuda.synchronize()
    assert sm.status() == 0
    return sm.mean.cpu().numpy(), float(sm.logL_out.item()), (xo.cpu().numpy() if xo is not None else None)


def _bytes(r):
    return S.request_bytes(r.K, r.N, r.model.d, r.model.prop_kind == W.PROP_GAUSS, r.x_ref is not None)


@pytest.mark.parametrize("compute", [dsmc.FP32, dsmc.BF16])
@pytest.mark.parametrize("tight,realtime", [(False, False), (True, False), (False, True)])
def test_same_alone_and_in_the_mix(compute, tight, realtime):
    reqs = _mix()
    sizes = [_bytes(r) for r in reqs]
    # tight: about a third of the mix fits at once, so requests wait for memory to free up
    budget = max(max(sizes), sum(sizes) // 3) if tight else 10**11
    srv = S.Server(hbm_budget_bytes=budget, precision=lambda m, N: compute, lane_workspaces_in_budget=False)
    res = {r.rid: r for r in srv.run(reqs, realtime=realtime)}
    assert sorted(res) == [r.rid for r in reqs]
    if tight:
        assert srv.sched.peak_active < len(reqs)      # the budget held requests back
        assert srv.sched.peak_used <= budget
    for r in reqs:
        mean, ll, xo = _alone(r, compute)
        got = res[r.rid]
        np.testing.assert_array_equal(got.mean, mean)
        assert got.logL == ll or (np.isnan(ll) and np.isnan(got.logL))
        if r.x_ref is not None:
            np.testing.assert_array_equal(got.x_ref_out, xo)
        assert got.finished >= got.admitted >= 0.0
