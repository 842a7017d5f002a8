"""Batched smoothing through the C ABI: many sequences of one model and N in one call, the
combinations of each level launched together.  Each sequence's draws depend only on its
own seed, counter base and combination ids, so every result equals the single-sequence
smoothing of that sequence alone (bit for bit), whatever else is in the batch."""
import numpy as np
import pytest
import torch

from oracle import kalman
from paper_2202_02264_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda").contiguous()


def _single(model, y, K, N, seed, base, compute, fused, x_ref=None):
    sm = dsmc.Smoother(model, K, N, seed=seed, compute=compute, fused_max_merges=fused)
    sm.set_seed(seed, counter_base=base)
    yd = dev(y)
    if x_ref is None:
        sm.smooth(yd)
        xo = None
    else:
        xo = torch.empty_like(x_ref)
        sm.conditional(yd, x_ref, xo)
    torch.cuda.synchronize()
    assert sm.status() == 0
    return sm.pairs.clone(), sm.mean.clone(), float(sm.logL_out.item()), xo


@pytest.mark.parametrize("name,N,compute,fused", [("lgssm_d4", 96, dsmc.FP32, 0),
                                                  ("lgssm_d8", 70, dsmc.FP32, 0),
                                                  ("sv", 64, dsmc.FP32, 0),
                                                  ("lgssm_d4", 128, dsmc.BF16, -1),
                                                  ("lgssm_d8", 256, dsmc.TF32, -1)])
def test_batch_equals_each_sequence_alone(name, N, compute, fused):
    Ks = [1, 2, 3, 7, 16, 33, 64, 100]
    rng = np.random.default_rng(7)
    base_wl = W.workload(name, K=max(Ks), N=N)
    model = base_wl.model
    ys = [W.simulate(model, K, 100 + i)[1] for i, K in enumerate(Ks)]
    seeds = [int(s) for s in rng.integers(1, 2**40, len(Ks))]
    bases = [0, 3, 0, 5, 0, 0, 11, 2]
    cond = [False, False, True, False, True, False, False, True] if N >= 2 else [False] * len(Ks)
    x_in = [dev(W.simulate(model, K, 500 + i)[0]) if c else None for i, (K, c) in enumerate(zip(Ks, cond))]
    x_out = [torch.empty_like(x) if x is not None else None for x in x_in]
    b = dsmc.BatchSmoother(model, Ks, N, seeds=seeds, compute=compute, fused_max_merges=fused)
    b.counter_base = bases
    b.set_inputs([dev(y) for y in ys], x_in, x_out)
    b.smooth()
    torch.cuda.synchronize()
    assert b.status() == 0
    for i, K in enumerate(Ks):
        p, m, ll, xo = _single(model, ys[i], K, N, seeds[i], bases[i], compute, fused, x_in[i])
        assert torch.equal(b.pairs[i], p), i
        assert torch.equal(b.mean[i], m), i
        assert float(b.logL_out[i].item()) == ll or (np.isnan(ll) and np.isnan(float(b.logL_out[i].item()))), i
        if cond[i]:
            assert torch.equal(x_out[i], xo), i


def test_batch_replay_in_a_cuda_graph():
    """dsmc_batch_run holds no host synchronisation: captured once in a CUDA graph, a replay
    recomputes the batch and gives the same results as the direct call."""
    Ks = [17, 40, 64, 5]
    model = W.lgssm_d4()
    N = 64
    ys = [dev(W.simulate(model, K, 900 + i)[1]) for i, K in enumerate(Ks)]
    b = dsmc.BatchSmoother(model, Ks, N, seeds=[5, 6, 7, 8])
    b.set_inputs(ys)
    b.prepare()
    b.run()
    torch.cuda.synchronize()
    ref = [m.clone() for m in b.mean]
    for m in b.mean:
        m.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    for a, r in zip(b.mean, ref):
        assert torch.equal(a, r)


def test_batch_means_vs_rts_ragged_lengths():
    """The configuration shape of the batched workload (uneven K including non-powers of
    two) at a reduced count: means within Monte Carlo error of the Kalman/RTS means."""
    model = W.lgssm_d4()
    Ks = [64, 100, 257, 513]
    N = 256
    R = 16
    ys = [W.simulate(model, K, 1300 + i)[1] for i, K in enumerate(Ks)]
    g = [[] for _ in Ks]
    b = dsmc.BatchSmoother(model, Ks, N, compute=dsmc.BF16)
    b.set_inputs([dev(y) for y in ys])
    for r in range(R):
        b.seeds = [7000 + 131 * r + i for i in range(len(Ks))]
        b.smooth()
        torch.cuda.synchronize()
        assert b.status() == 0
        for i in range(len(Ks)):
            g[i].append(b.mean[i].cpu().numpy().copy())
    from scipy import stats as _st
    zs, single = [], []
    for i, K in enumerate(Ks):
        ms, _, _ = kalman.rts_for(model, ys[i])
        G = np.array(g[i])
        sd = G.std(0, ddof=1)
        zs.append((np.abs(G.mean(0) - ms) / (sd / np.sqrt(R))).ravel())
        single.append((np.abs(G - ms[None]) <= 3 * sd[None]).ravel())
    # seed-averaged means: z is t-distributed with R - 1 degrees of freedom when unbiased
    z = np.concatenate(zs)
    p3 = 2 * _st.t.sf(3.0, R - 1)
    allowed = z.size * p3 + 4 * np.sqrt(z.size * p3) + 1
    assert (z > 3).sum() <= allowed, ((z > 3).sum(), allowed)
    assert z.max() < 7.0, z.max()
    assert np.concatenate(single).mean() >= 0.985
