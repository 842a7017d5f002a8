#!/usr/bin/env python
"""Throughput of the dSMC smoother (N*T/s) on GB300, with roofline, end-to-end and CPU
oracle baselines.

Default workload (``batched_lgssm_d4``): 256 independent sequences of the 4-dimensional
linear-Gaussian model with lengths uniform in [64, 4096], N = 512 particles, smoothed in one
batched call per step (one launch per level of Algorithm 6 for the whole batch; cross term
on the tensor cores in BF16 with FP32 accumulation).  The same line reports the plain form
(FP32, each sequence smoothed alone, one after another) and the smoothing-mean error of both
against Kalman/RTS.  ``--workload lgssm_d8`` times one sequence of the 8-dimensional model,
K = N = 1024 (cross term in TF32; ``--compute fp32`` for the CUDA-core form).

A step is one full smoothing (of the batch, or of the sequence): Algorithm 2 init, every
level (column/row terms, fused exp / tile sums, row CDF and three-stage pair draws) and the
trajectory resolve with fused means.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

Under torchrun each rank smooths its own independent batch (replicas, weak scaling); no
collective touches the data path, one barrier brackets the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dSMC N·T/s per GB300 (batched mixed vs plain) at fixed error; p50/p99 latency"
UNIT = "N·T/s"
MUFU_EX2_PER_CLK_SM = 32       # measured on GB300 (dsmc_profile_unit_rates), twice B200's 16
FMA_PER_CLK_SM = 128


def _sms() -> int:
    """SMs of the current device (queried; 152 on a GB300)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

# DRAM bytes (read + write) per launch of the cross-term / tile-sum kernel, mean over the
# ten levels of one lgssm_d8 K = N = 1024 smoothing, from one ncu capture of the kernel
# revision named; None once that kernel has changed since the counters were taken.
# The epilogue's exp split between MUFU and an FMA-pipe polynomial, with issue slots counted:
# per 32 pairs MUFU needs 4 cycles of its unit and ~1.6 issue slots; a polynomial exp ~8
# issue slots per 32.  The balanced split (22 % polynomial) bounds the rate at ~1.28x the
# MUFU-only peak.
COMBINED_EXP_FACTOR = 1.28

# ncu DRAM bytes per combination of the dominant kernel in the batched step, from one
# launch of 4096 combinations (working set above L2; profiles/kernels_batched_n64_N512.md),
# scaled by the timed step's combinations per launch.
TRAFFIC_PER_COMBINATION = {("batched_lgssm_d4", "bf16"): {"bytes": 52993, "kernel": "rowsum_tc_kernel<BF16, 1 K plane>"},
                           ("batched_lgssm_d4", "bf16", "fused"): {"bytes": 23150,
                                                                  "kernel": "merge_tc_fused_kernel<4, BF16>"}}

# ncu DRAM bytes per launch of the single-sequence workloads' dominant kernel (none current:
# the kernels changed since the last capture).
TRAFFIC_PER_LAUNCH = {}

WORKLOADS = {
    "batched_lgssm_d4": dict(kind="batch", n_seq=256, N=512, resampler="dense"),
    "serving": dict(kind="serving", n_req=300, rate=2000.0, resampler="dense"),
    "pg_sv": dict(kind="pg", K=4096, N=4096, sweeps=200, resampler="dense"),
    # particle Gibbs with parameter updates on the theta-logistic model (T + 1 = 120 as the
    # paper's nutria series; N is not stated there): Algorithm 4 proposals refreshed by one
    # linearisation pass per sweep, one conditional dSMC sweep, the parameter steps on the host
    "pg_theta": dict(kind="pg_theta", K=120, N=512, sweeps=2000, resampler="dense"),
    "lgssm_d8": dict(K=1024, N=1024, resampler="dense"),
    "lgssm_1d": dict(K=32, N=64, resampler="dense"),
    "sv": dict(K=4096, N=4096, resampler="dense"),
    # Algorithm 8 at N = 16384.  One-dimensional states: the bound uses the hull of the
    # transition means, so a particle far in the proposal's upper tail does not set it; a
    # genuinely dominant pair (two low-tail particles with a near-zero observation) still
    # leaves some combinations accepting ~1e-6 of their uniform proposals, hence the cap
    "sv_rs": dict(K=4096, N=16384, resampler="rs", rs_max_attempts=1 << 26, steps=3),
    # rejection with factorised pair proposals (I ~ e^{a_i}, J ~ e^{b'_j} e^{-dist_j^2 / 2Q})
    # at N = 16384 under the default attempt cap
    "sv_rsf": dict(K=4096, N=16384, resampler="rsf", steps=3),
    # systematic resampling on the dense sampler
    "sv_sys": dict(K=4096, N=4096, resampler="sys"),
    # the constrained random walk of the lazy-resampling experiment (sigma = 0.4, uniform
    # proposals on [-1, 1]): rejection with uniform and with factorised pair proposals, and
    # systematic resampling
    "crw_rs": dict(K=1024, N=4096, resampler="rs", steps=10),
    "crw_rsf": dict(K=1024, N=4096, resampler="rsf", steps=10),
    "crw_sys": dict(K=1024, N=4096, resampler="sys", steps=20),
    # the Poisson-count model of the Cox-process experiment (stationary Gaussian proposal)
    "cox": dict(K=1024, N=1024, resampler="dense"),
    # run time against the number of time steps on the same model (the paper's run-time
    # figure: logarithmic in K while the levels fill the device, then linear)
    "cox_scaling": dict(kind="scaling", Ks=(32, 64, 128, 256, 512, 1024, 2048, 4096, 16384),
                        Ns=(256, 1024, 4096)),
    # Algorithm 7 at N = 16384: B = 64 Metropolis-Hastings steps per slot (biased)
    "sv_mh": dict(K=4096, N=16384, resampler="mh", steps=10),
    "lgssm_d4": dict(K=512, N=512, resampler="dense"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def job_time(t_local: float, device) -> float:
    """The whole job's timed region: the slowest rank's time (a MAX all-reduce over the
    process group), or the local time when the job runs as a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def oracle_sample(wl, target_s=12.0, seed=1000):
    """The FP64 CPU oracle on a bounded sample of the workload: the first K' steps of the
    same sequence at the same N (whole smoothings), K' grown until ~target_s of work."""
    from oracle import core
    m, y, N = wl.model, wl.y.astype(np.float32).astype(np.float64), wl.N
    Kp = 2
    done_units, done_s, runs = 0, 0.0, []
    while True:
        Kp = min(Kp, wl.K)
        t0 = time.perf_counter()
        core.smooth(m, y[:Kp], Kp, N, seed)
        dt = time.perf_counter() - t0
        runs.append((Kp, dt))
        done_units += Kp * N
        done_s += dt
        if done_s >= target_s or Kp == wl.K:
            break
        Kp = Kp * 2 if dt < target_s / 8 else Kp
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    Klast, tlast = runs[-1]
    return {"value": Klast * N / tlast, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"whole smoothings of the first {Klast} of {wl.K} steps, N={N}, "
                      f"d={m.d}, FP64; {len(runs)} runs, {done_s:.1f} s total"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2202_02264_gb300 import workloads as W
    spec = WORKLOADS[args.workload]
    config = None
    if spec.get("kind") == "batch":   # the oracle on the batch's first sequence
        bw = W.batch_workload(args.n_seq or spec["n_seq"], spec["N"])
        wl = W.Workload(args.workload, bw.model, int(bw.Ks[0]), bw.N, bw.ys[0], None)
        Ks = [int(k) for k in bw.Ks]
        config = {"workload": args.workload, "n_seq": len(Ks), "sum_K": sum(Ks), "K_range": [min(Ks), max(Ks)],
                  "N": bw.N, "dx": bw.model.d, "resampler": "dense"}
    elif spec.get("kind") == "serving":   # the oracle on the stream's first request
        from paper_2202_02264_gb300 import serving as S
        r0 = S.request_stream(1, spec["rate"])[0]
        wl = W.Workload(args.workload, r0.model, r0.K, r0.N, r0.y, None)
    elif spec.get("kind") == "scaling":   # the oracle at the line's largest N and K
        wl = W.workload("cox", K=spec["Ks"][-1], N=spec["Ns"][-1])
    elif spec.get("kind") == "pg_theta":
        wl = W.workload("theta_logistic", K=spec["K"], N=spec["N"])
    else:
        wl = W.workload(re.sub(r"_(rsf|rs|mh|sys)$", "", args.workload), K=spec["K"], N=spec["N"])
    from oracle import core
    y = wl.y.astype(np.float32).astype(np.float64)
    # the workload's own sampler (Algorithm 1 multinomial or systematic, 8 or 7) and its
    # attempt cap / step count
    res = spec.get("resampler", "dense")
    lazy = ({"resampler": {"sys": "systematic"}.get(res, res),
             "rs_max_attempts": spec.get("rs_max_attempts", 0) or (64 if res == "mh" else 1 << 26)}
            if res in ("rs", "mh", "rsf", "sys") else {})
    # calibrate K' so that each step is a bounded slice of the workload (~2-4 s)
    Kp = 2
    while True:
        t0 = time.perf_counter()
        core.smooth(wl.model, y[:Kp], Kp, wl.N, 999, **lazy)
        dt = time.perf_counter() - t0
        if dt > 1.0 or Kp >= wl.K:
            break
        Kp = min(Kp * 2, wl.K)
    for w in range(args.warmup):
        core.smooth(wl.model, y[:Kp], Kp, wl.N, 900 + w, **lazy)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        core.smooth(wl.model, y[:Kp], Kp, wl.N, 1000 + s, **lazy)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * Kp * wl.N / tot
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(config or {"workload": args.workload, "K": wl.K, "N": wl.N, "dx": wl.model.d},
                           sample_K=Kp),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: a whole smoothing of the first {Kp} of {wl.K} "
                                       f"steps, N={wl.N}, FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch

    from paper_2202_02264_gb300 import dsmc, workloads as W

    world, rank, lrank = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = WORKLOADS[args.workload]
    base_name = re.sub(r"_(rsf|rs|mh|sys)$", "", args.workload)
    wl = W.workload(base_name, K=spec["K"], N=spec["N"])
    K, N = wl.K, wl.N
    resampler = {"rs": dsmc.RS, "mh": dsmc.MH, "rsf": dsmc.RS_FACTORED,
                 "sys": dsmc.SYSTEMATIC}.get(spec["resampler"], dsmc.MULTINOMIAL)
    lazy = resampler in (dsmc.RS, dsmc.MH, dsmc.RS_FACTORED)   # no N x N pass
    if lazy:
        args.compute = "fp32"   # the lazy samplers evaluate their proposed pairs in FP32
    compute = {"fp32": dsmc.FP32, "tf32": dsmc.TF32, "bf16": dsmc.BF16}[args.compute]
    sm = dsmc.Smoother(wl.model, K, N, seed=1000 + 7919 * rank, resampler=resampler, compute=compute,
                       rs_max_attempts=spec.get("rs_max_attempts", 0),
                       fused_max_merges=args.fused_max_merges or 0)
    y = torch.as_tensor(wl.y, dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 126 MB L2
    stream = torch.cuda.current_stream()

    def step(i):
        sm.set_seed(1000 + 7919 * rank, counter_base=i)
        sm.smooth(y)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    st = sm.status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

    clocks = ClockSampler(torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    dsmc.dsmc_profile_enable(True)
    for i in range(args.steps):
        flush.zero_()                      # L2 flushed between timed steps, outside the events
        ev[i][0].record(stream)
        step(args.warmup + i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    rs_ms, rs_n, rs_pairs, launches = dsmc.dsmc_profile_read()
    dsmc.dsmc_profile_enable(False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per_step = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(per_step) / 1e3
    t_total = job_time(t_total, dev)
    st = sm.status()
    if st != 0:
        raise RuntimeError(f"device status {st} after timed steps")
    value = world * args.steps * N * K / t_total
    acceptance = None
    if resampler in (dsmc.RS, dsmc.RS_FACTORED):   # the last timed smoothing's attempts
        att = dsmc.dsmc_lazy_attempts(sm.cfg, sm.hm, sm.ws)
        acceptance = {"attempts_per_smoothing": att, "slots_per_smoothing": (K - 1) * N,
                      "rate": (K - 1) * N / att if att else None,
                      "cap": spec.get("rs_max_attempts") or "default (2^26)"}

    # end to end through the C ABI with host buffers: H2D of y, smoothing, D2H of results
    y_host = torch.as_tensor(wl.y, dtype=torch.float32).pin_memory()
    mean_host = torch.empty((K, wl.model.d), dtype=torch.float64).pin_memory()
    logL_host = torch.empty((1,), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(e2e_steps)]
    for i in range(e2e_steps):
        flush.zero_()
        eev[i][0].record(stream)
        y.copy_(y_host, non_blocking=True)
        sm.set_seed(1000 + 7919 * rank, counter_base=10_000 + i)
        sm.smooth(y)
        mean_host.copy_(sm.mean, non_blocking=True)
        logL_host.copy_(sm.logL_out, non_blocking=True)
        eev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_t = sum(a.elapsed_time(b) for a, b in eev) / 1e3 / e2e_steps
    e2e = {"value": world * N * K / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": y_host.numel() * 4,
           "d2h_bytes_per_step": mean_host.numel() * 8 + 8}
    # per-kernel-kind breakdown of a few more steps (CUDA events around every launch; untimed)
    dsmc.dsmc_profile_breakdown_enable(True)
    for i in range(4):
        step(20_000 + i)
    torch.cuda.synchronize()
    breakdown = {k: {"ms": v["ms"] / 4, "launches": v["launches"] // 4}
                 for k, v in dsmc.dsmc_profile_breakdown_read().items()}
    dsmc.dsmc_profile_breakdown_enable(False)

    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ex2_peak = MUFU_EX2_PER_CLK_SM * _sms() * sm_max * 1e6 / 1e9       # G exp / s
    achieved = rs_pairs / (rs_ms / 1e3) / 1e9 if rs_ms > 0 else None   # G exp / s
    d = wl.model.d
    roofline = {"bound": "alu",
                "kernel": ("lazy sampler (Algorithm 8 or 7: proposed pairs only; no N x N pass to time)"
                           if lazy else
                           "rowsum_kernel (fused exp / tile sums)" if args.compute == "fp32"
                           else "rowsum_tc_kernel (tcgen05 cross term, fused exp / tile sums)"),
                "achieved": achieved, "peak": ex2_peak, "unit": "Gexp/s",
                "frac": achieved / ex2_peak if achieved else None,
                "peak_source": f"MUFU ex2 {MUFU_EX2_PER_CLK_SM}/clk/SM x {_sms()} SMs x {sm_max:.0f} MHz "
                               f"({src} max clock)",
                "combined_peak": ex2_peak * COMBINED_EXP_FACTOR,
                "frac_combined": achieved / (ex2_peak * COMBINED_EXP_FACTOR) if achieved else None,
                # the CUDA-core variant evaluates the d-term with FMAs: that pipe binds first
                "fma_bound_frac": (achieved / (FMA_PER_CLK_SM / (d + 2) * _sms() * sm_max * 1e-3)
                                   if achieved and args.compute == "fp32" else None),
                "avg_launch_ms": rs_ms / max(rs_n, 1), "launches": rs_n,
                "traffic": (TRAFFIC_PER_LAUNCH.get((args.workload, args.compute)) or {}).get("bytes"),
                "traffic_unit": "B per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32"}[args.compute],
            "data": "synthetic",
            "config": {"workload": args.workload, "K": K, "N": N, "dx": d,
                       "resampler": spec["resampler"],
                       "compute": "fp32 pair evaluations of the proposed pairs" if lazy else {"fp32": "fp32 cuda-core cross term",
                                   "tf32": "tf32 tcgen05 cross term, fp32 accumulate / exp",
                                   "bf16": "bf16 tcgen05 cross term, fp32 accumulate / exp"}[args.compute],
                       "l2": "flushed between timed steps (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
            "breakdown_ms_per_step": breakdown,
            "step_ms": {"median": float(np.median(per_step)), "p99": float(np.percentile(per_step, 99))}}
    if acceptance:
        line["acceptance"] = acceptance
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(wl)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def _rmse_vs_rts(model, ys, means):
    from oracle import kalman
    out = []
    for y, m in zip(ys, means):
        ms, _, _ = kalman.rts_for(model, y)
        out.append(float(np.sqrt(np.mean((np.asarray(m) - ms) ** 2))))
    return np.array(out)


def run_batched(args):
    """The batched workload: 256 sequences of the d = 4 linear-Gaussian model with uneven
    lengths in one batched call per step (one launch per level for the whole batch), against
    the plain form (FP32, each sequence smoothed alone, one after another)."""
    import torch

    from paper_2202_02264_gb300 import dsmc, workloads as W

    world, rank, lrank = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = WORKLOADS[args.workload]
    bw = W.batch_workload(args.n_seq or spec["n_seq"], spec["N"])
    model, N, Ks, d = bw.model, bw.N, [int(k) for k in bw.Ks], bw.model.d
    units = N * sum(Ks)
    compute = {"fp32": dsmc.FP32, "tf32": dsmc.TF32, "bf16": dsmc.BF16}[args.compute]
    seeds = [1000 + 7919 * rank + i for i in range(len(Ks))]
    from paper_2202_02264_gb300 import autotune
    if args.schedule:
        v = [int(x) for x in args.schedule.split(",")]
        tuned = {"fused_max_merges": v[0], "max_merges_per_launch": v[1], "tc_fused": v[2] if len(v) > 2 else 0,
                 "tile_cols": v[3] if len(v) > 3 else 0, "timings": {}}
    elif args.no_autotune:
        tuned = {"fused_max_merges": 0, "max_merges_per_launch": 0, "tc_fused": 0, "tile_cols": 0, "timings": {}}
    else:
        tuned = autotune.tune_batch(model, Ks, N, bw.ys, compute, use_cache=False)   # untimed
    b = dsmc.BatchSmoother(model, Ks, N, seeds=seeds, compute=compute,
                           fused_max_merges=tuned["fused_max_merges"],
                           max_merges_per_launch=tuned["max_merges_per_launch"],
                           tc_fused=tuned["tc_fused"], tile_cols=tuned.get("tile_cols", 0))
    ys = [torch.as_tensor(y, dtype=torch.float32, device=dev) for y in bw.ys]
    b.set_inputs(ys)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def prep(i):
        b.counter_base = [i] * len(Ks)
        b.prepare()

    for i in range(args.warmup):
        prep(i)
        b.run()
    torch.cuda.synchronize()
    if b.status() != 0:
        raise RuntimeError(f"device status {b.status()} after warm-up")
    # the whole batched step (every launch of every level) captured once as a CUDA graph, with
    # the CUDA events of the dominant kernel's launches captured into it; each timed step
    # uploads that step's descriptor tables (new counter bases), then replays the graph
    graph = None
    if not args.no_graph:
        prep(args.warmup)
        dsmc.dsmc_profile_enable(True)        # one eager step creates the event pool before capture
        b.run()
        torch.cuda.synchronize()
        prep(args.warmup)
        dsmc.dsmc_profile_enable(True)
        cap_stream = torch.cuda.Stream()
        cap_stream.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap_stream):
            with torch.cuda.graph(graph, stream=cap_stream):
                b.run()
        torch.cuda.current_stream().wait_stream(cap_stream)
        graph.replay()
        torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    if graph is None:
        dsmc.dsmc_profile_enable(True)
    for i in range(args.steps):
        prep(args.warmup + i)                 # descriptor upload (host tables), outside the events
        flush.zero_()                         # L2 flushed between timed steps, outside the events
        ev[i][0].record(stream)
        if graph is not None:
            graph.replay()
        else:
            b.run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    # with a graph the captured events hold the last replay's launches (one step's worth)
    rs_ms, rs_n, rs_pairs, launches = dsmc.dsmc_profile_read()
    dsmc.dsmc_profile_enable(False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per_step = [a.elapsed_time(c) for a, c in ev]
    t_total = sum(per_step) / 1e3
    t_total = job_time(t_total, dev)
    if b.status() != 0:
        raise RuntimeError(f"device status {b.status()} after timed steps")
    value = world * args.steps * units / t_total
    mixed_means = [m.cpu().numpy().copy() for m in b.mean[:32]]

    # end to end through the public API, wall clock: pinned host observations copied in, the
    # whole dsmc_smooth_batch call (its host-side descriptor tables and their upload included),
    # means and log L copied back to pinned host memory
    y_host = [torch.as_tensor(y, dtype=torch.float32).pin_memory() for y in bw.ys]
    m_host = [torch.empty((K, d), dtype=torch.float64).pin_memory() for K in Ks]
    l_host = torch.empty((len(Ks),), dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    t_e2e = 0.0
    for i in range(e2e_steps):
        b.counter_base = [10_000 + i] * len(Ks)
        flush.zero_()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for yd, yh in zip(ys, y_host):
            yd.copy_(yh, non_blocking=True)
        b.smooth()
        for mh, md in zip(m_host, b.mean):
            mh.copy_(md, non_blocking=True)
        l_host.copy_(b.logL_out, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e += time.perf_counter() - w0
    e2e = {"value": world * units * e2e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": sum(y.numel() * 4 for y in y_host),
           "d2h_bytes_per_step": sum(m.numel() * 8 for m in m_host) + l_host.numel() * 8}

    # per-kernel-kind breakdown of one more step (CUDA events around every launch; untimed)
    prep(20_000)
    dsmc.dsmc_profile_breakdown_enable(True)
    b.run()
    torch.cuda.synchronize()
    breakdown = dsmc.dsmc_profile_breakdown_read()
    dsmc.dsmc_profile_breakdown_enable(False)

    # the plain form (FP32, each sequence alone) and the accuracy of both forms
    plain_value, t_plain, accuracy = None, None, None
    if not args.no_compare:
        plain_value, t_plain, accuracy = _plain_and_accuracy(model, Ks, N, seeds, ys, bw, mixed_means, units, stream)
    roofline = _batch_roofline(args, rs_pairs, rs_ms, rs_n, N, tuned["tc_fused"], breakdown,
                               1 if graph is not None else args.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32"}[args.compute],
            "data": "synthetic",
            "config": {"workload": args.workload, "n_seq": len(Ks), "sum_K": sum(Ks), "K_range": [min(Ks), max(Ks)],
                       "N": N, "dx": d, "resampler": "dense",
                       "compute": f"{args.compute} cross term (fp32 accumulate / exp), batched: one launch "
                                  "per level for all sequences",
                       "l2": "flushed between timed steps (512 MiB write)",
                       "timed_step": ("one replay of the captured CUDA graph of the whole batched step "
                                      "(descriptor upload of the step's counter bases outside the events)"
                                      if graph is not None else "direct launches of the whole batched step"),
                       "parallelism": f"replicas x{world}",
                       "autotuned": {"fused_max_merges": tuned["fused_max_merges"],
                                     "max_merges_per_launch": tuned["max_merges_per_launch"],
                                     "tc_fused": tuned["tc_fused"],
                                     "tile_cols": tuned.get("tile_cols", 0),
                                     "candidates_ms": tuned["timings"]}},
            "plain_fp32_per_request": ({"value": plain_value, "unit": UNIT,
                                        "ms_per_batch": 1e3 * t_plain,
                                        "form": "FP32, each sequence smoothed alone (dsmc_smooth), in order"}
                                       if plain_value else None),
            "mixed_over_plain": value / world / plain_value if plain_value else None,
            "breakdown_ms_per_step": breakdown,
            "accuracy": accuracy,
            "roofline": roofline, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
            "step_ms": {"median": float(np.median(per_step)), "p99": float(np.percentile(per_step, 99))}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        wl = W.Workload("batched_lgssm_d4_seq0", model, Ks[0], N, bw.ys[0], None)
        line["cpu_baseline"] = oracle_sample(wl)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def _plain_and_accuracy(model, Ks, N, seeds, ys, bw, mixed_means, units, stream):
    """The plain form (FP32, each sequence smoothed alone with dsmc_smooth, one call after
    another) timed on the device, and the smoothing-mean RMSE of both forms against
    Kalman/RTS on the first 32 sequences."""
    import torch

    from paper_2202_02264_gb300 import dsmc
    Kmax = max(Ks)
    single = dsmc.Smoother(model, Kmax, N, seed=seeds[0], compute=dsmc.FP32)
    plain_means = []
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i, K in enumerate(Ks):
        cfg = dsmc.make_config(K, N, seeds[i], 0, dsmc.MULTINOMIAL, dsmc.FP32)
        dsmc.dsmc_smooth(cfg, single.hm, single.prop, ys[i], single.state, None, single.mean, None,
                         single.logL_out, single.ws)
        if i < 32:
            plain_means.append(single.mean[:K].clone())
    p1.record(stream)
    torch.cuda.synchronize()
    t_plain = p0.elapsed_time(p1) / 1e3
    plain_value = units / t_plain
    plain_means = [m.cpu().numpy() for m in plain_means]
    r_mixed = _rmse_vs_rts(model, bw.ys[:32], mixed_means)
    r_plain = _rmse_vs_rts(model, bw.ys[:32], plain_means)
    diff = r_mixed - r_plain
    accuracy = {"sequences": 32, "metric": "RMSE of smoothing means vs Kalman/RTS, mean over sequences",
                "mixed": float(r_mixed.mean()), "mixed_se": float(r_mixed.std(ddof=1) / np.sqrt(32)),
                "plain_fp32": float(r_plain.mean()), "plain_fp32_se": float(r_plain.std(ddof=1) / np.sqrt(32)),
                "difference": float(diff.mean()), "difference_se": float(diff.std(ddof=1) / np.sqrt(32))}
    accuracy["equal_within_2se"] = bool(abs(accuracy["difference"]) <= 2 * accuracy["difference_se"])
    return plain_value, t_plain, accuracy


def _batch_roofline(args, rs_pairs, rs_ms, rs_n, N, tc_fused=0, breakdown=None, steps_profiled=1):
    """Roofline of the dominant kernel of the batched step (the fused exp / tile-sum pass, or
    the fused tensor-core level kernel that also builds the operands and draws the pairs):
    algorithmic work = pair exponentials per launch, over its mean event-timed duration.
    frac_merge: the same work over the device time of every merge kernel of one step."""
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ex2_peak = MUFU_EX2_PER_CLK_SM * _sms() * sm_max * 1e6 / 1e9
    achieved = rs_pairs / (rs_ms / 1e3) / 1e9 if rs_ms > 0 else None
    if tc_fused > 0 and args.compute != "fp32":
        kname = ("merge_tc_fused_kernel (operand rows, tcgen05 cross term, exp / tile sums, row CDF "
                 "and pair draws of each combination on one SM)")
        per_comb = TRAFFIC_PER_COMBINATION.get((args.workload, args.compute, "fused"))
    else:
        kname = {"fp32": "rowsum_kernel (fused exp / tile sums)",
                 "tf32": "rowsum_tc_kernel (tcgen05 cross term, fused exp / tile sums)",
                 "bf16": "rowsum_tc_kernel (tcgen05 cross term, fused exp / tile sums)"}[args.compute]
        per_comb = TRAFFIC_PER_COMBINATION.get((args.workload, args.compute))
    combs_per_launch = rs_pairs / (N * N) / max(rs_n, 1)
    merge_ms = None
    if breakdown:
        merge_ms = sum(breakdown.get(k, {}).get("ms", 0.0)
                       for k in ("prologue", "tile_sums", "draws", "fused_levels", "fused_tc_levels"))
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": ex2_peak, "unit": "Gexp/s",
                "frac": achieved / ex2_peak if achieved else None,
                "peak_source": f"MUFU ex2 {MUFU_EX2_PER_CLK_SM}/clk/SM x {_sms()} SMs x {sm_max:.0f} MHz "
                               f"({src} max clock)",
                "combined_peak": ex2_peak * COMBINED_EXP_FACTOR,
                "frac_combined": achieved / (ex2_peak * COMBINED_EXP_FACTOR) if achieved else None,
                "avg_launch_ms": rs_ms / max(rs_n, 1), "launches": rs_n,
                "combinations_per_launch": combs_per_launch,
                "traffic": per_comb["bytes"] * combs_per_launch if per_comb else None,
                "traffic_unit": "B per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum per "
                                "combination, times combinations per launch)",
                "merge_ms_per_step": merge_ms,
                "frac_merge": ((rs_pairs / steps_profiled) / (merge_ms / 1e3) / 1e9 / ex2_peak
                               if merge_ms else None)}
    return roofline


def run_serving(args):
    """The serving workload: a Poisson stream of smoothing requests (70 % linear-Gaussian
    with d in {2, 8, 32}, 30 % stochastic volatility; K log-uniform in [64, 8192]; N in
    {256, 1024, 4096}) served by continuous batching under a 150 GB budget.  One pass at the
    stated arrival rate (2000 / s: above capacity, so latency includes queueing; its
    throughput is the saturation throughput), then the same requests at 70 % of the
    measured capacity."""
    import torch

    from paper_2202_02264_gb300 import dsmc, serving as S

    world, rank, lrank = _dist()
    torch.cuda.set_device(lrank if world > 1 else 0)
    spec = WORKLOADS[args.workload]
    n = spec["n_req"]
    reqs = S.request_stream(n, spec["rate"])
    units = sum(r.N * r.K for r in reqs)
    # warm-up: a short stream through the same lanes
    warm = S.request_stream(24, spec["rate"], seed=7, K_range=(64, 256))
    for i in range(args.warmup):
        S.Server().run(warm, realtime=False)
    torch.cuda.synchronize()

    def serve(stream):
        srv = S.Server(hbm_budget_bytes=150 * 10**9)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = srv.run(stream, realtime=True)
        t1 = time.perf_counter()
        lat = np.array([r.latency for r in res]) * 1e3
        return srv, res, t1 - t0, lat

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dsmc.dsmc_profile_enable(True)
    srv, res, makespan, lat = serve(reqs)
    rs_ms, rs_n, rs_pairs, launches = dsmc.dsmc_profile_read()
    dsmc.dsmc_profile_enable(False)
    clk = clocks.stop()
    value = units / makespan
    capacity = len(res) / makespan
    rate70 = 0.7 * capacity
    scale = spec["rate"] / rate70
    reqs70 = [S.Request(r.rid, r.lane, r.model, r.N, r.y, r.seed, r.arrival * scale) for r in reqs]
    _, res70, makespan70, lat70 = serve(reqs70)

    # device time per launch kind over one more pass of the stream (untimed; events around
    # every launch on the lanes' streams, summed over the lanes)
    dsmc.dsmc_profile_breakdown_enable(True)
    srv_b = S.Server(hbm_budget_bytes=150 * 10**9)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    srv_b.run(reqs, realtime=False)
    torch.cuda.synchronize()
    tb = time.perf_counter() - tb0
    serve_breakdown = {"kinds": dsmc.dsmc_profile_breakdown_read(), "wall_s": tb, "ticks": srv_b.ticks}
    dsmc.dsmc_profile_breakdown_enable(False)

    # plain: the same requests one after another through dsmc_smooth in FP32 (no batching,
    # no reduced precision), host observations in and host means out, wall clock
    plain = None
    if not args.no_compare:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in reqs:
            sm = dsmc.Smoother(r.model, r.K, r.N, seed=r.seed, compute=dsmc.FP32)
            yd = torch.as_tensor(r.y, dtype=torch.float32).to("cuda", non_blocking=True)
            sm.smooth(yd)
            _ = sm.mean.cpu(), sm.logL_out.cpu()
            if sm.status() != 0:
                raise RuntimeError(f"plain request {r.rid}: device status {sm.status()}")
        t_plain = time.perf_counter() - t0
        plain = {"value": units / t_plain, "unit": UNIT, "makespan_s": t_plain,
                 "form": "each request alone through dsmc_smooth, FP32 cross term, sequential"}

    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ex2_peak = MUFU_EX2_PER_CLK_SM * _sms() * sm_max * 1e6 / 1e9
    achieved = rs_pairs / (rs_ms / 1e3) / 1e9 if rs_ms > 0 else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
            "ms_per_step": 1e3 * makespan, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": args.workload, "requests": n, "arrival_rate_per_s": spec["rate"],
                       "mix": "70% linear-Gaussian d in {2, 8, 32}, 30% stochastic volatility",
                       "K": "log-uniform [64, 8192]", "N": [256, 1024, 4096], "sum_N_K": units,
                       "hbm_budget_bytes": 150 * 10**9,
                       "serving": "continuous batching, one lane per (model, N, precision), level by level"},
            "latency_ms": {
                "stated_rate": {"rate_per_s": spec["rate"], "p50": float(np.percentile(lat, 50)),
                                "p99": float(np.percentile(lat, 99)), "makespan_s": makespan,
                                "note": "offered load above capacity: latency includes queueing"},
                "at_70pct_capacity": {"rate_per_s": rate70, "p50": float(np.percentile(lat70, 50)),
                                      "p99": float(np.percentile(lat70, 99)), "makespan_s": makespan70,
                                      "throughput": units / makespan70}},
            "capacity_req_per_s": capacity,
            "plain_fp32_sequential": plain,
            "breakdown_all_requests": serve_breakdown,
            "mixed_over_plain": value / plain["value"] if plain else None,
            "peak_active_requests": srv.sched.peak_active, "peak_request_bytes": srv.sched.peak_used,
            "roofline": {"bound": "alu", "kernel": "rowsum_tc_kernel / rowsum_kernel (fused exp / tile sums)",
                         "achieved": achieved, "peak": ex2_peak, "unit": "Gexp/s",
                         "frac": achieved / ex2_peak if achieved else None,
                         "peak_source": f"MUFU ex2 {MUFU_EX2_PER_CLK_SM}/clk/SM x {_sms()} SMs x {sm_max:.0f} MHz "
                                        f"({src} max clock)",
                         "launches": rs_n, "traffic": None},
            "e2e": {"value": value, "unit": UNIT,
                    "h2d_bytes_per_step": sum(r.y.size * 4 for r in reqs),
                    "d2h_bytes_per_step": sum(r.K * r.model.d * 8 + 8 for r in reqs),
                    "note": "host observations in, host means and logL out, per request"},
            "clocks": clk, "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line))


def run_pg(args):
    """Particle Gibbs at fixed parameters on the stochastic-volatility model (K = N = 4096):
    each step is one conditional dSMC sweep (Section 3.2), the reference of the next sweep
    being the trajectory drawn at the root; reports sweeps / s, N*T/s and the per-t update
    rate (the fraction of sweeps in which x*_t changed)."""
    import torch

    from paper_2202_02264_gb300 import dsmc, workloads as W

    world, rank, lrank = _dist()
    torch.cuda.set_device(lrank if world > 1 else 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = WORKLOADS[args.workload]
    wl = W.workload("sv", K=spec["K"], N=spec["N"])
    K, N = wl.K, wl.N
    sweeps = spec["sweeps"] if args.steps is None else args.steps
    compute = {"fp32": dsmc.FP32, "tf32": dsmc.TF32, "bf16": dsmc.BF16}[args.compute]
    sm = dsmc.Smoother(wl.model, K, N, seed=2000 + rank, compute=compute)
    y = torch.as_tensor(wl.y, dtype=torch.float32, device=dev)
    xa = torch.full((K, 1), float(wl.model.mu), dtype=torch.float32, device=dev)
    xb = torch.empty_like(xa)
    changed = torch.zeros((K,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def sweep(s, count):
        nonlocal xa, xb
        sm.set_seed(2000 + rank, counter_base=s)
        sm.conditional(y, xa, xb)
        if count:
            changed.add_((xb != xa).any(1).to(torch.int32))
        xa, xb = xb, xa

    for s in range(args.warmup):
        sweep(s, True)   # also loads the counting ops' kernels before the timed region
    changed.zero_()
    torch.cuda.synchronize()
    if sm.status() != 0:
        raise RuntimeError(f"device status {sm.status()} after warm-up")
    clocks = ClockSampler(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    dsmc.dsmc_profile_enable(True)
    e0.record(stream)
    for s in range(sweeps):
        sweep(args.warmup + s, True)
    e1.record(stream)
    torch.cuda.synchronize()
    rs_ms, rs_n, rs_pairs, launches = dsmc.dsmc_profile_read()
    dsmc.dsmc_profile_enable(False)
    clk = clocks.stop()
    if sm.status() != 0:
        raise RuntimeError(f"device status {sm.status()} after the sweeps")
    t = e0.elapsed_time(e1) / 1e3
    rate = changed.cpu().numpy() / sweeps
    # device time per launch kind of one more (untimed) sweep
    dsmc.dsmc_profile_breakdown_enable(True)
    sweep(args.warmup + sweeps, False)
    torch.cuda.synchronize()
    breakdown = dsmc.dsmc_profile_breakdown_read()
    dsmc.dsmc_profile_breakdown_enable(False)
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ex2_peak = MUFU_EX2_PER_CLK_SM * _sms() * sm_max * 1e6 / 1e9
    achieved = rs_pairs / (rs_ms / 1e3) / 1e9 if rs_ms > 0 else None
    line = {"metric": METRIC, "value": sweeps * N * K / t, "unit": UNIT, "n_gpus": 1, "steps": sweeps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / sweeps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32"}[args.compute],
            "data": "synthetic",
            "config": {"workload": args.workload, "K": K, "N": N, "dx": 1, "model": "stochastic volatility",
                       "sweeps": sweeps, "resampler": "dense",
                       "form": "conditional dSMC sweeps at fixed parameters (particle Gibbs)"},
            "sweeps_per_s": sweeps / t,
            "update_rate": {"mean": float(rate.mean()), "min": float(rate.min()),
                            "p10": float(np.percentile(rate, 10)), "p50": float(np.percentile(rate, 50)),
                            "first_t": float(rate[0]), "last_t": float(rate[-1])},
            "roofline": {"bound": "alu", "kernel": "rowsum kernels (fused exp / tile sums)", "achieved": achieved,
                         "peak": ex2_peak, "unit": "Gexp/s", "frac": achieved / ex2_peak if achieved else None,
                         "peak_source": f"MUFU ex2 {MUFU_EX2_PER_CLK_SM}/clk/SM x {_sms()} SMs x {sm_max:.0f} MHz "
                                        f"({src} max clock)", "launches": rs_n, "traffic": None},
            "clocks": clk, "gpu_launches": launches, "breakdown_ms_per_sweep": breakdown}
    if rank == 0:
        print(json.dumps(line))


def run_scaling(args):
    """Smoothing time against K on the Poisson-count model (Section 5.1): for each N and K, the
    median CUDA-event time of whole smoothings (device-resident observations, L2 flushed
    between runs).  The line's value is N*T/s at the largest N and K."""
    import torch

    from paper_2202_02264_gb300 import dsmc, workloads as W

    torch.cuda.set_device(0)
    spec = WORKLOADS[args.workload]
    compute = {"fp32": dsmc.FP32, "tf32": dsmc.TF32, "bf16": dsmc.BF16}[args.compute]
    reps = args.steps if args.steps else 9
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    table, launches = {}, 0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for N in spec["Ns"]:
        row = {}
        for K in spec["Ks"]:
            wl = W.workload("cox", K=K, N=N)
            sm = dsmc.Smoother(wl.model, K, N, seed=3000, compute=compute)
            y = torch.as_tensor(wl.y, dtype=torch.float32, device="cuda")
            for w in range(args.warmup):
                sm.set_seed(3000, counter_base=w)
                sm.smooth(y)
            ts = []
            for r in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                sm.set_seed(3000, counter_base=100 + r)
                e0.record(stream)
                sm.smooth(y)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            if sm.status() != 0:
                raise RuntimeError(f"device status {sm.status()} at N={N}, K={K}")
            row[str(K)] = float(np.median(ts))
            del sm
        table[str(N)] = row
    clk = clocks.stop()
    Nl, Kl = spec["Ns"][-1], spec["Ks"][-1]
    ms = table[str(Nl)][str(Kl)]
    line = {"metric": METRIC, "value": Nl * Kl / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": reps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32"}[args.compute],
            "data": "synthetic (simulated Poisson counts)",
            "config": {"workload": args.workload, "model": "Poisson counts (Cox)", "resampler": "dense",
                       "Ks": list(spec["Ks"]), "Ns": list(spec["Ns"]),
                       "l2": "flushed between timed runs (512 MiB write)",
                       "value_at": {"N": Nl, "K": Kl}},
            "ms_per_smoothing": table, "clocks": clk}
    print(json.dumps(line))


def run_pg_theta(args):
    """Particle Gibbs with parameter updates on the theta-logistic model (Section 3.2,
    Section 5.2), K = 120: per sweep one pass of the linearised smoother from the previous
    proposals (Algorithm 4), one conditional dSMC sweep, the K values of x* to the host and the
    parameter steps there.  The timed region is the wall clock of whole sweeps (the parameter
    step depends on the sweep's x*, so every sweep synchronises once).  Reports sweeps / s,
    the seconds 10^5 Gibbs samples take, and the per-t update rate of x*."""
    import torch

    from paper_2202_02264_gb300 import dsmc, pgibbs as P, workloads as W

    world, rank, lrank = _dist()
    torch.cuda.set_device(lrank if world > 1 else 0)
    spec = WORKLOADS[args.workload]
    K, N = spec["K"], spec["N"]
    sweeps = spec["sweeps"] if args.steps is None else args.steps
    m = W.theta_logistic()
    _, y = W.simulate(m, K, 2264 + 7 + rank)
    compute = {"fp32": dsmc.FP32, "tf32": dsmc.TF32, "bf16": dsmc.BF16}[args.compute]
    g = P.ThetaLogisticGibbs(y[:, 0], N, P.ThetaState(0.0, 0.0, 0.5, 0.05, 0.05), seed=3000 + rank,
                             compute=compute)
    g.run(args.warmup)                     # the first sweep's 25 linearisation passes are here
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dsmc.dsmc_profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ch = g.run(sweeps, counter_base0=args.warmup)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    t = job_time(t, torch.device("cuda", torch.cuda.current_device()))
    _, _, _, launches = dsmc.dsmc_profile_read()
    dsmc.dsmc_profile_enable(False)
    clk = clocks.stop()
    rate = ch.updated / sweeps
    th = ch.theta[sweeps // 2:]
    line = {"metric": METRIC, "value": world * sweeps * N * K / t, "unit": UNIT, "n_gpus": world, "steps": sweeps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / sweeps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32"}[args.compute],
            "data": "synthetic (simulated from the theta-logistic model; the nutria series is not here)",
            "config": {"workload": args.workload, "K": K, "N": N, "dx": 1, "model": "theta-logistic",
                       "sweeps": sweeps, "resampler": "dense",
                       "form": "particle Gibbs: Algorithm 4 proposals (1 pass per sweep, 25 first), "
                               "conditional dSMC sweep, parameter steps (conjugate r^2, (tau0, tau1), q^2; "
                               "random-walk MH tau2)",
                       "timed": "wall clock of whole sweeps, host parameter steps included"},
            "sweeps_per_s": sweeps / t, "seconds_per_1e5_samples": 1e5 * t / sweeps,
            "paper_context": "480 s per 1e5 samples on an RTX 3090 (nutria data, N not stated)",
            "device_ms_per_sweep_dsmc": 1e3 * ch.device_s / sweeps,
            "update_rate": {"mean": float(rate.mean()), "min": float(rate.min()),
                            "p10": float(np.percentile(rate, 10)), "p50": float(np.percentile(rate, 50))},
            "posterior_mean_second_half": {k: float(np.mean([getattr(x, k) for x in th]))
                                           for k in ("tau0", "tau1", "tau2", "q2", "r2")},
            "clocks": clk, "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 10 batched smoothings, or 400 single smoothings)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_lgssm_d4", choices=sorted(WORKLOADS))
    ap.add_argument("--compute", default=None, choices=["fp32", "tf32", "bf16"],
                    help="cross-term precision (default: bf16 for the batched workload, tf32 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: default launch schedule")
    ap.add_argument("--no-graph", action="store_true", help="batched workload: time direct launches, not a graph")
    ap.add_argument("--schedule", default=None,
                    help="batched workload: fixed 'fused_max_merges,max_merges_per_launch[,tc_fused[,tile_cols]]' "
                         "instead of the autotuner")
    ap.add_argument("--fused-max-merges", type=int, default=None,
                    help="single-sequence workloads: levels with at most this many combinations run "
                         "fused (-1: never; default: the library's)")
    ap.add_argument("--no-compare", action="store_true",
                    help="batched workload: skip the plain-FP32 comparison and accuracy legs (profiling runs)")
    ap.add_argument("--n-seq", type=int, default=None, help="batched workload: fewer sequences (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    kind = WORKLOADS[args.workload].get("kind", "single")
    if args.steps is None and kind not in ("pg", "pg_theta", "scaling"):
        args.steps = WORKLOADS[args.workload].get("steps", {"batch": 10, "serving": 1}.get(kind, 400))
    if args.compute is None:
        args.compute = {"batch": "bf16", "pg": "fp32", "pg_theta": "fp32"}.get(kind, "tf32")
    if args.impl == "reference":
        run_reference(args)
    else:
        from oracle import core  # built here so cpu_baseline does not compile mid-run
        core.build()
        if kind == "batch":
            run_batched(args)
        elif kind == "serving":
            run_serving(args)
        elif kind == "pg":
            run_pg(args)
        elif kind == "pg_theta":
            run_pg_theta(args)
        elif kind == "scaling":
            run_scaling(args)
        else:
            run_ours(args)


if __name__ == "__main__":
    main()
