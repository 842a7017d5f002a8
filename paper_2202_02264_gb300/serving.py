"""Continuous-batching server for dSMC smoothing requests on one GPU.

A request is one sequence to smooth (model, N, observations, seed; optionally a reference
trajectory for a particle-Gibbs sweep).  Requests that share a model, N and precision form a
lane: one workspace and one CUDA stream.  A request advances one stage per tick of its lane
(Algorithm 2, then level 0, 1, ... of Algorithm 6, then the resolve that writes its means),
and every tick launches the stages of all the lane's requests together through
``dsmc_serve_tick``, so the levels of different requests share launches ("level by level"
batching).  Requests are admitted first come, first served while their device memory fits
the HBM budget; a finished request releases its memory, so requests that arrive while
others are on the GPU join the running lanes at the next tick.  Lanes run on their own
streams, so their work overlaps on the device.

Each request's result is the one ``dsmc_smooth`` gives for it alone with the same seed:
the draws depend only on the request's own seed and combination ids, and whether a level
runs fused depends only on that request.

``Scheduler`` holds the admission and stage bookkeeping (plain Python, no device);
``Server`` drives the lanes on the GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import workloads as W


@dataclass
class Request:
    rid: int
    lane: str                  # lane key: requests of one lane share model, N and precision
    model: W.SSM
    N: int
    y: np.ndarray              # [K][d] observations
    seed: int
    arrival: float = 0.0       # seconds since the start of the stream
    x_ref: Optional[np.ndarray] = None   # [K][d] reference for a particle-Gibbs sweep
    counter_base: int = 0

    @property
    def K(self) -> int:
        return int(self.y.shape[0])


@dataclass
class Result:
    rid: int
    mean: np.ndarray
    logL: float
    arrival: float
    admitted: float
    finished: float
    x_ref_out: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def levels(K: int) -> int:
    L = 0
    while (1 << L) < K:
        L += 1
    return L


def merges_at_level(K: int, level: int) -> int:
    size = 1 << level
    n = 0
    start = 0
    while start < K:
        if start + size < K:
            n += 1
        start += 2 * size
    return n


def request_bytes(K: int, N: int, d: int, gauss_prop: bool = False, conditional: bool = False) -> int:
    """Device bytes a request holds while admitted: observations, particles, leaf weights,
    block log-likelihoods, pairs, index maps, means (and proposal / reference arrays)."""
    b = K * d * 4 + K * N * d * 4 + K * N * 4 + K * 8 + max(K - 1, 0) * 2 * N * 4
    b += 16 * K * N + 8 + K * d * 8 + 8
    if gauss_prop:
        b += 2 * K * d * 4
    if conditional:
        b += 2 * K * d * 4
    return b


@dataclass
class _Slot:
    req: Request
    bytes: int
    L: int
    stage: int = -1            # -1: Algorithm 2; 0..L-1: level; L: resolve
    admitted: float = 0.0


class Scheduler:
    """First-come-first-served admission under a byte budget, and the stage of every
    admitted request.  ``lane_limit(lane)`` bounds the combinations one tick of a lane may
    hold (its workspace); a request whose largest level would not fit waits."""

    def __init__(self, budget_bytes: int, bytes_of: Callable[[Request], int],
                 lane_limit: Callable[[str], int] = lambda lane: 1 << 30):
        self.budget = int(budget_bytes)
        self.bytes_of = bytes_of
        self.lane_limit = lane_limit
        self.queue: deque[Request] = deque()
        self.active: dict[str, list[_Slot]] = {}
        self.used = 0
        self.draining = 0
        self.peak_used = 0
        self.peak_active = 0

    def submit(self, req: Request):
        if self.bytes_of(req) > self.budget:
            raise ValueError(f"request {req.rid} needs more than the whole budget")
        if merges_at_level(req.K, 0) > self.lane_limit(req.lane):
            raise ValueError(f"request {req.rid}: one level exceeds the lane's tick capacity")
        self.queue.append(req)

    def _lane_items(self, lane: str) -> int:
        # worst case of one tick: every active request at its level 0
        return sum(merges_at_level(s.req.K, 0) for s in self.active.get(lane, []))

    def admit(self, now: float) -> list[_Slot]:
        """Admit queued requests in arrival order while they fit (stops at the first that
        does not: no overtaking)."""
        out = []
        while self.queue and self.queue[0].arrival <= now:
            r = self.queue[0]
            nb = self.bytes_of(r)
            if self.used + nb > self.budget:
                break
            if self._lane_items(r.lane) + merges_at_level(r.K, 0) > self.lane_limit(r.lane):
                break
            self.queue.popleft()
            s = _Slot(r, nb, levels(r.K), -1, now)
            self.active.setdefault(r.lane, []).append(s)
            self.used += nb
            out.append(s)
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, sum(len(v) for v in self.active.values()))
        return out

    def tick_plan(self, lane: str) -> list[_Slot]:
        """The requests of a lane and their stages for the next tick."""
        return list(self.active.get(lane, []))

    def advance(self, lane: str) -> list[_Slot]:
        """After a tick: every request moves one stage; those past their resolve leave the
        lane (their bytes stay in use until ``release``).  Returns the finished ones."""
        done, keep = [], []
        for s in self.active.get(lane, []):
            if s.stage == s.L:
                done.append(s)
            else:
                s.stage += 1
                keep.append(s)
        self.active[lane] = keep
        self.draining += len(done)
        return done

    def release(self, slot: _Slot):
        """A finished request's results are on the host: its device memory is free."""
        self.used -= slot.bytes
        self.draining -= 1

    def busy(self) -> bool:
        return bool(self.queue) or any(self.active.values()) or self.draining > 0


class _Lane:
    """The device side of one lane: workspace, stream, and the buffers of its requests."""

    def __init__(self, key: str, model: W.SSM, N: int, compute: int, max_comb: int, device):
        import torch

        from . import dsmc
        self.torch, self.dsmc = torch, dsmc
        self.key, self.model, self.N, self.d = key, model, int(N), model.d
        self.hm = dsmc.HostModel(model)
        # launch cap from a ~1 GiB merge workspace: tile sums, terms, operands per combination
        per_comb = self.N * (4 * 8 + 8 * self.d + 16 + 4 * max(4, (self.N // 32 + 3) // 4 * 4)) + 4096
        cap = int(max(16, min(1024, (1 << 30) // per_comb)))
        self.cfg = dsmc.make_config(2, self.N, 0, 0, dsmc.MULTINOMIAL, compute, 0, cap)
        kind = W.PROP_GAUSS if model.prop_kind == W.PROP_GAUSS else W.PROP_OBS
        self.prop = dsmc.Proposal(kind, float(model.prop_scale), None, None, int(model.nu))
        self.max_comb = int(max_comb)
        self.ws = torch.empty((dsmc.dsmc_serve_workspace_size(self.cfg, self.hm, 4096, self.max_comb),),
                              dtype=torch.uint8, device=device)
        self.stream = torch.cuda.Stream(device=device)
        self.device = device
        self.bufs: dict[int, dict] = {}
        self.pending: list[tuple] = []    # (event, slot, host buffers)

    def workspace_bytes(self) -> int:
        return self.ws.numel()

    def attach(self, slot: _Slot):
        torch, r = self.torch, slot.req
        K, N, d = r.K, self.N, self.d
        f32, f64, i32 = torch.float32, torch.float64, torch.int32
        with torch.cuda.stream(self.stream):
            b = {"y": torch.as_tensor(np.asarray(r.y, np.float32), device=self.device),
                 "X": torch.empty((K, N, d), dtype=f32, device=self.device),
                 "logw": torch.empty((K, N), dtype=f32, device=self.device),
                 "logL": torch.empty((K,), dtype=f64, device=self.device),
                 "pairs": torch.empty((max(K - 1, 0), 2, N), dtype=i32, device=self.device),
                 "maps": torch.empty((self.dsmc.dsmc_seq_maps_bytes(K, N),), dtype=torch.uint8, device=self.device),
                 "mean": torch.empty((K, d), dtype=f64, device=self.device),
                 "logL_out": torch.empty((1,), dtype=f64, device=self.device)}
            if self.model.prop_kind == W.PROP_GAUSS:
                b["pm"] = torch.as_tensor(self.dsmc.proposal_rows(self.model.prop_mean, K, d), device=self.device)
                b["ps"] = torch.as_tensor(self.dsmc.proposal_rows(self.model.prop_std, K, d), device=self.device)
            if r.x_ref is not None:
                b["x_in"] = torch.as_tensor(np.asarray(r.x_ref, np.float32), device=self.device)
                b["x_out"] = torch.empty((K, d), dtype=f32, device=self.device)
        self.bufs[r.rid] = b

    def _seq(self, slot: _Slot):
        dsmc, r = self.dsmc, slot.req
        b = self.bufs[r.rid]
        st = dsmc.State(b["X"].data_ptr(), b["logw"].data_ptr(), b["logL"].data_ptr(),
                        b["pairs"].data_ptr() if b["pairs"].numel() else None)
        return dsmc.Seq(r.K, b["y"].data_ptr(), b["pm"].data_ptr() if "pm" in b else None,
                        b["ps"].data_ptr() if "ps" in b else None, st, b["mean"].data_ptr(), None,
                        b["logL_out"].data_ptr(), b["x_in"].data_ptr() if "x_in" in b else None,
                        b["x_out"].data_ptr() if "x_out" in b else None, int(r.seed) & (2**64 - 1),
                        int(r.counter_base), b["maps"].data_ptr())

    def tick(self, slots: list[_Slot]):
        torch, dsmc = self.torch, self.dsmc
        if not slots:
            return
        seqs = [self._seq(s) for s in slots]
        stages = [s.stage for s in slots]
        dsmc.dsmc_serve_tick(self.cfg, self.hm, self.prop, seqs, stages, self.ws, stream=self.stream)
        with torch.cuda.stream(self.stream):
            for s in slots:
                if s.stage == s.L:      # resolved: copy the results out behind the tick
                    b = self.bufs[s.req.rid]
                    host = {"mean": torch.empty(b["mean"].shape, dtype=torch.float64).pin_memory(),
                            "logL": torch.empty((1,), dtype=torch.float64).pin_memory()}
                    host["mean"].copy_(b["mean"], non_blocking=True)
                    host["logL"].copy_(b["logL_out"], non_blocking=True)
                    if "x_out" in b:
                        host["x_out"] = torch.empty(b["x_out"].shape, dtype=torch.float32).pin_memory()
                        host["x_out"].copy_(b["x_out"], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                    self.pending.append((ev, s, host))

    def collect(self, now_fn, release) -> list[Result]:
        out, keep = [], []
        for ev, s, host in self.pending:
            if ev.query():
                r = s.req
                out.append(Result(r.rid, host["mean"].numpy(), float(host["logL"][0]), r.arrival, s.admitted,
                                  now_fn(), host["x_out"].numpy() if "x_out" in host else None))
                del self.bufs[r.rid]
                release(s)
            else:
                keep.append((ev, s, host))
        self.pending = keep
        return out

    def status(self) -> int:
        return self.dsmc.dsmc_stream_status(self.ws, self.stream)


class Server:
    """Requests in, results out, on one GPU.  ``lane_of(req)`` gives (model, N, precision)
    for a lane key on first use."""

    def __init__(self, hbm_budget_bytes: int = 150 * 10**9, device="cuda", max_comb_per_tick: int = 1 << 16,
                 precision: Callable[[W.SSM, int], int] | None = None, lane_workspaces_in_budget: bool = True):
        from . import dsmc
        self.dsmc = dsmc
        self.device = device
        self.max_comb = int(max_comb_per_tick)
        self.precision = precision or (lambda m, N: dsmc.BF16)
        self.lanes: dict[str, _Lane] = {}

        def bytes_of(r: Request) -> int:
            return request_bytes(r.K, r.N, r.model.d, r.model.prop_kind == W.PROP_GAUSS, r.x_ref is not None)

        self.sched = Scheduler(hbm_budget_bytes, bytes_of, lambda lane: self.max_comb)
        self.ws_in_budget = lane_workspaces_in_budget
        self.results: list[Result] = []
        self.ticks = 0

    def _lane(self, r: Request) -> _Lane:
        if r.lane not in self.lanes:
            self.lanes[r.lane] = _Lane(r.lane, r.model, r.N, self.precision(r.model, r.N), self.max_comb,
                                       self.device)
            if self.ws_in_budget:
                self.sched.budget -= self.lanes[r.lane].workspace_bytes()
        return self.lanes[r.lane]

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve the requests (sorted by arrival).  realtime: arrivals follow the wall clock
        from the start of the call; otherwise every request is available at once."""
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            self._lane(r)
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0 if realtime else float("inf")

        def clock():
            return time.perf_counter() - t0

        i = 0
        while i < len(reqs) or self.sched.busy():
            t = now()
            while i < len(reqs) and reqs[i].arrival <= t:
                self.sched.submit(reqs[i])
                i += 1
            for s in self.sched.admit(t):
                s.admitted = clock()
                self.lanes[s.req.lane].attach(s)
            worked = False
            for key, lane in self.lanes.items():
                plan = self.sched.tick_plan(key)
                if plan:
                    lane.tick(plan)
                    self.sched.advance(key)
                    worked = True
            for lane in self.lanes.values():
                self.results.extend(lane.collect(clock, self.sched.release))
            self.ticks += 1
            if not worked and i < len(reqs) and realtime and not self.sched.busy():
                time.sleep(max(0.0, min(reqs[i].arrival - clock(), 0.001)))
            elif not worked:
                time.sleep(0.0002)
        torch.cuda.synchronize()
        for lane in self.lanes.values():
            st = lane.status()
            if st != 0:
                raise RuntimeError(f"lane {lane.key}: device status {st}")
        return self.results


# ---------------------------------------------------------------- the request stream
def lane_models():
    """The serving mix's models: the linear-Gaussian family at d = 2, 8, 32 (A = 0.5 I +
    0.05 sqrt(8/d) G, Q = I, R = 0.25 I) and stochastic volatility (mu = -1, phi = 0.95,
    sigma = 0.3)."""
    return {"lg2": W.lgssm_dn(2), "lg8": W.lgssm_d8(), "lg32": W.lgssm_dn(32), "sv": W.sv(1)}


def request_stream(n: int, rate: float, seed: int = 2269, Ns=(256, 1024, 4096), K_range=(64, 8192),
                   models=None) -> list[Request]:
    """n requests with Poisson arrivals at `rate` per second: 70 % linear-Gaussian with d
    uniform in {2, 8, 32}, 30 % stochastic volatility; K log-uniform in K_range; N uniform
    in Ns; observations simulated from the request's model (seed 50000 + id)."""
    rng = np.random.default_rng(seed)
    models = models or lane_models()
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        name = "sv" if rng.random() < 0.3 else ["lg2", "lg8", "lg32"][rng.integers(3)]
        K = int(np.exp(rng.uniform(np.log(K_range[0]), np.log(K_range[1]))))
        N = int(Ns[rng.integers(len(Ns))])
        m = models[name]
        _, y = W.simulate(m, K, 50000 + rid)
        out.append(Request(rid, f"{name}/N{N}", m, N, y, 1000 + rid, t))
    return out
