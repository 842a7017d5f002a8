"""Thin Python binding of the dSMC C ABI (include/dsmc.h).

Every function here only marshals arguments: tensors become device pointers, the
current PyTorch stream becomes the ``stream`` argument, and every step of the method runs
in the CUDA library.  There is no CPU fallback: if the library is not built or no CUDA
device is present, calls raise.

The functions keep the C names (``dsmc_init_particles``, ``dsmc_merge_level``,
``dsmc_smooth``, ``dsmc_conditional_smooth`` ...).  ``Smoother`` owns the device buffers
(allocated through PyTorch) for one (config, model) pair and calls them in order.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import build as _build
from . import workloads as W

OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "workspace too small",
          5: "CUDA error", 6: "non-finite log-weight", 7: "degenerate weights",
          8: "rejection-sampling attempt cap", 9: "timeout", 10: "lazy-sampler bound exceeded"}

FP32, TF32, BF16 = 0, 1, 2
MULTINOMIAL, RS, MH, SYSTEMATIC, RS_FACTORED = 0, 1, 2, 3, 4


class DsmcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code}) {detail}".strip())


class Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("dx", C.c_int),
                ("A", C.POINTER(C.c_double)), ("Q", C.POINTER(C.c_double)),
                ("R", C.POINTER(C.c_double)), ("m0", C.POINTER(C.c_double)),
                ("P0", C.POINTER(C.c_double)),
                ("mu", C.c_double), ("phi", C.c_double), ("sigma", C.c_double),
                ("lam", C.c_double), ("tau0", C.c_double), ("tau1", C.c_double), ("tau2", C.c_double),
                ("obs_sd", C.c_double), ("bound", C.c_double)]


class Proposal(C.Structure):
    _fields_ = [("kind", C.c_int), ("scale", C.c_double), ("mean", C.c_void_p),
                ("std", C.c_void_p), ("nu", C.c_int)]


class Config(C.Structure):
    _fields_ = [("K", C.c_int), ("N", C.c_int), ("compute", C.c_int), ("resampler", C.c_int),
                ("seed", C.c_uint64), ("counter_base", C.c_uint32),
                ("rs_max_attempts", C.c_uint32), ("max_merges_per_launch", C.c_int),
                ("fused_max_merges", C.c_int), ("tc_fused", C.c_int), ("tile_cols", C.c_int)]


class State(C.Structure):
    _fields_ = [("X", C.c_void_p), ("logw", C.c_void_p), ("logL", C.c_void_p),
                ("pairs", C.c_void_p)]


class Seq(C.Structure):
    """dsmc_seq_t: one sequence of a batched call."""
    _fields_ = [("K", C.c_int), ("y", C.c_void_p), ("prop_mean", C.c_void_p), ("prop_std", C.c_void_p),
                ("state", State), ("mean_out", C.c_void_p), ("m2_out", C.c_void_p),
                ("logL_out", C.c_void_p), ("x_ref_in", C.c_void_p), ("x_ref_out", C.c_void_p),
                ("seed", C.c_uint64), ("counter_base", C.c_uint32), ("maps", C.c_void_p)]


_lib = None
_lock = threading.Lock()

EXPORTS = ["dsmc_status_string", "dsmc_last_error", "dsmc_state_sizes", "dsmc_workspace_size",
           "dsmc_init_particles", "dsmc_merge_level", "dsmc_resolve", "dsmc_smooth",
           "dsmc_conditional_smooth", "dsmc_smooth_noalloc", "dsmc_stream_status",
           "dsmc_profile_enable",
           "dsmc_profile_read", "dsmc_debug_philox", "dsmc_debug_merge_weights",
           "dsmc_debug_stall_tensor_cores",
           "dsmc_batch_workspace_size", "dsmc_batch_prepare", "dsmc_batch_run", "dsmc_smooth_batch",
           "dsmc_seq_maps_bytes", "dsmc_serve_workspace_size", "dsmc_serve_tick",
           "dsmc_profile_breakdown_enable", "dsmc_profile_breakdown_read", "dsmc_profile_unit_rates",
           "dsmc_debug_lazy_weights", "dsmc_lazy_attempts", "dsmc_debug_row_shift", "dsmc_debug_keep_weights",
           "dsmc_gaussian_proposals_workspace_size", "dsmc_gaussian_proposals"]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = False) -> C.CDLL:
    """Load libdsmc.so (raises if it is missing; it never falls back to anything)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and _build.needs_build():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libdsmc.so is not built: run __graft_entry__.build() "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        torch.cuda.init() if torch.cuda.is_available() else None
        lib = C.CDLL(_build.LIB)
        vp, sz = C.c_void_p, C.c_size_t
        lib.dsmc_status_string.restype = C.c_char_p
        lib.dsmc_status_string.argtypes = [C.c_int]
        lib.dsmc_last_error.restype = C.c_char_p
        lib.dsmc_last_error.argtypes = []
        for name in EXPORTS[2:]:
            getattr(lib, name).restype = C.c_int
        cfgp, modp, prop_p, statp = C.POINTER(Config), C.POINTER(Model), C.POINTER(Proposal), C.POINTER(State)
        lib.dsmc_state_sizes.argtypes = [cfgp, modp, C.POINTER(C.c_size_t)]
        lib.dsmc_workspace_size.argtypes = [cfgp, modp, C.POINTER(C.c_size_t)]
        lib.dsmc_init_particles.argtypes = [cfgp, modp, prop_p, vp, vp, statp, vp, sz, vp]
        lib.dsmc_merge_level.argtypes = [cfgp, modp, prop_p, vp, C.c_int, C.c_int, statp, vp, sz, vp]
        lib.dsmc_resolve.argtypes = [cfgp, modp, statp, vp, vp, vp, vp, vp, sz, vp]
        lib.dsmc_smooth.argtypes = [cfgp, modp, prop_p, vp, statp, vp, vp, vp, vp, vp, sz, vp]
        lib.dsmc_conditional_smooth.argtypes = [cfgp, modp, prop_p, vp, vp, vp, statp, vp, vp, vp,
                                                vp, sz, vp]
        lib.dsmc_smooth_noalloc.argtypes = [cfgp, modp, prop_p, vp, statp, vp, vp, vp, vp,
                                             C.POINTER(C.c_int), vp]
        lib.dsmc_stream_status.argtypes = [vp, vp, C.POINTER(C.c_int)]
        lib.dsmc_profile_enable.argtypes = [C.c_int]
        lib.dsmc_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        lib.dsmc_debug_philox.argtypes = [vp, C.c_int64, C.c_uint64, vp, vp]
        lib.dsmc_debug_stall_tensor_cores.argtypes = [C.c_int]
        lib.dsmc_debug_keep_weights.argtypes = [C.c_int]
        lib.dsmc_gaussian_proposals_workspace_size.argtypes = [modp, C.c_int, C.POINTER(C.c_size_t)]
        lib.dsmc_gaussian_proposals.argtypes = [modp, C.c_int, vp, C.c_int, vp, vp, vp, vp, sz, vp]
        lib.dsmc_debug_merge_weights.argtypes = [cfgp, modp, C.c_int, C.c_int, vp, vp, vp, vp, vp,
                                                 vp, C.POINTER(C.c_int), vp, sz, vp]
        lib.dsmc_seq_maps_bytes.restype = C.c_size_t
        lib.dsmc_seq_maps_bytes.argtypes = [C.c_int, C.c_int]
        lib.dsmc_serve_workspace_size.argtypes = [cfgp, modp, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
        lib.dsmc_serve_tick.argtypes = [cfgp, modp, prop_p, C.c_int, C.POINTER(Seq), C.POINTER(C.c_int), vp, sz, vp]
        lib.dsmc_profile_breakdown_enable.argtypes = [C.c_int]
        lib.dsmc_profile_breakdown_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        lib.dsmc_profile_unit_rates.argtypes = [vp, C.POINTER(C.c_double), vp]
        lib.dsmc_debug_lazy_weights.argtypes = [cfgp, modp, C.c_int, C.c_int, vp, vp, vp, C.POINTER(C.c_int),
                                                vp, sz, vp]
        lib.dsmc_lazy_attempts.argtypes = [cfgp, modp, vp, sz, vp, C.POINTER(C.c_uint64)]
        lib.dsmc_debug_row_shift.argtypes = [cfgp, modp, C.c_int, C.c_int, vp, vp, vp, sz, vp]
        seqp = C.POINTER(Seq)
        lib.dsmc_batch_workspace_size.argtypes = [cfgp, modp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        for name in ("dsmc_batch_prepare", "dsmc_batch_run", "dsmc_smooth_batch"):
            getattr(lib, name).argtypes = [cfgp, modp, prop_p, C.c_int, seqp, vp, sz, vp]
        _lib = lib
        return lib


def _check(code: int, where: str):
    if code != OK:
        detail = load().dsmc_last_error().decode(errors="replace")
        raise DsmcError(code, where, detail)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class HostModel:
    """The C model struct plus the FP64 host arrays it points into."""

    def __init__(self, m: W.SSM):
        d = m.d
        self.m = m
        self._arrs = []

        def arr(x, shape):
            a = np.ascontiguousarray(np.asarray(x if x is not None else np.zeros(shape), np.float64).reshape(shape))
            self._arrs.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_double))

        extra = (float(getattr(m, "lam", 1.0)), float(getattr(m, "tau0", 0.0)), float(getattr(m, "tau1", 0.0)),
                 float(getattr(m, "tau2", 0.0)), float(getattr(m, "obs_sd", 1.0)), float(getattr(m, "bound", 1.0)))
        if m.kind == W.LGSSM:
            self.struct = Model(m.kind, d, arr(m.A, (d, d)), arr(m.Q, (d, d)), arr(m.R, (d, d)),
                                arr(m.m0, (d,)), arr(m.P0, (d, d)), 0.0, 0.0, 1.0, *extra)
        else:
            self.struct = Model(m.kind, d, None, None, None, None, None, m.mu, m.phi, m.sigma, *extra)


def make_config(K, N, seed, counter_base=0, resampler=MULTINOMIAL, compute=FP32,
                rs_max_attempts=0, max_merges_per_launch=0, fused_max_merges=0, tc_fused=0,
                tile_cols=0) -> Config:
    return Config(int(K), int(N), int(compute), int(resampler), int(seed) & (2**64 - 1),
                  int(counter_base), int(rs_max_attempts), int(max_merges_per_launch),
                  int(fused_max_merges), int(tc_fused), int(tile_cols))


def make_proposal(m: W.SSM, K: int, device="cuda"):
    """The C proposal struct and the device arrays it points into (kept alive by caller)."""
    if m.prop_kind in (W.PROP_OBS, W.PROP_UNIFORM):
        return Proposal(int(m.prop_kind), float(m.prop_scale), None, None, int(m.nu)), ()
    mean = torch.as_tensor(proposal_rows(m.prop_mean, K, m.d), device=device)
    std = torch.as_tensor(proposal_rows(m.prop_std, K, m.d), device=device)
    return Proposal(W.PROP_GAUSS, 1.0, mean.data_ptr(), std.data_ptr(), int(m.nu)), (mean, std)


def proposal_rows(a, K: int, d: int) -> np.ndarray:
    """K rows of a per-t proposal array as FP32 [K][d]; a single row is a stationary proposal
    and is repeated."""
    a = np.asarray(a, np.float32).reshape(-1, d)
    if a.shape[0] == 1:
        return np.repeat(a, K, axis=0)
    return np.ascontiguousarray(a[:K])


# ---------------------------------------------------------------- C-named wrappers
def dsmc_state_sizes(cfg: Config, model: HostModel):
    out = (C.c_size_t * 4)()
    _check(load().dsmc_state_sizes(C.byref(cfg), C.byref(model.struct), out), "dsmc_state_sizes")
    return list(out)


def dsmc_workspace_size(cfg: Config, model: HostModel) -> int:
    out = C.c_size_t(0)
    _check(load().dsmc_workspace_size(C.byref(cfg), C.byref(model.struct), C.byref(out)),
           "dsmc_workspace_size")
    return int(out.value)


def dsmc_init_particles(cfg, model, prop, y, x_ref, state, ws, stream=None):
    _check(load().dsmc_init_particles(C.byref(cfg), C.byref(model.struct), C.byref(prop), _ptr(y),
                                      _ptr(x_ref), C.byref(state), _ptr(ws), ws.numel(),
                                      _stream(stream)), "dsmc_init_particles")


def dsmc_merge_level(cfg, model, prop, y, level, conditional, state, ws, stream=None):
    _check(load().dsmc_merge_level(C.byref(cfg), C.byref(model.struct), C.byref(prop), _ptr(y),
                                   int(level), int(conditional), C.byref(state), _ptr(ws),
                                   ws.numel(), _stream(stream)), "dsmc_merge_level")


def dsmc_resolve(cfg, model, state, traj, mean, m2, x_star, ws, stream=None):
    _check(load().dsmc_resolve(C.byref(cfg), C.byref(model.struct), C.byref(state), _ptr(traj),
                               _ptr(mean), _ptr(m2), _ptr(x_star), _ptr(ws), ws.numel(),
                               _stream(stream)), "dsmc_resolve")


def dsmc_smooth(cfg, model, prop, y, state, traj, mean, m2, logL, ws, stream=None):
    _check(load().dsmc_smooth(C.byref(cfg), C.byref(model.struct), C.byref(prop), _ptr(y),
                              C.byref(state), _ptr(traj), _ptr(mean), _ptr(m2), _ptr(logL),
                              _ptr(ws), ws.numel(), _stream(stream)), "dsmc_smooth")


def dsmc_conditional_smooth(cfg, model, prop, y, x_ref_in, x_ref_out, state, traj, mean, logL,
                            ws, stream=None):
    _check(load().dsmc_conditional_smooth(C.byref(cfg), C.byref(model.struct), C.byref(prop),
                                          _ptr(y), _ptr(x_ref_in), _ptr(x_ref_out), C.byref(state),
                                          _ptr(traj), _ptr(mean), _ptr(logL), _ptr(ws), ws.numel(),
                                          _stream(stream)), "dsmc_conditional_smooth")


def dsmc_smooth_noalloc(cfg, model, prop, y, state, traj, mean, m2, logL, stream=None) -> int:
    """dsmc_smooth on the library's static scratch (no workspace argument, no allocation);
    returns the device status of the smoothing (the call synchronises the stream)."""
    st = C.c_int(0)
    _check(load().dsmc_smooth_noalloc(C.byref(cfg), C.byref(model.struct), C.byref(prop), _ptr(y),
                                      C.byref(state), _ptr(traj), _ptr(mean), _ptr(m2), _ptr(logL),
                                      C.byref(st), _stream(stream)), "dsmc_smooth_noalloc")
    return int(st.value)


def dsmc_gaussian_proposals_workspace_size(model: HostModel, K: int) -> int:
    out = C.c_size_t(0)
    _check(load().dsmc_gaussian_proposals_workspace_size(C.byref(model.struct), int(K), C.byref(out)),
           "dsmc_gaussian_proposals_workspace_size")
    return int(out.value)


def dsmc_gaussian_proposals(model: HostModel, y, iterations=1, init_mean=None, ws=None, stream=None):
    """Algorithm 4's Gaussian marginals (means, standard deviations [K][dx] FP32 device tensors)
    of the linearised smoother, for DSMC_PROP_GAUSS proposals."""
    K, d = y.shape
    if ws is None:
        ws = torch.empty((dsmc_gaussian_proposals_workspace_size(model, K),), dtype=torch.uint8, device=y.device)
    mean = torch.empty((K, d), dtype=torch.float32, device=y.device)
    std = torch.empty((K, d), dtype=torch.float32, device=y.device)
    _check(load().dsmc_gaussian_proposals(C.byref(model.struct), int(K), _ptr(y), int(iterations), _ptr(init_mean),
                                          _ptr(mean), _ptr(std), _ptr(ws), ws.numel(), _stream(stream)),
           "dsmc_gaussian_proposals")
    return mean, std, ws


def dsmc_stream_status(ws, stream=None) -> int:
    out = C.c_int(0)
    _check(load().dsmc_stream_status(_ptr(ws), _stream(stream), C.byref(out)), "dsmc_stream_status")
    return int(out.value)


def dsmc_profile_enable(enable: bool):
    _check(load().dsmc_profile_enable(1 if enable else 0), "dsmc_profile_enable")


def dsmc_profile_read():
    """(rowsum_ms, rowsum_launches, rowsum_pairs, all_launches) since profiling was enabled."""
    ms, n, pairs, alln = C.c_double(0), C.c_int64(0), C.c_double(0), C.c_int64(0)
    _check(load().dsmc_profile_read(C.byref(ms), C.byref(n), C.byref(pairs), C.byref(alln)),
           "dsmc_profile_read")
    return ms.value, n.value, pairs.value, alln.value


def dsmc_debug_stall_tensor_cores(enable: bool):
    _check(load().dsmc_debug_stall_tensor_cores(int(bool(enable))), "dsmc_debug_stall_tensor_cores")


def dsmc_debug_keep_weights(enable: bool):
    _check(load().dsmc_debug_keep_weights(int(bool(enable))), "dsmc_debug_keep_weights")


def dsmc_debug_philox(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    n = ctr.numel() // 4
    _check(load().dsmc_debug_philox(_ptr(ctr), n, int(seed), _ptr(out), _stream(stream)),
           "dsmc_debug_philox")
    return out


def dsmc_debug_merge_weights(cfg, model, level, m, ws,
                             want=("logW", "r", "rowsum", "tiles", "e", "ratio"), stream=None):
    N = cfg.N
    info = (C.c_int * 4)()
    # first call for the tile count
    _check(load().dsmc_debug_merge_weights(C.byref(cfg), C.byref(model.struct), int(level), int(m),
                                           None, None, None, None, None, None, info, _ptr(ws),
                                           ws.numel(),
                                           _stream(stream)), "dsmc_debug_merge_weights")
    B, nT = info[0], info[1]
    dev = ws.device
    out = {}
    out["logW"] = torch.empty((N, N), dtype=torch.float32, device=dev) if "logW" in want else None
    out["r"] = torch.empty((N,), dtype=torch.float32, device=dev) if "r" in want else None
    out["rowsum"] = torch.empty((N,), dtype=torch.float32, device=dev) if "rowsum" in want else None
    out["tiles"] = torch.empty((N, nT), dtype=torch.float32, device=dev) if "tiles" in want else None
    out["e"] = torch.empty((N, N), dtype=torch.float32, device=dev) if "e" in want else None
    out["ratio"] = torch.empty((N, N), dtype=torch.float32, device=dev) if "ratio" in want else None
    _check(load().dsmc_debug_merge_weights(C.byref(cfg), C.byref(model.struct), int(level), int(m),
                                           _ptr(out["logW"]), _ptr(out["r"]), _ptr(out["rowsum"]),
                                           _ptr(out["tiles"]),
                                           _ptr(out["e"]), _ptr(out["ratio"]), info, _ptr(ws),
                                           ws.numel(), _stream(stream)), "dsmc_debug_merge_weights")
    out.update(B=info[0], nT=info[1], gid=info[2], left_leaf=info[3])
    return out


def dsmc_debug_lazy_weights(cfg, model, level, m, ws, stream=None):
    """The factorised proposals (pa, pc [N]) and acceptance ratios (acc [N][N]) of one
    combination after dsmc_merge_level with DSMC_RS_FACTORED."""
    N = cfg.N
    info = (C.c_int * 4)()
    dev = ws.device
    out = {"pa": torch.empty((N,), dtype=torch.float32, device=dev),
           "pc": torch.empty((N,), dtype=torch.float32, device=dev),
           "acc": torch.empty((N, N), dtype=torch.float32, device=dev)}
    _check(load().dsmc_debug_lazy_weights(C.byref(cfg), C.byref(model.struct), int(level), int(m),
                                          _ptr(out["pa"]), _ptr(out["pc"]), _ptr(out["acc"]), info, _ptr(ws),
                                          ws.numel(), _stream(stream)), "dsmc_debug_lazy_weights")
    out.update(gid=info[2], left_leaf=info[3])
    return out


def dsmc_debug_row_shift(cfg, model, level, m, ws, stream=None):
    """(shift [N] FP64, delta [N] FP32): the per-row scale of the tile and element weights of
    one combination after dsmc_merge_level with a dense resampler."""
    N = cfg.N
    sh = torch.empty((N,), dtype=torch.float64, device=ws.device)
    dl = torch.empty((N,), dtype=torch.float32, device=ws.device)
    _check(load().dsmc_debug_row_shift(C.byref(cfg), C.byref(model.struct), int(level), int(m), _ptr(sh), _ptr(dl),
                                       _ptr(ws), ws.numel(), _stream(stream)), "dsmc_debug_row_shift")
    return sh, dl


def dsmc_lazy_attempts(cfg, model, ws, stream=None) -> int:
    out = C.c_uint64(0)
    _check(load().dsmc_lazy_attempts(C.byref(cfg), C.byref(model.struct), _ptr(ws), ws.numel(), _stream(stream),
                                     C.byref(out)), "dsmc_lazy_attempts")
    return int(out.value)


def dsmc_batch_workspace_size(cfg: Config, model: HostModel, Ks) -> int:
    K = (C.c_int * len(Ks))(*[int(k) for k in Ks])
    out = C.c_size_t(0)
    _check(load().dsmc_batch_workspace_size(C.byref(cfg), C.byref(model.struct), len(Ks), K, C.byref(out)),
           "dsmc_batch_workspace_size")
    return int(out.value)


def _batch_call(name, cfg, model, prop, seqs, ws, stream):
    arr = (Seq * len(seqs))(*seqs)
    _check(getattr(load(), name)(C.byref(cfg), C.byref(model.struct), C.byref(prop), len(seqs), arr, _ptr(ws),
                                 ws.numel(), _stream(stream)), name)


def dsmc_batch_prepare(cfg, model, prop, seqs, ws, stream=None):
    _batch_call("dsmc_batch_prepare", cfg, model, prop, seqs, ws, stream)


def dsmc_batch_run(cfg, model, prop, seqs, ws, stream=None):
    _batch_call("dsmc_batch_run", cfg, model, prop, seqs, ws, stream)


def dsmc_smooth_batch(cfg, model, prop, seqs, ws, stream=None):
    _batch_call("dsmc_smooth_batch", cfg, model, prop, seqs, ws, stream)


KINDS = ["init", "prologue", "tile_sums", "draws", "fused_levels", "resolve", "gather", "fused_tc_levels"]


def dsmc_profile_breakdown_enable(enable: bool):
    _check(load().dsmc_profile_breakdown_enable(1 if enable else 0), "dsmc_profile_breakdown_enable")


def dsmc_profile_breakdown_read() -> dict:
    ms = (C.c_double * 8)()
    n = (C.c_int64 * 8)()
    _check(load().dsmc_profile_breakdown_read(ms, n), "dsmc_profile_breakdown_read")
    return {KINDS[k]: {"ms": ms[k], "launches": int(n[k])} for k in range(8) if n[k] > 0}


UNIT_NAMES = ["ex2", "ffma", "ffma2_lanes", "fadd", "dfma"]


def dsmc_profile_unit_rates(stream=None) -> dict:
    """Results per second of the device's MUFU ex2, FFMA, FFMA2 (lanes), FADD and DFMA units."""
    sink = torch.zeros((1,), dtype=torch.float32, device="cuda")
    out = (C.c_double * len(UNIT_NAMES))()
    _check(load().dsmc_profile_unit_rates(_ptr(sink), out, _stream(stream)), "dsmc_profile_unit_rates")
    return {UNIT_NAMES[k]: out[k] for k in range(len(UNIT_NAMES))}


def dsmc_seq_maps_bytes(K: int, N: int) -> int:
    return int(load().dsmc_seq_maps_bytes(int(K), int(N)))


def dsmc_serve_workspace_size(cfg: Config, model: HostModel, max_seq: int, max_combinations: int) -> int:
    out = C.c_size_t(0)
    _check(load().dsmc_serve_workspace_size(C.byref(cfg), C.byref(model.struct), int(max_seq),
                                            int(max_combinations), C.byref(out)), "dsmc_serve_workspace_size")
    return int(out.value)


def dsmc_serve_tick(cfg, model, prop, seqs, stages, ws, stream=None):
    arr = (Seq * len(seqs))(*seqs)
    st = (C.c_int * len(stages))(*[int(s) for s in stages])
    _check(load().dsmc_serve_tick(C.byref(cfg), C.byref(model.struct), C.byref(prop), len(seqs), arr, st,
                                  _ptr(ws), ws.numel(), _stream(stream)), "dsmc_serve_tick")


# ---------------------------------------------------------------- buffer owner
class Smoother:
    """Device buffers for one (model, K, N) and the calls of the C ABI over them.

    Buffers are allocated once through PyTorch (the library allocates nothing)."""

    def __init__(self, model: W.SSM, K: int, N: int, seed: int = 0, resampler: int = MULTINOMIAL,
                 compute: int = FP32, rs_max_attempts: int = 0, max_merges_per_launch: int = 0,
                 device: str = "cuda", want_traj: bool = False, fused_max_merges: int = 0, tc_fused: int = 0,
                 tile_cols: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("dSMC needs a CUDA device; there is no CPU path")
        self.model = model
        self.hm = HostModel(model)
        self.K, self.N, self.d = int(K), int(N), model.d
        self.cfg = make_config(K, N, seed, 0, resampler, compute, rs_max_attempts, max_merges_per_launch,
                               fused_max_merges, tc_fused, tile_cols)
        self.prop, self._prop_keep = make_proposal(model, K, device)
        sizes = dsmc_state_sizes(self.cfg, self.hm)
        self.X = torch.empty((self.K, self.N, self.d), dtype=torch.float32, device=device)
        self.logw = torch.empty((self.K, self.N), dtype=torch.float32, device=device)
        self.logL = torch.empty((self.K,), dtype=torch.float64, device=device)
        self.pairs = torch.empty((max(self.K - 1, 0), 2, self.N), dtype=torch.int32, device=device)
        assert sizes[0] == self.X.numel() * 4 and sizes[3] == self.pairs.numel() * 4
        self.state = State(self.X.data_ptr(), self.logw.data_ptr(), self.logL.data_ptr(),
                           self.pairs.data_ptr() if self.pairs.numel() else None)
        wsb = dsmc_workspace_size(self.cfg, self.hm)
        self.ws = torch.empty((wsb,), dtype=torch.uint8, device=device)
        self.mean = torch.empty((self.K, self.d), dtype=torch.float64, device=device)
        self.m2 = torch.empty((self.K, self.d), dtype=torch.float64, device=device)
        self.logL_out = torch.empty((1,), dtype=torch.float64, device=device)
        self.traj = (torch.empty((self.K, self.N, self.d), dtype=torch.float32, device=device)
                     if want_traj else None)
        self.x_star = torch.empty((self.K, self.d), dtype=torch.float32, device=device)

    def set_model(self, model: W.SSM, prop_mean: torch.Tensor = None, prop_std: torch.Tensor = None):
        """Swap the model parameters (same kind and dimension: the buffers stay).  With device
        FP32 [K][d] tensors prop_mean / prop_std the proposal is DSMC_PROP_GAUSS over them, kept
        on the device (no host round trip), e.g. dsmc_gaussian_proposals' outputs."""
        if model.kind != self.model.kind or model.d != self.d:
            raise ValueError("set_model keeps the model kind and dimension")
        self.model = model
        self.hm = HostModel(model)
        if prop_mean is None:
            self.prop, self._prop_keep = make_proposal(model, self.K, self.X.device)
        else:
            if prop_mean.shape != (self.K, self.d) or prop_std.shape != (self.K, self.d) or \
                    prop_mean.dtype != torch.float32 or prop_std.dtype != torch.float32:
                raise ValueError("proposal arrays must be FP32 [K][d]")
            pm, ps = prop_mean.contiguous(), prop_std.contiguous()
            self.prop, self._prop_keep = Proposal(W.PROP_GAUSS, 1.0, pm.data_ptr(), ps.data_ptr(), int(model.nu)), \
                (pm, ps)

    @property
    def levels(self) -> int:
        L = 0
        while (1 << L) < self.K:
            L += 1
        return L

    def set_seed(self, seed: int, counter_base: int = 0):
        self.cfg.seed = int(seed) & (2**64 - 1)
        self.cfg.counter_base = int(counter_base)

    def smooth(self, y: torch.Tensor, stream=None):
        dsmc_smooth(self.cfg, self.hm, self.prop, y, self.state, self.traj, self.mean, self.m2,
                    self.logL_out, self.ws, stream)
        return self.mean

    def conditional(self, y: torch.Tensor, x_ref_in: torch.Tensor, x_ref_out: torch.Tensor, stream=None):
        dsmc_conditional_smooth(self.cfg, self.hm, self.prop, y, x_ref_in, x_ref_out, self.state,
                                self.traj, self.mean, self.logL_out, self.ws, stream)
        return x_ref_out

    def init(self, y, x_ref=None, stream=None):
        dsmc_init_particles(self.cfg, self.hm, self.prop, y, x_ref, self.state, self.ws, stream)

    def merge_level(self, y, level, conditional=False, stream=None):
        dsmc_merge_level(self.cfg, self.hm, self.prop, y, level, conditional, self.state, self.ws, stream)

    def resolve(self, x_star=False, stream=None):
        dsmc_resolve(self.cfg, self.hm, self.state, self.traj, self.mean, self.m2,
                     self.x_star if x_star else None, self.ws, stream)

    def status(self, stream=None) -> int:
        return dsmc_stream_status(self.ws, stream)


class BatchSmoother:
    """Device buffers for a batch of sequences of one model and N (lengths Ks, observations
    ys), and the batched calls over them.  Each sequence gets its own seed (seeds[i]) and
    counter base; ``run`` launches without host synchronisation (CUDA-graph capturable)
    after ``prepare``."""

    def __init__(self, model: W.SSM, Ks, N: int, seeds=None, resampler: int = MULTINOMIAL,
                 compute: int = FP32, max_merges_per_launch: int = 0, fused_max_merges: int = 0,
                 device: str = "cuda", want_m2: bool = False, tc_fused: int = 0, tile_cols: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("dSMC needs a CUDA device; there is no CPU path")
        self.model = model
        self.hm = HostModel(model)
        self.Ks = [int(k) for k in Ks]
        self.N, self.d = int(N), model.d
        n = len(self.Ks)
        self.seeds = list(seeds) if seeds is not None else [1000 + i for i in range(n)]
        self.counter_base = [0] * n
        self.cfg = make_config(max(self.Ks), N, 0, 0, resampler, compute, 0, max_merges_per_launch,
                               fused_max_merges, tc_fused, tile_cols)
        if model.prop_kind == W.PROP_GAUSS:
            self.prop = Proposal(W.PROP_GAUSS, 1.0, None, None, int(model.nu))
        else:
            self.prop = Proposal(int(model.prop_kind), float(model.prop_scale), None, None, int(model.nu))
        f32, f64, i32 = torch.float32, torch.float64, torch.int32
        dev = device
        self.X = [torch.empty((k, N, self.d), dtype=f32, device=dev) for k in self.Ks]
        self.logw = [torch.empty((k, N), dtype=f32, device=dev) for k in self.Ks]
        self.logL = [torch.empty((k,), dtype=f64, device=dev) for k in self.Ks]
        self.pairs = [torch.empty((max(k - 1, 0), 2, N), dtype=i32, device=dev) for k in self.Ks]
        self.mean = [torch.empty((k, self.d), dtype=f64, device=dev) for k in self.Ks]
        self.m2 = [torch.empty((k, self.d), dtype=f64, device=dev) for k in self.Ks] if want_m2 else None
        self.logL_out = torch.empty((n,), dtype=f64, device=dev)
        self.y = [None] * n
        self.pm = [None] * n
        self.ps = [None] * n
        self.x_in = [None] * n
        self.x_out = [None] * n
        self.ws = torch.empty((dsmc_batch_workspace_size(self.cfg, self.hm, self.Ks),), dtype=torch.uint8,
                              device=dev)

    def set_inputs(self, ys, x_ref_in=None, x_ref_out=None):
        """Observations (device [K_i][d] FP32 tensors) and, for a particle-Gibbs sweep, the
        references in and out per sequence (None entries: plain smoothing)."""
        n = len(self.Ks)
        for i in range(n):
            self.y[i] = ys[i]
            if self.model.prop_kind == W.PROP_GAUSS:
                K = self.Ks[i]
                self.pm[i] = torch.as_tensor(proposal_rows(self.model.prop_mean, K, self.d), device=ys[i].device)
                self.ps[i] = torch.as_tensor(proposal_rows(self.model.prop_std, K, self.d), device=ys[i].device)
            self.x_in[i] = x_ref_in[i] if x_ref_in is not None else None
            self.x_out[i] = x_ref_out[i] if x_ref_out is not None else None

    def seqs(self):
        out = []
        for i, K in enumerate(self.Ks):
            st = State(self.X[i].data_ptr(), self.logw[i].data_ptr(), self.logL[i].data_ptr(),
                       self.pairs[i].data_ptr() if self.pairs[i].numel() else None)
            out.append(Seq(K, self.y[i].data_ptr(),
                           self.pm[i].data_ptr() if self.pm[i] is not None else None,
                           self.ps[i].data_ptr() if self.ps[i] is not None else None, st,
                           self.mean[i].data_ptr(), self.m2[i].data_ptr() if self.m2 is not None else None,
                           self.logL_out.data_ptr() + 8 * i,
                           self.x_in[i].data_ptr() if self.x_in[i] is not None else None,
                           self.x_out[i].data_ptr() if self.x_out[i] is not None else None,
                           int(self.seeds[i]) & (2**64 - 1), int(self.counter_base[i]), None))
        return out

    def prepare(self, stream=None):
        dsmc_batch_prepare(self.cfg, self.hm, self.prop, self.seqs(), self.ws, stream)

    def run(self, stream=None):
        dsmc_batch_run(self.cfg, self.hm, self.prop, self.seqs(), self.ws, stream)

    def smooth(self, stream=None):
        dsmc_smooth_batch(self.cfg, self.hm, self.prop, self.seqs(), self.ws, stream)
        return self.mean

    def status(self, stream=None) -> int:
        return dsmc_stream_status(self.ws, stream)
