"""ctypes binding of the FP64 C oracle ``dsmc_oracle.c`` (test infrastructure only).

Each function names the passage of the paper it follows; the C source carries the steps.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR = {0: "ok", 1: "invalid argument", 3: "out of memory", 7: "degenerate weights",
       8: "rejection-sampling attempt cap reached"}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP contraction off, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def build_variant(replacements, out_dir: str) -> str:
    """Compile a copy of the oracle source with textual replacements [(old, new), ...]
    (each old text must occur) into out_dir; returns the library path."""
    src = open(_SRC).read()
    for old, new in replacements:
        if old not in src:
            raise ValueError(f"replacement target not found: {old!r}")
        src = src.replace(old, new)
    c_path = os.path.join(out_dir, "oracle_variant.c")
    so_path = os.path.join(out_dir, "liboracle_variant.so")
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                           "-o", so_path, c_path, "-lm"])
    return so_path


class Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int),
                ("A", C.POINTER(C.c_double)), ("Q", C.POINTER(C.c_double)),
                ("R", C.POINTER(C.c_double)), ("m0", C.POINTER(C.c_double)),
                ("P0", C.POINTER(C.c_double)),
                ("mu", C.c_double), ("phi", C.c_double), ("sigma", C.c_double),
                ("prop_kind", C.c_int), ("prop_scale", C.c_double),
                ("prop_mean", C.POINTER(C.c_double)), ("prop_std", C.POINTER(C.c_double)),
                ("nu", C.c_int), ("lam", C.c_double), ("tau0", C.c_double), ("tau1", C.c_double),
                ("tau2", C.c_double), ("obs_sd", C.c_double), ("bound", C.c_double)]


class Config(C.Structure):
    _fields_ = [("K", C.c_int), ("N", C.c_int), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32),
                ("counter_base", C.c_uint32), ("resampler", C.c_int),
                ("rs_max_attempts", C.c_uint32), ("conditional", C.c_int)]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _setup(C.CDLL(build()))
    return _lib


def load_variant(path: str):
    """A separately compiled copy of the oracle (tests plant mistakes in such copies to show
    that a pin rejects them); use it through ``variant``."""
    return _setup(C.CDLL(path))


class variant:
    """Context manager: the module's functions call the given oracle library inside it."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _lib
        _lib_handle()
        self.saved = _lib
        _lib = self.lib
        return self.lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _setup(lib):
    """Argument types of the oracle's exported functions."""
    dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
    u64p, fp = C.POINTER(C.c_uint64), C.POINTER(C.c_float)
    lib.orc_philox4x32_10.argtypes = [up, up, up]
    lib.orc_philox_many.argtypes = [C.c_int64, up, up, up]
    lib.orc_init.argtypes = [C.POINTER(Model), C.POINTER(Config), dp, dp, dp, dp, dp]
    lib.orc_smooth.argtypes = [C.POINTER(Model), C.POINTER(Config), dp, dp, dp, ip, dp, dp,
                               dp, dp, dp, u64p]
    lib.orc_logw_matrix.argtypes = [C.POINTER(Model), C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                    dp, dp, dp, dp, dp]
    lib.orc_model_logdens.argtypes = [C.POINTER(Model), C.c_int, dp, C.c_int, dp, dp, dp]
    lib.orc_num_levels.argtypes = [C.c_int]
    lib.orc_merges_at_level.argtypes = [C.c_int, C.c_int]
    lib.orc_dense_pairs.argtypes = [C.c_int, dp, C.c_uint32, C.c_uint32, C.c_uint32,
                                    C.c_uint32, C.c_int, C.c_int, ip, ip]
    lib.orc_rs_pairs.argtypes = [C.c_int, dp, C.c_double, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip, u64p]
    lib.orc_kp_dense_pairs.argtypes = [C.c_int, C.c_int, fp, fp, fp, C.c_uint32,
                                       C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int,
                                       ip, ip]
    lib.orc_kp_rs_pairs.argtypes = [C.c_int, fp, C.c_uint32, C.c_uint32, C.c_uint32,
                                    C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip, up]
    lib.orc_rs_bounds.argtypes = [C.POINTER(Model), C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                  dp, dp, dp, dp, dp]
    lib.orc_mh_pairs.argtypes = [C.c_int, dp, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip]
    lib.orc_kp_mh_pairs.argtypes = [C.c_int, fp, C.c_uint32, C.c_uint32, C.c_uint32,
                                    C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip]
    lib.orc_sys_pairs.argtypes = [C.c_int, dp, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_int, C.c_int, ip, ip]
    lib.orc_kp_sys_pairs.argtypes = [C.c_int, C.c_int, fp, fp, fp, C.c_uint32,
                                     C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int,
                                     ip, ip]
    lib.orc_rsf_pairs.argtypes = [C.c_int, dp, dp, dp, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip, u64p]
    lib.orc_kp_rsf_pairs.argtypes = [C.c_int, fp, fp, fp, C.c_uint32, C.c_uint32, C.c_uint32,
                                     C.c_uint32, C.c_int, C.c_int, C.c_uint32, ip, ip, up]
    return lib


def _p(a, ctype=C.c_double):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


class _Keep:
    """Holds the arrays a Model struct points into."""

    def __init__(self, model, K, y):
        d = model.d
        z = np.zeros((d, d))
        self.A = np.ascontiguousarray(model.A if model.A is not None else z, np.float64)
        self.Q = np.ascontiguousarray(model.Q if model.Q is not None else np.eye(d), np.float64)
        self.R = np.ascontiguousarray(model.R if model.R is not None else np.eye(d), np.float64)
        self.m0 = np.ascontiguousarray(model.m0 if model.m0 is not None else np.zeros(d), np.float64)
        self.P0 = np.ascontiguousarray(model.P0 if model.P0 is not None else np.eye(d), np.float64)
        if model.prop_kind == 1:
            self.pm = np.ascontiguousarray(np.asarray(model.prop_mean, np.float64)[:K], np.float64)
            self.ps = np.ascontiguousarray(np.asarray(model.prop_std, np.float64)[:K], np.float64)
            if self.pm.shape != (K, d) or self.ps.shape != (K, d):
                raise ValueError("proposal arrays must be [K][d]")
        else:
            self.pm = self.ps = None
        self.y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(K, d))
        self.struct = Model(model.kind, d, _p(self.A), _p(self.Q), _p(self.R), _p(self.m0),
                            _p(self.P0), model.mu, model.phi, model.sigma, model.prop_kind,
                            model.prop_scale, _p(self.pm), _p(self.ps), model.nu,
                            float(getattr(model, "lam", 1.0)), float(getattr(model, "tau0", 0.0)),
                            float(getattr(model, "tau1", 0.0)), float(getattr(model, "tau2", 0.0)),
                            float(getattr(model, "obs_sd", 1.0)), float(getattr(model, "bound", 1.0)))


def _seed_words(seed: int):
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def _check(st, what):
    if st not in (0, 8):
        raise RuntimeError(f"oracle {what}: {ERR.get(st, st)}")
    return st


def philox(ctr, key):
    """Philox4x32-10 of one counter (4 words) under one key (2 words)."""
    lib = _lib_handle()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def philox_many(ctrs, key):
    lib = _lib_handle()
    c = np.ascontiguousarray(ctrs, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros_like(c)
    lib.orc_philox_many(c.shape[0], _p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def num_levels(K: int) -> int:
    return _lib_handle().orc_num_levels(K)


def merges_at_level(K: int, l: int) -> int:
    return _lib_handle().orc_merges_at_level(K, l)


def init(model, y, K, N, seed, counter_base=0, x_ref=None):
    """Algorithm 2 (and its conditional form, Section 3.2): particles [K][N][d],
    normalised leaf log-weights [K][N], log L_t [K]."""
    lib = _lib_handle()
    keep = _Keep(model, K, y)
    lo, hi = _seed_words(seed)
    cf = Config(K, N, lo, hi, counter_base, 0, 1 << 20, 0 if x_ref is None else 1)
    X = np.zeros((K, N, model.d))
    lw = np.zeros((K, N))
    lL = np.zeros(K)
    xr = None if x_ref is None else np.ascontiguousarray(np.asarray(x_ref, np.float64).reshape(K, model.d))
    _check(lib.orc_init(C.byref(keep.struct), C.byref(cf), _p(keep.y), _p(xr), _p(X), _p(lw), _p(lL)), "init")
    return X, lw, lL


RESAMPLERS = {"dense": 0, "rs": 1, "mh": 2, "systematic": 3, "rsf": 4}


def smooth(model, y, K, N, seed, counter_base=0, resampler="dense", rs_max_attempts=1 << 20,
           x_ref=None, want_traj=False, want_pairs=False):
    """Full dSMC smoother: Algorithm 2, then Algorithm 6 over Combine (Algorithm 1) or
    ConditionalCombine (Algorithm 5), with multinomial, systematic, rejection (Algorithm 8,
    uniform or factorised pair proposals) or Metropolis-Hastings (Algorithm 7,
    B = rs_max_attempts steps) draws.

    Returns a dict with mean [K][d], m2 [K][d], logL, and optionally traj [K][N][d],
    pairs [K-1][2][N], X_leaf [K][N][d], x_star [K][d], rs_attempts, status."""
    lib = _lib_handle()
    keep = _Keep(model, K, y)
    lo, hi = _seed_words(seed)
    cond = x_ref is not None
    cf = Config(K, N, lo, hi, counter_base, RESAMPLERS[resampler], rs_max_attempts, 1 if cond else 0)
    d = model.d
    mean = np.zeros((K, d))
    m2 = np.zeros((K, d))
    logL = np.zeros(1)
    X = np.zeros((K, N, d)) if (want_traj or cond) else None
    traj = np.zeros((K, N, d)) if want_traj else None
    pairs = np.zeros((max(K - 1, 0), 2, N), np.int32) if (want_pairs or cond) else None
    xr = np.ascontiguousarray(np.asarray(x_ref, np.float64).reshape(K, d)) if cond else None
    xs = np.zeros((K, d)) if cond else None
    att = np.zeros(1, np.uint64)
    st = _check(lib.orc_smooth(C.byref(keep.struct), C.byref(cf), _p(keep.y), _p(xr), _p(X),
                               _p(pairs, C.c_int32) if pairs is not None and pairs.size else None,
                               _p(traj), _p(mean), _p(m2), _p(logL), _p(xs), _p(att, C.c_uint64)),
                "smooth")
    out = dict(mean=mean, m2=m2, logL=float(logL[0]), status=st, rs_attempts=int(att[0]))
    if want_traj:
        out["traj"] = traj
        out["X_leaf"] = X
    if want_pairs or cond:
        out["pairs"] = pairs
    if cond:
        out["x_star"] = xs
    return out


def logw_matrix(model, y, K, c, xl, xr, wl, wr):
    """logW[i][j] = log omega_c(xl_i, xr_j) + wl_i + wr_j in FP64 (Eq. normalized-weights,
    Proposition 2)."""
    lib = _lib_handle()
    keep = _Keep(model, K, y)
    xl = np.ascontiguousarray(xl, np.float64)
    xr = np.ascontiguousarray(xr, np.float64)
    wl = np.ascontiguousarray(wl, np.float64)
    wr = np.ascontiguousarray(wr, np.float64)
    Nl, Nr = wl.shape[0], wr.shape[0]
    out = np.zeros((Nl, Nr))
    _check(lib.orc_logw_matrix(C.byref(keep.struct), K, _p(keep.y), c, Nl, Nr, _p(xl), _p(xr),
                               _p(wl), _p(wr), _p(out)), "logw_matrix")
    return out


def rs_bounds(model, y, K, c, xl, xr, wl, wr):
    """(finite-set bound, hull bound) of Algorithm 8 for one combination, FP64."""
    lib = _lib_handle()
    keep = _Keep(model, K, y)
    xl = np.ascontiguousarray(xl, np.float64)
    xr = np.ascontiguousarray(xr, np.float64)
    wl = np.ascontiguousarray(wl, np.float64)
    wr = np.ascontiguousarray(wr, np.float64)
    out = np.zeros(2)
    _check(lib.orc_rs_bounds(C.byref(keep.struct), K, _p(keep.y), c, wl.shape[0], wr.shape[0], _p(xl),
                             _p(xr), _p(wl), _p(wr), _p(out)), "rs_bounds")
    return float(out[0]), float(out[1])


def model_logdens(model, y, K, t, xprev, x):
    """(log f(x|xprev), log h_t(x), log nu_t(x), log q_t(x), log f_max)."""
    lib = _lib_handle()
    keep = _Keep(model, K, y)
    a = np.ascontiguousarray(xprev, np.float64)
    b = np.ascontiguousarray(x, np.float64)
    out = np.zeros(5)
    _check(lib.orc_model_logdens(C.byref(keep.struct), K, _p(keep.y), t, _p(a), _p(b), _p(out)), "logdens")
    return out


def dense_pairs(logW, seed, gid, n0, n1, counter_base=0):
    """Multinomial draws (inverse CDF on the flattened matrix) for slots [n0, n1)."""
    lib = _lib_handle()
    W = np.ascontiguousarray(logW, np.float64)
    N = W.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_dense_pairs(N, _p(W), lo, hi, counter_base, gid, n0, n1, _p(li, C.c_int32),
                               _p(ri, C.c_int32)), "dense_pairs")
    return li, ri


def rs_pairs(logW, logbar, seed, gid, n0, n1, max_attempts=1 << 20, counter_base=0):
    """Algorithm 8 draws for slots [n0, n1) from a given log-weight matrix and bound."""
    lib = _lib_handle()
    W = np.ascontiguousarray(logW, np.float64)
    N = W.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    att = np.zeros(1, np.uint64)
    lo, hi = _seed_words(seed)
    st = _check(lib.orc_rs_pairs(N, _p(W), logbar, lo, hi, counter_base, gid, n0, n1, max_attempts,
                                 _p(li, C.c_int32), _p(ri, C.c_int32), _p(att, C.c_uint64)), "rs_pairs")
    return li, ri, int(att[0]), st


def mh_pairs(logW, seed, gid, n0, n1, B, counter_base=0):
    """Algorithm 7 draws for slots [n0, n1): B Metropolis-Hastings steps from (n, n) on a
    given log-weight matrix."""
    lib = _lib_handle()
    W = np.ascontiguousarray(logW, np.float64)
    N = W.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_mh_pairs(N, _p(W), lo, hi, counter_base, gid, n0, n1, B,
                            _p(li, C.c_int32), _p(ri, C.c_int32)), "mh_pairs")
    return li, ri


def kp_mh_pairs(ratio, seed, gid, n0, n1, B, counter_base=0):
    """Device-precision Algorithm 7 on the device's own FP32 ratios [N][N]."""
    lib = _lib_handle()
    q = np.ascontiguousarray(ratio, np.float32)
    N = q.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_kp_mh_pairs(N, _p(q, C.c_float), lo, hi, counter_base, gid, n0, n1, B,
                               _p(li, C.c_int32), _p(ri, C.c_int32)), "kp_mh_pairs")
    return li, ri


def kp_dense_pairs(r, t, e, B, seed, gid, n0, n1, counter_base=0):
    """Device-precision three-stage sampler (row / tile / column, exact fixed point) on the
    device's own FP32 weights: r [N] row weights, t [N][nT] tile weights, e [N][N] element
    weights."""
    lib = _lib_handle()
    r = np.ascontiguousarray(r, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    e = np.ascontiguousarray(e, np.float32)
    N = r.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_kp_dense_pairs(N, B, _p(r, C.c_float), _p(t, C.c_float), _p(e, C.c_float), lo, hi,
                                  counter_base, gid, n0, n1, _p(li, C.c_int32), _p(ri, C.c_int32)),
           "kp_dense_pairs")
    return li, ri


def kp_rs_pairs(ratio, seed, gid, n0, n1, max_attempts=1 << 20, counter_base=0):
    """Device-precision Algorithm 8 on the device's own FP32 acceptance ratios [N][N]."""
    lib = _lib_handle()
    q = np.ascontiguousarray(ratio, np.float32)
    N = q.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    att = np.zeros(n1 - n0, np.uint32)
    lo, hi = _seed_words(seed)
    st = _check(lib.orc_kp_rs_pairs(N, _p(q, C.c_float), lo, hi, counter_base, gid, n0, n1,
                                    max_attempts, _p(li, C.c_int32), _p(ri, C.c_int32),
                                    _p(att, C.c_uint32)), "kp_rs_pairs")
    return li, ri, att, st


def sys_pairs(logW, seed, gid, n0, n1, counter_base=0):
    """Systematic draws (positions (k + U) / N of the flattened CDF) for slots [n0, n1)."""
    lib = _lib_handle()
    W = np.ascontiguousarray(logW, np.float64)
    N = W.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_sys_pairs(N, _p(W), lo, hi, counter_base, gid, n0, n1, _p(li, C.c_int32),
                             _p(ri, C.c_int32)), "sys_pairs")
    return li, ri


def kp_sys_pairs(r, t, e, B, seed, gid, n0, n1, counter_base=0):
    """Device-precision systematic three-stage sampler on the device's own FP32 weights."""
    lib = _lib_handle()
    r = np.ascontiguousarray(r, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    e = np.ascontiguousarray(e, np.float32)
    N = r.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    lo, hi = _seed_words(seed)
    _check(lib.orc_kp_sys_pairs(N, B, _p(r, C.c_float), _p(t, C.c_float), _p(e, C.c_float), lo, hi,
                                counter_base, gid, n0, n1, _p(li, C.c_int32), _p(ri, C.c_int32)),
           "kp_sys_pairs")
    return li, ri


def rsf_pairs(la, lc, lacc, seed, gid, n0, n1, max_attempts=1 << 20, counter_base=0):
    """Rejection draws with factorised proposals (rows by exp(la), columns by exp(lc),
    acceptance exp(lacc) <= 1) for slots [n0, n1), FP64."""
    lib = _lib_handle()
    la = np.ascontiguousarray(la, np.float64)
    lc = np.ascontiguousarray(lc, np.float64)
    A = np.ascontiguousarray(lacc, np.float64)
    N = la.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    att = np.zeros(1, np.uint64)
    lo, hi = _seed_words(seed)
    st = _check(lib.orc_rsf_pairs(N, _p(la), _p(lc), _p(A), lo, hi, counter_base, gid, n0, n1, max_attempts,
                                  _p(li, C.c_int32), _p(ri, C.c_int32), _p(att, C.c_uint64)), "rsf_pairs")
    return li, ri, int(att[0]), st


def kp_rsf_pairs(ra, rc, acc, seed, gid, n0, n1, max_attempts=1 << 20, counter_base=0):
    """Device-precision factorised-proposal rejection sampler on the device's own FP32 row
    and column proposal weights and acceptance ratios."""
    lib = _lib_handle()
    ra = np.ascontiguousarray(ra, np.float32)
    rc = np.ascontiguousarray(rc, np.float32)
    A = np.ascontiguousarray(acc, np.float32)
    N = ra.shape[0]
    li = np.zeros(n1 - n0, np.int32)
    ri = np.zeros(n1 - n0, np.int32)
    att = np.zeros(n1 - n0, np.uint32)
    lo, hi = _seed_words(seed)
    st = _check(lib.orc_kp_rsf_pairs(N, _p(ra, C.c_float), _p(rc, C.c_float), _p(A, C.c_float), lo, hi,
                                     counter_base, gid, n0, n1, max_attempts, _p(li, C.c_int32),
                                     _p(ri, C.c_int32), _p(att, C.c_uint32)), "kp_rsf_pairs")
    return li, ri, att, st
