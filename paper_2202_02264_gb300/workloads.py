"""Seeded synthetic workloads: state-space models and simulated observations.

This module holds model parameters and the simulation of observations from them (the
state-space model of Eq. (ssm) in Section 1 of the paper).  It holds none of dSMC's own
arithmetic, so that both the CUDA path and the CPU oracle can draw their inputs from it.

Workloads (T in the paper's experiments is read as the number of time steps K):
  * ``lgssm_1d``   x_0 ~ N(0,1), x_t = 0.9 x_{t-1} + N(0,1), y_t = x_t + N(0, 0.5^2);
                   proposal q_t = N(y_t, 1).  K = 32, N = 64.
  * ``lgssm_d8``   d_x = d_y = 8, A = 0.5 I + 0.05 G (G iid N(0,1), seed 2202), Q = I,
                   R = 0.25 I, x_0 ~ N(0, I), q_t = N(y_t, I).  K = N = 1024.
  * ``sv``         stochastic volatility, mu = -1, phi = 0.95, sigma = 0.3, d = 1;
                   q_t = nu_t = stationary N(mu, sigma^2 / (1 - phi^2)) (the choice of the
                   paper's Cox experiment).  K = 4096, N = 4096 dense / 16384 lazy.
  * ``lgssm_d4``   d = 4, A = 0.8 I, Q = I, R = 0.5 I, x_0 ~ N(0, I), q_t = N(y_t, I).
Observations use seed 2264 + workload index; algorithm seeds are 1000 + replicate.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

LGSSM = 0
SV = 1
COX = 2              # Section 5.1: Poisson counts, Gaussian autoregression
THETA_LOGISTIC = 3   # Section 5.2: theta-logistic population dynamics
CRW = 4              # Section 5.3: random walk constrained to [-bound, bound]

PROP_OBS = 0      # q_t = N(y_t, scale^2 I)
PROP_GAUSS = 1    # q_t = N(mean_t, diag(std_t^2)), arrays [K][d]
PROP_UNIFORM = 2  # q_t = U([-scale, scale]^d)

NU_EQ_Q = 0     # nu_t = q_t for t >= 1
NU_PROP_H = 1   # nu_t proportional to h_t(y_t | .)


@dataclass
class SSM:
    """A state-space model with its proposal (Definition 1 and Algorithm 2 inputs)."""

    kind: int
    d: int
    A: Optional[np.ndarray] = None
    Q: Optional[np.ndarray] = None
    R: Optional[np.ndarray] = None
    m0: Optional[np.ndarray] = None
    P0: Optional[np.ndarray] = None
    mu: float = 0.0
    phi: float = 0.0
    sigma: float = 1.0
    lam: float = 1.0      # COX
    tau0: float = 0.0     # THETA_LOGISTIC
    tau1: float = 0.0
    tau2: float = 0.0
    obs_sd: float = 1.0
    bound: float = 1.0    # CRW
    prop_kind: int = PROP_OBS
    prop_scale: float = 1.0
    prop_mean: Optional[np.ndarray] = None  # [K][d]
    prop_std: Optional[np.ndarray] = None   # [K][d]
    nu: int = NU_EQ_Q
    name: str = ""

    def proposal_arrays(self, y: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Per-t proposal mean and standard deviation, [K][d] each."""
        K = y.shape[0]
        if self.prop_kind == PROP_OBS:
            return y.astype(np.float64).copy(), np.full((K, self.d), self.prop_scale)
        return (np.asarray(self.prop_mean, np.float64)[:K].copy(),
                np.asarray(self.prop_std, np.float64)[:K].copy())


def lgssm(A, Q, R, m0=None, P0=None, prop_scale=1.0, nu=NU_EQ_Q, name="lgssm") -> SSM:
    A = np.atleast_2d(np.asarray(A, np.float64))
    d = A.shape[0]
    Q = np.atleast_2d(np.asarray(Q, np.float64))
    R = np.atleast_2d(np.asarray(R, np.float64))
    m0 = np.zeros(d) if m0 is None else np.asarray(m0, np.float64).reshape(d)
    P0 = np.eye(d) if P0 is None else np.atleast_2d(np.asarray(P0, np.float64))
    return SSM(kind=LGSSM, d=d, A=A, Q=Q, R=R, m0=m0, P0=P0, prop_kind=PROP_OBS,
               prop_scale=float(prop_scale), nu=nu, name=name)


def lgssm_1d(nu=NU_EQ_Q) -> SSM:
    return lgssm([[0.9]], [[1.0]], [[0.25]], [0.0], [[1.0]], 1.0, nu, "lgssm_1d")


def random_transition(d: int, seed: int = 2202, base: float = 0.5, scale: float = 0.05) -> np.ndarray:
    """A = base I + scale * G with G iid N(0,1); the spectral radius is checked below 1."""
    G = np.random.default_rng(seed).standard_normal((d, d))
    A = base * np.eye(d) + scale * G
    rho = max(abs(np.linalg.eigvals(A)))
    if rho >= 1.0:
        raise ValueError(f"transition matrix not stable (rho={rho})")
    return A


def lgssm_d8(nu=NU_EQ_Q) -> SSM:
    d = 8
    return lgssm(random_transition(d), np.eye(d), 0.25 * np.eye(d), np.zeros(d), np.eye(d),
                 1.0, nu, "lgssm_d8")


def lgssm_dn(d: int, nu=NU_EQ_Q) -> SSM:
    """The d = 8 model family at another dimension: A = 0.5 I + 0.05 sqrt(8/d) G."""
    A = random_transition(d, scale=0.05 * np.sqrt(8.0 / d))
    return lgssm(A, np.eye(d), 0.25 * np.eye(d), np.zeros(d), np.eye(d), 1.0, nu, f"lgssm_d{d}")


def lgssm_d4(nu=NU_EQ_Q) -> SSM:
    d = 4
    return lgssm(0.8 * np.eye(d), np.eye(d), 0.5 * np.eye(d), np.zeros(d), np.eye(d), 1.0, nu,
                 "lgssm_d4")


def sv(K: int, mu=-1.0, phi=0.95, sigma=0.3, nu=NU_EQ_Q) -> SSM:
    """Stochastic volatility with the stationary law as proposal for every t."""
    s0 = sigma / np.sqrt(1.0 - phi * phi)
    return SSM(kind=SV, d=1, mu=float(mu), phi=float(phi), sigma=float(sigma),
               prop_kind=PROP_GAUSS, prop_mean=np.full((K, 1), mu),
               prop_std=np.full((K, 1), s0), nu=nu, name="sv")


def cox(K: int, mu=0.5, phi=0.9, sigma=0.35, lam=1.0) -> SSM:
    """The Poisson-count model of Section 5.1 with the stationary law as q_t = nu_t."""
    s0 = sigma / np.sqrt(1.0 - phi * phi)
    return SSM(kind=COX, d=1, mu=float(mu), phi=float(phi), sigma=float(sigma), lam=float(lam),
               prop_kind=PROP_GAUSS, prop_mean=np.full((K, 1), mu), prop_std=np.full((K, 1), s0),
               nu=NU_EQ_Q, name="cox")


def theta_logistic(tau0=0.15, tau1=0.12, tau2=0.25, q=0.12, r=0.25, prop_scale=0.5) -> SSM:
    """The theta-logistic model of Section 5.2 (log-population), observation-centred
    proposals N(y_t, prop_scale^2)."""
    return SSM(kind=THETA_LOGISTIC, d=1, sigma=float(q), tau0=float(tau0), tau1=float(tau1), tau2=float(tau2),
               obs_sd=float(r), prop_kind=PROP_OBS, prop_scale=float(prop_scale), nu=NU_EQ_Q,
               name="theta_logistic")


def crw(sigma=0.4, bound=1.0) -> SSM:
    """The constrained random walk of Section 5.3 with the uniform proposal on the constraint."""
    return SSM(kind=CRW, d=1, sigma=float(sigma), bound=float(bound), prop_kind=PROP_UNIFORM,
               prop_scale=float(bound), nu=NU_EQ_Q, name="crw")


def simulate(model: SSM, K: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Draw (x_{0:K-1}, y_{0:K-1}) from the model, FP64, shapes [K][d].  For the constrained
    random walk y is all zero (the model has no observations) and x is one path of the
    unconstrained walk."""
    rng = np.random.default_rng(seed)
    d = model.d
    x = np.zeros((K, d))
    y = np.zeros((K, d))
    if model.kind == COX:
        s0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
        x[0, 0] = model.mu + s0 * rng.standard_normal()
        for t in range(1, K):
            x[t, 0] = (model.mu + model.phi * (model.lam * x[t - 1, 0] - model.mu)
                       + model.sigma * rng.standard_normal())
        y[:, 0] = rng.poisson(np.exp(x[:, 0]))
        return x, y
    if model.kind == THETA_LOGISTIC:
        x[0, 0] = rng.standard_normal()
        for t in range(1, K):
            xp = x[t - 1, 0]
            x[t, 0] = xp + model.tau0 - model.tau1 * np.exp(model.tau2 * xp) + model.sigma * rng.standard_normal()
        y[:, 0] = x[:, 0] + model.obs_sd * rng.standard_normal(K)
        return x, y
    if model.kind == CRW:
        x[0, 0] = rng.standard_normal()
        for t in range(1, K):
            x[t, 0] = x[t - 1, 0] + model.sigma * rng.standard_normal()
        return x, y
    if model.kind == LGSSM:
        Lq = np.linalg.cholesky(model.Q)
        Lr = np.linalg.cholesky(model.R)
        L0 = np.linalg.cholesky(model.P0)
        x[0] = model.m0 + L0 @ rng.standard_normal(d)
        for t in range(1, K):
            x[t] = model.A @ x[t - 1] + Lq @ rng.standard_normal(d)
        y = x + rng.standard_normal((K, d)) @ Lr.T
    else:
        s0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
        x[0, 0] = model.mu + s0 * rng.standard_normal()
        for t in range(1, K):
            x[t, 0] = model.mu + model.phi * (x[t - 1, 0] - model.mu) + model.sigma * rng.standard_normal()
        y[:, 0] = np.exp(x[:, 0] / 2.0) * rng.standard_normal(K)
    return x, y


@dataclass
class Workload:
    name: str
    model: SSM
    K: int
    N: int
    y: np.ndarray = field(repr=False)
    x_true: np.ndarray = field(repr=False)


def workload(name: str, K: Optional[int] = None, N: Optional[int] = None) -> Workload:
    """The named synthetic workload, optionally at another K or N."""
    if name == "lgssm_1d":
        K = 32 if K is None else K
        N = 64 if N is None else N
        m, seed = lgssm_1d(), 2264 + 1
    elif name == "lgssm_d8":
        K = 1024 if K is None else K
        N = 1024 if N is None else N
        m, seed = lgssm_d8(), 2264 + 2
    elif name == "sv":
        K = 4096 if K is None else K
        N = 4096 if N is None else N
        m, seed = sv(K), 2264 + 3
    elif name == "lgssm_d4":
        K = 512 if K is None else K
        N = 512 if N is None else N
        m, seed = lgssm_d4(), 2264 + 4
    elif name == "cox":
        K = 256 if K is None else K
        N = 512 if N is None else N
        m, seed = cox(K), 2264 + 40
    elif name == "theta_logistic":
        K = 120 if K is None else K
        N = 256 if N is None else N
        m, seed = theta_logistic(), 2264 + 41
    elif name == "crw":
        K = 64 if K is None else K
        N = 1024 if N is None else N
        m, seed = crw(), 2264 + 42
    elif name in ("lgssm_d2", "lgssm_d16", "lgssm_d32"):
        dd = int(name[len("lgssm_d"):])
        K = 256 if K is None else K
        N = 256 if N is None else N
        m, seed = lgssm_dn(dd), 2264 + 5 + dd
    else:
        raise KeyError(name)
    x, y = simulate(m, K, seed)
    return Workload(name, m, K, N, y, x)


def batched_lengths(n_seq: int = 256, lo: int = 64, hi: int = 4096, seed: int = 2264 + 4) -> np.ndarray:
    """Sequence lengths K_i drawn uniformly in [lo, hi] (includes non-powers of two)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n_seq)


@dataclass
class BatchWorkload:
    name: str
    model: SSM
    N: int
    Ks: np.ndarray
    ys: list = field(repr=False)


def batch_workload(n_seq: int = 256, N: int = 512, lo: int = 64, hi: int = 4096) -> BatchWorkload:
    """The batched workload: n_seq independent sequences of the d = 4 linear-Gaussian model
    (A = 0.8 I, Q = I, R = 0.5 I), lengths uniform in [lo, hi] (seed 2268), sequence i's
    observations simulated with seed 40000 + i."""
    m = lgssm_d4()
    Ks = batched_lengths(n_seq, lo, hi)
    ys = [simulate(m, int(K), 40000 + i)[1] for i, K in enumerate(Ks)]
    return BatchWorkload("batched_lgssm_d4", m, int(N), Ks, ys)
