"""Parallel-in-time particle Gibbs with parameter updates (Section 3.2) on the theta-logistic
model of Section 5.2.

One sweep:
  1. (optional) the Gaussian proposals of Algorithm 4 for the current parameters: one pass of
     the iterated extended smoother started from the previous pass's means (the paper runs
     25 passes for the first sweep and one per sweep afterwards);
  2. one conditional dSMC sweep on the device (dsmc_conditional_smooth): the reference
     trajectory x* is kept in slot 0 of every combination and the next one is drawn from
     the root's weights;
  3. the parameters given x* and y, each from its full conditional:
       r^2 | x, y          ~ InvGamma(a + K/2, b + sum_t (y_t - x_t)^2 / 2)
       (tau0, tau1) | ...  Gaussian: the regression of x_t - x_{t-1} on [1, -exp(tau2 x_{t-1})]
                           with noise q^2 and an N(0, s^2 I) prior
       q^2 | x, tau        ~ InvGamma(a + (K-1)/2, b + sum_t residual_t^2 / 2)
       tau2 | ...          random-walk Metropolis-Hastings under a half-normal prior.
The dSMC sweep is the device's work; the parameter step is O(K) scalar arithmetic on the
host on the K values of x* (a transfer of K floats per sweep).  The priors are a reading:
the paper takes its priors from the references it cites and does not restate them.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import dsmc, workloads as W


@dataclass
class ThetaPrior:
    s_tau: float = 1.0        # N(0, s^2) for tau0, tau1; half-normal scale for tau2
    a: float = 2.0            # InvGamma(a, b) for q^2 and r^2
    b: float = 0.05
    rw_tau2: float = 0.05     # random-walk step of tau2


@dataclass
class ThetaState:
    tau0: float
    tau1: float
    tau2: float
    q2: float
    r2: float

    def model(self, prop_scale: float = 0.5) -> W.SSM:
        return W.theta_logistic(self.tau0, self.tau1, self.tau2, float(np.sqrt(self.q2)), float(np.sqrt(self.r2)),
                                prop_scale)


def _inv_gamma(rng, shape, rate):
    return rate / rng.gamma(shape)


def update_r2(rng, prior: ThetaPrior, x, y):
    K = x.shape[0]
    return _inv_gamma(rng, prior.a + 0.5 * K, prior.b + 0.5 * float(((y - x) ** 2).sum()))


def regression(x, tau2):
    """Design [1, -exp(tau2 x_{t-1})] and response x_t - x_{t-1} of the transition."""
    Z = np.stack([np.ones(x.shape[0] - 1), -np.exp(tau2 * x[:-1])], axis=1)
    return Z, x[1:] - x[:-1]


def update_tau01(rng, prior: ThetaPrior, x, tau2, q2):
    Z, dlt = regression(x, tau2)
    prec = np.eye(2) / prior.s_tau ** 2 + Z.T @ Z / q2
    cov = np.linalg.inv(prec)
    mean = cov @ (Z.T @ dlt / q2)
    t = rng.multivariate_normal(mean, cov)
    return float(t[0]), float(t[1])


def update_q2(rng, prior: ThetaPrior, x, tau0, tau1, tau2):
    Z, dlt = regression(x, tau2)
    res = dlt - Z @ np.array([tau0, tau1])
    return _inv_gamma(rng, prior.a + 0.5 * res.shape[0], prior.b + 0.5 * float((res ** 2).sum()))


def log_target_tau2(prior: ThetaPrior, x, tau0, tau1, tau2, q2):
    if tau2 <= 0.0:
        return -np.inf
    Z, dlt = regression(x, tau2)
    res = dlt - Z @ np.array([tau0, tau1])
    return -0.5 * float((res ** 2).sum()) / q2 - 0.5 * (tau2 / prior.s_tau) ** 2


def update_tau2(rng, prior: ThetaPrior, x, tau0, tau1, tau2, q2):
    prop = tau2 + prior.rw_tau2 * rng.standard_normal()
    lp = log_target_tau2(prior, x, tau0, tau1, prop, q2) - log_target_tau2(prior, x, tau0, tau1, tau2, q2)
    return prop if np.log(rng.uniform()) < lp else tau2


def update_parameters(rng, prior: ThetaPrior, th: ThetaState, x, y) -> ThetaState:
    r2 = update_r2(rng, prior, x, y)
    tau0, tau1 = update_tau01(rng, prior, x, th.tau2, th.q2)
    q2 = update_q2(rng, prior, x, tau0, tau1, th.tau2)
    tau2 = update_tau2(rng, prior, x, tau0, tau1, th.tau2, q2)
    return ThetaState(tau0, tau1, tau2, q2, r2)


@dataclass
class Chain:
    theta: list = field(default_factory=list)     # ThetaState per sweep
    updated: np.ndarray = None                    # [K] count of sweeps where x*_t moved
    x: list = field(default_factory=list)         # x* per sweep
    sweeps: int = 0
    device_s: float = 0.0
    wall_s: float = 0.0


class ThetaLogisticGibbs:
    """Particle Gibbs on the theta-logistic model with N particles per time step."""

    def __init__(self, y: np.ndarray, N: int, theta0: ThetaState, prior: ThetaPrior = ThetaPrior(), seed: int = 1,
                 pit_proposals: bool = True, pit_first_passes: int = 25, compute: int = dsmc.FP32,
                 update_theta: bool = True):
        self.y = np.asarray(y, np.float64).reshape(-1)
        self.K = self.y.shape[0]
        self.N = int(N)
        self.prior = prior
        self.rng = np.random.default_rng(seed)
        self.theta = theta0
        self.pit = pit_proposals
        self.pit_first = pit_first_passes
        self.compute = compute
        self.seed = seed
        self.yd = torch.as_tensor(self.y[:, None], dtype=torch.float32, device="cuda")
        self.x_ref = self.yd.clone()             # the first reference: the observations
        self.x_next = torch.empty_like(self.x_ref)
        self.pit_mean = None
        self.pit_ws = None
        self.sm = None
        self.update_theta = update_theta   # False: x-steps only, a chain on p(x | y, theta0)

    def _proposals(self, m: W.SSM):
        """Algorithm 4's Gaussian marginals for the current parameters (device tensors), or None
        for the model's own observation-centred proposal."""
        if not self.pit:
            return None, None
        passes = self.pit_first if self.pit_mean is None else 1
        mean, std, self.pit_ws = dsmc.dsmc_gaussian_proposals(dsmc.HostModel(m), self.yd, iterations=passes,
                                                              init_mean=self.pit_mean, ws=self.pit_ws)
        self.pit_mean = mean
        return mean, std

    def run(self, sweeps: int, counter_base0: int = 0) -> Chain:
        ch = Chain(updated=np.zeros(self.K))
        prev = self.x_ref.cpu().numpy()[:, 0].copy()
        t0 = time.perf_counter()
        for s in range(sweeps):
            m = self.theta.model()
            pm, ps = self._proposals(m)
            if self.sm is None:  # device buffers once; the parameters and proposals change every sweep
                self.sm = dsmc.Smoother(m, self.K, self.N, seed=self.seed, compute=self.compute)
            self.sm.set_model(m, pm, ps)
            sm = self.sm
            sm.set_seed(self.seed, counter_base=(counter_base0 + s) % (1 << 28))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sm.conditional(self.yd, self.x_ref, self.x_next)
            e1.record()
            x = self.x_next.cpu().numpy()[:, 0].astype(np.float64)
            ch.device_s += e0.elapsed_time(e1) / 1e3
            if sm.status() != 0:
                raise RuntimeError(f"device status {sm.status()} in sweep {s}")
            ch.updated += (x != prev)
            prev = x
            self.x_ref, self.x_next = self.x_next, self.x_ref
            if self.update_theta:
                self.theta = update_parameters(self.rng, self.prior, self.theta, x, self.y)
            ch.theta.append(self.theta)
            ch.x.append(x)
        ch.sweeps = sweeps
        ch.wall_s = time.perf_counter() - t0
        return ch
