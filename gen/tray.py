"""Seeded synthetic inputs for the distillation-column (tray) workloads.

The column model is the one of Sec. VI-A of Pacaud & Shin (arXiv 2403.15913):
32 trays, relative volatility alpha = 1.6, distillate flow D = 0.2, feed flow
F = 0.4, reflux ratio bounded by 1 <= u <= 5.  The paper leaves the tray
holdups M_n, the feed composition x_f, the set-points and the initial profile
unstated; the values chosen here are documented constants (M_n = 1,
x_f = 0.5, xbar = 0.5, ubar = 2, xbar_{n,0} = 0.3).

Nothing in this module evaluates the model or its derivatives: it only fixes
constants, the variable/constraint index layout, and draws seeded random
iterates, multipliers, barrier diagonals and right-hand sides.  Both the CPU
oracle and the CUDA path consume these draws.

Variable layout (stage-major): stage t = 0..T owns the block
    [x_{1,t} .. x_{k,t}, y_{1,t} .. y_{k,t}, u_t]      (2k+1 entries)
so n = (2k+1)(T+1).
Constraint layout: stage t owns 2k rows; the first k are the initial condition
(t = 0) or the implicit-Euler dynamics (t >= 1), the next k the vapour-liquid
equilibrium; so m = 2k(T+1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class TrayParams:
    """Constants of one distillation-column instance (Sec. VI-A)."""
    k: int = 32            # number of trays
    T: int = 50            # number of implicit-Euler stages after t = 0
    h: float = 0.1         # time step
    alpha: float = 1.6     # relative volatility
    D: float = 0.2         # distillate flow rate
    F: float = 0.4         # feed flow rate
    xf: float = 0.5        # feed composition (not given in the paper)
    M: float = 1.0         # tray holdup M_n, same on every tray (not given)
    xbar: float = 0.5      # composition set-point (not given)
    ubar: float = 2.0      # reflux set-point (not given)
    rho: float = 1.0       # control weight (paper: rho = 1)
    x0bar: float = 0.3     # initial composition on every tray (not given)
    x_lo: float = 0.0
    x_hi: float = 1.0
    u_lo: float = 1.0
    u_hi: float = 5.0

    @property
    def feed(self) -> int:
        """Zero-based index of the feed tray (tray k/2 + 1 in 1-based terms)."""
        return self.k // 2

    @property
    def nstage(self) -> int:
        return 2 * self.k + 1

    @property
    def n(self) -> int:
        return (2 * self.k + 1) * (self.T + 1)

    @property
    def m(self) -> int:
        return 2 * self.k * (self.T + 1)

    def as_array(self) -> np.ndarray:
        """Packed float64 parameter vector, in the order the C-ABI expects."""
        return np.array([self.k, self.T, self.h, self.alpha, self.D, self.F,
                         self.xf, self.M, self.xbar, self.ubar, self.rho,
                         self.x0bar, self.x_lo, self.x_hi, self.u_lo,
                         self.u_hi], dtype=np.float64)


def x_index(p: TrayParams, t, i):
    return t * p.nstage + i


def y_index(p: TrayParams, t, i):
    return t * p.nstage + p.k + i


def u_index(p: TrayParams, t):
    return t * p.nstage + 2 * p.k


def bounds(p: TrayParams):
    """Lower/upper variable bounds: 0 <= x, y <= 1 and 1 <= u <= 5."""
    lo = np.empty(p.n)
    hi = np.empty(p.n)
    blk_lo = np.concatenate([np.full(2 * p.k, p.x_lo), [p.u_lo]])
    blk_hi = np.concatenate([np.full(2 * p.k, p.x_hi), [p.u_hi]])
    lo[:] = np.tile(blk_lo, p.T + 1)
    hi[:] = np.tile(blk_hi, p.T + 1)
    return lo, hi


@dataclass
class KKTPoint:
    """A seeded primal-dual point at which one KKT system is formed."""
    params: TrayParams
    w: np.ndarray          # primal variables, length n
    lam: np.ndarray        # equality multipliers, length m
    sigma: np.ndarray      # barrier diagonal Sigma_x, length n
    rx: np.ndarray         # N(0,1) right-hand side, primal rows (length n)
    ry: np.ndarray         # N(0,1) right-hand side, dual rows (length m)
    seed: int = 0
    extra: dict = field(default_factory=dict)


def kkt_point(p: TrayParams, seed: int = 0,
              sigma_range=(1e-6, 1e6)) -> KKTPoint:
    """Seeded KKT data: x, y ~ U(0.05, 0.95), u ~ U(1.05, 4.95),
    multipliers ~ N(0, 1), Sigma_x log-uniform on sigma_range, and an
    N(0, 1) right-hand side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.empty(p.n)
    states = rng.uniform(0.05, 0.95, size=(p.T + 1, 2 * p.k))
    ctrl = rng.uniform(1.05, 4.95, size=(p.T + 1,))
    w.reshape(p.T + 1, p.nstage)[:, :2 * p.k] = states
    w.reshape(p.T + 1, p.nstage)[:, 2 * p.k] = ctrl
    lam = rng.standard_normal(p.m)
    lo, hi = np.log10(sigma_range[0]), np.log10(sigma_range[1])
    sigma = 10.0 ** rng.uniform(lo, hi, size=p.n)
    rx = rng.standard_normal(p.n)
    ry = rng.standard_normal(p.m)
    return KKTPoint(p, w, lam, sigma, rx, ry, seed)


def ipm_start(p: TrayParams) -> np.ndarray:
    """Starting primal point of the IPM runs: every composition (x and y) at
    xbar_{n,0}, every control at ubar.  Multipliers start at zero."""
    w = np.empty(p.n)
    blk = np.concatenate([np.full(2 * p.k, p.x0bar), [p.ubar]])
    w[:] = np.tile(blk, p.T + 1)
    return w
