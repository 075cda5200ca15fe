"""Oracle O7: a minimal primal-dual filter line-search interior-point method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. III of the paper: the barrier problem is solved by Newton steps on
F_mu(w) = 0 (Eq. smoothkkt), each step a solution of the condensed KKT system
(Eq. kkt:condensed) with the bound terms folded into Sigma_x; the step length
comes from a fraction-to-boundary rule and the filter line search of Wachter &
Biegler (2006), which MadNLP implements.  The paper gives no parameter values;
the defaults below are that reference's published defaults.  This is the
basic form: monotone barrier update, no second-order correction, no
restoration phase (a failed line search stops the run with status "stall").

Problem:   min f(x)  s.t.  c(x) = 0,  x_L <= x <= x_U          (equality mode)
Lifted-KKT solves instead the relaxed problem of Eq. (problemrelaxation):
           min f(x)  s.t.  c(x) - s = 0,  -tau <= s <= tau       (relaxed mode)
whose condensed system is [[H, J^T], [J, -Sigma_s^{-1}]] (C = Sigma_s^{-1},
D = Sigma_s in the Lifted-KKT matrix H + J^T D J).

Iteration (one call of ``step``):
  1. evaluate f, grad f, c, J at x and W = Hess(f + y^T c) at (x, y);
  2. optimality error E_0 (scaled as in the reference); stop when E_0 <= tol;
  3. while E_mu <= kappa_eps mu: mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu)),
     reset the filter;
  4. Sigma_x = z_L/(x - x_L) + z_U/(x_U - x);  r_x = -(grad phi_mu + J^T y);
     relaxed: Sigma_s likewise on s, r_y = -(c - s) - Sigma_s^{-1}(grad_s phi - y);
     equality: r_y = -c;
  5. factor with the smallest delta_x of the inertia-correction ladder that
     gives a positive definite condensed matrix; solve for (dx, dy);
  6. recover ds = Sigma_s^{-1}(dy - grad_s phi + y) and the bound-multiplier
     steps dz = mu/gap - z -/+ Sigma dx;
  7. fraction to boundary with tau_ftb = max(0.99, 1 - mu) for the primal
     (x, s) and dual (z, v) steps;
  8. backtracking filter line search on (theta, phi) with theta = ||c - s||_1,
     phi = f - mu sum log(gaps); switching condition + Armijo for f-type steps;
  9. update; bound multipliers are kept within [mu/(kappa_Sigma gap),
     kappa_Sigma mu/gap].

Parity: pinned by tests (closed-form box-constrained QP; the optimum of a tiny
column instance against scipy's trust-constr; equal iteration counts and
iterates for the exact dense solver and HyKKT; the barrier parameters drawn,
in order, from the published Fiacco-McCormick sequence; accepted steps equal
to the fraction-to-boundary step halved once per rejected trial) and by
worked single steps with a prescribed direction, whose outcomes were worked
out by hand from the cited method's definitions: Armijo acceptance of f-type
steps, filter and theta_max rejection, the switching condition and the
theta_min test, filter augmentation by h-type steps only and its reset at
each barrier decrease, the l1 constraint violation, the barrier-update
threshold kappa_eps, the scaling s_d / s_c of the optimality error, tau =
max(tau_min, 1 - mu), the dual step length from both bound multipliers, the
primal step length for y, and the kappa_Sigma multiplier safeguard.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from oracle import kkt as okkt
from oracle.cholesky import NotPositiveDefinite


@dataclass
class IPMOptions:
    tol: float = 1e-8
    max_iter: int = 200
    mu_init: float = 0.1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    s_max: float = 100.0
    bound_push: float = 1e-2       # kappa_1
    bound_frac: float = 1e-2       # kappa_2
    kappa_sigma: float = 1e10
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-8
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-8
    max_ls: int = 40
    # inertia correction
    delta_w0: float = 1e-4
    delta_min: float = 1e-20
    delta_max: float = 1e40
    kappa_w_minus: float = 1.0 / 3.0
    kappa_w_plus: float = 8.0
    kappa_w_plus_bar: float = 100.0
    # relaxation of Lifted-KKT
    relaxed: bool = False
    tau_relax: float = 1e-8


@dataclass
class IterInfo:
    it: int
    mu: float
    inf_pr: float
    inf_du: float
    compl: float
    err0: float
    obj: float
    alpha_pr: float = 0.0
    alpha_du: float = 0.0
    delta_x: float = 0.0
    ls: int = 0
    status: str = "ok"
    extra: dict = field(default_factory=dict)


def _push(x, lo, hi, k1, k2):
    """Move x strictly inside [lo, hi] (Wachter-Biegler Sec. 3.6)."""
    pl = np.minimum(k1 * np.maximum(1.0, np.abs(lo)), k2 * (hi - lo))
    pu = np.minimum(k1 * np.maximum(1.0, np.abs(hi)), k2 * (hi - lo))
    return np.minimum(np.maximum(x, lo + pl), hi - pu)


def _max_step(v, dv, lo, hi, tau):
    """Largest alpha in (0, 1] with lo + (1-tau)(v-lo) <= v + alpha dv <=
    hi - (1-tau)(hi-v)."""
    a = 1.0
    neg = dv < 0
    if np.any(neg):
        a = min(a, float(np.min(-tau * (v[neg] - lo[neg]) / dv[neg])))
    pos = dv > 0
    if np.any(pos):
        a = min(a, float(np.min(tau * (hi[pos] - v[pos]) / dv[pos])))
    return a


def _max_step_pos(z, dz, tau):
    neg = dz < 0
    if not np.any(neg):
        return 1.0
    return min(1.0, float(np.min(-tau * z[neg] / dz[neg])))


class KKTLinearSolver:
    """Linear solves of the IPM: the exact dense solve, Lifted-KKT or HyKKT
    from ``oracle.kkt`` (sparse symbolic analysis done once)."""

    def __init__(self, kind, n, m, Wpat, Jpat, sym=None, gamma=1e4, tol_refine=1e-10,
                 max_refine=20):
        self.kind, self.n, self.m = kind, n, m
        self.sym = sym
        self.gamma = gamma
        self.tol_refine, self.max_refine = tol_refine, max_refine
        self.stats = []

    def solve(self, W, J, sigma, delta_x, rx, ry, C=None):
        """Returns (dx, dy); raises NotPositiveDefinite when the condensed
        matrix is not positive definite (or K_orig has the wrong inertia
        for the dense solver)."""
        n, m = self.n, self.m
        if self.kind == "dense":
            K = okkt.kkt_matrix(n, m, W, J, sigma, delta_x, C)
            Hd = okkt.hessian_block(n, W, sigma, delta_x).toarray()
            Jd = okkt.jacobian_matrix(n, m, J).toarray()
            Cd = np.zeros(m) if C is None else np.asarray(C)
            # positive definiteness of H + J^T C^{-1} J (relaxed) or of the
            # reduced Hessian (equality) by dense Cholesky of H + g J^T J
            Kg = Hd + (Jd.T * (1.0 / Cd if C is not None else 1e8)) @ Jd
            try:
                np.linalg.cholesky(Kg)
            except np.linalg.LinAlgError:
                raise NotPositiveDefinite(-1)
            v = okkt.dense_solve(K, np.concatenate([rx, ry]))
            return v[:n], v[n:]
        if self.kind == "lifted":
            D = 1.0 / np.asarray(C) if C is not None else np.full(m, 1e8)
            dx, dy, info = okkt.lifted_solve(self.sym, n, m, W, J, sigma, delta_x, D, rx, ry,
                                             C=C, tol=self.tol_refine, max_refine=self.max_refine)
        else:
            dx, dy, info = okkt.hykkt_solve(self.sym, n, m, W, J, sigma, delta_x, self.gamma,
                                            rx, ry, tol=self.tol_refine,
                                            max_refine=self.max_refine)
        self.stats.append(info)
        return dx, dy


class IPM:
    """Minimal filter line-search IPM over a model with the methods
    ``f, grad, cons, jac_csr, hess_lower_csc`` and attributes
    ``n, m, x_lo, x_hi``."""

    def __init__(self, model, linsolver, opt: IPMOptions, x0):
        self.mdl, self.ls, self.o = model, linsolver, opt
        o = opt
        n, m = model.n, model.m
        self.x = _push(np.asarray(x0, dtype=float), model.x_lo, model.x_hi, o.bound_push,
                       o.bound_frac)
        self.y = np.zeros(m)
        self.zl = np.ones(n)
        self.zu = np.ones(n)
        if o.relaxed:
            self.s_lo = np.full(m, -o.tau_relax)
            self.s_hi = np.full(m, o.tau_relax)
            self.s = _push(model.cons(self.x), self.s_lo, self.s_hi, o.bound_push, o.bound_frac)
            self.vl = np.ones(m)
            self.vu = np.ones(m)
        self.mu = o.mu_init
        self.filter = []
        self.delta_last = 0.0
        self.it = 0
        th0 = self._theta(self.x, self.s if o.relaxed else None)
        self.theta_max = 1e4 * max(1.0, th0)
        self.theta_min = 1e-4 * max(1.0, th0)
        self.done = False
        self.history = []

    # ------------------------------------------------------------ measures
    def _theta(self, x, s):
        c = self.mdl.cons(x)
        if s is not None:
            c = c - s
        return float(np.sum(np.abs(c)))

    def _phi(self, x, s, mu):
        m = self.mdl
        v = m.f(x) - mu * np.sum(np.log(x - m.x_lo)) - mu * np.sum(np.log(m.x_hi - x))
        if s is not None:
            v -= mu * (np.sum(np.log(s - self.s_lo)) + np.sum(np.log(self.s_hi - s)))
        return float(v)

    def _errors(self, g, c, Jm, mu):
        o, m = self.o, self.mdl
        x = self.x
        du = g + Jm.T @ self.y - self.zl + self.zu
        cl = self.zl * (x - m.x_lo) - mu
        cu = self.zu * (m.x_hi - x) - mu
        pr = c.copy()
        dual_parts = [np.abs(du)]
        comp_parts = [np.abs(cl), np.abs(cu)]
        sum_mult = np.sum(np.abs(self.y)) + np.sum(self.zl) + np.sum(self.zu)
        sum_z = np.sum(self.zl) + np.sum(self.zu)
        cnt_mult = m.m + 2 * m.n
        cnt_z = 2 * m.n
        if o.relaxed:
            pr = pr - self.s
            dual_parts.append(np.abs(-self.y - self.vl + self.vu))
            comp_parts.append(np.abs(self.vl * (self.s - self.s_lo) - mu))
            comp_parts.append(np.abs(self.vu * (self.s_hi - self.s) - mu))
            sum_mult += np.sum(self.vl) + np.sum(self.vu)
            sum_z += np.sum(self.vl) + np.sum(self.vu)
            cnt_mult += 2 * m.m
            cnt_z += 2 * m.m
        s_d = max(o.s_max, sum_mult / cnt_mult) / o.s_max
        s_c = max(o.s_max, sum_z / cnt_z) / o.s_max
        inf_du = max(float(np.max(p)) for p in dual_parts)
        inf_pr = float(np.max(np.abs(pr)))
        compl = max(float(np.max(p)) for p in comp_parts)
        return max(inf_du / s_d, inf_pr, compl / s_c), inf_pr, inf_du, compl

    # ------------------------------------------------------------ one step
    def step(self):
        o, mdl = self.o, self.mdl
        n, m = mdl.n, mdl.m
        x = self.x
        f = mdl.f(x)
        g = mdl.grad(x)
        c = mdl.cons(x)
        J = mdl.jac_csr(x)
        W = mdl.hess_lower_csc(x, self.y)
        Jm = okkt.jacobian_matrix(n, m, J)
        err0, inf_pr, inf_du, compl = self._errors(g, c, Jm, 0.0)
        info = IterInfo(self.it, self.mu, inf_pr, inf_du, compl, err0, f)
        if err0 <= o.tol:
            self.done = True
            info.status = "converged"
            self.history.append(info)
            return info
        while self.mu > o.tol / 10:
            errmu = self._errors(g, c, Jm, self.mu)[0]
            if errmu > o.kappa_eps * self.mu:
                break
            self.mu = max(o.tol / 10, min(o.kappa_mu * self.mu, self.mu ** o.theta_mu))
            self.filter = []
        mu = self.mu
        gl, gu = x - mdl.x_lo, mdl.x_hi - x
        sigma = self.zl / gl + self.zu / gu
        gphi = g - mu / gl + mu / gu
        rx = -(gphi + Jm.T @ self.y)
        C = None
        if o.relaxed:
            s = self.s
            hl, hu = s - self.s_lo, self.s_hi - s
            sig_s = self.vl / hl + self.vu / hu
            gphi_s = -mu / hl + mu / hu
            ry = -(c - s) - (gphi_s - self.y) / sig_s
            C = 1.0 / sig_s
        else:
            ry = -c
        # inertia correction ladder
        dx = dy = None
        delta = 0.0
        while True:
            try:
                dx, dy = self.ls.solve(W, J, sigma, delta, rx, ry, C)
                break
            except NotPositiveDefinite:
                if delta == 0.0:
                    delta = o.delta_w0 if self.delta_last == 0.0 else max(
                        o.delta_min, o.kappa_w_minus * self.delta_last)
                else:
                    delta *= o.kappa_w_plus_bar if self.delta_last == 0.0 else o.kappa_w_plus
                if delta > o.delta_max:
                    info.status = "inertia"
                    self.done = True
                    self.history.append(info)
                    return info
        if delta > 0:
            self.delta_last = delta
        info.delta_x = delta
        dzl = mu / gl - self.zl - (self.zl / gl) * dx
        dzu = mu / gu - self.zu + (self.zu / gu) * dx
        tau = max(o.tau_min, 1.0 - mu)
        a_pr = _max_step(x, dx, mdl.x_lo, mdl.x_hi, tau)
        a_du = min(_max_step_pos(self.zl, dzl, tau), _max_step_pos(self.zu, dzu, tau))
        ds = None
        if o.relaxed:
            ds = (dy - gphi_s + self.y) / sig_s
            dvl = mu / hl - self.vl - (self.vl / hl) * ds
            dvu = mu / hu - self.vu + (self.vu / hu) * ds
            a_pr = min(a_pr, _max_step(s, ds, self.s_lo, self.s_hi, tau))
            a_du = min(a_du, _max_step_pos(self.vl, dvl, tau), _max_step_pos(self.vu, dvu, tau))
        # filter line search
        s0 = self.s if o.relaxed else None
        th = self._theta(x, s0)
        ph = self._phi(x, s0, mu)
        dphi = float(gphi @ dx)
        if o.relaxed:
            dphi += float(gphi_s @ ds)
        alpha = a_pr
        info.extra["alpha_max"] = a_pr
        accepted = False
        ls = 0
        for ls in range(1, o.max_ls + 1):
            xt = x + alpha * dx
            st = (s0 + alpha * ds) if o.relaxed else None
            tht = self._theta(xt, st)
            pht = self._phi(xt, st, mu)
            ok = tht <= self.theta_max and all(tht < tf or pht < pf for tf, pf in self.filter)
            f_type = False
            if ok:
                switching = dphi < 0 and alpha * (-dphi) ** o.s_phi > o.delta * th ** o.s_theta
                if th <= self.theta_min and switching:
                    ok = pht <= ph + o.eta_phi * alpha * dphi
                    f_type = True
                else:
                    ok = tht <= (1 - o.gamma_theta) * th or pht <= ph - o.gamma_phi * th
            if ok:
                if not f_type:
                    self.filter.append(((1 - o.gamma_theta) * th, ph - o.gamma_phi * th))
                accepted = True
                break
            alpha *= 0.5
        info.ls = ls
        if not accepted:
            info.status = "stall"
            self.done = True
            self.history.append(info)
            return info
        info.alpha_pr, info.alpha_du = alpha, a_du
        self.x = x + alpha * dx
        self.y = self.y + alpha * dy
        self.zl = self.zl + a_du * dzl
        self.zu = self.zu + a_du * dzu
        k = o.kappa_sigma
        gl, gu = self.x - mdl.x_lo, mdl.x_hi - self.x
        self.zl = np.maximum(np.minimum(self.zl, k * mu / gl), mu / (k * gl))
        self.zu = np.maximum(np.minimum(self.zu, k * mu / gu), mu / (k * gu))
        if o.relaxed:
            self.s = s0 + alpha * ds
            self.vl = self.vl + a_du * dvl
            self.vu = self.vu + a_du * dvu
            hl, hu = self.s - self.s_lo, self.s_hi - self.s
            self.vl = np.maximum(np.minimum(self.vl, k * mu / hl), mu / (k * hl))
            self.vu = np.maximum(np.minimum(self.vu, k * mu / hu), mu / (k * hu))
        self.it += 1
        self.history.append(info)
        return info

    def solve(self):
        while not self.done and self.it < self.o.max_iter:
            self.step()
        return self.history[-1]


class TrayModel:
    """The column model of ``oracle.tray`` behind the IPM interface."""

    def __init__(self, p, x0=None):
        from gen.tray import bounds
        from oracle import tray
        self.p, self.t = p, tray
        self.x0 = None if x0 is None else np.asarray(x0, dtype=float)   # per-tray initial state
        self.n, self.m = p.n, p.m
        self.x_lo, self.x_hi = bounds(p)

    def f(self, x):
        return float(self.t.objective(self.p, x))

    def grad(self, x):
        return self.t.objective_grad(self.p, x)

    def cons(self, x):
        return self.t.constraints(self.p, x, self.x0)

    def jac_csr(self, x):
        return self.t.jacobian_csr(self.p, x)

    def hess_lower_csc(self, x, y):
        return self.t.hessian_lower_csc(self.p, x, y, 1.0)
