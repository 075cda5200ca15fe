"""Oracle O1: the distillation-column model of Sec. VI-A and its derivatives.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper writes the column as an index-1 DAE discretised in time:

* flows  L_t = u_t D,  V_t = L_t + D,  S_t = F + L_t
* vapour-liquid equilibrium  y = alpha x / (1 + (alpha - 1) x)
* tray balances M_n xdot_n = g_n(x_t, y_t, u_t):
    condenser (n = 1)        V (y_2 - x_1)
    rectifying (2..feed-1)   L (x_{n-1} - x_n) - V (y_n - y_{n+1})
    feed tray                F x_f + L x_{n-1} - S x_n - V (y_n - y_{n+1})
    stripping (feed+1..k-1)  S (x_{n-1} - x_n) - V (y_n - y_{n+1})
    reboiler (n = k)         S x_{k-1} - (F - D) x_k - V y_k
  (the reboiler line of the paper has unbalanced parentheses and a stray D_t;
  this reading is the one that conserves mass: the total inflow S equals the
  outflow (F - D) + V, checked by a test)
* implicit Euler  x_t - x_{t-1} - h g(x_t, y_t, u_t) / M = 0,  x_0 = xbar_0
* objective  sum_{t=0..T} ( ||x_t - xbar||^2 + rho (u_t - ubar)^2 )

Every function accepts complex arrays so that tests can differentiate it by
the complex step.  Parity: pinned (complex step, mass balance, closed forms of
the equilibrium curve).
"""
from __future__ import annotations

import numpy as np

from gen.tray import TrayParams


# ---------------------------------------------------------------- helpers
def split(p: TrayParams, w):
    """Views (x[t, i], y[t, i], u[t]) of the stage-major primal vector."""
    blk = w.reshape(p.T + 1, p.nstage)
    return blk[:, :p.k], blk[:, p.k:2 * p.k], blk[:, 2 * p.k]


def flows(p: TrayParams, u):
    """L_t, V_t, S_t of Sec. VI-A."""
    L = u * p.D
    V = L + p.D
    S = p.F + L
    return L, V, S


def vle(p: TrayParams, x):
    """Equilibrium vapour fraction y = alpha x / (1 + (alpha-1) x)."""
    return p.alpha * x / (1.0 + (p.alpha - 1.0) * x)


def vle_d1(p: TrayParams, x):
    return p.alpha / (1.0 + (p.alpha - 1.0) * x) ** 2


def vle_d2(p: TrayParams, x):
    return -2.0 * p.alpha * (p.alpha - 1.0) / (1.0 + (p.alpha - 1.0) * x) ** 3


def balance(p: TrayParams, x, y, u):
    """g_n = M_n xdot_n for every tray (columns) and stage (rows)."""
    L, V, S = flows(p, u)
    k, kf = p.k, p.feed
    g = np.zeros(x.shape, dtype=np.result_type(x, y, u))
    for n in range(k):
        if n == 0:
            g[:, n] = V * (y[:, 1] - x[:, 0])
        elif n < kf:
            g[:, n] = L * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n + 1])
        elif n == kf:
            g[:, n] = (p.F * p.xf + L * x[:, n - 1] - S * x[:, n]
                       - V * (y[:, n] - y[:, n + 1]))
        elif n < k - 1:
            g[:, n] = S * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n + 1])
        else:
            g[:, n] = S * x[:, n - 1] - (p.F - p.D) * x[:, n] - V * y[:, n]
    return g


def balance_partials(p: TrayParams, x, y, u, n):
    """First partials of g_n w.r.t. the variables of its own stage, as a list
    of (kind, tray, value-per-stage).  kind is 'x', 'y' or 'u'."""
    L, V, S = flows(p, u)
    k, kf = p.k, p.feed
    D = p.D
    out = []
    if n == 0:
        out.append(('x', 0, -V))
        out.append(('y', 1, V))
        out.append(('u', None, D * (y[:, 1] - x[:, 0])))
        return out
    if n == k - 1:
        out.append(('x', n - 1, S))
        out.append(('x', n, -(p.F - p.D) + 0.0 * u))
        out.append(('y', n, -V))
        out.append(('u', None, D * x[:, n - 1] - D * y[:, n]))
        return out
    liq_in = L if n <= kf else S          # coefficient of x_{n-1}
    liq_out = L if n < kf else S          # coefficient of -x_n
    out.append(('x', n - 1, liq_in))
    out.append(('x', n, -liq_out))
    out.append(('y', n, -V))
    out.append(('y', n + 1, V))
    out.append(('u', None, D * (x[:, n - 1] - x[:, n]) - D * (y[:, n] - y[:, n + 1])))
    return out


def balance_second(p: TrayParams, n):
    """Nonzero second partials of g_n: all are (u, v) cross terms with a
    constant value; returned as a list of (kind, tray, value)."""
    k, D = p.k, p.D
    if n == 0:
        return [('x', 0, -D), ('y', 1, D)]
    if n == k - 1:
        return [('x', n - 1, D), ('y', n, -D)]
    return [('x', n - 1, D), ('x', n, -D), ('y', n, -D), ('y', n + 1, D)]


def _col(p, kind, t, i):
    if kind == 'x':
        return t * p.nstage + i
    if kind == 'y':
        return t * p.nstage + p.k + i
    return t * p.nstage + 2 * p.k


def dyn_row(p, t, n):
    return t * 2 * p.k + n


def eq_row(p, t, n):
    return t * 2 * p.k + p.k + n


# ---------------------------------------------------------------- model
def objective(p: TrayParams, w):
    x, y, u = split(p, w)
    return np.sum((x - p.xbar) ** 2) + p.rho * np.sum((u - p.ubar) ** 2)


def objective_grad(p: TrayParams, w):
    x, y, u = split(p, w)
    g = np.zeros(p.n, dtype=w.dtype)
    gx, gy, gu = split(p, g)
    gx[:] = 2.0 * (x - p.xbar)
    gu[:] = 2.0 * p.rho * (u - p.ubar)
    return g


def constraints(p: TrayParams, w, x0=None):
    """c(w), length m: initial condition / dynamics rows then equilibrium
    rows, stage by stage.  The initial condition pins the stage-0
    compositions to x0 (one value per tray; default x0bar on every tray):
    in receding-horizon use x0 is the measured state of the column."""
    x, y, u = split(p, w)
    c = np.zeros(p.m, dtype=w.dtype)
    cb = c.reshape(p.T + 1, 2 * p.k)
    cb[0, :p.k] = x[0] - (p.x0bar if x0 is None else np.asarray(x0, dtype=float))
    g = balance(p, x[1:], y[1:], u[1:])
    cb[1:, :p.k] = x[1:] - x[:-1] - (p.h / p.M) * g
    cb[:, p.k:] = y - vle(p, x)
    return c


def jacobian_coo(p: TrayParams, w):
    """Jacobian of c as COO triplets (row, col, value); one entry per
    structural nonzero."""
    x, y, u = split(p, w)
    rows, cols, vals = [], [], []
    T, k = p.T, p.k
    ts = np.arange(T + 1)
    hm = p.h / p.M

    def add(r, c, v):
        rows.append(np.asarray(r))
        cols.append(np.asarray(c))
        vals.append(np.broadcast_to(np.asarray(v), np.shape(r)).astype(w.dtype))

    for n in range(k):                   # initial condition, stage 0
        add(np.array([dyn_row(p, 0, n)]), np.array([_col(p, 'x', 0, n)]), np.ones(1))
    t1 = ts[1:]
    for n in range(k):                   # dynamics, stages 1..T
        r = dyn_row(p, t1, n)
        add(r, _col(p, 'x', t1 - 1, n), -np.ones(T))
        diag_done = False
        for kind, i, v in balance_partials(p, x[1:], y[1:], u[1:], n):
            val = -hm * v
            if kind == 'x' and i == n:
                val = 1.0 + val
                diag_done = True
            add(r, _col(p, kind, t1, i), val)
        assert diag_done
    for n in range(k):                   # equilibrium, stages 0..T
        r = eq_row(p, ts, n)
        add(r, _col(p, 'x', ts, n), -vle_d1(p, x[:, n]))
        add(r, _col(p, 'y', ts, n), np.ones(T + 1))
    return (np.concatenate(rows).astype(np.int64),
            np.concatenate(cols).astype(np.int64), np.concatenate(vals))


def jacobian_csr(p: TrayParams, w):
    """CSR (rowptr, colind, val) of the Jacobian, columns ascending in every
    row."""
    r, c, v = jacobian_coo(p, w)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(p.m + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c, v


def hessian_lower_csc(p: TrayParams, w, lam, obj_weight=1.0):
    """Lower triangle of W = obj_weight * Hess f + sum_r lam_r Hess c_r as
    CSC (colptr, rowind, val), rows ascending in every column.

    The pattern is fixed: every diagonal entry, plus (u_t, x_{i,t}) and
    (u_t, y_{i,t}) for every tray i and stage t (some of these are
    structurally zero for the column model and are stored as explicit zeros).
    """
    x, y, u = split(p, w)
    T, k = p.T, p.k
    dt = np.result_type(w, lam)
    diag = np.zeros(p.n, dtype=dt)
    ux = np.zeros((T + 1, k), dtype=dt)      # W[u_t, x_{i,t}]
    uy = np.zeros((T + 1, k), dtype=dt)      # W[u_t, y_{i,t}]
    dx, dy, du = split(p, diag)
    dx += obj_weight * 2.0
    du += obj_weight * 2.0 * p.rho
    lamb = lam.reshape(T + 1, 2 * k)
    # equilibrium rows: Hess(y - vle(x)) = -vle''(x) on (x, x)
    dx -= lamb[:, k:] * vle_d2(p, x)
    # dynamics rows (t >= 1): Hess(x_t - x_{t-1} - h g / M) = -(h/M) Hess g
    hm = p.h / p.M
    for n in range(k):
        ln = lamb[1:, n]
        for kind, i, v in balance_second(p, n):
            if kind == 'x':
                ux[1:, i] += -hm * v * ln
            else:
                uy[1:, i] += -hm * v * ln
    # assemble CSC: per stage the columns x_0..x_{k-1}, y_0..y_{k-1}, u
    colptr = [0]
    rowind = []
    val = []
    for t in range(T + 1):
        ucol = _col(p, 'u', t, None)
        for i in range(k):
            c = _col(p, 'x', t, i)
            rowind += [c, ucol]
            val += [diag[c], ux[t, i]]
            colptr.append(colptr[-1] + 2)
        for i in range(k):
            c = _col(p, 'y', t, i)
            rowind += [c, ucol]
            val += [diag[c], uy[t, i]]
            colptr.append(colptr[-1] + 2)
        rowind.append(ucol)
        val.append(diag[ucol])
        colptr.append(colptr[-1] + 1)
    return (np.array(colptr, dtype=np.int64), np.array(rowind, dtype=np.int64),
            np.array(val, dtype=dt))


def lagrangian_grad(p: TrayParams, w, lam, obj_weight=1.0):
    """obj_weight * grad f + J^T lam (used by complex-step pins of W)."""
    r, c, v = jacobian_coo(p, w)
    g = obj_weight * objective_grad(p, w)
    jt = np.zeros(p.n, dtype=np.result_type(v, lam))
    np.add.at(jt, c, v * lam[r])
    return g + jt


def mass_balance_residual(p: TrayParams, x, y, u):
    """sum_n M_n xdot_n - (F x_f - D x_1 - (F - D) x_k); zero for every
    state when the tray balances conserve mass."""
    g = balance(p, x, y, u)
    return g.sum(axis=1) - (p.F * p.xf - p.D * x[:, 0] - (p.F - p.D) * x[:, -1])
