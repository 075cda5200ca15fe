"""Oracle O2/O5/O6: the KKT systems of Sec. III-IV and the two hybrid solvers.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sign convention (fixed for the whole project): a KKT solve returns the
solution of

    [ W + Sigma_x + delta_x I    J^T ] [dx]   [r_x]
    [ J                          -C  ] [dy] = [r_y]          (K_orig)

which is the condensed system Eq. (kkt:condensed) with the bound terms of the
variables folded into Sigma_x (the column model has no general inequality
h(x), only variable bounds) and with an optional dual block -C (C = 0 for the
equality-constrained system; C = D^{-1} for the relaxed problem of Lifted-KKT,
Eq. problemrelaxation).  Callers pass r = -F_mu.

* ``dense_solve``: the plain definition, the unique solution of K_orig v = b
  by the Bunch-Kaufman LDL^T of ``oracle.ldlt`` (up to 2,500 unknowns; above
  that LAPACK's LU solves the same definition, because the unblocked
  elimination would take minutes), followed by two steps of FP64
  refinement.
* ``inertia``: Sylvester's law on the blocks of D of the same LDL^T
  (Eq. inertia).
* ``lifted_solve``: Lifted-KKT (Sec. IV-A, Sec. V-B).  The preconditioner
  M = [[H, J^T], [J, -D^{-1}]] is applied by one Cholesky solve with the
  condensed matrix K_D = H + J^T D J (Eq. liftedkkt) and
  dy = D (J dx - r_y); Richardson iterations v <- v + M^{-1}(b - K_orig v)
  polish the step on K_orig (Sec. V-B).
* ``hykkt_solve``: HyKKT (Sec. IV-B).  K_gamma = H + gamma J^T J
  (Eq. hykkt) is factorised; CG on S_gamma = J K_gamma^{-1} J^T
  (Eq. schurcomp) gives dy, then dx = K_gamma^{-1}(r_gamma - J^T dy) with
  r_gamma = r_x + gamma J^T r_y.  The signs follow from the convention above
  (the printed right-hand side of the recovery step is garbled).

Refinement stops at eta <= tol, after max_refine sweeps, or when eta fails
to drop below 0.9 times its previous value twice in a row (stagnation; the
paper only names Richardson iterations, Sec. V-B).

Backward error (Rigal-Gaches, normwise):
    eta = ||b - K_orig v||_inf / (||K_orig||_inf ||v||_inf + ||b||_inf).

Parity: pinned (LAPACK cross-checks of both dense solve routes, Haynsworth inertia, equality of the
three solutions for every gamma, eigenvalues of gamma S_gamma -> 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from oracle import ldlt
from oracle.cholesky import SparseCholesky, NotPositiveDefinite


# -------------------------------------------------------------- matrices
def csc_lower_to_coo(n, colptr, rowind, val):
    cols = np.repeat(np.arange(n), np.diff(colptr))
    return np.asarray(rowind), cols, np.asarray(val)


def hessian_block(n, W, sigma, delta_x):
    """H = W + diag(Sigma_x) + delta_x I as a full symmetric scipy matrix."""
    r, c, v = csc_lower_to_coo(n, *W)
    off = r != c
    rows = np.concatenate([r, c[off], np.arange(n)])
    cols = np.concatenate([c, r[off], np.arange(n)])
    vals = np.concatenate([v, v[off], np.asarray(sigma) + delta_x])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def jacobian_matrix(n, m, J):
    rowptr, colind, val = J
    return sp.csr_matrix((np.asarray(val), np.asarray(colind),
                          np.asarray(rowptr)), shape=(m, n))


def kkt_matrix(n, m, W, J, sigma, delta_x, C=None):
    """K_orig as a scipy sparse matrix (both triangles)."""
    H = hessian_block(n, W, sigma, delta_x)
    Jm = jacobian_matrix(n, m, J)
    Cm = sp.diags(np.zeros(m) if C is None else -np.asarray(C))
    return sp.bmat([[H, Jm.T], [Jm, Cm]], format="csr")


def condensed_coo(n, W, J, sigma, delta_x, D):
    """Lower-triangle-agnostic COO triplets of K_D = H + J^T diag(D) J."""
    H = hessian_block(n, W, sigma, delta_x)
    Jm = sp.csr_matrix(jacobian_matrix(n, len(D), J))
    K = (H + Jm.T @ sp.diags(np.asarray(D)) @ Jm).tocoo()
    return K.row.astype(np.int64), K.col.astype(np.int64), K.data


def inf_norm(K):
    return float(np.max(np.asarray(abs(K).sum(axis=1)).ravel()))


def backward_error(K, v, b, knorm=None):
    r = b - K @ v
    kn = inf_norm(K) if knorm is None else knorm
    return float(np.max(np.abs(r)) / (kn * np.max(np.abs(v)) + np.max(np.abs(b))))


# --------------------------------------------------------------- dense O2
def dense_solve(K, b, refine_steps=2, ldlt_max=2500):
    """Plain definition of the KKT step: the solution of the dense K_orig by
    its Bunch-Kaufman LDL^T (LAPACK's LU above ``ldlt_max`` unknowns), then
    ``refine_steps`` Richardson steps in FP64."""
    Kd = K.toarray() if sp.issparse(K) else np.asarray(K, dtype=np.float64)
    if Kd.shape[0] <= ldlt_max:
        solve = ldlt.factor(Kd).solve
    else:
        lu = scipy.linalg.lu_factor(Kd)
        solve = lambda r: scipy.linalg.lu_solve(lu, r)
    v = solve(b)
    for _ in range(refine_steps):
        v = v + solve(b - Kd @ v)
    return v


def inertia(K):
    """(n_plus, n_zero, n_minus) of a symmetric matrix: Sylvester's law of
    inertia on the blocks of its Bunch-Kaufman LDL^T."""
    return ldlt.factor(K).inertia()


# ------------------------------------------------------------ hybrid O5/O6
@dataclass
class SolveInfo:
    refine_iters: int = 0
    cg_iters: int = 0
    bwd_err: float = np.inf
    status: str = "ok"
    etas: list = None


def _factor(sym, n, rows, cols, vals):
    return SparseCholesky(sym, n, rows, cols, vals)


def lifted_solve(sym, n, m, W, J, sigma, delta_x, D, rx, ry, C=None,
                 tol=1e-10, max_refine=20):
    """Lifted-KKT step with Richardson refinement on K_orig (target dual
    block -C; C = None means the equality system)."""
    D = np.asarray(D, dtype=np.float64)
    chol = _factor(sym, n, *condensed_coo(n, W, J, sigma, delta_x, D))
    Jm = jacobian_matrix(n, m, J)
    K = kkt_matrix(n, m, W, J, sigma, delta_x, C)
    knorm = inf_norm(K)
    b = np.concatenate([rx, ry])

    def precond(r):
        r1, r2 = r[:n], r[n:]
        dx = chol.solve(r1 + Jm.T @ (D * r2))
        dy = D * (Jm @ dx - r2)
        return np.concatenate([dx, dy])

    return _richardson(precond, K, knorm, b, tol, max_refine, n)


def _richardson(precond, K, knorm, b, tol, max_refine, n, info=None):
    info = info or SolveInfo()
    v = np.zeros_like(b)
    r = b.copy()
    etas = []
    slow = 0
    for it in range(max_refine + 1):
        v = v + precond(r)
        r = b - K @ v
        eta = float(np.max(np.abs(r)) / (knorm * np.max(np.abs(v)) + np.max(np.abs(b))))
        etas.append(eta)
        info.refine_iters = it
        if eta <= tol:
            break
        if len(etas) >= 2 and eta > 0.9 * etas[-2]:
            slow += 1
            if slow >= 2:
                info.status = "stall"
                break
        else:
            slow = 0
    else:
        info.status = "maxit"
    info.bwd_err = etas[-1]
    info.etas = etas
    return v[:n], v[n:], info


def conjugate_gradient(apply_S, rhs, tol=1e-10, max_iter=200):
    """Plain CG from x0 = 0, stopping at ||r||_2 <= tol ||rhs||_2."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    stop = tol * np.sqrt(float(rhs @ rhs))
    it = 0
    while np.sqrt(rr) > stop and it < max_iter:
        Sp = apply_S(p)
        alpha = rr / float(p @ Sp)
        x += alpha * p
        r -= alpha * Sp
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) <= stop


def hykkt_solve(sym, n, m, W, J, sigma, delta_x, gamma, rx, ry,
                tol_cg=1e-10, max_cg=200, tol=1e-10, max_refine=20):
    """HyKKT step (equality system, C = 0) with Richardson polish."""
    chol = _factor(sym, n, *condensed_coo(n, W, J, sigma, delta_x,
                                          np.full(m, float(gamma))))
    Jm = jacobian_matrix(n, m, J)
    K = kkt_matrix(n, m, W, J, sigma, delta_x, None)
    knorm = inf_norm(K)
    b = np.concatenate([rx, ry])
    info = SolveInfo()

    def inner(r):
        r1, r2 = r[:n], r[n:]
        r_gamma = r1 + gamma * (Jm.T @ r2)
        q = chol.solve(r_gamma)
        rhs = Jm @ q - r2
        dy, its, ok = conjugate_gradient(lambda p: Jm @ chol.solve(Jm.T @ p),
                                         rhs, tol_cg, max_cg)
        info.cg_iters += its
        if not ok:
            info.status = "cg_maxit"
        dx = chol.solve(r_gamma - Jm.T @ dy)
        return np.concatenate([dx, dy])

    return _richardson(inner, K, knorm, b, tol, max_refine, n, info)
