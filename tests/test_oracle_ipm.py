"""Pins of the oracle's minimal filter IPM: a box-constrained QP with a
closed-form optimum, the optimum of a tiny column instance against scipy's
trust-constr (an independent algorithm), equal iterates for the exact dense
solver and HyKKT, and the relaxed (Lifted-KKT) problem's O(tau) gap."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from gen.tray import TrayParams, ipm_start
from oracle import ipm, symbolic, tray


class SimplexQP:
    """min 1/2 ||x - a||^2  s.t.  sum(x) = b,  0 <= x <= 1."""

    def __init__(self, a, b):
        self.a, self.b = np.asarray(a, float), float(b)
        self.n, self.m = len(a), 1
        self.x_lo, self.x_hi = np.zeros(self.n), np.ones(self.n)

    def f(self, x):
        return 0.5 * float(np.sum((x - self.a) ** 2))

    def grad(self, x):
        return x - self.a

    def cons(self, x):
        return np.array([np.sum(x) - self.b])

    def jac_csr(self, x):
        return (np.array([0, self.n]), np.arange(self.n), np.ones(self.n))

    def hess_lower_csc(self, x, y):
        return (np.arange(self.n + 1), np.arange(self.n), np.ones(self.n))

    def closed_form(self):
        # x_i = clip(a_i - lam, 0, 1) with sum(x) = b: bisection on lam
        lo, hi = np.min(self.a) - 2, np.max(self.a) + 2
        for _ in range(200):
            lam = 0.5 * (lo + hi)
            if np.sum(np.clip(self.a - lam, 0, 1)) > self.b:
                lo = lam
            else:
                hi = lam
        return np.clip(self.a - lam, 0, 1)


# Fiacco-McCormick barrier sequence of the cited filter method with mu_0 = 0.1,
# kappa_mu = 0.2, theta_mu = 1.5: 0.1, then min(0.2 mu, mu^1.5) at every
# update, never below tol/10 (tol = 1e-10): 0.1, 0.02, 0.02^1.5, ...
MU_SEQUENCE = [0.1, 0.02, 2.828427124746191e-03, 1.5042412372345582e-04,
               1.8449144625279508e-06, 2.5059035596800618e-09, 1e-11]


def test_barrier_parameter_follows_the_published_sequence():
    a = np.random.default_rng(5).uniform(-0.5, 1.5, 12)
    qp = SimplexQP(a, 4.0)
    lin = ipm.KKTLinearSolver("dense", qp.n, qp.m, None, None)
    s = ipm.IPM(qp, lin, ipm.IPMOptions(tol=1e-10), np.full(qp.n, 0.5))
    assert s.solve().status == "converged"
    used = [h.mu for h in s.history]
    seen = []
    for u in used:
        assert any(u == pytest.approx(v, rel=1e-12) for v in MU_SEQUENCE), u
        if not seen or u != seen[-1]:
            seen.append(u)
    # monotone and without skipping a value of the sequence
    idx = [next(i for i, v in enumerate(MU_SEQUENCE) if u == pytest.approx(v, rel=1e-12))
           for u in seen]
    assert idx == list(range(idx[0], idx[0] + len(idx)))
    assert len(seen) >= 4


def test_backtracking_halves_the_fraction_to_boundary_step():
    """Every accepted step is the largest fraction-to-boundary step halved
    once per rejected trial."""
    s, last = _tray_ipm(TrayParams(k=4, T=3), "lifted", relaxed=True)
    assert last.status == "converged"
    steps = [h for h in s.history if h.status == "ok"]
    assert any(h.ls > 1 for h in steps)
    for h in steps:
        assert h.alpha_pr == h.extra["alpha_max"] * 0.5 ** (h.ls - 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qp_closed_form(seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-0.5, 1.5, 12)
    qp = SimplexQP(a, 4.0)
    lin = ipm.KKTLinearSolver("dense", qp.n, qp.m, None, None)
    s = ipm.IPM(qp, lin, ipm.IPMOptions(tol=1e-10), np.full(qp.n, 0.5))
    last = s.solve()
    assert last.status == "converged"
    assert np.max(np.abs(s.x - qp.closed_form())) < 1e-8


def test_qp_relaxed_gap_is_order_tau():
    rng = np.random.default_rng(5)
    qp = SimplexQP(rng.uniform(-0.5, 1.5, 10), 3.0)
    lin = ipm.KKTLinearSolver("dense", qp.n, qp.m, None, None)
    s = ipm.IPM(qp, lin, ipm.IPMOptions(tol=1e-10, relaxed=True, tau_relax=1e-6),
                np.full(qp.n, 0.5))
    assert s.solve().status == "converged"
    assert abs(np.sum(s.x) - 3.0) <= 1e-6 * (1 + 1e-9)
    assert np.max(np.abs(s.x - qp.closed_form())) < 1e-5


def _tray_ipm(p, kind, relaxed=False, tol=1e-8):
    mdl = ipm.TrayModel(p)
    x0 = ipm_start(p)
    W = tray.hessian_lower_csc(p, x0, np.zeros(p.m))
    J = tray.jacobian_csr(p, x0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], leaf_size=16, relax_cols=16,
                           relax_zeros=64, max_width=16)
    lin = ipm.KKTLinearSolver(kind, p.n, p.m, None, None, sym=sym, gamma=1e4)
    s = ipm.IPM(mdl, lin, ipm.IPMOptions(tol=tol, relaxed=relaxed), x0)
    return s, s.solve()


def test_hykkt_cg_needs_few_iterations_at_large_gamma():
    """Sec. V-B: with gamma = 1e7 the unpreconditioned CG on S_gamma takes
    fewer than 10 iterations on average over the IPM's linear solves (the
    eigenvalues of gamma S_gamma cluster at 1)."""
    p = TrayParams(k=16, T=20)
    mdl = ipm.TrayModel(p)
    x0 = ipm_start(p)
    W = tray.hessian_lower_csc(p, x0, np.zeros(p.m))
    J = tray.jacobian_csr(p, x0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], leaf_size=16, relax_cols=16,
                           relax_zeros=64, max_width=16)
    lin = ipm.KKTLinearSolver("hykkt", p.n, p.m, None, None, sym=sym, gamma=1e7)
    s = ipm.IPM(mdl, lin, ipm.IPMOptions(tol=1e-8), x0)
    assert s.solve().status == "converged"
    per_solve = [i.cg_iters / (i.refine_iters + 1) for i in lin.stats]
    assert len(per_solve) >= 3 and np.mean(per_solve) < 10


def test_tray_optimum_matches_scipy():
    p = TrayParams(k=4, T=3)
    s, last = _tray_ipm(p, "hykkt", tol=1e-9)
    assert last.status == "converged"
    from gen.tray import bounds
    lo, hi = bounds(p)
    x0 = np.clip(ipm_start(p), lo + 1e-3, hi - 1e-3)
    res = so.minimize(lambda x: tray.objective(p, x), x0,
                      jac=lambda x: tray.objective_grad(p, x), method="trust-constr",
                      constraints=[so.NonlinearConstraint(
                          lambda x: tray.constraints(p, x), 0.0, 0.0,
                          jac=lambda x: sp.csr_matrix((tray.jacobian_csr(p, x)[2],
                                                       tray.jacobian_csr(p, x)[1],
                                                       tray.jacobian_csr(p, x)[0]),
                                                      shape=(p.m, p.n)))],
                      bounds=so.Bounds(lo, hi), options=dict(gtol=1e-12, xtol=1e-14,
                                                             maxiter=3000))
    assert np.max(np.abs(tray.constraints(p, res.x))) < 1e-8
    assert abs(res.fun - last.obj) <= 1e-7 * abs(last.obj)
    assert np.max(np.abs(res.x - s.x)) < 1e-5


def test_dense_and_hykkt_take_identical_steps():
    """Table II: HyKKT converges in the same number of iterations as an
    exact solve of the same KKT system."""
    p = TrayParams(k=6, T=4)
    s1, l1 = _tray_ipm(p, "dense")
    s2, l2 = _tray_ipm(p, "hykkt")
    assert l1.status == l2.status == "converged"
    assert l1.it == l2.it
    assert np.max(np.abs(s1.x - s2.x)) < 1e-9
    assert abs(l1.obj - l2.obj) <= 1e-12 * abs(l1.obj)


def test_lifted_solves_relaxed_problem():
    """Lifted-KKT solves the relaxed problem (Eq. problemrelaxation): its
    optimum is within O(tau) of the equality-constrained one."""
    p = TrayParams(k=6, T=4)
    s1, l1 = _tray_ipm(p, "hykkt")
    s2, l2 = _tray_ipm(p, "lifted", relaxed=True)
    assert l2.status == "converged"
    assert np.max(np.abs(tray.constraints(p, s2.x))) <= 1e-8 * (1 + 1e-6)
    assert abs(l1.obj - l2.obj) <= 1e-6 * abs(l1.obj)
    assert l2.it >= l1.it


def test_kkt_residual_at_convergence():
    p = TrayParams(k=4, T=5)
    s, last = _tray_ipm(p, "hykkt", tol=1e-8)
    assert last.status == "converged" and last.err0 <= 1e-8
    g = tray.objective_grad(p, s.x)
    r, c, v = tray.jacobian_coo(p, s.x)
    jty = np.zeros(p.n)
    np.add.at(jty, c, v * s.y[r])
    # stationarity with the bound multipliers (up to the scaled tolerance)
    assert np.max(np.abs(g + jty - s.zl + s.zu)) < 1e-6
