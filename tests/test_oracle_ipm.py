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


# ---------------------------------------------------------------------------
# Worked single steps of the filter line search (Wachter & Biegler 2006,
# Sec. 2.3-2.5 and 3.9: the method the paper's IPM follows, Sec. III).  Each
# case fixes the iterate and the Newton direction (a prescribed linear
# solver), takes ONE step and compares the outcome with values worked out by
# hand from the method's definitions; the comments give the arithmetic.

class LineModel:
    """min x_1^2  s.t.  x_{j+1} - b_j = 0 (j < m),  lo <= x <= hi.

    The constraints are linear and each fixes one trailing variable, so
    theta = ||c||_1 can be set freely through the iterate."""

    def __init__(self, n, b, lo, hi):
        self.n, self.m = n, len(b)
        self.b = np.asarray(b, float)
        self.x_lo = np.broadcast_to(np.asarray(lo, float), (n,)).copy()
        self.x_hi = np.broadcast_to(np.asarray(hi, float), (n,)).copy()

    def f(self, x):
        return float(x[0] ** 2)

    def grad(self, x):
        g = np.zeros(self.n)
        g[0] = 2.0 * x[0]
        return g

    def cons(self, x):
        return x[1:1 + self.m] - self.b

    def jac_csr(self, x):
        return (np.arange(self.m + 1), np.arange(1, self.m + 1), np.ones(self.m))

    def hess_lower_csc(self, x, y):
        v = np.zeros(self.n)
        v[0] = 2.0
        return (np.arange(self.n + 1), np.arange(self.n), v)


class PrescribedStep:
    """Linear solver stand-in: returns a fixed (dx, dy)."""

    def __init__(self, dx, dy):
        self.dx, self.dy = np.asarray(dx, float), np.asarray(dy, float)

    def solve(self, W, J, sigma, delta_x, rx, ry, C=None):
        return self.dx.copy(), self.dy.copy()


def _one_step_ipm(mdl, x0, dx, dy, mu, **opts):
    s = ipm.IPM(mdl, PrescribedStep(dx, dy), ipm.IPMOptions(**opts), np.asarray(x0, float))
    assert np.array_equal(s.x, x0)           # x0 lies inside the bound push
    s.mu = mu
    return s


def test_f_type_step_is_accepted_by_the_armijo_condition():
    """theta = 0 <= theta_min and dphi < 0: the switching condition holds, so
    the trial must give sufficient decrease of phi (Armijo).  x = (1, 1),
    bounds [-10, 10], mu = 1e-3, dx = (-1.9, 0):
      phi(x) = 1 - mu (2 ln 11 + 2 ln 9) = 0.990810;
      dphi = -1.9 (2 - mu/11 + mu/9) = -3.800038;
      alpha = 1:   phi = 0.81 - mu (ln 9.1 + ln 11 + ln 10.9 + ln 9) = 0.800808;
      alpha = 1/2: phi = 0.0025 - mu (ln 10.05 + ln 11 + ln 9.95 + ln 9) = -0.006700.
    With the published eta_phi = 1e-8 the full step passes (0.8008 <= 0.99081);
    with eta_phi = 1/2 it must fail (0.8008 > phi + dphi/2 = -0.9092) and the
    halved step pass (-0.0067 <= phi + dphi/4 = 0.0408).  An f-type step
    leaves the filter unchanged."""
    mdl = LineModel(2, [1.0], -10.0, 10.0)
    for eta_phi, ls, alpha, x1 in ((1e-8, 1, 1.0, -0.9), (0.5, 2, 0.5, 0.05)):
        s = _one_step_ipm(mdl, [1.0, 1.0], [-1.9, 0.0], [0.0], 1e-3, eta_phi=eta_phi)
        h = s.step()
        assert h.status == "ok" and s.mu == 1e-3
        assert (h.ls, h.alpha_pr) == (ls, alpha)
        assert s.x[0] == pytest.approx(x1, rel=1e-14)
        assert s.filter == []


def test_h_type_step_augments_the_filter_with_the_l1_violation():
    """theta = ||c||_1: c = (3, -4) gives theta = 7 (not the 2-norm 5).
    theta > theta_min = 7e-4, so the step is h-type: accepted when
    theta_trial <= (1 - gamma_theta) theta, and the filter gains
    ((1 - 1e-5) 7, phi - 1e-8 * 7) = (6.99993, 0.986409645) with
    phi = 1 - mu (ln 11 + ln 14 + ln 8 + ln 9 + ln 6 + ln 12) = 0.986409715
    at x = (1, 4, -2), bounds [-10, 10], mu = 1e-3."""
    mdl = LineModel(3, [1.0, 2.0], -10.0, 10.0)
    s = _one_step_ipm(mdl, [1.0, 4.0, -2.0], [0.0, -3.0, 4.0], [0.0, 0.0], 1e-3)
    h = s.step()
    assert (h.status, h.ls, h.alpha_pr) == ("ok", 1, 1.0)
    assert np.array_equal(s.x, [1.0, 1.0, 2.0])
    assert len(s.filter) == 1
    assert s.filter[0][0] == pytest.approx(6.99993, rel=1e-15)
    assert s.filter[0][1] == pytest.approx(0.9864096451595542, rel=1e-14)


def test_filter_and_theta_max_reject_trial_points():
    """x = (1, 4), c = 3, dx = (0, -5): the full step gives theta = 2 (x_2 =
    -1), the halved one 0.5.  Without a filter the full step is accepted
    (2 <= 2.99997).  A trial is acceptable to the filter only if it beats
    EVERY entry in theta or in phi: with entries (1, -1e9) and (10, 1e9) the
    full step fails the first one and the halved step (0.5 < 1, 0.5 < 10)
    passes both.  theta_max = 1.5 rejects the full step on its own."""
    mdl = LineModel(2, [1.0], -10.0, 10.0)
    s = _one_step_ipm(mdl, [1.0, 4.0], [0.0, -5.0], [0.0], 1e-3)
    h = s.step()
    assert (h.ls, h.alpha_pr) == (1, 1.0) and len(s.filter) == 1
    assert s.filter[0][0] == pytest.approx(2.99997, rel=1e-15)

    s = _one_step_ipm(mdl, [1.0, 4.0], [0.0, -5.0], [0.0], 1e-3)
    s.filter = [(1.0, -1e9), (10.0, 1e9)]
    h = s.step()
    assert (h.ls, h.alpha_pr) == (2, 0.5)
    assert len(s.filter) == 3 and s.x[1] == 1.5

    s = _one_step_ipm(mdl, [1.0, 4.0], [0.0, -5.0], [0.0], 1e-3)
    s.theta_max = 1.5
    h = s.step()
    assert (h.ls, h.alpha_pr) == (2, 0.5)


def test_switching_condition_decides_between_f_and_h_type():
    """theta = 1e-5 <= theta_min = 1e-4 at x = (1, 1 + 1e-5).  The switching
    condition alpha (-dphi)^s_phi > delta theta^s_theta (s_phi = 2.3,
    s_theta = 1.1, delta = 1) compares with 1e-5^1.1 = 3.2e-6:
      dx = (-1e-5, -1e-5): dphi ~ -2e-5, (2e-5)^2.3 = 1.6e-11: fails -> h-type,
        the accepted step (theta 0 <= 0.99999e-5) augments the filter;
      dx = (-1.9, -1e-5): dphi ~ -3.8, 3.8^2.3 = 21.6: holds -> f-type, accepted
        by Armijo (phi drops by ~0.19), the filter stays empty.
    At x = (1, 1 + 2e-3) theta = 2e-3 > theta_min: the step is h-type even
    though dx = (-1.9, -2e-3) satisfies the switching condition (21.6 >
    2e-3^1.1 = 1.1e-3), so it augments the filter."""
    mdl = LineModel(2, [1.0], -10.0, 10.0)
    x0 = [1.0, 1.0 + 1e-5]
    s = _one_step_ipm(mdl, x0, [-1e-5, -1e-5], [0.0], 1e-3)
    assert s.theta_min == 1e-4
    h = s.step()
    assert (h.ls, h.alpha_pr) == (1, 1.0)
    assert len(s.filter) == 1 and s.filter[0][0] == pytest.approx(0.99999e-5, rel=1e-9)
    s = _one_step_ipm(mdl, x0, [-1.9, -1e-5], [0.0], 1e-3)
    h = s.step()
    assert (h.ls, h.alpha_pr) == (1, 1.0) and s.filter == []
    s = _one_step_ipm(mdl, [1.0, 1.0 + 2e-3], [-1.9, -2e-3], [0.0], 1e-3)
    assert s.theta_min == 1e-4
    h = s.step()
    assert (h.ls, h.alpha_pr) == (1, 1.0)
    assert len(s.filter) == 1 and s.filter[0][0] == pytest.approx(0.99999 * 2e-3, rel=1e-9)


def test_step_lengths_multiplier_update_and_safeguard():
    """x = (0.5, 1), bounds (0, -10) .. (1, 10), mu = 1e-3, dx = (-1, 0),
    dy = 0.5, y = 0.2, z_L = (1, 1e12), z_U = (1, 1).
    * tau = max(tau_min, 1 - mu) = 0.999, so the primal step stops at
      alpha_max = 0.999 * 0.5 = 0.4995 (not 0.495 with tau_min alone);
    * dz_U,1 = mu/0.5 - 1 + (1/0.5)(-1) = -2.998 limits the dual step to
      0.999 / 2.998 = 0.333222 (z_L alone would allow ~0.999);
    * the full fraction-to-boundary step is f-type and accepted, and the
      equality multipliers move with the PRIMAL step: y = 0.2 + 0.4995 * 0.5
      = 0.44975;
    * z_L,2 = 1e12 + 0.333 (-1e12) = 6.7e11 exceeds kappa_Sigma mu / (x_2 -
      lo_2) = 1e10 * 1e-3 / 11 = 909090.9 and is reset to it;
      z_U,1 = 1 + 0.333222 * (-2.998) = 0.001 stays inside its interval."""
    mdl = LineModel(2, [1.0], [0.0, -10.0], [1.0, 10.0])
    s = _one_step_ipm(mdl, [0.5, 1.0], [-1.0, 0.0], [0.5], 1e-3)
    s.y = np.array([0.2])
    s.zl = np.array([1.0, 1e12])
    h = s.step()
    assert h.status == "ok" and s.mu == 1e-3
    assert h.extra["alpha_max"] == pytest.approx(0.4995, rel=1e-15)
    assert (h.ls, h.alpha_pr) == (1, h.extra["alpha_max"])
    assert h.alpha_du == pytest.approx(0.33322214809873246, rel=1e-14)
    assert s.y[0] == pytest.approx(0.44975, rel=1e-15)
    assert s.zl[1] == pytest.approx(909090.9090909091, rel=1e-14)
    assert s.zu[0] == pytest.approx(0.001, rel=1e-9)


def test_upper_multiplier_safeguard():
    """The same rule on z_U: x = (0.5, 1), dx = (+1, 0) (now z_L,1 limits the
    dual step: dz_L,1 = 0.002 - 1 - 2 = -2.998), z_U,2 = 1e12 falls to
    6.7e11 and is reset to kappa_Sigma mu / (hi_2 - x_2) = 1e7 / 9."""
    mdl = LineModel(2, [1.0], [0.0, -10.0], [1.0, 10.0])
    s = _one_step_ipm(mdl, [0.5, 1.0], [1.0, 0.0], [0.0], 1e-3)
    s.zu = np.array([1.0, 1e12])
    h = s.step()
    assert h.status == "ok"
    assert h.alpha_du == pytest.approx(0.33322214809873246, rel=1e-14)
    assert s.zu[1] == pytest.approx(1111111.111111111, rel=1e-14)


def test_optimality_error_scaling():
    """E_mu = max(inf_du / s_d, inf_pr, compl / s_c) with
    s_d = max(s_max, sum|multipliers| / count) / s_max and
    s_c = max(s_max, sum z / count) / s_max, s_max = 100.
    x = (0.5, 1), bounds (0, -10) .. (1, 10), grad f = (1, 0), c = 0:
    (a) y = 3000, z = 1: dual residual (1, 3000); s_d = (3004 / 5) / 100 =
        6.008, s_c = 1; complementarity max(0.5, 11, 0.5, 9) = 11;
        E_0 = 3000 / 6.008 = 499.334;
    (b) y = 0, z = 1000: dual residual (1, 0), s_d = 8; s_c = 10,
        complementarity 1000 * 11 = 11000: E_0 = 1100."""
    mdl = LineModel(2, [1.0], [0.0, -10.0], [1.0, 10.0])
    s = _one_step_ipm(mdl, [0.5, 1.0], [0.0, 0.0], [0.0], 1e-3)
    g, c = mdl.grad(s.x), mdl.cons(s.x)
    Jm = sp.csr_matrix((np.ones(1), np.array([1]), np.array([0, 1])), shape=(1, 2))
    s.y = np.array([3000.0])
    err, pr, du, co = s._errors(g, c, Jm, 0.0)
    assert (pr, du, co) == (0.0, 3000.0, 11.0)
    assert err == pytest.approx(499.33422103861517, rel=1e-15)
    s.y = np.array([0.0])
    s.zl = np.full(2, 1000.0)
    s.zu = np.full(2, 1000.0)
    err, pr, du, co = s._errors(g, c, Jm, 0.0)
    assert (du, co) == (1.0, 11000.0)
    assert err == pytest.approx(1100.0, rel=1e-15)


def test_barrier_update_threshold_and_filter_reset():
    """mu is decreased while E_mu <= kappa_eps mu (kappa_eps = 10), and each
    decrease resets the filter.  x = (0.5, 1.5) (c = 0.5), z_L = (0.7, 0.01),
    z_U = (0.2, 0.01): dual residual (1 - 0.7 + 0.2, 0) = 0.5 and
    complementarity <= 0.25 at mu = 0.1, so E_0.1 = 0.5 <= 1: mu becomes
    min(0.2 * 0.1, 0.1^1.5) = 0.02; there E_0.02 = 0.5 > 0.2 stops the
    decrease.  The old filter entry is gone and the h-type step adds one."""
    mdl = LineModel(2, [1.0], [0.0, -10.0], [1.0, 10.0])
    s = _one_step_ipm(mdl, [0.5, 1.5], [0.0, -0.5], [0.0], 0.1)
    s.zl = np.array([0.7, 0.01])
    s.zu = np.array([0.2, 0.01])
    s.filter = [(100.0, 1e9)]
    h = s.step()
    assert h.status == "ok" and h.mu == 0.1
    assert s.mu == pytest.approx(0.02, rel=1e-15)
    assert len(s.filter) == 1 and s.filter[0][0] == pytest.approx(0.499995, rel=1e-15)
