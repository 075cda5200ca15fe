"""Pins of the oracle's numeric Cholesky and KKT solvers: dense Cholesky and
LAPACK cross-checks, the first failing pivot, condensation recovery
(Eq. kkt:condensed), Haynsworth inertia, HyKKT equivalence for every gamma
(Eq. hykkt), the spectrum of gamma S_gamma (Sec. IV-B), Lifted-KKT
refinement (Sec. V-B)."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen.tray import TrayParams, kkt_point
from oracle import cholesky, kkt, symbolic, tray


def _tray_case(k=8, T=6, seed=0, sigma_range=(1e-6, 1e6)):
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, seed, sigma_range)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    return p, pt, W, J


def _sym(p, W, J, **kw):
    return symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **kw)


def _spd_case(delta_x=10.0, D=1e2, **kw):
    p, pt, W, J = _tray_case(**kw)
    Kr, Kc, Kv = kkt.condensed_coo(p.n, W, J, pt.sigma, delta_x, np.full(p.m, D))
    return p, pt, W, J, Kr, Kc, Kv


@pytest.mark.parametrize("relax", [dict(), dict(relax_cols=48, relax_zeros=1024, max_width=16)])
def test_cholesky_matches_dense(relax):
    p, pt, W, J, Kr, Kc, Kv = _spd_case()
    sym = _sym(p, W, J, leaf_size=16, **relax)
    ch = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    K = sp.coo_matrix((Kv, (Kr, Kc)), shape=(p.n, p.n)).toarray()
    Kp = K[np.ix_(sym.perm, sym.perm)]
    L = cholesky.to_dense_L(p.n, sym.structs, ch.vals)
    Ld = np.linalg.cholesky(Kp)
    assert np.max(np.abs(L - Ld)) <= 1e-12 * np.max(np.abs(Ld))
    assert np.linalg.norm(Kp - L @ L.T) <= 1e-13 * np.linalg.norm(Kp)
    b = np.random.default_rng(1).standard_normal(p.n)
    assert np.allclose(ch.solve(b), np.linalg.solve(K, b), rtol=1e-9, atol=1e-12)


def test_cholesky_reports_first_failing_column():
    p, pt, W, J, Kr, Kc, Kv = _spd_case(delta_x=0.0, D=1.0)
    sym = _sym(p, W, J, leaf_size=16)
    K = sp.coo_matrix((Kv, (Kr, Kc)), shape=(p.n, p.n)).toarray()
    Kp = K[np.ix_(sym.perm, sym.perm)]
    # make the leading minor of order j0+1 indefinite: subtract from the
    # pivot column j0 more than its Schur complement value
    j0 = p.n // 3
    s = Kp[j0, j0] - Kp[j0, :j0] @ np.linalg.solve(Kp[:j0, :j0], Kp[:j0, j0])
    shift = s + 1.0
    K2 = K.copy()
    K2[sym.perm[j0], sym.perm[j0]] -= shift
    r, c = np.nonzero(K2)
    with pytest.raises(cholesky.NotPositiveDefinite) as e:
        cholesky.SparseCholesky(sym, p.n, r, c, K2[r, c])
    assert e.value.column == j0
    # the library's definition of the failing column equals the first
    # leading principal minor that is not positive definite
    Kp2 = K2[np.ix_(sym.perm, sym.perm)]
    first = next(j for j in range(p.n)
                 if np.min(np.linalg.eigvalsh(Kp2[:j + 1, :j + 1])) <= 0)
    assert first == j0


def test_cholesky_exact_zero_pivot_fails():
    """[[1, 1], [1, 1]] is positive semidefinite: the second pivot is
    exactly 1 - 1 * 1 = 0, which is not positive."""
    structs = [np.array([0, 1]), np.array([1])]
    with pytest.raises(cholesky.NotPositiveDefinite) as e:
        cholesky.factor(2, structs, [{0: 1.0, 1: 1.0}, {1: 1.0}])
    assert e.value.column == 1
    vals = cholesky.factor(2, structs, [{0: 4.0, 1: 2.0}, {1: 5.0}])
    assert np.array_equal(vals[0], [2.0, 1.0]) and np.array_equal(vals[1], [2.0])


def test_cholesky_sums_duplicate_triplets():
    """K given as the concatenated triplets of its summands (as assembly
    produces it: W, the diagonal, J^T D J) factors like K itself."""
    p, pt, W, J, Kr, Kc, Kv = _spd_case()
    sym = _sym(p, W, J, leaf_size=16)
    ref = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    rng = np.random.default_rng(3)
    split = rng.uniform(0.2, 0.8, len(Kv))
    two = cholesky.SparseCholesky(sym, p.n, np.concatenate([Kr, Kr]), np.concatenate([Kc, Kc]),
                                  np.concatenate([Kv * split, Kv * (1.0 - split)]))
    for a, b in zip(ref.vals, two.vals):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.max(np.abs(a)))


def test_dense_solve_small_closed_form():
    # [[2, 1], [1, 0]] [x; y] = [3; 1]  ->  x = 1, y = 1
    K = np.array([[2.0, 1.0], [1.0, 0.0]])
    for steps in range(4):          # any number of refinement steps, odd or even
        v = kkt.dense_solve(K, np.array([3.0, 1.0]), refine_steps=steps)
        assert np.allclose(v, [1.0, 1.0], rtol=0, atol=1e-15), steps
    assert kkt.inertia(K) == (1, 0, 1)


def test_backward_error_and_norm_worked_values():
    """Rigal-Gaches normwise backward error
    eta = ||b - K v||_inf / (||K||_inf ||v||_inf + ||b||_inf) and the
    infinity norm (largest absolute row sum) on hand-computed cases."""
    K = np.array([[1.0, -2.0], [3.0, 4.0]])
    assert kkt.inf_norm(K) == 7.0
    import scipy.sparse as sps
    assert kkt.inf_norm(sps.csr_matrix(K)) == 7.0
    # K = I: v = (1, 0), b = (2, 0): residual 1, eta = 1 / (1 * 1 + 2)
    assert kkt.backward_error(np.eye(2), np.array([1.0, 0.0]), np.array([2.0, 0.0])) == 1.0 / 3.0
    # v = 0 is never better than eta = 1
    assert kkt.backward_error(K, np.zeros(2), np.array([1.0, -5.0])) == 1.0
    # an exact solution has eta = 0
    assert kkt.backward_error(K, np.array([1.0, 1.0]), np.array([-1.0, 7.0])) == 0.0


def test_condensation_recovers_augmented_solution():
    """Eq. (kkt:augmented) solved densely equals the condensed solve of
    Eq. (kkt:condensed) plus the recovery d_s = -r4 - H d_x,
    d_z = -r2 - D_s d_s, on a random system with slacks."""
    rng = np.random.default_rng(7)
    n, me, mi = 9, 3, 4
    A = rng.standard_normal((n, n))
    W = A @ A.T + np.eye(n)
    G = rng.standard_normal((me, n))
    H = rng.standard_normal((mi, n))
    Ds = np.diag(rng.uniform(0.5, 3.0, mi))
    Z = np.zeros
    Kaug = np.block([[W, Z((n, mi)), G.T, H.T],
                     [Z((mi, n)), Ds, Z((mi, me)), np.eye(mi)],
                     [G, Z((me, mi)), Z((me, me)), Z((me, mi))],
                     [H, np.eye(mi), Z((mi, me)), Z((mi, mi))]])
    r1, r2, r3, r4 = (rng.standard_normal(s) for s in (n, mi, me, mi))
    d = np.linalg.solve(Kaug, -np.concatenate([r1, r2, r3, r4]))
    dx, ds, dy, dz = np.split(d, [n, n + mi, n + mi + me])
    Kk = W + H.T @ Ds @ H
    Kc = np.block([[Kk, G.T], [G, Z((me, me))]])
    e = np.linalg.solve(Kc, -np.concatenate([r1 + H.T @ (Ds @ r4 - r2), r3]))
    assert np.allclose(e[:n], dx) and np.allclose(e[n:], dy)
    ds2 = -r4 - H @ e[:n]
    dz2 = -r2 - Ds @ ds2
    assert np.allclose(ds2, ds) and np.allclose(dz2, dz)
    # Haynsworth: In(K_aug) = (n + mi, 0, mi + me) <=> In(K_cond) = (n, 0, me)
    assert kkt.inertia(Kaug) == (n + mi, 0, mi + me)
    assert kkt.inertia(Kc) == (n, 0, me)
    ev = np.linalg.eigvalsh(Kaug)
    assert (np.sum(ev > 0), np.sum(ev < 0)) == (n + mi, mi + me)


def test_tray_kkt_inertia_and_schur_spectrum():
    p, pt, W, J = _tray_case(k=4, T=3, sigma_range=(1e-1, 1e1))
    delta_x = 50.0          # enough to make W + Sigma + delta_x I positive
    K = kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    assert kkt.inertia(K) == (p.n, 0, p.m)
    Hd = kkt.hessian_block(p.n, W, pt.sigma, delta_x).toarray()
    Jd = kkt.jacobian_matrix(p.n, p.m, J).toarray()
    errs = []
    for gamma in (1e2, 1e4, 1e7):
        Kg = Hd + gamma * Jd.T @ Jd
        S = Jd @ np.linalg.solve(Kg, Jd.T)
        ev = np.linalg.eigvalsh(0.5 * (S + S.T))
        errs.append(np.max(np.abs(gamma * ev - 1.0)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


@pytest.mark.parametrize("gamma", [1e2, 1e4, 1e7])
def test_hykkt_equals_dense(gamma):
    p, pt, W, J = _tray_case(k=6, T=5, seed=2, sigma_range=(1e-2, 1e2))
    sym = _sym(p, W, J, leaf_size=16)
    delta_x = 20.0
    K = kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    b = np.concatenate([pt.rx, pt.ry])
    v = kkt.dense_solve(K, b)
    dx, dy, info = kkt.hykkt_solve(sym, p.n, p.m, W, J, pt.sigma, delta_x,
                                   gamma, pt.rx, pt.ry)
    assert info.status == "ok" and info.bwd_err <= 1e-10
    vv = np.concatenate([dx, dy])
    assert np.max(np.abs(vv - v)) <= 1e-7 * np.max(np.abs(v))


@pytest.mark.parametrize("gamma", [1e2, 1e4, 1e7])
def test_hykkt_inner_solve_is_exact_without_refinement(gamma):
    """For every gamma, K_gamma and the Schur complement S_gamma reproduce
    the KKT solution exactly (Eq. hykkt, Eq. schurcomp): one inner solve
    with CG run to 1e-12 already gives the dense solution, no Richardson
    sweep needed."""
    p, pt, W, J = _tray_case(k=6, T=5, seed=2, sigma_range=(1e-2, 1e2))
    sym = _sym(p, W, J, leaf_size=16)
    delta_x = 20.0
    K = kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    v = kkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]))
    dx, dy, info = kkt.hykkt_solve(sym, p.n, p.m, W, J, pt.sigma, delta_x, gamma,
                                   pt.rx, pt.ry, tol_cg=1e-12, max_refine=0)
    assert info.status == "ok" and info.refine_iters == 0
    assert info.bwd_err <= 1e-12
    assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-9 * np.max(np.abs(v))


def test_lifted_relaxed_target_is_exact():
    """With target C = D^{-1} the condensed solve is exact (Eq. liftedkkt)."""
    p, pt, W, J = _tray_case(k=6, T=4, seed=4)
    sym = _sym(p, W, J, leaf_size=16)
    D = np.full(p.m, 1e6)
    K = kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 30.0, C=1.0 / D)
    b = np.concatenate([pt.rx, pt.ry])
    v = kkt.dense_solve(K, b)
    dx, dy, info = kkt.lifted_solve(sym, p.n, p.m, W, J, pt.sigma, 30.0, D,
                                    pt.rx, pt.ry, C=1.0 / D)
    assert info.refine_iters <= 1 and info.bwd_err <= 1e-12
    assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-8 * np.max(np.abs(v))


def test_lifted_refinement_converges_on_original_system():
    """Lifted-KKT with D = 1/delta preconditions K_orig; Richardson reaches
    eta <= 1e-10 and the solution equals the dense one."""
    p, pt, W, J = _tray_case(k=6, T=4, seed=6, sigma_range=(1e-2, 1e2))
    sym = _sym(p, W, J, leaf_size=16)
    delta_x = 30.0
    K = kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    b = np.concatenate([pt.rx, pt.ry])
    v = kkt.dense_solve(K, b)
    dx, dy, info = kkt.lifted_solve(sym, p.n, p.m, W, J, pt.sigma, delta_x,
                                    np.full(p.m, 1e8), pt.rx, pt.ry)
    assert info.status == "ok" and info.bwd_err <= 1e-10
    assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-6 * np.max(np.abs(v))
    # error contracts at least geometrically
    assert all(b2 < b1 for b1, b2 in zip(info.etas, info.etas[1:]))


@pytest.mark.parametrize("delta", [1e-4, 1e-3])
def test_lifted_refinement_rate_closed_form(delta):
    """Richardson with the Lifted-KKT preconditioner M = [[H, J^T], [J,
    -delta I]] on K_orig = [[H, J^T], [J, 0]] maps the error by
    M^{-1}(M - K_orig), whose nonzero eigenvalues are delta / (delta + mu_j)
    for the eigenvalues mu_j of J H^{-1} J^T (Sec. IV-A, V-B): the backward
    error contracts asymptotically by delta / (delta + mu_min)."""
    p, pt, W, J = _tray_case(k=6, T=4, seed=6, sigma_range=(1e-2, 1e2))
    sym = _sym(p, W, J, leaf_size=16)
    delta_x = 30.0
    H = kkt.hessian_block(p.n, W, pt.sigma, delta_x).toarray()
    Jd = kkt.jacobian_matrix(p.n, p.m, J).toarray()
    mu_min = np.linalg.eigvalsh(Jd @ np.linalg.solve(H, Jd.T))[0]
    rho = delta / (delta + mu_min)
    dx, dy, info = kkt.lifted_solve(sym, p.n, p.m, W, J, pt.sigma, delta_x,
                                    np.full(p.m, 1.0 / delta), pt.rx, pt.ry,
                                    tol=1e-14, max_refine=60)
    etas = np.array(info.etas)
    etas = etas[etas > 1e-13]                 # above the rounding floor
    assert len(etas) >= 6
    ratios = etas[1:] / etas[:-1]
    assert abs(ratios[-1] / rho - 1.0) < 0.05, (ratios[-4:], rho)
    assert np.all(ratios <= rho * 1.01)       # the slowest mode bounds every step


def test_cg_exact_in_n_steps():
    """CG on an SPD 3x3 system terminates in at most 3 steps (exact
    arithmetic property, here to rounding)."""
    A = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    b = np.array([1.0, 2.0, 3.0])
    x, it, ok = kkt.conjugate_gradient(lambda v: A @ v, b, tol=1e-14)
    assert ok and it <= 4 and np.allclose(A @ x, b, atol=1e-13)
