"""Pins of the oracle's dense Bunch-Kaufman LDL^T (the dense solution and the
inertia of the indefinite KKT matrix, Eq. inertia): factorisation residual at
unit-roundoff level with every pivot case exercised, the negative determinant
of every 2x2 block, inertia against LAPACK eigenvalues, solutions against
LAPACK's LU, no pivoting on diagonally dominant SPD matrices (against a
Cholesky factor), and the textbook 2x2 pivot."""
import numpy as np
import pytest
import scipy.linalg

from gen.tray import TrayParams, kkt_point
from oracle import kkt, ldlt, tray

U = np.finfo(np.float64).eps / 2


def _sym_indefinite(rng, N):
    A = rng.standard_normal((N, N))
    return A + A.T


def _tray_kkt(k=4, T=5, seed=0, delta_x=20.0):
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, seed, (1e-2, 1e2))
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    return p, kkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x).toarray()


def _residual(K, F):
    P = K[np.ix_(F.perm, F.perm)]
    return np.linalg.norm(P - F.L @ F.D() @ F.L.T) / np.linalg.norm(K)


def test_factorisation_residual_and_every_pivot_case():
    rng = np.random.default_rng(11)
    seen = set()
    mats = [_sym_indefinite(rng, N) for N in (5, 17, 40, 80) for _ in range(3)]
    mats.append(_tray_kkt()[1])
    for K in mats:
        F = ldlt.factor(K)
        N = K.shape[0]
        assert sorted(F.perm.tolist()) == list(range(N))
        assert np.allclose(np.triu(F.L, 1), 0.0) and np.all(np.diag(F.L) == 1.0)
        assert sum(s for _, s in F.blocks) == N
        assert _residual(K, F) <= 20 * N * U
        seen.update(F.kinds)
    # the four non-degenerate cases of the pivot rule all occurred
    assert {ldlt.PIV_KK, ldlt.PIV_KK_SIGMA, ldlt.PIV_RR, ldlt.PIV_2X2} <= seen


def test_two_by_two_blocks_have_negative_determinant():
    # |A_kk A_rr| < alpha^2 lambda^2 < A_rk^2 whenever the rule picks 2x2
    rng = np.random.default_rng(3)
    count = 0
    for _ in range(10):
        F = ldlt.factor(_sym_indefinite(rng, 30))
        for k, s in F.blocks:
            if s == 2:
                count += 1
                assert F.d[k] * F.d[k + 1] - F.e[k] ** 2 < 0
    assert count > 0


def test_inertia_matches_eigenvalues():
    rng = np.random.default_rng(5)
    for N, npos in ((7, 3), (25, 20), (60, 1), (60, 59)):
        Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
        lam = rng.uniform(0.1, 10.0, N) * np.where(np.arange(N) < npos, 1.0, -1.0)
        K = (Q * lam) @ Q.T
        K = 0.5 * (K + K.T)
        assert ldlt.factor(K).inertia() == (npos, 0, N - npos)
        ev = np.linalg.eigvalsh(K)
        assert (int(np.sum(ev > 0)), int(np.sum(ev < 0))) == (npos, N - npos)


def test_inertia_counts_exact_zero_rows():
    # zero rows and columns stay exactly zero through the elimination
    rng = np.random.default_rng(8)
    M = _sym_indefinite(rng, 9)
    ev = np.linalg.eigvalsh(M)
    K = np.zeros((13, 13))
    K[:9, :9] = M
    q = rng.permutation(13)
    K = K[np.ix_(q, q)]
    assert ldlt.factor(K).inertia() == (int(np.sum(ev > 0)), 4, int(np.sum(ev < 0)))


def test_tray_kkt_inertia_is_n_0_m():
    p, K = _tray_kkt(k=4, T=5)
    F = ldlt.factor(K)
    assert F.inertia() == (p.n, 0, p.m)
    ev = np.linalg.eigvalsh(K)
    assert (int(np.sum(ev > 0)), int(np.sum(ev < 0))) == (p.n, p.m)


@pytest.mark.parametrize("N", [1, 2, 9, 64, 150])
def test_solve_matches_lapack(N):
    rng = np.random.default_rng(N)
    K = _sym_indefinite(rng, N)
    b = rng.standard_normal(N)
    x = ldlt.factor(K).solve(b)
    ref = scipy.linalg.lu_solve(scipy.linalg.lu_factor(K), b)
    cond = np.linalg.cond(K)
    assert np.max(np.abs(x - ref)) <= 1e3 * N * U * cond * np.max(np.abs(ref))


def test_diagonally_dominant_spd_needs_no_pivoting():
    rng = np.random.default_rng(2)
    N = 30
    B = rng.uniform(-1.0, 1.0, (N, N))
    K = 0.5 * (B + B.T) + 2.0 * N * np.eye(N)
    F = ldlt.factor(K)
    assert F.kinds == [ldlt.PIV_KK] * N
    assert np.array_equal(F.perm, np.arange(N))
    Lc = np.linalg.cholesky(K)
    g = np.diag(Lc)
    assert np.allclose(F.L, Lc / g, rtol=0, atol=1e-14)
    assert np.allclose(F.d, g * g, rtol=1e-14, atol=0)
    assert np.all(F.e == 0.0)


def test_textbook_two_by_two_pivot():
    K = np.array([[0.0, 1.0], [1.0, 0.0]])
    F = ldlt.factor(K)
    assert F.blocks == [(0, 2)] and F.kinds == [ldlt.PIV_2X2]
    assert F.inertia() == (1, 0, 1)
    assert np.allclose(F.solve(np.array([2.0, 3.0])), [3.0, 2.0], rtol=0, atol=0)
    # a zero diagonal with a dominant coupling swaps a 1x1 pivot in instead:
    # lambda = 1 at r = 1; sigma = 1; |A_rr| = 5 >= alpha
    K = np.array([[0.0, 1.0], [1.0, 5.0]])
    F = ldlt.factor(K)
    assert F.kinds[0] == ldlt.PIV_RR and F.perm.tolist() == [1, 0]
    assert F.inertia() == (1, 0, 1)
    assert np.allclose(F.solve(np.array([1.0, 7.0])), np.linalg.solve(K, [1.0, 7.0]))


@pytest.mark.parametrize("K, kind, perm0", [
    # |A_00| = 2 >= alpha * lambda = alpha
    ([[2.0, 1.0], [1.0, 0.0]], ldlt.PIV_KK, 0),
    # |A_00| = 0.5 < alpha; r = 1, sigma = max(|A_01|, |A_21|) = 2,
    # |A_00| sigma = 1 >= alpha lambda^2 = alpha: keep A_00
    ([[0.5, 1.0, 0.0], [1.0, 0.0, 2.0], [0.0, 2.0, 0.0]], ldlt.PIV_KK_SIGMA, 0),
    # sigma = |A_01| = 1 (A_rr is not part of sigma), |A_00| sigma < alpha,
    # |A_11| = 10 >= alpha sigma: A_11 is the pivot
    ([[0.5, 1.0], [1.0, 10.0]], ldlt.PIV_RR, 1),
    # lambda = 2: |A_00| sigma = 2 < alpha lambda^2 = 2.56 (though >= alpha
    # lambda), then |A_11| = 3 >= alpha sigma: A_11 is the pivot
    ([[1.0, 2.0], [2.0, 3.0]], ldlt.PIV_RR, 1),
    # lambda = 3 at r = 2, sigma = max(|A_02|, |A_12|) = 3, |A_22| = 1 < alpha 3
    ([[0.1, 1.0, 3.0], [1.0, 5.0, 3.0], [3.0, 3.0, 1.0]], ldlt.PIV_2X2, 0),
    # lambda = 2 at r = 2, sigma = |A_12| = 5: alpha lambda <= |A_22| = 2 <
    # alpha sigma, so the 2x2 pivot, not A_22
    ([[0.1, 1.0, 2.0], [1.0, 0.0, 5.0], [2.0, 5.0, 2.0]], ldlt.PIV_2X2, 0),
])
def test_pivot_rule_worked_cases(K, kind, perm0):
    K = np.array(K)
    F = ldlt.factor(K)
    assert F.kinds[0] == kind and F.perm[0] == perm0
    if kind == ldlt.PIV_2X2:
        assert F.perm[1] == 2          # r swapped into position k + 1
    assert _residual(K, F) <= 10 * U


def test_dense_solve_routes_agree():
    p, K = _tray_kkt(k=4, T=5)
    b = np.random.default_rng(4).standard_normal(K.shape[0])
    v1 = kkt.dense_solve(K, b)
    v2 = kkt.dense_solve(K, b, ldlt_max=0)
    assert np.max(np.abs(v1 - v2)) <= 1e-10 * np.max(np.abs(v2))
    assert kkt.backward_error(K, v1, b) <= 1e-15
