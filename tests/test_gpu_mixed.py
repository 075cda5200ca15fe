"""Mixed-precision factorization (kkt_options.precision = 1): the supernodal
factor in FP32, refinement in FP64 against the FP64 system, FP64 refactor
when the FP32 factor fails or does not refine to the tolerance.  The
answer must meet the same FP64 bar as the FP64 path (eta <= 1e-10, checked
again by the oracle); the FP32 factor itself is compared with the oracle's
FP64 factor to single-precision accuracy."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cholesky, kkt as okkt, symbolic
from tests.gpu_common import ensure_built, instance, oracle_eta, solver_for, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _factor(p, pt, W, J, D, delta_x, precision=1, **o):
    torch = torch_cuda()
    opts = dict(OPTS)
    opts.update(o)
    s = solver_for(p, W, J, scheme=opts.pop("scheme", "lifted"), precision=precision, **opts)
    st = s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  None if D is None else to_dev(torch, D), delta_x)
    return s, st


def _oracle_factor(p, pt, W, J, D, delta_x):
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    Kr, Kc, Kv = okkt.condensed_coo(p.n, W, J, pt.sigma, delta_x, D)
    return sym, (Kr, Kc, Kv), cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)


@pytest.mark.parametrize("k,T", [(32, 50), (7, 13)])
def test_fp32_factor_matches_oracle(k, T):
    """Every entry of the FP32 factor agrees with the oracle's FP64 factor to
    a few hundred single-precision units (K well conditioned here)."""
    p, pt, W, J = instance(k, T, seed=1, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e2)
    s, st = _factor(p, pt, W, J, D, 10.0)
    assert st == 0 and s.info.status_detail == 1
    colptr, rowind, val = s.factor_export()
    sym, _, ch = _oracle_factor(p, pt, W, J, D, 10.0)
    worst = 0.0
    for j in range(p.n):
        ref = dict(zip(sym.structs[j].tolist(), ch.vals[j].tolist()))
        scale = max(abs(v) for v in ref.values())
        rows = rowind[colptr[j]:colptr[j + 1]].tolist()
        assert set(ref) <= set(rows)
        for r, v in zip(rows, val[colptr[j]:colptr[j + 1]].tolist()):
            worst = max(worst, abs(v - ref.get(r, 0.0)) / scale)
    assert worst <= 3e-5, worst
    assert worst > 1e-12          # it really is the single-precision factor


def test_fp32_relaxed_target_refines_in_fp32():
    """Relaxed target with D = 1e2: K_delta is the exact Schur complement, the
    FP32 factor is a contraction for the FP64 refinement, which reaches
    eta <= 1e-10 without falling back."""
    p, pt, W, J = instance(8, 9, 4, sigma_range=(1e-2, 1e2))
    torch = torch_cuda()
    D = np.full(p.m, 1e2) * (1 + np.arange(p.m) % 3)
    s, st = _factor(p, pt, W, J, D, 30.0, target_relaxed=1)
    assert st == 0 and s.info.status_detail == 1
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert st == 0 and s.info.status_detail == 1
    assert s.info.bwd_err <= 1e-10 and 1 <= s.info.refine_iters <= 12
    K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 30.0, C=1.0 / D)
    v = okkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]))
    g = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    assert np.max(np.abs(g - v)) <= 1e-9 * np.max(np.abs(v))
    assert s.stats()["fp64_fallbacks"] == 0 and s.stats()["fp32_factors"] == 1


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
@pytest.mark.parametrize("seed", [0, 1])
def test_fp32_config1_meets_fp64_bar(scheme, seed):
    """32 trays, T = 50, Sigma in [1e-6, 1e6]: whatever precision ends up
    carrying the solve, the backward error recomputed by the oracle is
    <= 1e-10 (the FP64 bar)."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, seed)
    s, st = _factor(p, pt, W, J, None, 0.0, scheme=scheme, gamma=1e7, max_cg=500)
    assert st == 0 and s.info.status_detail in (1, 2)
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert st == 0 and s.info.bwd_err <= 1e-10
    assert s.info.status_detail in (1, 2)
    assert oracle_eta(p, W, J, pt.sigma, 0.0, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry) <= 1e-10


def test_fp32_fallback_refactors_in_fp64():
    """A tolerance one FP32 solve cannot meet with no refinement allowed: the
    solve refactorises in FP64 (status_detail 2), and the factor in use is
    then the FP64 one, equal to the oracle's to FP64 accuracy."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, 1, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e2)
    s, st = _factor(p, pt, W, J, D, 10.0, tol_refine=1e-14, max_refine=0)
    assert st == 0 and s.info.status_detail == 1
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert s.info.status_detail == 2
    assert s.stats()["fp64_fallbacks"] == 1
    colptr, rowind, val = s.factor_export()
    sym, _, ch = _oracle_factor(p, pt, W, J, D, 10.0)
    worst = 0.0
    for j in range(p.n):
        ref = dict(zip(sym.structs[j].tolist(), ch.vals[j].tolist()))
        scale = max(abs(v) for v in ref.values())
        for r, v in zip(rowind[colptr[j]:colptr[j + 1]].tolist(), val[colptr[j]:colptr[j + 1]].tolist()):
            worst = max(worst, abs(v - ref.get(r, 0.0)) / scale)
    assert worst <= 1e-11


def test_fp32_not_spd_falls_back_then_reports_oracle_column():
    """An indefinite K: the FP32 pivot fails, the FP64 refactor fails at the
    column the oracle's factorization names."""
    p, pt, W, J = instance(8, 12, seed=2)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    Wv = W[2].copy()
    Wv[W[0][int(sym.perm[p.n // 2])]] -= 1e12
    Kr, Kc, Kv = okkt.condensed_coo(p.n, (W[0], W[1], Wv), J, pt.sigma, 0.0, np.full(p.m, 1e2))
    with pytest.raises(cholesky.NotPositiveDefinite) as e:
        cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    s, st = _factor(p, pt, (W[0], W[1], Wv), J, np.full(p.m, 1e2), 0.0)
    assert st == -4
    assert s.info.status_detail == 2 and s.info.failed_col == e.value.column


def test_fp32_backsolve():
    """K^{-1} b with the FP32 factor: single-precision backward error on K."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e2)
    s, st = _factor(p, pt, W, J, D, 10.0)
    assert st == 0 and s.info.status_detail == 1
    b = np.random.default_rng(3).standard_normal(p.n)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s.backsolve(to_dev(torch, b), x)
    _, (Kr, Kc, Kv), _ = _oracle_factor(p, pt, W, J, D, 10.0)
    K = sp.coo_matrix((Kv, (Kr, Kc)), shape=(p.n, p.n)).tocsr()
    xg = x.cpu().numpy()
    res = np.max(np.abs(K @ xg - b)) / (okkt.inf_norm(K) * np.max(np.abs(xg)) + np.max(np.abs(b)))
    assert res <= 1e-6, res
    assert res > 1e-14


@pytest.mark.parametrize("precision", [0, 1])
def test_sigma_1e8_span_meets_bar(precision):
    """Sigma log-uniform on [1e-8, 1e8] (late-IPM conditioning) at 32 trays,
    T = 50: both precisions meet eta <= 1e-10, as does the dense LU
    solution.  K_orig is nearly singular here (||v|| ~ 1e9 for an N(0,1)
    right-hand side), so solutions with the same backward error differ at
    O(1) relative and no forward agreement is asserted."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-8, 1e8))
    s, st = _factor(p, pt, W, J, None, 0.0, precision=precision)
    delta_x = 0.0
    while st == -4:
        delta_x = 1e-4 if delta_x == 0 else delta_x * 8
        st = s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma), None, delta_x)
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert st == 0 and s.info.bwd_err <= 1e-10
    g = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    assert oracle_eta(p, W, J, pt.sigma, delta_x, g[:p.n], g[p.n:], pt.rx, pt.ry) <= 1e-10
    K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    b = np.concatenate([pt.rx, pt.ry])
    v = okkt.dense_solve(K, b, refine_steps=4)
    assert okkt.backward_error(K, v, b) <= 1e-10


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_full_size_mixed_precision_workload(scheme):
    """The mixed-precision workload (32 trays, T = 20000, n = 1,300,065,
    Sigma on [1e-8, 1e8]) with precision = 1: the backward error recomputed
    by the oracle on the CPU is <= 1e-10 whichever factor carried the solve."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 20000, 0, sigma_range=(1e-8, 1e8))
    s = solver_for(p, W, J, scheme=scheme, gamma=1e4, max_cg=500, precision=1, **OPTS)
    Wv, Jv, sigma = to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma)
    st = s.factor(Wv, Jv, sigma, None, 0.0)
    delta_x = 0.0
    while st == -4:
        delta_x = 1e-4 if delta_x == 0 else delta_x * 8
        st = s.factor(Wv, Jv, sigma, None, delta_x)
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert st == 0 and s.info.bwd_err <= 1e-10
    assert s.info.status_detail in (1, 2)
    eta = oracle_eta(p, W, J, pt.sigma, delta_x, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry)
    assert eta <= 1e-10


# ---- double-float factor (precision = 2): pairs of FP32 numbers, ~48 bits

@pytest.mark.parametrize("k,T", [(32, 50), (7, 13)])
def test_df64_factor_matches_oracle(k, T):
    """The double-float factor agrees with the oracle's FP64 factor to
    ~1e-13 relative (unit roundoff ~2^-47), and is not the FP64 factor."""
    p, pt, W, J = instance(k, T, seed=1, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e2)
    s, st = _factor(p, pt, W, J, D, 10.0, precision=2)
    assert st == 0 and s.info.status_detail == 3
    colptr, rowind, val = s.factor_export()
    sym, _, ch = _oracle_factor(p, pt, W, J, D, 10.0)
    worst = 0.0
    for j in range(p.n):
        ref = dict(zip(sym.structs[j].tolist(), ch.vals[j].tolist()))
        scale = max(abs(v) for v in ref.values())
        for r, v in zip(rowind[colptr[j]:colptr[j + 1]].tolist(), val[colptr[j]:colptr[j + 1]].tolist()):
            worst = max(worst, abs(v - ref.get(r, 0.0)) / scale)
    assert worst <= 1e-12, worst
    assert worst > 1e-16


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
@pytest.mark.parametrize("seed", [0, 1])
def test_df64_config1_meets_fp64_bar(scheme, seed):
    """32 trays, T = 50, Sigma on [1e-6, 1e6], delta = 1e-8 (the case where
    an FP32 factor falls back): the double-float factor carries the solve to
    eta <= 1e-10 without falling back; the oracle confirms eta."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, seed)
    s, st = _factor(p, pt, W, J, None, 0.0, precision=2, scheme=scheme, gamma=1e7, max_cg=500)
    assert st == 0 and s.info.status_detail == 3
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert st == 0 and s.info.bwd_err <= 1e-10 and s.info.status_detail == 3
    assert oracle_eta(p, W, J, pt.sigma, 0.0, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry) <= 1e-10


def test_df64_ipm_matches_fp64_ipm():
    """The device IPM with double-float factors takes the FP64 IPM's
    iterations to the same optimum (16 trays, T = 40)."""
    torch_cuda()
    from gen.tray import TrayParams
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=16, T=40)
    out = {}
    for prec in (0, 2):
        g = IPMSolver(p.as_array(), scheme="lifted", precision=prec, **OPTS)
        g.init()
        h = g.solve()
        assert h[-1]["status"] == 1
        out[prec] = (h[-1]["iter"], h[-1]["objective"], g.get()[0].cpu().numpy())
        g.close()
    assert abs(out[2][0] - out[0][0]) <= 1
    assert abs(out[2][1] - out[0][1]) <= 1e-8 * abs(out[0][1])
    assert np.max(np.abs(out[2][2] - out[0][2])) <= 1e-6


def test_set_precision_switches_between_the_analysed_and_fp64():
    """kkt_set_precision: an FP32-analysed context factorises in FP64 after
    kkt_set_precision(0) (no reduced-precision factor counted, the FP64
    backward error) and in FP32 again after kkt_set_precision(1); an FP64
    context accepts only 0."""
    torch = torch_cuda()
    from paper_2403_15913_gb300 import _native as nat
    p, pt, W, J = instance(16, 30, 4, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", precision=1, **OPTS)
    L = nat.lib()
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    vals = (to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma))
    for prec, want in ((0, 0), (1, 1), (0, 0)):
        assert L.kkt_set_precision(s._ctx, prec) == 0
        s.reset_stats()
        assert s.factor(*vals, None, 10.0) == 0
        assert s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy) == 0
        assert s.stats()["fp32_factors"] == want
        assert s.info.status_detail == want
        assert oracle_eta(p, W, J, pt.sigma, 10.0, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry) <= 1e-10
    assert L.kkt_set_precision(s._ctx, 2) == nat.KKT_ERR_ARG
    s.close()
    s64 = solver_for(p, W, J, scheme="lifted", **OPTS)
    assert L.kkt_set_precision(s64._ctx, 1) == nat.KKT_ERR_ARG
    assert L.kkt_set_precision(s64._ctx, 0) == 0
    s64.close()
