"""GPU parity of the KKT hot path against the oracle, through the C ABI:
model evaluation kernels, numeric factor, failing pivot, Lifted-KKT and
HyKKT steps (backward error and agreement with the dense oracle solution),
edge cases and the full-size workload (properties that hold at any size)."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen.tray import TrayParams, kkt_point
from oracle import cholesky, kkt as okkt, symbolic, tray as otray
from tests.gpu_common import (ensure_built, instance, oracle_eta, solver_for, to_dev,
                              torch_cuda)

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# the last case has non-default holdup, control weight, step, volatility and
# feed composition, so a constant dropped on either side cannot hide behind 1
@pytest.mark.parametrize("k,T,kw", [(32, 50, {}), (5, 7, {}), (32, 0, {}), (3, 4, {}),
                                    (6, 5, dict(M=2.0, rho=0.7, h=0.05, alpha=1.9, xf=0.4))])
def test_tray_eval_matches_oracle(k, T, kw):
    torch = torch_cuda()
    from paper_2403_15913_gb300 import TrayModel
    p = TrayParams(k=k, T=T, **kw)
    pt = kkt_point(p, 11)
    tm = TrayModel(p.as_array())
    w, lam = to_dev(torch, pt.w), to_dev(torch, pt.lam)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    c = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    Jv = torch.zeros(tm.nnzJ, dtype=torch.float64, device="cuda")
    Wv = torch.zeros(tm.nnzW, dtype=torch.float64, device="cuda")
    tm.eval(w, lam, 0.7, f, g, c, Jv, Wv)
    torch.cuda.synchronize()
    of = otray.objective(p, pt.w)
    og = otray.objective_grad(p, pt.w)
    oc = otray.constraints(p, pt.w)
    oJ = otray.jacobian_csr(p, pt.w)[2]
    oW = otray.hessian_lower_csc(p, pt.w, pt.lam, 0.7)[2]
    tol = 1e-14
    assert abs(f.item() - of) <= tol * abs(of) * 10
    for dev, ref in ((g, og), (c, oc), (Jv, oJ), (Wv, oW)):
        d = dev.cpu().numpy()
        assert d.shape == ref.shape
        assert np.max(np.abs(d - ref)) <= tol * max(1.0, np.max(np.abs(ref)))


def _dense_factor_parity(p, pt, W, J, delta_x, D, opts):
    torch = torch_cuda()
    s = solver_for(p, W, J, scheme="lifted", **opts)
    st = s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  to_dev(torch, np.full(p.m, D)), delta_x)
    assert st == 0
    colptr, rowind, val = s.factor_export()
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **opts)
    Kr, Kc, Kv = okkt.condensed_coo(p.n, W, J, pt.sigma, delta_x, np.full(p.m, D))
    ch = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    worst = 0.0
    for j in range(p.n):
        rows = rowind[colptr[j]:colptr[j + 1]]
        vals = val[colptr[j]:colptr[j + 1]]
        ref = dict(zip(sym.structs[j].tolist(), ch.vals[j].tolist()))
        scale = max(abs(v) for v in ref.values())
        for r, v in zip(rows.tolist(), vals.tolist()):
            worst = max(worst, abs(v - ref.get(r, 0.0)) / scale)
        assert set(ref) <= set(rows.tolist())
    return worst


@pytest.mark.parametrize("k,T,opts", [
    (32, 50, OPTS),
    (32, 40, dict(leaf_size=64, relax_cols=48, relax_zeros=1024, max_width=64)),
    (7, 13, dict(leaf_size=16, relax_cols=16, relax_zeros=40, max_width=8)),
    (32, 20, dict(leaf_size=64, relax_cols=0, relax_zeros=0, max_width=64)),
    # 64-column separators: the split levels (diagonal block, lanes-over-rows
    # TRSM, SYRK) and the narrow-level cluster kernel
    (64, 24, OPTS),
    (64, 100, OPTS),
])
def test_factor_matches_oracle(k, T, opts):
    p, pt, W, J = instance(k, T, seed=1, sigma_range=(1e-2, 1e2))
    worst = _dense_factor_parity(p, pt, W, J, 10.0, 1e2, opts)
    assert worst <= 1e-11


def test_not_spd_reports_oracle_column():
    torch = torch_cuda()
    p, pt, W, J = instance(8, 12, seed=2)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    # W with a strongly negative diagonal on one variable
    Wv = W[2].copy()
    v = int(sym.perm[p.n // 2])
    first = W[0][v]
    Wv[first] -= 1e12
    Kr, Kc, Kv = okkt.condensed_coo(p.n, (W[0], W[1], Wv), J, pt.sigma, 0.0, np.full(p.m, 1e2))
    with pytest.raises(cholesky.NotPositiveDefinite) as e:
        cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    s = solver_for(p, W, J, scheme="lifted", **OPTS)
    st = s.factor(to_dev(torch, Wv), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  to_dev(torch, np.full(p.m, 1e2)), 0.0)
    assert st == -4
    assert s.info.failed_col == e.value.column
    # a solve without a successful factor is refused
    from paper_2403_15913_gb300 import KKTError
    z = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    zy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    with pytest.raises(KKTError):
        s.solve(z, zy, z.clone(), zy.clone())


@pytest.mark.parametrize("where,bad", [("W", np.nan), ("J", np.inf), ("sigma", np.nan),
                                       ("sigma", -np.inf)])
def test_nonfinite_values_report_oracle_column(where, bad):
    """A NaN or infinity injected on the host into W, J or Sigma reaches a
    pivot: the factor reports KKT_ERR_NOT_SPD at the oracle's first failing
    column (the library never returns a factor built on it)."""
    torch = torch_cuda()
    p, pt, W, J = instance(8, 12, seed=3, sigma_range=(1e-2, 1e2))
    Wv, Jv, sig = W[2].copy(), J[2].copy(), pt.sigma.copy()
    target = {"W": Wv, "J": Jv, "sigma": sig}[where]
    target[len(target) // 2] = bad
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    Kr, Kc, Kv = okkt.condensed_coo(p.n, (W[0], W[1], Wv), (J[0], J[1], Jv), sig, 1.0,
                                    np.full(p.m, 1e2))
    with pytest.raises(cholesky.NotPositiveDefinite) as e, np.errstate(invalid="ignore"):
        cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    s = solver_for(p, W, J, scheme="lifted", **OPTS)
    st = s.factor(to_dev(torch, Wv), to_dev(torch, Jv), to_dev(torch, sig),
                  to_dev(torch, np.full(p.m, 1e2)), 1.0)
    assert st == -4
    assert s.info.failed_col == e.value.column


@pytest.mark.parametrize("staged", [3, 2, 1, 0])
@pytest.mark.parametrize("sig,D,dx0", [((1e-2, 1e2), 1e2, 10.0), ((1e-6, 1e6), 1e8, 0.0)])
def test_backsolve_matches_oracle(sig, D, dx0, staged):
    """K^{-1} b by the supernodal triangular solves equals the oracle's
    left-looking factor + column substitutions (dataflow, staged and plain
    level kernels)."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, 0, sigma_range=sig)
    s = solver_for(p, W, J, scheme="lifted", staged_solve=staged, **OPTS)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, np.full(p.m, D)), dx0) == 0
    b = np.random.default_rng(3).standard_normal(p.n)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s.backsolve(to_dev(torch, b), x)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    Kr, Kc, Kv = okkt.condensed_coo(p.n, W, J, pt.sigma, dx0, np.full(p.m, D))
    ref = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv).solve(b)
    K = sp.coo_matrix((Kv, (Kr, Kc)), shape=(p.n, p.n)).tocsr()
    xg = x.cpu().numpy()
    # backward error of the GPU solve on K, and agreement with the oracle's
    res = np.max(np.abs(K @ xg - b)) / (okkt.inf_norm(K) * np.max(np.abs(xg)) + np.max(np.abs(b)))
    assert res <= 1e-15, res
    if D < 1e3:
        assert np.max(np.abs(xg - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("k,T,opts", [(32, 50, OPTS), (8, 400, dict(leaf_size=16, subtree_cols=16)),
                                       (16, 120, dict(subtree_cols=0))])
def test_dataflow_solves_repeat_and_match_the_oracle(k, T, opts, mode):
    """The dataflow triangular solves (staged_solve 2: one launch per
    direction; 3: the subtree tasks in their own launches) re-arm their
    arrival counters and epochs: five solves in a row with different right-
    hand sides each match the oracle's factor substitution, on a tree with
    subtree tasks and many levels, and on one without subtree tasks; each
    K^{-1} costs four launches (gather, forward, backward, scatter), two
    more with the subtree tasks apart."""
    torch = torch_cuda()
    p, pt, W, J = instance(k, T, 1, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", staged_solve=mode, **opts)
    D = np.full(p.m, 1e2)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma), to_dev(torch, D), 1.0) == 0
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)   # K^{-1} b does not depend on the ordering
    Kr, Kc, Kv = okkt.condensed_coo(p.n, W, J, pt.sigma, 1.0, D)
    chol = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv)
    rng = np.random.default_rng(11)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    for rep in range(5):
        b = rng.standard_normal(p.n) * 10.0 ** rep
        s.reset_stats()
        s.backsolve(to_dev(torch, b), x)
        assert s.stats()["launches"] in ((4,) if mode == 2 else (4, 6))
        ref = chol.solve(b)
        xg = x.cpu().numpy()
        assert np.max(np.abs(xg - ref)) <= 1e-10 * np.max(np.abs(ref)), rep
    s.close()


def _solve(p, pt, W, J, scheme, delta_x=0.0, D=None, **opts):
    torch = torch_cuda()
    o = dict(OPTS)
    o.update(opts)
    s = solver_for(p, W, J, scheme=scheme, **o)
    st = s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  None if D is None else to_dev(torch, D), delta_x)
    assert st == 0, s.last_error()
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    ds = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy, ds)
    return st, s.info.as_dict(), dx.cpu().numpy(), dy.cpu().numpy(), ds.cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lifted_config1_backward_error(seed):
    """Config 1 (32 trays, T = 50, Sigma in [1e-6, 1e6], delta = 1e-8):
    eta <= 1e-10 reported by the library and recomputed by the oracle."""
    p, pt, W, J = instance(32, 50, seed)
    st, info, dx, dy, _ = _solve(p, pt, W, J, "lifted")
    assert st == 0 and info["bwd_err"] <= 1e-10
    assert oracle_eta(p, W, J, pt.sigma, 0.0, dx, dy, pt.rx, pt.ry) <= 1e-10


@pytest.mark.parametrize("seed", [0, 1])
def test_lifted_config1_agrees_with_dense(seed):
    """Refined to the floor of the FP64 residual (stopped by stagnation),
    Lifted-KKT agrees with the dense LU solution of K_orig to 1e-8 relative
    although cond(K_orig) ~ 1e14 here."""
    p, pt, W, J = instance(32, 50, seed)
    st, info, dx, dy, _ = _solve(p, pt, W, J, "lifted", tol_refine=1e-40, max_refine=40)
    assert st in (0, -5, -6)
    K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 0.0)
    v = okkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]), refine_steps=4)
    err = np.max(np.abs(np.concatenate([dx, dy]) - v)) / np.max(np.abs(v))
    assert err <= 1e-8, (err, info)


@pytest.mark.parametrize("gamma", [1e7, 1e4])
def test_hykkt_config1(gamma):
    p, pt, W, J = instance(32, 50, 0)
    st, info, dx, dy, _ = _solve(p, pt, W, J, "hykkt", gamma=gamma, max_cg=500)
    assert info["bwd_err"] <= 1e-10
    assert oracle_eta(p, W, J, pt.sigma, 0.0, dx, dy, pt.rx, pt.ry) <= 1e-10
    if gamma == 1e7:
        K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 0.0)
        v = okkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]), refine_steps=4)
        err = np.max(np.abs(np.concatenate([dx, dy]) - v)) / np.max(np.abs(v))
        assert err <= 1e-8
        assert info["cg_iters"] <= 60


def test_hykkt_matches_oracle_iterations():
    """Same algorithm, same stopping rule: CG iteration counts of the GPU
    and the oracle agree within one (rounding may move the last test)."""
    p, pt, W, J = instance(32, 20, 3, sigma_range=(1e-2, 1e2))
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    ox, oy, oinfo = okkt.hykkt_solve(sym, p.n, p.m, W, J, pt.sigma, 0.0, 1e4, pt.rx, pt.ry)
    st, info, dx, dy, _ = _solve(p, pt, W, J, "hykkt", gamma=1e4)
    assert abs(info["cg_iters"] - oinfo.cg_iters) <= 1
    v = np.concatenate([ox, oy])
    assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-8 * np.max(np.abs(v))


def test_lifted_relaxed_target_exact():
    p, pt, W, J = instance(8, 9, 4, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e6) * (1 + np.arange(p.m) % 3)
    st, info, dx, dy, ds = _solve(p, pt, W, J, "lifted", delta_x=30.0, D=D, target_relaxed=1)
    assert st == 0 and info["refine_iters"] <= 1
    K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 30.0, C=1.0 / D)
    v = okkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]))
    assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-9 * np.max(np.abs(v))
    Jm = okkt.jacobian_matrix(p.n, p.m, J)
    assert np.allclose(ds, Jm @ dx - pt.ry, rtol=1e-12, atol=1e-12 * np.max(np.abs(ds)))


@pytest.mark.parametrize("k,T", [(3, 0), (4, 1), (32, 0)])
def test_edge_sizes(k, T):
    """Degenerate horizons: one stage, two stages, tiny columns."""
    p, pt, W, J = instance(k, T, 5, sigma_range=(1e-2, 1e2))
    for scheme in ("lifted", "hykkt"):
        st, info, dx, dy, _ = _solve(p, pt, W, J, scheme, delta_x=10.0, gamma=1e7,
                                     tol_refine=1e-16)
        assert st == 0
        K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, 10.0)
        v = okkt.dense_solve(K, np.concatenate([pt.rx, pt.ry]))
        assert np.max(np.abs(np.concatenate([dx, dy]) - v)) <= 1e-8 * np.max(np.abs(v))


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (5, 3), (9, 8)])
def test_smallest_general_patterns(n, m):
    """Systems that are not column models, down to one variable and one
    constraint (one supernode, a 1 x 1 Schur complement), with every J row
    touching one or two variables."""
    torch = torch_cuda()
    from paper_2403_15913_gb300 import KKTSolver
    rng = np.random.default_rng(10 * n + m)
    lower = [sorted(set([j] + [int(i) for i in rng.integers(j, n, 2)])) for j in range(n)]
    Wc = np.cumsum([0] + [len(l) for l in lower]).astype(np.int64)
    Wr = np.concatenate(lower).astype(np.int64)
    Wv = np.array([float(n + 1) if i == j else rng.uniform(-1, 1)
                   for j in range(n) for i in lower[j]])
    # row r touches variable r % n (so J has full row rank for m <= n) and maybe one more
    rows = [sorted(set([r % n] + ([int(rng.integers(0, n))] if rng.random() < 0.5 else [])))
            for r in range(m)]
    Jr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    Jc = np.concatenate(rows).astype(np.int64)
    Jv = rng.uniform(0.5, 1.5, len(Jc)) * rng.choice([-1.0, 1.0], len(Jc))
    sigma = rng.uniform(0.1, 1.0, n)
    rx, ry = rng.standard_normal(n), rng.standard_normal(m)
    K = okkt.kkt_matrix(n, m, (Wc, Wr, Wv), (Jr, Jc, Jv), sigma, 0.0)
    v = okkt.dense_solve(K, np.concatenate([rx, ry]))
    for scheme in ("lifted", "hykkt"):
        s = KKTSolver(n, m, Wc, Wr, Jr, Jc, scheme=scheme, gamma=1e4, tol_refine=1e-14, **OPTS)
        assert s.factor(to_dev(torch, Wv), to_dev(torch, Jv), to_dev(torch, sigma), None, 0.0) == 0
        dx = torch.zeros(n, dtype=torch.float64, device="cuda")
        dy = torch.zeros(m, dtype=torch.float64, device="cuda")
        st = s.solve(to_dev(torch, rx), to_dev(torch, ry), dx, dy)
        assert st in (0, -6), s.last_error()       # STALL: at the rounding floor
        got = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
        assert np.max(np.abs(got - v)) <= 1e-9 * np.max(np.abs(v)), scheme
        s.close()


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_full_size_workload_backward_error(scheme):
    """The benchmark workload (32 trays, T = 5000, n = 325,065) in the
    benchmark's launch configuration: the backward error recomputed by the
    oracle on the CPU is <= 1e-10 (inputs computed by the oracle model)."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 5000, 0)
    s = solver_for(p, W, J, scheme=scheme, gamma=1e7, max_cg=500, **OPTS)
    Wv, Jv, sigma = to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma)
    st = s.factor(Wv, Jv, sigma, None, 0.0)
    delta_x = 0.0
    while st == -4:
        delta_x = 1e-4 if delta_x == 0 else delta_x * 8
        st = s.factor(Wv, Jv, sigma, None, delta_x)
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert s.info.bwd_err <= 1e-10
    eta = oracle_eta(p, W, J, pt.sigma, delta_x, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry)
    assert eta <= 1e-10
