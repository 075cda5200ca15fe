"""Block cyclic reduction (solver = 1) of the stage-block-tridiagonal
condensed matrix against the oracle: K^{-1} b, Lifted-KKT and HyKKT steps,
the IPM, pivot failure, and the patterns it must reject."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen.tray import TrayParams, ipm_start
from oracle import cholesky, ipm as oipm, kkt as okkt, symbolic, tray
from tests.gpu_common import ensure_built, instance, oracle_eta, solver_for, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def bcr(p, W, J, **o):
    return solver_for(p, W, J, solver=1, block=2 * p.k + 1, **OPTS, **o)


@pytest.mark.parametrize("k,T", [(32, 50), (5, 7), (3, 0), (4, 1), (16, 64)])
def test_bcr_backsolve_matches_oracle(k, T):
    """K^{-1} b by block cyclic reduction: backward error ~1e-16 on K and
    agreement with the oracle's sparse Cholesky solve."""
    torch = torch_cuda()
    p, pt, W, J = instance(k, T, 0, sigma_range=(1e-2, 1e2))
    D = np.full(p.m, 1e2)
    s = bcr(p, W, J, scheme="lifted")
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, D), 10.0) == 0
    b = np.random.default_rng(4).standard_normal(p.n)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s.backsolve(to_dev(torch, b), x)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    Kr, Kc, Kv = okkt.condensed_coo(p.n, W, J, pt.sigma, 10.0, D)
    ref = cholesky.SparseCholesky(sym, p.n, Kr, Kc, Kv).solve(b)
    K = sp.coo_matrix((Kv, (Kr, Kc)), shape=(p.n, p.n)).tocsr()
    xg = x.cpu().numpy()
    res = np.max(np.abs(K @ xg - b)) / (okkt.inf_norm(K) * np.max(np.abs(xg)) + np.max(np.abs(b)))
    assert res <= 1e-15, res
    assert np.max(np.abs(xg - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
@pytest.mark.parametrize("seed", [0, 1])
def test_bcr_kkt_step_config1(scheme, seed):
    """32 trays, T = 50, Sigma on [1e-6, 1e6]: eta <= 1e-10 recomputed by the
    oracle, and the same step as the supernodal path to 1e-8 relative."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 50, seed)
    out = {}
    for solver in (0, 1):
        o = dict(OPTS, scheme=scheme, gamma=1e7, max_cg=500, solver=solver, block=2 * p.k + 1)
        s = solver_for(p, W, J, **o)
        assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma), None, 0.0) == 0
        dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
        st = s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
        assert st == 0 and s.info.bwd_err <= 1e-10
        out[solver] = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
        assert oracle_eta(p, W, J, pt.sigma, 0.0, out[solver][:p.n], out[solver][p.n:], pt.rx, pt.ry) <= 1e-10
    assert np.max(np.abs(out[1] - out[0])) <= 1e-8 * np.max(np.abs(out[0]))


def test_bcr_not_spd():
    torch = torch_cuda()
    p, pt, W, J = instance(8, 12, seed=2)
    Wv = W[2].copy()
    Wv[W[0][p.n // 2]] -= 1e12
    s = bcr(p, W, J, scheme="lifted")
    st = s.factor(to_dev(torch, Wv), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  to_dev(torch, np.full(p.m, 1e2)), 0.0)
    assert st == -4 and 0 <= s.info.failed_col < p.n


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_bcr_ipm_matches_oracle(scheme):
    torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=8, T=10)
    w0 = ipm_start(p)
    W = tray.hessian_lower_csc(p, w0, np.zeros(p.m))
    J = tray.jacobian_csr(p, w0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    lin = oipm.KKTLinearSolver(scheme, p.n, p.m, None, None, sym=sym, gamma=1e4)
    o = oipm.IPM(oipm.TrayModel(p), lin, oipm.IPMOptions(relaxed=(scheme == "lifted")), w0)
    last = o.solve()
    g = IPMSolver(p.as_array(), scheme=scheme, solver=1, block=2 * p.k + 1, **OPTS)
    g.init()
    hist = g.solve()
    assert hist[-1]["status"] == 1 and hist[-1]["iter"] == last.it
    assert abs(hist[-1]["objective"] - last.obj) <= 1e-8 * abs(last.obj)
    assert np.max(np.abs(g.get()[0].cpu().numpy() - o.x)) <= 1e-6


def test_bcr_rejects_other_patterns():
    torch_cuda()
    from paper_2403_15913_gb300 import KKTError
    p, pt, W, J = instance(8, 6, 0)
    with pytest.raises(KKTError):   # block does not divide n
        solver_for(p, W, J, solver=1, block=2 * p.k, **OPTS)
    with pytest.raises(KKTError):   # blocks of 7 straddle stages of 17: not block tridiagonal
        solver_for(p, W, J, solver=1, block=7, **OPTS)


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_bcr_full_size_workload(scheme):
    """T = 5000 (n = 325,065): eta <= 1e-10 recomputed by the oracle."""
    torch = torch_cuda()
    p, pt, W, J = instance(32, 5000, 0)
    s = bcr(p, W, J, scheme=scheme, gamma=1e7, max_cg=500)
    Wv, Jv, sigma = to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma)
    st = s.factor(Wv, Jv, sigma, None, 0.0)
    delta_x = 0.0
    while st == -4:
        delta_x = 1e-4 if delta_x == 0 else delta_x * 8
        st = s.factor(Wv, Jv, sigma, None, delta_x)
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    assert s.info.bwd_err <= 1e-10
    assert oracle_eta(p, W, J, pt.sigma, delta_x, dx.cpu().numpy(), dy.cpu().numpy(), pt.rx, pt.ry) <= 1e-10
