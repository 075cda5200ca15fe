"""GPU IPM driver against the oracle IPM (same algorithm, same linear
solver family): same iteration count, same optimum; at the benchmark size,
the solution is checked by the oracle model (constraint violation, objective
and stationarity) on the CPU."""
import numpy as np
import pytest

from gen.tray import TrayParams, ipm_start
from oracle import ipm as oipm, symbolic, tray
from tests.gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _oracle(p, scheme):
    mdl = oipm.TrayModel(p)
    x0 = ipm_start(p)
    W = tray.hessian_lower_csc(p, x0, np.zeros(p.m))
    J = tray.jacobian_csr(p, x0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    lin = oipm.KKTLinearSolver(scheme, p.n, p.m, None, None, sym=sym, gamma=1e4)
    s = oipm.IPM(mdl, lin, oipm.IPMOptions(relaxed=(scheme == "lifted")), x0)
    return s, s.solve()


@pytest.mark.parametrize("scheme", ["hykkt", "lifted"])
@pytest.mark.parametrize("k,T", [(8, 10), (32, 20)])
def test_gpu_ipm_matches_oracle(scheme, k, T):
    torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=k, T=T)
    os_, olast = _oracle(p, scheme)
    assert olast.status == "converged"
    g = IPMSolver(p.as_array(), scheme=scheme, **OPTS)
    g.init()
    hist = g.solve()
    assert hist[-1]["status"] == 1, hist[-1]
    iters = hist[-1]["iter"]
    assert iters == olast.it, (iters, olast.it)
    x, y, zl, zu, s = g.get()
    x = x.cpu().numpy()
    assert abs(hist[-1]["objective"] - olast.obj) <= 1e-8 * abs(olast.obj)
    assert np.max(np.abs(x - os_.x)) <= 1e-6
    # the first iterations follow the same path
    for a, b in zip(hist[:3], os_.history[:3]):
        assert abs(a["objective"] - b.obj) <= 1e-9 * max(1.0, abs(b.obj))


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_gpu_ipm_full_size(scheme):
    """Benchmark workload (32 trays, T = 5000): the IPM converges and the
    oracle model confirms feasibility and stationarity of the result."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=32, T=5000)
    g = IPMSolver(p.as_array(), scheme=scheme, **OPTS)
    g.init()
    hist = g.solve()
    assert hist[-1]["status"] == 1, hist[-1]
    x, y, zl, zu, s = g.get()
    x, y, zl, zu = (t.cpu().numpy() for t in (x, y, zl, zu))
    c = tray.constraints(p, x)
    tol_c = 2e-8 * (1 + 1e-6) if scheme == "lifted" else 1e-8   # |c| <= tau + tol (relaxed)
    assert np.max(np.abs(c)) <= tol_c
    assert abs(tray.objective(p, x) - hist[-1]["objective"]) <= 1e-10 * abs(hist[-1]["objective"])
    r, cc, v = tray.jacobian_coo(p, x)
    jty = np.zeros(p.n)
    np.add.at(jty, cc, v * y[r])
    du = tray.objective_grad(p, x) + jty - zl + zu
    assert np.max(np.abs(du)) <= 1e-6
    assert all(h["bwd_err"] <= 1e-10 for h in hist[:-1])
