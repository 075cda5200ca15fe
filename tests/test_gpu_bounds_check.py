"""The bounds-check build of the library (-DKKT_BOUNDS_CHECK=1): on sound
maps it factorises and solves exactly like the ordinary build (the oracle's
backward error bound holds); with one entry of the Schur-update row map
pointing one row past its target supernode -- a wrong index that still lies
inside the factor storage, so nothing is accessed out of bounds even where
a check were missing -- kkt_factor returns KKT_ERR_INTERNAL and names the
map, and the context works again once the entry is restored."""
import numpy as np
import pytest

from gen.tray import TrayParams, kkt_point
from oracle import kkt as okkt
from oracle import tray
from tests.gpu_common import to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked_lib():
    torch_cuda()
    from paper_2403_15913_gb300 import _native as nat
    from paper_2403_15913_gb300 import build
    L = nat.load(build.build(debug_checks=True))
    prev = nat.lib()
    nat._lib = L
    try:
        yield nat
    finally:
        nat._lib = prev


def _case(torch, nat, **opts):
    from paper_2403_15913_gb300 import KKTSolver
    p = TrayParams(k=8, T=20)
    pt = kkt_point(p, 3, sigma_range=(1e-2, 1e2))
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    s = KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1], scheme="lifted", **opts)
    vals = (to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma))
    return p, pt, W, J, s, vals


def test_checked_build_solves_like_the_ordinary_build(checked_lib):
    torch = torch_cuda()
    nat = checked_lib
    p, pt, W, J, s, (Wv, Jv, sv) = _case(torch, nat)
    delta_x = 10.0
    assert s.factor(Wv, Jv, sv, None, delta_x) == nat.KKT_OK
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    assert s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy) == nat.KKT_OK
    K = okkt.kkt_matrix(p.n, p.m, W, J, pt.sigma, delta_x)
    v = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    assert okkt.backward_error(K, v, np.concatenate([pt.rx, pt.ry])) <= 1e-10
    s.close()


def test_corrupted_row_map_is_reported_and_recoverable(checked_lib):
    torch = torch_cuda()
    nat = checked_lib
    from paper_2403_15913_gb300 import KKTError
    p, pt, W, J, s, (Wv, Jv, sv) = _case(torch, nat)
    L = nat.lib()
    assert L.kkt_debug_corrupt_map(s._ctx, 1) == nat.KKT_OK
    with pytest.raises(KKTError) as e:
        s.factor(Wv, Jv, sv, None, 10.0)
    assert e.value.status == nat.KKT_ERR_INTERNAL
    assert "relative row" in str(e.value)
    assert L.kkt_debug_corrupt_map(s._ctx, 0) == nat.KKT_OK
    assert s.factor(Wv, Jv, sv, None, 10.0) == nat.KKT_OK
    s.close()


def test_dataflow_wait_that_runs_out_is_reported_and_recoverable(checked_lib):
    """The waits of the dataflow triangular solves are bounded: with the
    arrival count of the tree's last item raised by one (no solve can meet
    it) the wait gives up after about a second, the kernel still completes,
    and the solve returns KKT_ERR_TIMEOUT; once restored, the context solves
    correctly again (its counters were reset)."""
    import time
    torch = torch_cuda()
    nat = checked_lib
    from paper_2403_15913_gb300 import KKTError
    p, pt, W, J, s, (Wv, Jv, sv) = _case(torch, nat, staged_solve=2)
    L = nat.lib()
    delta_x = 10.0
    assert s.factor(Wv, Jv, sv, None, delta_x) == nat.KKT_OK
    b = np.random.default_rng(5).standard_normal(p.n)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    assert L.kkt_debug_corrupt_map(s._ctx, 2) == nat.KKT_OK
    t0 = time.perf_counter()
    with pytest.raises(KKTError) as e:
        s.backsolve(to_dev(torch, b), x)
    waited = time.perf_counter() - t0
    assert e.value.status == nat.KKT_ERR_TIMEOUT
    assert "gave up" in str(e.value)
    assert 0.5 <= waited <= 20.0, waited
    assert L.kkt_debug_corrupt_map(s._ctx, 0) == nat.KKT_OK
    Kc = okkt.condensed_coo(p.n, W, J, pt.sigma, delta_x, np.full(p.m, 1e8))   # D = 1/delta (delta = 1e-8)
    import scipy.sparse as sp
    K = sp.coo_matrix((Kc[2], (Kc[0], Kc[1])), shape=(p.n, p.n)).tocsr()
    for _ in range(2):
        x.zero_()
        s.backsolve(to_dev(torch, b), x)
        xg = x.cpu().numpy()
        res = np.max(np.abs(K @ xg - b)) / (okkt.inf_norm(K) * np.max(np.abs(xg)) + np.max(np.abs(b)))
        assert res <= 1e-15, res
    s.close()


def test_ordinary_build_has_no_test_hook():
    torch_cuda()
    from paper_2403_15913_gb300 import _native as nat
    from paper_2403_15913_gb300 import build
    L = nat.load(build.LIB_PATH)
    assert L.kkt_debug_corrupt_map(None, 1) == nat.KKT_ERR_STATE
