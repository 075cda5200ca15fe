"""Receding-horizon serving: per-tray initial state against the oracle IPM,
shifted warm starts, the same answer alone and in a busy mix of concurrent
clients, admission under a device-memory budget (eviction), per-client
order."""
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


def x0_for(k, seed):
    return np.random.default_rng(seed).uniform(0.15, 0.85, k)


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_initial_state_matches_oracle_ipm(scheme):
    """A per-tray initial state: the device IPM and the oracle IPM take the
    same iterations to the same optimum, whose stage-0 compositions are x0."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=8, T=10)
    x0 = x0_for(p.k, 1)
    mdl = oipm.TrayModel(p, x0)
    w0 = ipm_start(p)
    W = tray.hessian_lower_csc(p, w0, np.zeros(p.m))
    J = tray.jacobian_csr(p, w0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **OPTS)
    lin = oipm.KKTLinearSolver(scheme, p.n, p.m, None, None, sym=sym, gamma=1e4)
    o = oipm.IPM(mdl, lin, oipm.IPMOptions(relaxed=(scheme == "lifted")), w0)
    last = o.solve()
    assert last.status == "converged"
    g = IPMSolver(p.as_array(), scheme=scheme, **OPTS)
    g.set_initial_state(x0)
    g.init()
    hist = g.solve()
    assert hist[-1]["status"] == 1
    assert hist[-1]["iter"] == last.it
    x = g.get()[0].cpu().numpy()
    assert abs(hist[-1]["objective"] - last.obj) <= 1e-8 * abs(last.obj)
    assert np.max(np.abs(x - o.x)) <= 1e-6
    tol = 1e-8 if scheme == "hykkt" else 2e-8    # relaxed equalities: |c| <= tau
    assert np.max(np.abs(x[:p.k] - x0)) <= tol


def test_shifted_warm_start_reaches_cold_optimum():
    """Second receding-horizon solve: from the previous solution shifted one
    stage, with stage 0 pinned to stage 1 of that solution, the IPM reaches
    the optimum a cold start reaches."""
    torch = torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver
    p = TrayParams(k=16, T=30)
    a = IPMSolver(p.as_array(), scheme="lifted", **OPTS)
    a.set_initial_state(x0_for(p.k, 2))
    a.init()
    assert a.solve()[-1]["status"] == 1
    prev = a.get()[0].clone()
    x1 = prev[2 * p.k + 1:2 * p.k + 1 + p.k].cpu().numpy()
    a.set_initial_state(x1)
    a.init_shifted(prev)
    hw = a.solve()
    assert hw[-1]["status"] == 1
    xw = a.get()[0].cpu().numpy()
    b = IPMSolver(p.as_array(), scheme="lifted", **OPTS)
    b.set_initial_state(x1)
    b.init()
    hc = b.solve()
    assert hc[-1]["status"] == 1
    xc = b.get()[0].cpu().numpy()
    assert np.max(np.abs(xw - xc)) <= 1e-6
    assert abs(hw[-1]["objective"] - hc[-1]["objective"]) <= 1e-8 * abs(hc[-1]["objective"])
    # full warm start: the first solve's whole primal-dual iterate shifted
    # one stage, small barrier parameter; fewer iterations, same optimum
    c = IPMSolver(p.as_array(), scheme="lifted", **OPTS)
    c.set_initial_state(x0_for(p.k, 2))
    c.init()
    assert c.solve()[-1]["status"] == 1
    c.set_initial_state(x1)
    c.init_warm(1e-4)
    hf = c.solve()
    assert hf[-1]["status"] == 1
    xf = c.get()[0].cpu().numpy()
    assert np.max(np.abs(xf - xc)) <= 1e-6
    assert hf[-1]["iter"] < hc[-1]["iter"], (hf[-1]["iter"], hc[-1]["iter"])


def _clients(rng, count):
    return [TrayParams(k=int(rng.choice([8, 16])), T=int(rng.integers(10, 41))) for _ in range(count)]


def test_same_answer_alone_and_in_the_mix():
    """The target request solved on an idle 1-slot server and on an 8-slot
    server busy with 40 requests of 10 other clients: same iterations and
    the same solution to 1e-7 (only the order of atomic updates in the
    factorisation differs, as between two runs alone)."""
    torch_cuda()
    from paper_2403_15913_gb300 import NMPCServer
    rng = np.random.default_rng(5)
    target = TrayParams(k=16, T=25)
    x0 = x0_for(target.k, 3)
    alone = NMPCServer(slots=1)
    c = alone.add_client(target.as_array())
    ra, xa = alone.wait(alone.submit(c, x0, keep_solution=True), want_solution=True)
    alone.close()
    mix = NMPCServer(slots=8)
    others = [mix.add_client(p.as_array()) for p in _clients(rng, 10)]
    ct = mix.add_client(target.as_array())
    tickets = [mix.submit(others[i % 10]) for i in range(20)]
    tt = mix.submit(ct, x0, keep_solution=True)
    tickets += [mix.submit(others[i % 10]) for i in range(20)]
    rm, xm = mix.wait(tt, want_solution=True)
    for t in tickets:
        assert mix.wait(t)["status"] == 1
    st = mix.stats()
    mix.close()
    assert ra["status"] == 1 and rm["status"] == 1
    assert ra["iters"] == rm["iters"]
    assert np.max(np.abs(xa - xm)) <= 1e-7
    assert st["completed"] == 41 and st["failed"] == 0


def test_budget_admission_evicts_and_keeps_order():
    """A budget that holds about two contexts: contexts are evicted and
    recreated, the resident peak stays within the budget, every request
    converges, and each client's requests run in submission order."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMSolver, NMPCServer
    rng = np.random.default_rng(9)
    params = [TrayParams(k=16, T=int(rng.integers(20, 41))) for _ in range(6)]
    big = max(params, key=lambda q: q.n)
    probe = IPMSolver(big.as_array(), scheme="lifted", **OPTS)
    one = probe.device_bytes() + big.n * 8
    probe.close() if hasattr(probe, "close") else None
    budget_gb = 2.5 * one / 1e9
    srv = NMPCServer(slots=4, hbm_budget_gb=budget_gb)
    cl = [srv.add_client(q.as_array()) for q in params]
    tickets = [srv.submit(cl[i % 6]) for i in range(24)]
    res = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 1 for r in res)
    assert st["evictions"] > 0 and st["contexts_created"] > 6
    assert st["peak_resident_bytes"] <= budget_gb * 1e9
    by_client = {}
    for r in res:
        by_client.setdefault(r["client"], []).append(r)
    for rs in by_client.values():
        rs.sort(key=lambda r: r["id"])
        for a, b in zip(rs, rs[1:]):
            assert b["t_start_ms"] >= a["t_done_ms"]
