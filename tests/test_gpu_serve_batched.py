"""Batched serving (kkt_server_options.batch > 0): cohorts of clients share
one batched IPM whose every iteration factorises and solves the union of
their running requests' KKT systems once, with requests joining and leaving
between iterations.  Each request's result must be the one it gets alone:
the same iterations and solution as on an idle per-instance server, alone
in its cohort and in a busy mix; with the FP32 factor and FP64 refinement
the optimum is the FP64 one; a cohort budget evicts whole cohorts and keeps
each client's requests in order; a member that joins a running batch
follows the single-problem IPM."""
import numpy as np
import pytest

from gen.tray import TrayParams
from tests.gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def x0_for(k, seed):
    return np.random.default_rng(seed).uniform(0.15, 0.85, k)


def _clients(rng, count):
    return [TrayParams(k=int(rng.choice([8, 16])), T=int(rng.integers(10, 41))) for _ in range(count)]


def _alone(target, x0, **srv):
    from paper_2403_15913_gb300 import NMPCServer
    s = NMPCServer(**srv)
    c = s.add_client(target.as_array())
    r, x = s.wait(s.submit(c, x0, keep_solution=True), want_solution=True)
    s.close()
    return r, x


def test_batched_server_same_answer_alone_and_in_the_mix():
    """The target request: on an idle per-instance server, alone in a batched
    server, and in a batched server whose three cohorts are busy with 40
    requests of 11 other clients -- same status, iterations and solution to
    1e-7."""
    torch_cuda()
    from paper_2403_15913_gb300 import NMPCServer
    rng = np.random.default_rng(5)
    target = TrayParams(k=16, T=25)
    x0 = x0_for(target.k, 3)
    ra, xa = _alone(target, x0, slots=1)
    rb, xb = _alone(target, x0, slots=1, batch=4)
    mix = NMPCServer(slots=3, batch=4)
    others = [mix.add_client(p.as_array()) for p in _clients(rng, 11)]
    ct = mix.add_client(target.as_array())
    tickets = [mix.submit(others[i % 11]) for i in range(20)]
    tt = mix.submit(ct, x0, keep_solution=True)
    tickets += [mix.submit(others[i % 11]) for i in range(20)]
    rm, xm = mix.wait(tt, want_solution=True)
    res = [mix.wait(t) for t in tickets]
    st = mix.stats()
    mix.close()
    assert all(r["status"] == 1 for r in res)
    assert ra["status"] == 1 and rb["status"] == 1 and rm["status"] == 1
    assert ra["iters"] == rb["iters"] == rm["iters"], (ra["iters"], rb["iters"], rm["iters"])
    assert np.max(np.abs(xa - xb)) <= 1e-7
    assert np.max(np.abs(xa - xm)) <= 1e-7
    assert abs(ra["objective"] - rm["objective"]) <= 1e-8 * abs(ra["objective"])
    assert st["completed"] == 41 and st["failed"] == 0
    assert st["contexts_created"] == 3   # cohorts of 4, 4, 4 clients


def test_batched_fp32_factor_reaches_the_fp64_optimum():
    """Batched serving with the FP32 factor of the union and FP64 refinement:
    every request converges to tol, and its optimum agrees with the FP64
    per-instance server's to 1e-8 in the objective (equal accuracy)."""
    torch_cuda()
    from paper_2403_15913_gb300 import NMPCServer
    rng = np.random.default_rng(7)
    params = _clients(rng, 6)
    x0s = [x0_for(p.k, 10 + i) for i, p in enumerate(params)]
    out = {}
    for name, kw in (("fp64", dict(slots=2)), ("fp32", dict(slots=2, batch=3, precision=1))):
        s = NMPCServer(**kw)
        cl = [s.add_client(p.as_array()) for p in params]
        tk = [s.submit(cl[i], x0s[i], keep_solution=True) for i in range(6)]
        out[name] = [s.wait(t, want_solution=True) for t in tk]
        s.close()
    for (r64, x64), (r32, x32) in zip(out["fp64"], out["fp32"]):
        assert r64["status"] == 1 and r32["status"] == 1
        assert abs(r32["objective"] - r64["objective"]) <= 1e-8 * abs(r64["objective"])
        assert np.max(np.abs(x32 - x64)) <= 1e-5


def test_batched_warm_starts_follow_the_per_instance_server():
    """Three receding-horizon requests per client (each warm-started from the
    client's previous solution): the batched server takes the same
    iterations and reaches the same solutions as the per-instance one."""
    torch_cuda()
    from paper_2403_15913_gb300 import NMPCServer
    rng = np.random.default_rng(11)
    params = _clients(rng, 4)
    out = {}
    for name, kw in (("single", dict(slots=2)), ("batched", dict(slots=1, batch=4))):
        s = NMPCServer(**kw)
        cl = [s.add_client(p.as_array()) for p in params]
        res = []
        for rnd in range(3):
            tk = [s.submit(cl[i], x0_for(params[i].k, 100 * rnd + i) if rnd == 0 else None, keep_solution=True)
                  for i in range(4)]
            res.append([s.wait(t, want_solution=True) for t in tk])
        out[name] = res
        s.close()
    for rnd in range(3):
        for (ra, xa), (rb, xb) in zip(out["single"][rnd], out["batched"][rnd]):
            assert ra["status"] == 1 and rb["status"] == 1
            assert ra["iters"] == rb["iters"], (rnd, ra["iters"], rb["iters"])
            assert (ra["warm"], rb["warm"]) == ((0, 0) if rnd == 0 else (1, 1))
            assert np.max(np.abs(xa - xb)) <= 1e-7


def test_batched_budget_evicts_cohorts_and_keeps_order():
    """A budget that holds about one cohort, requests in rounds over all six
    clients of two cohorts: cohorts are evicted and rebuilt every round (a
    cohort runs every queued request of its clients before it is released),
    the resident peak stays within the budget, every request converges and
    each client's requests run in submission order."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch, NMPCServer
    rng = np.random.default_rng(9)
    params = [TrayParams(k=16, T=int(rng.integers(20, 41))) for _ in range(6)]
    one = 0
    for part in (params[:3], params[3:]):
        probe = IPMBatch([p.as_array() for p in part], scheme="lifted", **OPTS)
        one = max(one, probe.device_bytes() + sum(p.n for p in part) * 8)
        probe.close()
    budget_gb = 1.6 * one / 1e9
    srv = NMPCServer(slots=2, batch=3, hbm_budget_gb=budget_gb)
    cl = [srv.add_client(q.as_array()) for q in params]
    res = []
    for _ in range(4):
        tickets = [srv.submit(cl[i]) for i in range(6)]
        res += [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 1 for r in res)
    assert st["evictions"] >= 3 and st["contexts_created"] >= 4
    assert st["peak_resident_bytes"] <= budget_gb * 1e9
    by_client = {}
    for r in res:
        by_client.setdefault(r["client"], []).append(r)
    for rs in by_client.values():
        rs.sort(key=lambda r: r["id"])
        for a, b in zip(rs, rs[1:]):
            assert b["t_start_ms"] >= a["t_done_ms"]


def test_member_joining_a_running_batch_follows_the_single_ipm():
    """Continuous batching in kkt_ipm_batch: member 1 starts three
    iterations after member 0 and member 2 after member 0 converged; each
    takes the single-problem IPM's iterations to its optimum."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch, IPMSolver
    ps = [TrayParams(k=8, T=20), TrayParams(k=16, T=12), TrayParams(k=8, T=30)]
    b = IPMBatch([p.as_array() for p in ps], scheme="lifted", **OPTS)
    b.members[0].init()
    b.start_member(0)
    ticks = 0
    while True:
        if ticks == 3:
            b.members[1].init()
            b.start_member(1)
        if b.member_status(0)[0] != 0 and b.member_status(2)[0] == -8:
            b.members[2].init()
            b.start_member(2)
        st = b.step()
        ticks += 1
        if st == 1 and all(b.member_status(i)[0] != 0 for i in range(3)) and b.member_status(2)[0] != -8:
            break
        assert st in (0, 1) and ticks < 200
    for i, p in enumerate(ps):
        g = IPMSolver(p.as_array(), scheme="lifted", **OPTS)
        g.init()
        hist = g.solve()
        status, iters = b.member_status(i)
        assert status == 1 and hist[-1]["status"] == 1
        assert iters == hist[-1]["iter"], (i, iters, hist[-1]["iter"])
        assert np.max(np.abs(b.members[i].get()[0].cpu().numpy() - g.get()[0].cpu().numpy())) <= 1e-6
        g.close()
    b.close()


def test_batched_hykkt_server_follows_the_per_instance_server():
    """HyKKT in batched serving (CG per instance on the union's factor):
    each request takes the per-instance server's iterations to its optimum."""
    torch_cuda()
    from paper_2403_15913_gb300 import NMPCServer
    rng = np.random.default_rng(13)
    params = _clients(rng, 5)
    x0s = [x0_for(p.k, 40 + i) for i, p in enumerate(params)]
    out = {}
    for name, kw in (("single", dict(slots=2)), ("batched", dict(slots=2, batch=3))):
        s = NMPCServer(scheme="hykkt", **kw)
        cl = [s.add_client(p.as_array()) for p in params]
        tk = [s.submit(cl[i], x0s[i], keep_solution=True) for i in range(5)]
        out[name] = [s.wait(t, want_solution=True) for t in tk]
        s.close()
    for (ra, xa), (rb, xb) in zip(out["single"], out["batched"]):
        assert ra["status"] == 1 and rb["status"] == 1
        assert ra["iters"] == rb["iters"], (ra["iters"], rb["iters"])
        assert abs(ra["objective"] - rb["objective"]) <= 1e-8 * abs(ra["objective"])
        assert np.max(np.abs(xa - xb)) <= 1e-6
