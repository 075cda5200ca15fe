"""The one-graph step (kkt_factor_solve): the factorisation and the refined
solve of a batch as one CUDA graph launch, the refinement sweeps and the CG
iterations as conditional WHILE nodes.  It must give what kkt_factor_batch +
kkt_solve give (same stopping rules, same per-instance results), meet the
FP64 bar on every instance (eta <= 1e-10 recomputed by the oracle), replay
correctly with new values in the same buffers, and keep failures per
instance."""
import numpy as np
import pytest

from tests.gpu_common import ensure_built, oracle_eta, solver_for, to_dev, torch_cuda
from tests.test_gpu_batch import OPTS, SPECS, batch_solver, cat, make_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _inputs(torch, batch, Wscale=1.0):
    Wv = cat(torch, [W[2] * Wscale for _, _, W, _ in batch])
    Jv = cat(torch, [J[2] for _, _, _, J in batch])
    sig = cat(torch, [pt.sigma for _, pt, _, _ in batch])
    rx = cat(torch, [pt.rx for _, pt, _, _ in batch])
    ry = cat(torch, [pt.ry for _, pt, _, _ in batch])
    return Wv, Jv, sig, rx, ry


def _split(s, dx, dy, count):
    xo, yo = s.layout()
    return ([dx[xo[i]:xo[i + 1]].cpu().numpy() for i in range(count)],
            [dy[yo[i]:yo[i + 1]].cpu().numpy() for i in range(count)])


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_graph_step_matches_factor_then_solve(scheme):
    """Same statuses, refinement sweeps within one (CG iterations within
    one), solutions within the step-agreement bar 1e-8 relative (the two
    factors differ only by the order of atomic updates), eta <= 1e-10 by
    the oracle, and one graph launch per call."""
    torch = torch_cuda()
    batch = make_batch(SPECS)
    o = dict(scheme=scheme, gamma=1e7, max_cg=500)
    delta = np.full(len(batch), 10.0)
    Wv, Jv, sig, rx, ry = _inputs(torch, batch)
    ref = batch_solver(batch, **o)
    assert ref.factor_batch(Wv, Jv, sig, None, delta) == 0
    dx0 = torch.zeros(ref.n, dtype=torch.float64, device="cuda")
    dy0 = torch.zeros(ref.m, dtype=torch.float64, device="cuda")
    assert ref.solve(rx, ry, dx0, dy0) == 0
    r0 = ref.results()

    s = batch_solver(batch, **o)
    dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    assert s.factor_solve(Wv, Jv, sig, None, delta, rx, ry, dx, dy) == 0
    r = s.results()
    assert np.array_equal(r["status"], r0["status"])
    assert np.all(np.abs(r["refine_iters"] - r0["refine_iters"]) <= 1)
    if scheme == "hykkt":
        assert np.all(np.abs(r["cg_iters"] - r0["cg_iters"]) <= len(SPECS))
        assert np.all(r["cg_iters"] > 0)
    assert np.all(r["bwd_err"] <= 1e-10) and np.all(r["failed_col"] == -1)
    g = np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()])
    v = np.concatenate([dx0.cpu().numpy(), dy0.cpu().numpy()])
    assert np.max(np.abs(g - v)) <= 1e-8 * np.max(np.abs(v))
    xs, ys = _split(s, dx, dy, len(batch))
    for i, (p, pt, W, J) in enumerate(batch):
        assert oracle_eta(p, W, J, pt.sigma, 10.0, xs[i], ys[i], pt.rx, pt.ry) <= 1e-10
    st = s.stats()
    assert st["graph_steps"] == 1 and st["factor_calls"] == 1 and st["launches"] > 0


def test_graph_step_replays_with_new_values():
    """Second and third calls on the same buffers replay the captured graph
    (new W values, new right-hand sides, new delta_x): each result meets
    the bar against its own system."""
    torch = torch_cuda()
    batch = make_batch(SPECS[:4], seed0=5)
    s = batch_solver(batch, scheme="lifted")
    Wv, Jv, sig, rx, ry = _inputs(torch, batch)
    dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(1)
    for call, (scale, dval) in enumerate([(1.0, 10.0), (1.5, 3.0), (0.5, 30.0)]):
        Wn, _, _, rxn, ryn = _inputs(torch, batch, Wscale=scale)
        Wv.copy_(Wn)
        rx.copy_(rxn * (1 + call))
        ry.copy_(ryn * (1 - 0.5 * call))
        delta = np.full(len(batch), dval) * (1 + rng.random(len(batch)))
        assert s.factor_solve(Wv, Jv, sig, None, delta, rx, ry, dx, dy) == 0
        xs, ys = _split(s, dx, dy, len(batch))
        for i, (p, pt, W, J) in enumerate(batch):
            Ws = (W[0], W[1], W[2] * scale)
            assert oracle_eta(p, Ws, J, pt.sigma, delta[i], xs[i], ys[i], pt.rx * (1 + call),
                              pt.ry * (1 - 0.5 * call)) <= 1e-10, (call, i)
    assert s.stats()["graph_steps"] == 3


def test_graph_step_failure_is_per_instance():
    """An indefinite instance fails alone (NOT_SPD, its first failing
    column in its own range); the others are solved to the bar; a larger
    delta_x for that instance alone repairs it on the next replay."""
    torch = torch_cuda()
    batch = make_batch(SPECS[:5])
    p, pt, W, J = batch[2]
    Wbad = W[2].copy()
    Wbad[W[0][p.n // 2]] -= 1e12
    batch[2] = (p, pt, (W[0], W[1], Wbad), J)
    s = batch_solver(batch, scheme="lifted")
    Wv, Jv, sig, rx, ry = _inputs(torch, batch)
    dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    delta = np.full(len(batch), 1.0)
    assert s.factor_solve(Wv, Jv, sig, None, delta, rx, ry, dx, dy) == -4
    r = s.results()
    xo, _ = s.layout()
    assert xo[2] <= r["failed_col"][2] < xo[3] and np.all(np.delete(r["failed_col"], 2) == -1)
    assert r["status"][2] == -4 and np.all(np.delete(r["status"], 2) == 0)
    xs, ys = _split(s, dx, dy, len(batch))
    for i in (0, 1, 3, 4):
        q, qt, Wq, Jq = batch[i]
        assert oracle_eta(q, Wq, Jq, qt.sigma, 1.0, xs[i], ys[i], qt.rx, qt.ry) <= 1e-10
    delta[2] = 1e13
    assert s.factor_solve(Wv, Jv, sig, None, delta, rx, ry, dx, dy) == 0
    xs, ys = _split(s, dx, dy, len(batch))
    for i, (q, qt, Wq, Jq) in enumerate(batch):
        assert oracle_eta(q, Wq, Jq, qt.sigma, delta[i], xs[i], ys[i], qt.rx, qt.ry) <= 1e-10


def test_graph_step_single_system_and_relaxed_target():
    """A kkt_analyse context (one system, delta_x a float) with the relaxed
    target C = 1/D: the same answer as factor + solve, eta <= 1e-10 on the
    relaxed system; kkt_solve can follow with the factor left behind."""
    torch = torch_cuda()
    (p, pt, W, J), = make_batch([(32, 40)], seed0=9)
    D = np.full(p.m, 1e2)
    o = dict(OPTS, scheme="lifted", target_relaxed=1)
    a = solver_for(p, W, J, **o)
    args = [to_dev(torch, v) for v in (W[2], J[2], pt.sigma, D)]
    rx, ry = to_dev(torch, pt.rx), to_dev(torch, pt.ry)
    assert a.factor(*args, 10.0) == 0
    ax = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    ay = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    assert a.solve(rx, ry, ax, ay) == 0
    b = solver_for(p, W, J, **o)
    bx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    by = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    assert b.factor_solve(*args, 10.0, rx, ry, bx, by) == 0
    assert b.info.bwd_err <= 1e-10 and b.info.delta_x == 10.0
    v = np.concatenate([ax.cpu().numpy(), ay.cpu().numpy()])
    g = np.concatenate([bx.cpu().numpy(), by.cpu().numpy()])
    assert np.max(np.abs(g - v)) <= 1e-8 * np.max(np.abs(v))
    assert oracle_eta(p, W, J, pt.sigma, 10.0, g[:p.n], g[p.n:], pt.rx, pt.ry, C=1.0 / D) <= 1e-10
    cx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    cy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    assert b.solve(rx, ry, cx, cy) == 0
    c = np.concatenate([cx.cpu().numpy(), cy.cpu().numpy()])
    assert np.max(np.abs(c - g)) <= 1e-8 * np.max(np.abs(g))


def test_graph_step_rejects_other_settings():
    """FP32 factors and the block-tridiagonal solver are not captured: the
    call is refused with KKT_ERR_ARG before any work."""
    torch = torch_cuda()
    from paper_2403_15913_gb300 import KKTError
    batch = make_batch(SPECS[:2])
    s = batch_solver(batch, scheme="lifted", precision=1)
    Wv, Jv, sig, rx, ry = _inputs(torch, batch)
    dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    with pytest.raises(KKTError):
        s.factor_solve(Wv, Jv, sig, None, np.ones(2), rx, ry, dx, dy)
