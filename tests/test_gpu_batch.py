"""Batches of uneven KKT systems solved together (kkt_analyse_batch): every
instance meets the FP64 bar (eta <= 1e-10, recomputed by the oracle on that
instance alone), gets the same answer alone and in the batch, and fails or
succeeds on its own (per-instance pivots and delta_x)."""
import numpy as np
import pytest

from gen.tray import TrayParams, kkt_point
from oracle import kkt as okkt
from oracle import tray as otray
from tests.gpu_common import ensure_built, oracle_eta, solver_for, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def make_batch(specs, sigma_range=(1e-2, 1e2), seed0=0):
    """specs: [(k, T)]; every instance its own seeded KKT point."""
    out = []
    for i, (k, T) in enumerate(specs):
        p = TrayParams(k=k, T=T)
        pt = kkt_point(p, seed0 + i, sigma_range)
        W = otray.hessian_lower_csc(p, pt.w, pt.lam)
        J = otray.jacobian_csr(p, pt.w)
        out.append((p, pt, W, J))
    return out


def cat(torch, parts):
    return to_dev(torch, np.concatenate(parts))


def batch_solver(batch, **o):
    from paper_2403_15913_gb300 import KKTBatchSolver
    opts = dict(OPTS)
    opts.update(o)
    return KKTBatchSolver([(p.n, p.m, W[0], W[1], J[0], J[1]) for p, pt, W, J in batch], **opts)


def run_batch(batch, delta=None, D=None, ramp=False, **o):
    """Factor and solve the batch; with ramp, instances whose pivot fails get
    delta_x = 1e-4, then x8, until every instance factors (inertia
    correction per instance)."""
    torch = torch_cuda()
    s = batch_solver(batch, **o)
    Wv = cat(torch, [W[2] for _, _, W, _ in batch])
    Jv = cat(torch, [J[2] for _, _, _, J in batch])
    sig = cat(torch, [pt.sigma for _, pt, _, _ in batch])
    Dv = None if D is None else cat(torch, D)
    st = s.factor_batch(Wv, Jv, sig, Dv, delta)
    while ramp and st == -4:
        delta = np.zeros(len(batch)) if delta is None else delta
        bad = s.results()["failed_col"] >= 0
        delta[bad] = np.where(delta[bad] == 0, 1e-4, delta[bad] * 8)
        st = s.factor_batch(Wv, Jv, sig, Dv, delta)
    s.delta_used = np.zeros(len(batch)) if delta is None else delta
    dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    sst = None
    if st == 0 or s.results()["failed_col"].min() < 0:
        sst = s.solve(cat(torch, [pt.rx for _, pt, _, _ in batch]),
                      cat(torch, [pt.ry for _, pt, _, _ in batch]), dx, dy)
    xo, yo = s.layout()
    xs = [dx[xo[i]:xo[i + 1]].cpu().numpy() for i in range(len(batch))]
    ys = [dy[yo[i]:yo[i + 1]].cpu().numpy() for i in range(len(batch))]
    return s, st, sst, xs, ys


def run_alone(p, pt, W, J, delta_x=0.0, D=None, **o):
    torch = torch_cuda()
    opts = dict(OPTS)
    opts.update(o)
    s = solver_for(p, W, J, **opts)
    st = s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                  None if D is None else to_dev(torch, D), delta_x)
    assert st == 0
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    s.solve(to_dev(torch, pt.rx), to_dev(torch, pt.ry), dx, dy)
    return s.info.as_dict(), dx.cpu().numpy(), dy.cpu().numpy()


SPECS = [(16, 20), (32, 7), (24, 33), (48, 5), (64, 3), (16, 0), (32, 26), (24, 1)]


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_batch_each_instance_meets_bar_and_matches_alone(scheme):
    """Each instance: eta <= 1e-10 (library and oracle), and the batch answer
    equals the instance solved alone to the step-agreement bar 1e-8 relative
    (they differ only by the order of atomic updates, amplified in dy by
    D = 1/delta = 1e8: ~2e-10 observed); refinement sweeps and CG iterations
    within one."""
    batch = make_batch(SPECS)
    o = dict(scheme=scheme, gamma=1e7, max_cg=500)
    D = None
    delta = np.full(len(batch), 10.0)
    s, st, sst, xs, ys = run_batch(batch, delta=delta, D=D, **o)
    assert st == 0 and sst == 0
    r = s.results()
    assert np.all(r["status"] == 0) and np.all(r["bwd_err"] <= 1e-10)
    for i, (p, pt, W, J) in enumerate(batch):
        assert oracle_eta(p, W, J, pt.sigma, 10.0, xs[i], ys[i], pt.rx, pt.ry) <= 1e-10
        info, ax, ay = run_alone(p, pt, W, J, 10.0, None, **o)
        v, g = np.concatenate([ax, ay]), np.concatenate([xs[i], ys[i]])
        assert np.max(np.abs(g - v)) <= 1e-8 * np.max(np.abs(v)), i
        assert abs(int(r["refine_iters"][i]) - info["refine_iters"]) <= 1, i
        if scheme == "hykkt":
            assert abs(int(r["cg_iters"][i]) - info["cg_iters"]) <= 1, i


def test_batch_config1_conditioning():
    """Sigma on [1e-6, 1e6], delta = 1e-8, delta_x = 0: every instance
    reaches eta <= 1e-10 (oracle recomputed) in the batch."""
    batch = make_batch([(32, 50), (16, 12), (48, 30), (24, 44)], sigma_range=(1e-6, 1e6), seed0=7)
    s, st, sst, xs, ys = run_batch(batch, ramp=True, scheme="lifted")
    assert st == 0 and sst == 0
    for i, (p, pt, W, J) in enumerate(batch):
        assert oracle_eta(p, W, J, pt.sigma, s.delta_used[i], xs[i], ys[i], pt.rx, pt.ry) <= 1e-10


def test_batch_failure_is_per_instance():
    """Instance 2 indefinite: its pivot fails (column of the union in its own
    range), the others are solved; raising delta_x for instance 2 alone
    repairs it."""
    torch = torch_cuda()
    batch = make_batch(SPECS[:5])
    p, pt, W, J = batch[2]
    Wv = W[2].copy()
    Wv[W[0][p.n // 2]] -= 1e12
    batch[2] = (p, pt, (W[0], W[1], Wv), J)
    D = None
    delta = np.full(len(batch), 1.0)
    s, st, sst, xs, ys = run_batch(batch, delta=delta, D=D)
    assert st == -4
    r = s.results()
    assert r["failed_col"][2] >= 0 and np.all(np.delete(r["failed_col"], 2) == -1)
    xo, _ = s.layout()
    assert xo[2] <= r["failed_col"][2] < xo[3]
    assert sst == -4 and r["status"][2] == -4
    assert np.all(np.delete(r["status"], 2) == 0)
    for i in (0, 1, 3, 4):
        q, qt, Wq, Jq = batch[i]
        assert oracle_eta(q, Wq, Jq, qt.sigma, 1.0, xs[i], ys[i], qt.rx, qt.ry) <= 1e-10
    # per-instance delta_x: only instance 2 is shifted
    delta[2] = 1e13
    s2, st2, sst2, xs2, ys2 = run_batch(batch, delta=delta, D=D)
    assert st2 == 0 and sst2 == 0
    for i, (q, qt, Wq, Jq) in enumerate(batch):
        assert oracle_eta(q, Wq, Jq, qt.sigma, delta[i], xs2[i], ys2[i], qt.rx, qt.ry) <= 1e-10
        if i != 2:
            v = np.concatenate([xs[i], ys[i]])
            assert np.max(np.abs(np.concatenate([xs2[i], ys2[i]]) - v)) <= 1e-8 * np.max(np.abs(v))


def test_batch_mixed_precision():
    """FP32 factor of the whole batch, relaxed target with D = 1e2 (K_delta
    is then the exact Schur complement and FP32 refines without fallback):
    every instance meets eta <= 1e-10 on its relaxed system."""
    batch = make_batch(SPECS, sigma_range=(1e-2, 1e2), seed0=3)
    D = [np.full(p.m, 1e2) for p, _, _, _ in batch]
    s, st, sst, xs, ys = run_batch(batch, delta=np.full(len(batch), 10.0), D=D, precision=1,
                                   target_relaxed=1)
    assert st == 0 and sst == 0 and s.info.status_detail == 1
    for i, (p, pt, W, J) in enumerate(batch):
        assert oracle_eta(p, W, J, pt.sigma, 10.0, xs[i], ys[i], pt.rx, pt.ry, C=1.0 / D[i]) <= 1e-10


def test_batch_256_uneven_instances():
    """256 instances, trays uniform in {16, 24, 32, 48, 64}, horizons uniform
    in [20, 400] (the batched workload): every instance reports eta <= 1e-10
    and the oracle confirms it on eight of them."""
    torch = torch_cuda()
    rng = np.random.default_rng(2024)
    specs = [(int(rng.choice([16, 24, 32, 48, 64])), int(rng.integers(20, 401))) for _ in range(256)]
    batch = make_batch(specs, sigma_range=(1e-6, 1e6), seed0=100)
    s, st, sst, xs, ys = run_batch(batch, ramp=True, scheme="lifted")
    assert st == 0 and sst == 0
    r = s.results()
    assert np.all(r["status"] == 0) and np.all(r["bwd_err"] <= 1e-10)
    for i in rng.choice(256, 8, replace=False):
        p, pt, W, J = batch[i]
        assert oracle_eta(p, W, J, pt.sigma, s.delta_used[i], xs[i], ys[i], pt.rx, pt.ry) <= 1e-10


def test_autotuned_partition_solves_batch():
    """The autotuner returns one of its candidate partitions, and the batch
    analysed with it still meets the bar on every instance."""
    torch = torch_cuda()
    from paper_2403_15913_gb300 import autotune_batch
    batch = make_batch(SPECS, sigma_range=(1e-2, 1e2), seed0=11)
    inst = [(p.n, p.m, W[0], W[1], J[0], J[1]) for p, pt, W, J in batch]
    opts, ms = autotune_batch(inst, sample=4, **OPTS)
    assert ms > 0 and np.isfinite(ms)
    cands = {(32, 128, 64, 48), (16, 64, 64, 48), (48, 1024, 64, 48), (64, 4096, 64, 48),
             (32, 128, 32, 48), (32, 128, 64, 0), (32, 128, 64, 24), (0, 0, 64, 48)}
    assert (opts["relax_cols"], opts["relax_zeros"], opts["max_width"], opts["subtree_cols"]) in cands
    s, st, sst, xs, ys = run_batch(batch, delta=np.full(len(batch), 10.0), **opts)
    assert st == 0 and sst == 0
    for i, (p, pt, W, J) in enumerate(batch):
        assert oracle_eta(p, W, J, pt.sigma, 10.0, xs[i], ys[i], pt.rx, pt.ry) <= 1e-10



@pytest.mark.parametrize("precision", [0, 1])
def test_switched_off_instance_is_skipped_and_solves_to_zero(precision):
    """kkt_batch_set_active: with instance 1 of three switched off, the
    factorisation does no work for it (and does not fail on its values,
    which have a negative diagonal), its zero right-hand side solves to
    zero, and instances 0 and 2 get the answers they get alone (the step
    agreement bar, 1e-8 relative); switched back on, instance 1 solves like
    alone too."""
    torch = torch_cuda()
    import ctypes
    from paper_2403_15913_gb300 import _native as nat
    batch = make_batch([(8, 10), (16, 25), (8, 30)], seed0=20)
    ref = [run_alone(p, pt, W, J, 10.0, precision=precision)[1:] for p, pt, W, J in batch]
    s = batch_solver(batch, precision=precision)
    L = nat.lib()
    Wv = cat(torch, [W[2] for _, _, W, _ in batch])
    Jv = cat(torch, [J[2] for _, _, _, J in batch])
    sig = [pt.sigma.copy() for _, pt, _, _ in batch]
    good_sig = cat(torch, sig)
    sig[1][:] = -1.0                      # instance 1 would fail its first pivot
    bad_sig = cat(torch, sig)
    rx = [pt.rx.copy() for _, pt, _, _ in batch]
    ry = [pt.ry.copy() for _, pt, _, _ in batch]
    rx1, ry1 = [a.copy() for a in rx], [a.copy() for a in ry]
    rx1[1][:] = 0.0
    ry1[1][:] = 0.0
    xo, yo = s.layout()
    for on, sv, (bx, by) in (([1, 0, 1], bad_sig, (rx1, ry1)), ([1, 1, 1], good_sig, (rx, ry))):
        act = np.array(on, np.int32)
        assert L.kkt_batch_set_active(s._ctx, nat.ptr_i32(act)) == 0
        assert s.factor_batch(Wv, Jv, sv, None, np.full(3, 10.0)) == 0
        dx = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        dy = torch.zeros(s.m, dtype=torch.float64, device="cuda")
        assert s.solve(cat(torch, bx), cat(torch, by), dx, dy) == 0
        for i in range(3):
            xi = dx[xo[i]:xo[i + 1]].cpu().numpy()
            yi = dy[yo[i]:yo[i + 1]].cpu().numpy()
            if on[i]:
                v, r = np.concatenate([xi, yi]), np.concatenate(ref[i])
                assert np.max(np.abs(v - r)) <= 1e-8 * np.max(np.abs(r)), i
            else:
                assert not np.any(xi) and not np.any(yi)
    assert L.kkt_batch_set_active(s._ctx, None) == 0
    s.close()
