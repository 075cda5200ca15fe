"""Batched lock-step IPM (kkt_ipm_batch_*): several column problems of
uneven sizes, one batched KKT factor and solve per iteration.  Each member
must follow the single-problem IPM (same iteration count, same optimum),
which is itself asserted equal to the oracle IPM elsewhere; with the FP32
factor and FP64 refinement the members still converge to the same optimum;
a member steps only with its batch."""
import numpy as np
import pytest

from gen.tray import TrayParams
from tests.gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu

OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)
SPECS = [(8, 10), (16, 25), (32, 20), (8, 40), (24, 12)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _single(p, scheme, **o):
    from paper_2403_15913_gb300 import IPMSolver
    g = IPMSolver(p.as_array(), scheme=scheme, **OPTS, **o)
    g.init()
    hist = g.solve()
    x = g.get()[0].cpu().numpy()
    g.close()
    return hist[-1], x


@pytest.mark.parametrize("scheme", ["lifted", "hykkt"])
def test_batch_members_follow_the_single_ipm(scheme):
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch
    ps = [TrayParams(k=k, T=T) for k, T in SPECS]
    b = IPMBatch([p.as_array() for p in ps], scheme=scheme, **OPTS)
    b.init()
    status, iters = b.solve()
    assert np.all(status == 1), status
    st = b.kkt_stats()
    assert st["factor_calls"] >= iters.max()
    if scheme == "lifted":
        assert st["graph_steps"] == st["factor_calls"]   # FP64: one graph launch per KKT step
    for i, p in enumerate(ps):
        last, xs = _single(p, scheme)
        assert last["status"] == 1
        assert iters[i] == last["iter"], (i, iters[i], last["iter"])
        info = b.info(i)
        assert abs(info["objective"] - last["objective"]) <= 1e-8 * abs(last["objective"])
        xb = b.members[i].get()[0].cpu().numpy()
        assert np.max(np.abs(xb - xs)) <= 1e-6
    b.close()


def test_batch_fp32_factor_reaches_the_fp64_optimum():
    """Lifted-KKT, FP32 factor of the union with FP64 refinement (fallback to
    FP64 when it does not refine): every member converges to tol and its
    objective agrees with the FP64 single-problem IPM to 1e-8."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch
    ps = [TrayParams(k=k, T=T) for k, T in SPECS]
    b = IPMBatch([p.as_array() for p in ps], scheme="lifted", precision=1, **OPTS)
    b.init()
    status, iters = b.solve()
    assert np.all(status == 1), status
    assert b.kkt_stats()["fp32_factors"] > 0
    for i, p in enumerate(ps):
        last, xs = _single(p, "lifted")
        info = b.info(i)
        assert info["err0"] <= 1e-8
        assert abs(info["objective"] - last["objective"]) <= 1e-8 * abs(last["objective"])
        xb = b.members[i].get()[0].cpu().numpy()
        assert np.max(np.abs(xb - xs)) <= 1e-5
    b.close()


def test_batch_warm_started_receding_horizon():
    """A second solve after a shifted warm start of every member (the NMPC
    pattern): converges again, in fewer iterations than the cold solve in
    total."""
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch
    ps = [TrayParams(k=k, T=T) for k, T in SPECS]
    b = IPMBatch([p.as_array() for p in ps], scheme="lifted", **OPTS)
    b.init()
    s0, it0 = b.solve()
    assert np.all(s0 == 1)
    for mem in b.members:
        mem.init_warm(mu=1e-4, recenter=True)
    s1, it1 = b.solve()
    assert np.all(s1 == 1)
    assert it1.sum() < it0.sum(), (it0, it1)
    b.close()


def test_member_does_not_step_alone():
    torch_cuda()
    from paper_2403_15913_gb300 import IPMBatch
    b = IPMBatch([TrayParams(k=8, T=10).as_array(), TrayParams(k=8, T=12).as_array()], scheme="lifted", **OPTS)
    b.init()
    assert b.members[0].step() == -8   # KKT_ERR_STATE
    b.close()
