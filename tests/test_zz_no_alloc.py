"""The allocation-free backsolve, called through the C ABI, gives the same
K^{-1} b as the ordinary backsolve, on two calls in a row.

This variant exists for callers that must not allocate device memory while
they run (for example a control loop that may not call the allocator after
start-up); its scratch vector is a fixed array inside the library.  The file
name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import ensure_built, instance, solver_for, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_backsolve_noalloc_matches_backsolve():
    torch = torch_cuda()
    ensure_built()
    from paper_2403_15913_gb300 import _native as nat
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", leaf_size=64, relax_cols=48, relax_zeros=1024,
                   max_width=64)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, np.full(p.m, 1e2)), 10.0) == 0
    L = nat.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(9)
    for call in range(2):
        b = to_dev(torch, rng.standard_normal(p.n))
        ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        out = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
        s.backsolve(b, ref)
        st = L.kkt_backsolve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, L.kkt_last_error(s._ctx)
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r)), call


def test_backsolve_noalloc_fp32_factor():
    """With an FP32 factor (precision = 1) the static scratch holds the FP32
    permuted vector; the result equals the ordinary backsolve up to the
    order of FP32 atomic updates in the forward solve."""
    torch = torch_cuda()
    ensure_built()
    from paper_2403_15913_gb300 import _native as nat
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", precision=1)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, np.full(p.m, 1e2)), 10.0) == 0
    assert s.info.status_detail == 1
    L = nat.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    b = to_dev(torch, np.random.default_rng(10).standard_normal(p.n))
    ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    out = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
    s.backsolve(b, ref)
    st = L.kkt_backsolve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0, L.kkt_last_error(s._ctx)
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert np.max(np.abs(o - r)) <= 1e-5 * np.max(np.abs(r))


def test_backsolve_noalloc_df64_factor():
    """Double-float factor (precision = 2): the scratch holds the permuted
    vector as float pairs; same result as the ordinary backsolve."""
    torch = torch_cuda()
    ensure_built()
    from paper_2403_15913_gb300 import _native as nat
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", precision=2)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, np.full(p.m, 1e2)), 10.0) == 0
    assert s.info.status_detail == 3
    L = nat.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    b = to_dev(torch, np.random.default_rng(12).standard_normal(p.n))
    ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    out = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
    s.backsolve(b, ref)
    st = L.kkt_backsolve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0, L.kkt_last_error(s._ctx)
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r))


def test_backsolve_noalloc_block_cyclic_reduction():
    """Block cyclic reduction (solver = 1): the static scratch holds the
    right-hand side in natural order while it is solved in place; two calls
    in a row give the ordinary backsolve's result."""
    torch = torch_cuda()
    ensure_built()
    from paper_2403_15913_gb300 import _native as nat
    p, pt, W, J = instance(32, 50, 0, sigma_range=(1e-2, 1e2))
    s = solver_for(p, W, J, scheme="lifted", solver=1, block=2 * p.k + 1)
    assert s.factor(to_dev(torch, W[2]), to_dev(torch, J[2]), to_dev(torch, pt.sigma),
                    to_dev(torch, np.full(p.m, 1e2)), 10.0) == 0
    L = nat.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(13)
    for call in range(2):
        b = to_dev(torch, rng.standard_normal(p.n))
        ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        out = torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda")
        s.backsolve(b, ref)
        st = L.kkt_backsolve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, L.kkt_last_error(s._ctx)
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.array_equal(o, r), call
