"""Helpers shared by the GPU parity tests: build the same seeded instance
for the oracle (CPU) and the CUDA path, move oracle-computed inputs to the
device."""
import numpy as np

from gen.tray import TrayParams, kkt_point
from oracle import kkt as okkt
from oracle import tray as otray


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def ensure_built():
    import os
    from paper_2403_15913_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2403_15913_gb300 import build
        build.build()


def instance(k=32, T=50, seed=0, sigma_range=(1e-6, 1e6)):
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, seed, sigma_range)
    W = otray.hessian_lower_csc(p, pt.w, pt.lam)
    J = otray.jacobian_csr(p, pt.w)
    return p, pt, W, J


def to_dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def solver_for(p, W, J, **opts):
    from paper_2403_15913_gb300 import KKTSolver
    return KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1], **opts)


def oracle_eta(p, W, J, sigma, delta_x, dx, dy, rx, ry, C=None):
    K = okkt.kkt_matrix(p.n, p.m, W, J, sigma, delta_x, C)
    return okkt.backward_error(K, np.concatenate([dx, dy]), np.concatenate([rx, ry]))
