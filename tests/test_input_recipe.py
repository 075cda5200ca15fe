"""The seeded synthetic inputs follow the workload recipe: sizes of the
column at each horizon, the distributions of the KKT-point draws, the IPM
start, and the instance mixes of the batched and serving workloads.  Same
seed, same data; different seed, different data."""
import os
import sys

import numpy as np
import pytest

from gen.tray import TrayParams, bounds, ipm_start, kkt_point

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("T,n,m", [(50, 3_315, 3_264), (5_000, 325_065, 320_064),
                                   (20_000, 1_300_065, 1_280_064)])
def test_sizes_of_the_configured_horizons(T, n, m):
    p = TrayParams(k=32, T=T)
    assert (p.n, p.m) == (n, m)


def test_kkt_point_distributions():
    p = TrayParams(k=32, T=400)
    pt = kkt_point(p, 3)
    blk = pt.w.reshape(p.T + 1, p.nstage)
    comp, ctrl = blk[:, :2 * p.k], blk[:, 2 * p.k]
    assert comp.min() >= 0.05 and comp.max() <= 0.95
    assert ctrl.min() >= 1.05 and ctrl.max() <= 4.95
    # uniform: mean and spread of U(a, b)
    assert abs(comp.mean() - 0.5) < 0.01 and abs(comp.std() - 0.9 / np.sqrt(12)) < 0.01
    assert abs(ctrl.mean() - 3.0) < 0.1
    # multipliers and right-hand sides N(0, 1)
    for v in (pt.lam, pt.rx, pt.ry):
        assert abs(v.mean()) < 0.03 and abs(v.std() - 1.0) < 0.03
    # Sigma_x log-uniform on [1e-6, 1e6]: log10 uniform on [-6, 6]
    ls = np.log10(pt.sigma)
    assert ls.min() >= -6 and ls.max() <= 6
    assert abs(ls.mean()) < 0.1 and abs(ls.std() - 12 / np.sqrt(12)) < 0.05
    wide = kkt_point(p, 3, sigma_range=(1e-8, 1e8)).sigma
    assert np.log10(wide).min() >= -8 and np.log10(wide).max() <= 8
    assert np.log10(wide).max() - np.log10(wide).min() > 15


def test_kkt_point_is_seeded():
    p = TrayParams(k=8, T=10)
    a, b, c = kkt_point(p, 7), kkt_point(p, 7), kkt_point(p, 8)
    for f in ("w", "lam", "sigma", "rx", "ry"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(getattr(a, f), getattr(c, f))


def test_ipm_start_and_bounds():
    p = TrayParams(k=4, T=3)
    w = ipm_start(p).reshape(p.T + 1, p.nstage)
    assert np.all(w[:, :2 * p.k] == p.x0bar) and np.all(w[:, 2 * p.k] == p.ubar)
    lo, hi = bounds(p)
    lo, hi = lo.reshape(p.T + 1, p.nstage), hi.reshape(p.T + 1, p.nstage)
    assert np.all(lo[:, :2 * p.k] == 0.0) and np.all(hi[:, :2 * p.k] == 1.0)
    assert np.all(lo[:, 2 * p.k] == 1.0) and np.all(hi[:, 2 * p.k] == 5.0)


def test_batched_workload_mix():
    sys.path.insert(0, ROOT)
    import bench
    specs = bench.batch_specs(256, 0)
    assert len(specs) == 256
    ks = {k for k, _ in specs}
    Ts = np.array([T for _, T in specs])
    assert ks == {16, 24, 32, 48, 64}
    assert Ts.min() >= 20 and Ts.max() <= 400 and Ts.max() - Ts.min() > 300
    n = [TrayParams(k=k, T=T).n for k, T in specs]
    # per-instance n between the extremes (2*16+1)*21 and (2*64+1)*401
    assert min(n) >= 693 and max(n) <= 51_729
    assert bench.batch_specs(256, 0) == specs and bench.batch_specs(256, 1) != specs
