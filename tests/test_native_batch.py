"""CPU checks of the batch analysis: the concatenation of per-instance
analyses (run on host threads) equals, bit for bit, the oracle's analysis of
the block-diagonal union's pattern, for uneven tray instances and random
patterns (some of them disconnected)."""
import os

import numpy as np
import pytest

from gen.tray import TrayParams, kkt_point
from oracle import symbolic, tray


@pytest.fixture(scope="module")
def nat():
    from paper_2403_15913_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2403_15913_gb300 import build
        build.build()
    _native.lib()
    return _native


def tray_pattern(k, T):
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    return p.n, p.m, W[0], W[1], J[0], J[1]


def random_pattern(rng):
    n = int(rng.integers(5, 120))
    m = int(rng.integers(0, n))
    colptr, rowind = [0], []
    for j in range(n):
        rows = sorted(set([j] + [int(i) for i in rng.integers(j, n, rng.integers(0, 2))]))
        rowind += rows
        colptr.append(len(rowind))
    rowptr, colind = [0], []
    for _ in range(m):
        cols = sorted(set(int(c) for c in rng.integers(0, n, rng.integers(1, 4))))
        colind += cols
        rowptr.append(len(colind))
    return n, m, *(np.array(a, dtype=np.int64) for a in (colptr, rowind, rowptr, colind))


def union(instances):
    """Block-diagonal union of the patterns (plain concatenation with offsets)."""
    Wc, Wr, Jr, Jc = [0], [], [0], []
    x0 = 0
    for n, m, wc, wr, jr, jc in instances:
        w0, j0 = Wc[-1], Jr[-1]
        Wc += [w0 + int(v) for v in wc[1:]]
        Wr += [int(v) + x0 for v in wr]
        Jr += [j0 + int(v) for v in jr[1:]]
        Jc += [int(v) + x0 for v in jc]
        x0 += n
    return x0, len(Jr) - 1, *(np.array(a, dtype=np.int64) for a in (Wc, Wr, Jr, Jc))


def check_batch(instances, opts):
    from paper_2403_15913_gb300 import KKTBatchSolver
    s = KKTBatchSolver(instances, host_only=True, **opts)
    n, m, Wc, Wr, Jr, Jc = union(instances)
    assert (s.n, s.m) == (n, m)
    xo, yo = s.layout()
    assert np.array_equal(xo, np.concatenate([[0], np.cumsum([x[0] for x in instances])]))
    assert np.array_equal(yo, np.concatenate([[0], np.cumsum([x[1] for x in instances])]))
    g = s.symbolic()
    o = symbolic.analyse(n, Wc, Wr, Jr, Jc, **opts)
    assert np.array_equal(g["perm"], o.perm)
    assert np.array_equal(g["parent"], o.parent)
    assert np.array_equal(g["colcount"], o.colcount)
    assert np.array_equal(g["sn_ptr"], o.sn_ptr)
    assert np.array_equal(g["sn_rows"], np.concatenate(o.sn_rows))
    sz = s.sizes()
    assert sz.nnz_L == o.nnz_L and sz.flops == o.flops
    s.close()


OPTS = dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64)


def test_batch_of_uneven_trays_equals_union_analysis(nat):
    insts = [tray_pattern(k, T) for k, T in ((16, 5), (32, 3), (24, 0), (48, 2), (16, 9), (64, 1))]
    check_batch(insts, OPTS)


@pytest.mark.parametrize("seed", range(6))
def test_batch_of_random_patterns_equals_union_analysis(nat, seed):
    rng = np.random.default_rng(500 + seed)
    insts = [random_pattern(rng) for _ in range(int(rng.integers(1, 7)))]
    opts = dict(leaf_size=int(rng.integers(1, 30)), relax_cols=int(rng.integers(0, 20)),
                relax_zeros=int(rng.integers(0, 100)), max_width=int(rng.integers(1, 16)))
    check_batch(insts, opts)


def test_batch_of_one_equals_single_analysis(nat):
    from paper_2403_15913_gb300 import KKTBatchSolver, KKTSolver
    inst = tray_pattern(8, 6)
    a = KKTBatchSolver([inst], host_only=True, **OPTS).symbolic()
    b = KKTSolver(*inst, host_only=True, **OPTS).symbolic()
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_batch_rejects_bad_instances(nat):
    from paper_2403_15913_gb300 import KKTBatchSolver, KKTError
    good = tray_pattern(4, 1)
    bad = (3, 1, [0, 1, 2, 3], [0, 1, 2], [0, 1], [7])   # J column out of range
    with pytest.raises(KKTError) as e:
        KKTBatchSolver([good, bad], host_only=True, **OPTS)
    assert "instance 1" in str(e.value)
    with pytest.raises(KKTError):
        KKTBatchSolver([], host_only=True, **OPTS)
