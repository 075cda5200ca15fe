"""CPU-side checks of the CUDA library: it loads, exports every symbol the
header declares, and its host logic (tray pattern, symbolic analysis) agrees
bit-exactly with the oracle."""
import os
import re

import numpy as np
import pytest

from gen.tray import TrayParams, kkt_point
from oracle import symbolic, tray

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nat():
    from paper_2403_15913_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2403_15913_gb300 import build
        build.build()
    _native.lib()
    return _native


def test_library_exports_every_declared_symbol(nat):
    header = open(os.path.join(ROOT, "include", "kkt.h")).read()
    declared = set(re.findall(r"\b(kkt_[a-z_]+)\s*\(", header))
    assert declared, "no declarations found"
    L = nat.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(nat.EXPORTED)


@pytest.mark.parametrize("k,T", [(32, 3), (8, 10), (5, 1)])
def test_tray_pattern_matches_oracle(nat, k, T):
    from paper_2403_15913_gb300 import TrayModel
    p = TrayParams(k=k, T=T)
    tm = TrayModel(p.as_array())
    assert (tm.n, tm.m) == (p.n, p.m)
    Wc, Wr, Jr, Jc = tm.pattern()
    pt = kkt_point(p, 0)
    oW = tray.hessian_lower_csc(p, pt.w, pt.lam)
    oJ = tray.jacobian_csr(p, pt.w)
    assert np.array_equal(Wc, oW[0]) and np.array_equal(Wr, oW[1])
    assert np.array_equal(Jr, oJ[0]) and np.array_equal(Jc, oJ[1])


def _compare(p_or_adj, pats, n, **opts):
    from paper_2403_15913_gb300 import KKTSolver
    Wc, Wr, Jr, Jc = pats
    m = len(Jr) - 1
    s = KKTSolver(n, m, Wc, Wr, Jr, Jc, host_only=True, **opts)
    g = s.symbolic()
    o = symbolic.analyse(n, Wc, Wr, Jr, Jc, leaf_size=opts["leaf_size"],
                         relax_cols=opts["relax_cols"], relax_zeros=opts["relax_zeros"],
                         max_width=opts["max_width"])
    assert np.array_equal(g["perm"], o.perm)
    assert np.array_equal(g["parent"], o.parent)
    assert np.array_equal(g["colcount"], o.colcount)
    assert np.array_equal(g["sn_ptr"], o.sn_ptr)
    rows = np.concatenate(o.sn_rows)
    assert np.array_equal(g["sn_rows"], rows)
    assert np.array_equal(np.diff(g["sn_rowptr"]), [len(r) for r in o.sn_rows])
    sz = s.sizes()
    assert sz.nnz_L == o.nnz_L and sz.flops == o.flops
    s.close()


OPTS = [dict(leaf_size=64, relax_cols=32, relax_zeros=128, max_width=64),
        dict(leaf_size=64, relax_cols=48, relax_zeros=1024, max_width=64),
        dict(leaf_size=64, relax_cols=0, relax_zeros=0, max_width=64),
        dict(leaf_size=16, relax_cols=16, relax_zeros=40, max_width=8),
        dict(leaf_size=128, relax_cols=64, relax_zeros=4000, max_width=32)]


@pytest.mark.parametrize("opts", OPTS)
@pytest.mark.parametrize("k,T", [(32, 50), (8, 40), (32, 1), (4, 0)])
def test_symbolic_bit_exact_tray(nat, opts, k, T):
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    _compare(p, (W[0], W[1], J[0], J[1]), p.n, **opts)


@pytest.mark.parametrize("seed", range(10))
def test_symbolic_bit_exact_random(nat, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 300))
    m = int(rng.integers(0, n))
    # random lower W pattern with diagonal, random J rows of 1..5 entries
    colptr = [0]
    rowind = []
    for j in range(n):
        rows = sorted(set([j] + [int(i) for i in rng.integers(j, n, rng.integers(0, 3))]))
        rowind += rows
        colptr.append(len(rowind))
    rowptr = [0]
    colind = []
    for r in range(m):
        cols = sorted(set(int(c) for c in rng.integers(0, n, rng.integers(1, 6))))
        colind += cols
        rowptr.append(len(colind))
    pats = tuple(np.array(a, dtype=np.int64) for a in (colptr, rowind, rowptr, colind))
    opts = dict(leaf_size=int(rng.integers(1, 40)), relax_cols=int(rng.integers(0, 30)),
                relax_zeros=int(rng.integers(0, 200)), max_width=int(rng.integers(1, 20)))
    _compare(None, pats, n, **opts)


def test_analyse_rejects_bad_patterns(nat):
    from paper_2403_15913_gb300 import KKTSolver, KKTError
    with pytest.raises(KKTError):   # upper-triangular W entry
        KKTSolver(3, 0, [0, 2, 3, 4], [0, 1, 0, 2], [0], [], host_only=True)
    with pytest.raises(KKTError):   # J column out of range
        KKTSolver(3, 1, [0, 1, 2, 3], [0, 1, 2], [0, 1], [7], host_only=True)
    # a J row naming a column twice (its products J_ra J_rb would be wrong)
    with pytest.raises(KKTError) as e:
        KKTSolver(5, 1, np.arange(6), np.arange(5), [0, 3], [3, 3, 4], host_only=True)
    assert e.value.status == nat.KKT_ERR_ARG and "repeats" in str(e.value)
    from paper_2403_15913_gb300 import KKTBatchSolver
    good = (np.arange(6), np.arange(5), np.array([0, 2]), np.array([3, 4]))
    bad = (np.arange(6), np.arange(5), np.array([0, 3]), np.array([3, 3, 4]))
    with pytest.raises(KKTError):
        KKTBatchSolver([(5, 1) + good, (5, 1) + bad], host_only=True)


# the hand-worked graphs of the oracle's symbolic pins (even-length path,
# pendant at the separator level, pseudo-peripheral choice, fill in minimum
# degree), each as the pattern of W with no J, at the smallest leaf size
WORKED_GRAPHS = [
    (6, [(i, i + 1) for i in range(5)]),
    (6, [(0, 1), (1, 2), (2, 3), (3, 4), (1, 5)]),
    (7, [(0, 1), (0, 4), (1, 3), (1, 6), (2, 4), (2, 5), (4, 5)]),
    (6, [(0, 1), (0, 3), (1, 5), (2, 3), (2, 4), (2, 5)]),
    (15, [(i, i + 1) for i in range(14)]),
]


@pytest.mark.parametrize("leaf", [1, 3])
@pytest.mark.parametrize("n,edges", WORKED_GRAPHS)
def test_symbolic_bit_exact_worked_graphs(nat, n, edges, leaf):
    lower = [set([j]) for j in range(n)]
    for a, b in edges:
        lower[min(a, b)].add(max(a, b))
    colptr = np.cumsum([0] + [len(s) for s in lower])
    rowind = np.concatenate([sorted(s) for s in lower])
    pats = (colptr.astype(np.int64), rowind.astype(np.int64), np.zeros(1, np.int64),
            np.zeros(0, np.int64))
    _compare(None, pats, n, leaf_size=leaf, relax_cols=0, relax_zeros=0, max_width=0)


def test_missing_library_fails_loudly(nat, monkeypatch):
    """Without the CUDA library every entry point raises: there is no CPU
    or library fallback behind the binding."""
    from paper_2403_15913_gb300 import KKTSolver
    monkeypatch.setattr(nat, "_lib", None)
    monkeypatch.setattr(nat, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libkkt_gb300.so"))
    p = TrayParams(k=3, T=1)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    with pytest.raises(RuntimeError, match="missing"):
        KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1], host_only=True)


def test_product_package_imports_no_oracle_or_fallback():
    """The binding marshals arguments only: no module of the package imports
    the oracle, or a compiler or library that could stand in for the
    kernels."""
    pkg = os.path.join(ROOT, "paper_2403_15913_gb300")
    banned = re.compile(r"^\s*(from|import)\s+(oracle|triton|numba|cupy)\b|torch\.compile|scipy",
                        re.M)
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert not banned.search(src), name


@pytest.mark.parametrize("k,T,opts", [(32, 500, OPTS[0]), (16, 1500, OPTS[3]), (32, 500, OPTS[2]),
                                    (32, 1600, OPTS[0])])
def test_symbolic_bit_exact_parallel_recursion(nat, k, T, opts):
    """Columns large enough that the top of the nested-dissection recursion
    runs sibling components on threads (and, from 100,000 variables, the
    graph's adjacency lists are built on threads): the analysis equals the
    oracle's, every time (repeated to expose any dependence on thread
    timing)."""
    from paper_2403_15913_gb300 import KKTSolver
    p = TrayParams(k=k, T=T)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    o = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **opts)
    rows = np.concatenate(o.sn_rows)
    for _ in range(5):
        s = KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1], host_only=True, **opts)
        g = s.symbolic()
        assert np.array_equal(g["perm"], o.perm)
        assert np.array_equal(g["parent"], o.parent)
        assert np.array_equal(g["sn_ptr"], o.sn_ptr)
        assert np.array_equal(g["sn_rows"], rows)
        s.close()


def test_device_analysis_without_a_gpu_returns_a_status(nat):
    """Where no GPU can be used, the device analysis ends with a CUDA status
    and its message (the binding raises KKTError): no crash, no fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2403_15913_gb300 import KKTError, KKTSolver
    p = TrayParams(k=3, T=2)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    with pytest.raises(KKTError) as e:
        KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1])
    assert e.value.status == nat.KKT_ERR_CUDA


# the library's default partition (kkt_default_options), written out for the oracle
DEFAULT_PARTITION = dict(leaf_size=8, relax_cols=32, relax_zeros=128, max_width=32)


def _bench_column_parity(nat, T, opts=None):
    from paper_2403_15913_gb300 import KKTSolver
    p = TrayParams(k=32, T=T)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    o = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **(opts or DEFAULT_PARTITION))
    s = KKTSolver(p.n, p.m, W[0], W[1], J[0], J[1], host_only=True, **(opts or {}))
    g = s.symbolic()
    assert np.array_equal(g["perm"], o.perm)
    assert np.array_equal(g["parent"], o.parent)
    assert np.array_equal(g["colcount"], o.colcount)
    assert np.array_equal(g["sn_ptr"], o.sn_ptr)
    assert np.array_equal(g["sn_rows"], np.concatenate(o.sn_rows))
    sz = s.sizes()
    assert sz.nnz_L == o.nnz_L and sz.flops == o.flops
    s.close()


@pytest.mark.parametrize("opts", [None, OPTS[0]], ids=["defaults", "leaf64"])
def test_symbolic_bit_exact_benchmark_column(nat, opts):
    """The benchmark's column (32 trays, T = 5000: n = 325,065) with the
    library's default options (no options passed; the oracle gets them
    written out) and with ND leaves of 64: the threaded nested dissection
    and the threaded adjacency build give the oracle's analysis bit for
    bit."""
    _bench_column_parity(nat, 5000, opts)


@pytest.mark.slow
def test_symbolic_bit_exact_largest_column(nat):
    """The mixed-precision workload's column (32 trays, T = 20000: n =
    1,300,065) with the default options, bit for bit against the oracle
    (about two minutes of oracle time)."""
    _bench_column_parity(nat, 20000)
