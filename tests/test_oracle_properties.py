"""Property-based checks (hypothesis) of the oracle's dense LDL^T and of the
library's host analysis against the oracle's, on arbitrary small inputs:
factorisation residual, 2x2-block determinant sign, inertia against the
eigenvalues (well-separated spectra and exact zero rows), and bit-exact
symbolic analysis on arbitrary graphs and option sets."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import ldlt, symbolic  # noqa: E402

U = np.finfo(np.float64).eps / 2


@st.composite
def symmetric(draw, nmax=24):
    n = draw(st.integers(1, nmax))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) * 10.0 ** rng.integers(-3, 4, (n, n))
    zero = rng.random(n) < draw(st.sampled_from([0.0, 0.2]))
    K = A + A.T
    K[zero, :] = 0.0
    K[:, zero] = 0.0
    return K, int(zero.sum())


@settings(max_examples=60, deadline=None, derandomize=True)
@given(symmetric())
def test_ldlt_factorises_any_symmetric_matrix(case):
    K, _ = case
    F = ldlt.factor(K)
    N = K.shape[0]
    P = K[np.ix_(F.perm, F.perm)]
    R = P - F.L @ F.D() @ F.L.T
    assert np.linalg.norm(R) <= 50 * N * U * max(np.linalg.norm(K), np.finfo(float).tiny) * \
        max(1.0, np.max(np.abs(F.L))) ** 2
    for k, s in F.blocks:
        if s == 2:
            assert F.d[k] * F.d[k + 1] - F.e[k] ** 2 < 0


@settings(max_examples=60, deadline=None, derandomize=True)
@given(st.integers(1, 20), st.integers(0, 2**31 - 1), st.integers(0, 4))
def test_ldlt_inertia_counts_eigenvalue_signs(n, seed, nzero):
    rng = np.random.default_rng(seed)
    npos = int(rng.integers(0, n + 1))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.1, 10.0, n) * np.where(np.arange(n) < npos, 1.0, -1.0)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    K = np.zeros((n + nzero, n + nzero))
    K[:n, :n] = M
    q = rng.permutation(n + nzero)
    K = K[np.ix_(q, q)]
    assert ldlt.factor(K).inertia() == (npos, nzero, n - npos)


@st.composite
def pattern(draw):
    n = draw(st.integers(1, 60))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    m = int(rng.integers(0, n + 1))
    lower = [sorted(set([j] + [int(i) for i in rng.integers(j, n, rng.integers(0, 3))]))
             for j in range(n)]
    rows = [sorted(set(int(c) for c in rng.integers(0, n, rng.integers(1, 5)))) for _ in range(m)]
    colptr = np.cumsum([0] + [len(l) for l in lower]).astype(np.int64)
    rowind = np.concatenate(lower).astype(np.int64)
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    colind = (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int64)
    opts = dict(leaf_size=draw(st.integers(1, 40)), relax_cols=draw(st.integers(0, 40)),
                relax_zeros=draw(st.integers(0, 300)), max_width=draw(st.integers(1, 64)))
    return n, m, (colptr, rowind, rowptr, colind), opts


@pytest.fixture(scope="module")
def nat():
    import os
    from paper_2403_15913_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2403_15913_gb300 import build
        build.build()
    _native.lib()
    return _native


@settings(max_examples=80, deadline=None, derandomize=True)
@given(case=pattern())
def test_host_analysis_is_bit_exact_on_any_graph(nat, case):
    from paper_2403_15913_gb300 import KKTSolver
    n, m, (Wc, Wr, Jr, Jc), opts = case
    s = KKTSolver(n, m, Wc, Wr, Jr, Jc, host_only=True, **opts)
    g = s.symbolic()
    o = symbolic.analyse(n, Wc, Wr, Jr, Jc, **opts)
    assert np.array_equal(g["perm"], o.perm)
    assert np.array_equal(g["parent"], o.parent)
    assert np.array_equal(g["colcount"], o.colcount)
    assert np.array_equal(g["sn_ptr"], o.sn_ptr)
    assert np.array_equal(g["sn_rows"], np.concatenate(o.sn_rows))
    s.close()
