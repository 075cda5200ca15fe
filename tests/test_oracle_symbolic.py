"""Pins of the oracle's symbolic analysis: permutation validity, textbook
nested dissection of a path, the elimination game on tiny graphs (fill,
etree, column counts), supernode partition and containment invariants."""
import itertools

import numpy as np
import pytest

from gen.tray import TrayParams, kkt_point
from oracle import symbolic, tray


def _graph_from_edges(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return [sorted(s) for s in adj]


def _patterns_from_adj(adj):
    """Express an undirected graph as (lower CSC of W, empty J)."""
    n = len(adj)
    colptr = [0]
    rowind = []
    for j in range(n):
        rows = [j] + [i for i in adj[j] if i > j]
        rowind += rows
        colptr.append(len(rowind))
    return (np.array(colptr), np.array(rowind), np.zeros(1, np.int64),
            np.zeros(0, np.int64))


def _elimination_game(adj, perm):
    """Brute-force symbolic factorisation: eliminate nodes in order, adding
    fill edges among the remaining neighbours.  Returns struct(L(:, j))."""
    n = len(adj)
    iperm = np.empty(n, dtype=int)
    iperm[perm] = np.arange(n)
    g = [set(int(iperm[a]) for a in adj[perm[j]]) for j in range(n)]
    structs = []
    for j in range(n):
        later = sorted(i for i in g[j] if i > j)
        structs.append([j] + later)
        for a, b in itertools.combinations(later, 2):
            g[a].add(b)
            g[b].add(a)
    return structs


def test_path_textbook_nested_dissection():
    n = 7
    adj = _graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    perm = symbolic.nested_dissection(adj, leaf_size=1)
    assert perm.tolist() == [0, 2, 1, 4, 6, 5, 3]
    n = 15
    adj = _graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    perm = symbolic.nested_dissection(adj, leaf_size=1)
    assert perm.tolist() == [0, 2, 1, 4, 6, 5, 3, 8, 10, 9, 12, 14, 13, 11, 7]


def test_minimum_degree_star_and_ties():
    # star centred at 0 with leaves 1..4: leaves 1, 2, 3 go first (degree 1);
    # then centre 0 and leaf 4 both have degree 1 and the tie goes to 0
    adj = _graph_from_edges(5, [(0, i) for i in range(1, 5)])
    assert symbolic.minimum_degree(adj, set(range(5))) == [1, 2, 3, 0, 4]
    # a 4-cycle 0-1-2-3: all degree 2, eliminate 0 (fill 1-3), then 1 (deg 2,
    # ties to smallest), then 2, 3
    adj = _graph_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    assert symbolic.minimum_degree(adj, set(range(4))) == [0, 1, 2, 3]


def test_path_of_even_length_splits_at_lower_middle():
    # 0-1-2-3-4-5: five levels from node 0 (e = 5), separator level
    # floor(5/2) = 2; then {0, 1} has e = 1 (a leaf) and {3, 4, 5} splits at 4
    adj = _graph_from_edges(6, [(i, i + 1) for i in range(5)])
    assert symbolic.nested_dissection(adj, leaf_size=1).tolist() == [0, 1, 3, 5, 4, 2]


def test_separator_takes_only_nodes_facing_the_next_level():
    # path 0-1-2-3-4 with a pendant 5 on node 1: levels from 0 are {0}, {1},
    # {2, 5}, {3}, {4} (node 4's structure is no deeper); the middle level is
    # {2, 5} but only 2 touches level 3, so the separator is {2}
    adj = _graph_from_edges(6, [(0, 1), (1, 2), (2, 3), (3, 4), (1, 5)])
    assert symbolic.nested_dissection(adj, leaf_size=1).tolist() == [0, 5, 1, 3, 4, 2]


def test_pseudo_peripheral_node_worked_case():
    # from 0: last level {2, 3, 5, 6}; degree-1 nodes 3 and 6, tie to 3;
    # eccentricity of 3 is 4 > 2; from 3 the last level is {2, 5} (degree 2
    # each, tie to 2), whose eccentricity is not larger: node 3
    adj = _graph_from_edges(7, [(0, 1), (0, 4), (1, 3), (1, 6), (2, 4), (2, 5), (4, 5)])
    r, levels = symbolic.pseudo_peripheral(adj, set(range(7)))
    assert r == 3
    assert [sorted(l) for l in levels] == [[3], [1], [0, 6], [4], [2, 5]]


def test_minimum_degree_counts_fill():
    # degrees 2,2,3,2,1,2: eliminate 4; then all degree 2, eliminate 0, which
    # joins 1 and 3; 1 (degree 2: 3, 5) next, which joins 3 and 5; then 2,
    # 3, 5 (without the fill edges 3 would go before 2)
    adj = _graph_from_edges(6, [(0, 1), (0, 3), (1, 5), (2, 3), (2, 4), (2, 5)])
    assert symbolic.minimum_degree(adj, set(range(6))) == [4, 0, 1, 2, 3, 5]


def test_graph_is_pattern_of_W_plus_JtJ():
    """Adjacency of pattern(W + J^T J) against a sparse product of the
    patterns (positive values, so no cancellation)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(4)
    n, m = 30, 18
    Wd = np.tril(rng.random((n, n)) < 0.08)
    np.fill_diagonal(Wd, True)
    Jd = rng.random((m, n)) < 0.12
    Wc = sp.csc_matrix(Wd.astype(float))
    Jc = sp.csr_matrix(Jd.astype(float))
    adj = symbolic.kkt_graph(n, Wc.indptr, Wc.indices, Jc.indptr, Jc.indices)
    P = (abs(Wc) + abs(Wc).T + Jc.T @ Jc).toarray() != 0
    np.fill_diagonal(P, False)
    for v in range(n):
        assert adj[v] == np.nonzero(P[v])[0].tolist()


def test_postorder_visits_children_in_increasing_index():
    # node 3 has children 0 and 2, node 2 has child 1
    assert symbolic.postorder(np.array([3, 2, 3, -1])).tolist() == [0, 1, 2, 3]
    # two roots, 2 (children 0, 1) and 4 (child 3)
    assert symbolic.postorder(np.array([2, 2, -1, 4, -1])).tolist() == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("parent,cc,ptr", [
    # chain 0 -> 1 -> 2 with nested structures: one supernode
    ([1, 2, -1], [3, 2, 1], [0, 3]),
    # column 1 holds a row that column 0 lacks (cc equal): 0 stands alone
    ([1, 2, -1], [2, 2, 1], [0, 1, 3]),
    # node 2 has two children: neither joins it
    ([2, 2, -1], [2, 2, 1], [0, 1, 2, 3]),
])
def test_fundamental_supernodes_worked_cases(parent, cc, ptr):
    assert symbolic.fundamental_supernodes(np.array(parent), np.array(cc)) == ptr


@pytest.mark.parametrize("zeros,ptr", [(0, [0, 1, 3]), (1, [0, 3])])
def test_relaxation_counts_explicit_zeros(zeros, ptr):
    # fundamental supernodes {0}, {1}, {2} with rows {0, 2}, {1, 2}, {2} and
    # parent(0) = parent(1) = 2.  Backward: {1} joins {2} with no zero (3 of
    # 3 panel slots are in L); {0} joining {1, 2} gives a 3 x 3 lower
    # triangle of 6 slots with 5 entries of L: one explicit zero, (1, 0)
    rows = [np.array([0, 2]), np.array([1, 2]), np.array([2])]
    got = symbolic.relax_and_split([0, 1, 2, 3], np.array([2, 2, 1]), np.array([2, 2, -1]),
                                   rows, relax_cols=8, relax_zeros=zeros, max_width=0)
    assert got == ptr


@pytest.mark.parametrize("seed", range(12))
def test_elimination_game_matches(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 40))
    edges = [(int(a), int(b)) for a, b in rng.integers(0, n, (2 * n, 2))]
    adj = _graph_from_edges(n, edges)
    pats = _patterns_from_adj(adj)
    sym = symbolic.analyse(n, *pats, leaf_size=int(rng.integers(1, 9)))
    assert sorted(sym.perm.tolist()) == list(range(n))
    game = _elimination_game(adj, sym.perm)
    for j in range(n):
        assert sym.structs[j].tolist() == game[j]
        below = game[j][1:]
        assert sym.parent[j] == (below[0] if below else -1)
        assert sym.colcount[j] == len(game[j])
    # the final labels are a postorder: every subtree is the contiguous range
    # of labels ending at its root
    size = np.ones(n, dtype=int)
    for j in range(n):
        if sym.parent[j] >= 0:
            size[sym.parent[j]] += size[j]
    for j in range(n):
        lo = j - size[j] + 1
        for i in range(lo, j):
            a = i
            while a != -1 and a != j:
                a = sym.parent[a]
            assert a == j


@pytest.mark.parametrize("relax", [(0, 0, 0), (48, 1024, 64), (16, 40, 5)])
def test_supernode_invariants_tray(relax):
    p = TrayParams(k=8, T=12)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    rc, rz, mw = relax
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], leaf_size=16,
                           relax_cols=rc, relax_zeros=rz, max_width=mw)
    ptr = sym.sn_ptr
    assert ptr[0] == 0 and ptr[-1] == p.n and np.all(np.diff(ptr) > 0)
    if mw:
        assert np.max(np.diff(ptr)) <= mw
    ns = len(ptr) - 1
    snode = np.repeat(np.arange(ns), np.diff(ptr))
    for s in range(ns):
        f, l = ptr[s], ptr[s + 1] - 1
        rows = sym.sn_rows[s]
        assert rows[:l - f + 1].tolist() == list(range(f, l + 1))
        # every column's true structure is inside the panel
        for j in range(f, l + 1):
            assert set(sym.structs[j].tolist()) <= set(rows.tolist())
        below = rows[rows > l]
        if len(below):
            par = sym.sn_parent[s]
            assert par == snode[below[0]]
            prow = set(sym.sn_rows[par].tolist())
            assert set(below.tolist()) <= prow
        else:
            assert sym.sn_parent[s] == -1
    if rc == 0 and mw == 0:   # fundamental rule
        for j in range(p.n - 1):
            same = snode[j] == snode[j + 1]
            nchild = np.sum(sym.parent == j + 1)
            rule = (sym.parent[j] == j + 1 and sym.colcount[j] == sym.colcount[j + 1] + 1
                    and nchild == 1)
            assert same == rule


def test_tray_separators_are_small():
    """For the tray chain every nested-dissection separator is bounded by the
    size of one stage (2k+1)."""
    p = TrayParams(k=8, T=30)
    pt = kkt_point(p, 0)
    W = tray.hessian_lower_csc(p, pt.w, pt.lam)
    J = tray.jacobian_csr(p, pt.w)
    adj = symbolic.kkt_graph(p.n, W[0], W[1], J[0], J[1])
    seps = []
    orig = symbolic.nd_component

    def spy(adj_, comp, leaf):
        out = orig(adj_, comp, leaf)
        if len(comp) > leaf:
            _, levels = symbolic.pseudo_peripheral(adj_, comp)
            if len(levels) - 1 >= 2:
                lv = (len(levels) - 1) // 2
                below = set(levels[lv + 1])
                seps.append(sum(1 for v in levels[lv] if any(w in below for w in adj_[v])))
        return out
    symbolic.nd_component = spy
    try:
        symbolic.nested_dissection(adj, leaf_size=16)
    finally:
        symbolic.nd_component = orig
    assert seps and max(seps) <= 2 * p.k + 1
