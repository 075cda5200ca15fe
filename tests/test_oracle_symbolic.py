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
