"""Oracle O3: symbolic analysis of the condensed matrix K (Sec. V-B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes the symbolic factorisation of K once, because the pattern
of the condensed matrix does not change across IPM iterations (Sec. V-B), and
reuses it for every refactorisation.  cuDSS's own ordering is not described,
so the ordering is fixed here by a fully specified rule that the library's
host analysis must reproduce exactly:

1. Graph.  G = pattern(W + J^T J) without self loops, undirected.
2. Ordering: level-structure nested dissection (George & Liu, 1981).
   * Work on connected components, in increasing order of their smallest node.
   * A component with at most ``leaf_size`` nodes is ordered by exact minimum
     degree on its own induced subgraph (ties: smallest original index; no
     supervariables, no absorption).
   * Otherwise find a pseudo-peripheral node: start from the smallest node
     r; repeat { build the BFS level structure of r; among the last level take
     the node v of minimum degree inside the component (ties: smallest
     index); if the level structure of v has more levels, r <- v, else stop }.
   * With levels L_0..L_e of r: if e < 2 order the component as a leaf;
     otherwise l = floor(e/2) and the separator is
     { v in L_l : v has a neighbour in L_{l+1} }.
   * Order the rest of the component recursively (its components in
     increasing order of their smallest node), then the separator, in
     increasing node index.
3. Elimination tree of P K P^T (Liu's algorithm; unique for a given pattern).
4. Postorder: depth-first, children visited in increasing index, roots in
   increasing index; the final permutation composes ND and the postorder.
5. Column structures and counts of L by set union over the etree children.
6. Supernodes.  Fundamental: column j+1 joins the supernode of j iff
   parent(j) = j+1, cc(j) = cc(j+1) + 1 and j+1 has exactly one child.
   Relaxation (one written rule, one backward pass over the fundamental
   supernodes): s is merged into the (possibly already merged) supernode
   that follows it when parent(last(s)) lies in that supernode and the
   merged supernode would have at most ``relax_cols`` columns and at most
   ``relax_zeros`` explicit zeros in its panel's lower trapezoid.
   Finally supernodes wider than ``max_width`` columns are cut into pieces
   of ``max_width`` columns from their first column.
7. Supernode row structure, by the supernodal recursion
   rows(s) = cols(s) u {i > last(s): K(i, j) != 0, j in s}
             u U_{child supernodes c} {i in rows(c): i > last(s)}.

Parity: pinned by tests (permutation validity, the elimination game on tiny
graphs, textbook nested dissection of a path, etree/column-count identities
against a dense symbolic factorisation, supernode containment).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# ------------------------------------------------------------------ graph
def kkt_graph(n, W_colptr, W_rowind, J_rowptr, J_colind):
    """Adjacency (sorted lists) of pattern(W + J^T J) without self loops."""
    adj = [set() for _ in range(n)]
    for j in range(n):
        for p in range(W_colptr[j], W_colptr[j + 1]):
            i = int(W_rowind[p])
            if i != j:
                adj[i].add(j)
                adj[j].add(i)
    m = len(J_rowptr) - 1
    for r in range(m):
        cols = [int(c) for c in J_colind[J_rowptr[r]:J_rowptr[r + 1]]]
        for a in cols:
            for b in cols:
                if a != b:
                    adj[a].add(b)
    return [sorted(s) for s in adj]


# ------------------------------------------------------------ ordering
def components(adj, nodes):
    """Connected components of the subgraph induced by ``nodes`` (a set),
    each returned as a set, in increasing order of their smallest node."""
    seen = set()
    comps = []
    for s in sorted(nodes):
        if s in seen:
            continue
        comp = {s}
        seen.add(s)
        stack = [s]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w in nodes and w not in seen:
                    seen.add(w)
                    comp.add(w)
                    stack.append(w)
        comps.append(comp)
    return comps


def bfs_levels(adj, root, comp):
    """Rooted level structure L_0 .. L_e of ``root`` inside ``comp``."""
    levels = [[root]]
    seen = {root}
    while True:
        nxt = set()
        for v in levels[-1]:
            for w in adj[v]:
                if w in comp and w not in seen:
                    nxt.add(w)
        if not nxt:
            return levels
        seen |= nxt
        levels.append(sorted(nxt))


def degree_in(adj, v, comp):
    return sum(1 for w in adj[v] if w in comp)


def pseudo_peripheral(adj, comp):
    """George-Liu pseudo-peripheral node search, started at the smallest
    node of the component.  Returns the node and its level structure."""
    r = min(comp)
    levels = bfs_levels(adj, r, comp)
    while True:
        last = levels[-1]
        v = min(last, key=lambda w: (degree_in(adj, w, comp), w))
        lv = bfs_levels(adj, v, comp)
        if len(lv) > len(levels):
            r, levels = v, lv
        else:
            return r, levels


def minimum_degree(adj, comp):
    """Exact minimum-degree elimination order of the subgraph induced by
    ``comp``: repeatedly eliminate the node of smallest current degree
    (ties: smallest index), turning its neighbourhood into a clique."""
    g = {v: {w for w in adj[v] if w in comp} for v in comp}
    order = []
    while g:
        v = min(g, key=lambda w: (len(g[w]), w))
        nb = g.pop(v)
        for a in nb:
            g[a].discard(v)
            g[a] |= (nb - {a})
        order.append(v)
    return order


def nd_component(adj, comp, leaf_size):
    if len(comp) <= leaf_size:
        return minimum_degree(adj, comp)
    _, levels = pseudo_peripheral(adj, comp)
    e = len(levels) - 1
    if e < 2:
        return minimum_degree(adj, comp)
    lv = e // 2
    below = set(levels[lv + 1])
    sep = sorted(v for v in levels[lv] if any(w in below for w in adj[v]))
    rest = comp - set(sep)
    out = []
    for c in components(adj, rest):
        out += nd_component(adj, c, leaf_size)
    return out + sep


def nested_dissection(adj, leaf_size=64):
    """Permutation ``perm`` (new -> old) of the pinned nested dissection."""
    n = len(adj)
    out = []
    for c in components(adj, set(range(n))):
        out += nd_component(adj, c, leaf_size)
    assert sorted(out) == list(range(n))
    return np.array(out, dtype=np.int64)


# ------------------------------------------------- elimination tree etc.
def permuted_lower_neighbours(adj, perm):
    """For every new column j, the sorted new indices i < j adjacent to it."""
    n = len(adj)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    out = []
    for j in range(n):
        out.append(sorted(int(iperm[a]) for a in adj[perm[j]] if iperm[a] < j))
    return out


def etree(adj, perm):
    """Elimination tree of P K P^T by Liu's algorithm with path compression:
    parent[j] = -1 for roots."""
    n = len(adj)
    up = permuted_lower_neighbours(adj, perm)
    parent = [-1] * n
    ancestor = [-1] * n
    for j in range(n):
        for i in up[j]:
            r = i
            while ancestor[r] != -1 and ancestor[r] != j:
                nxt = ancestor[r]
                ancestor[r] = j
                r = nxt
            if ancestor[r] == -1:
                ancestor[r] = j
                parent[r] = j
    return np.array(parent, dtype=np.int64)


def postorder(parent):
    """Depth-first postorder; children and roots visited in increasing
    index.  Returns post (post[k] = node visited k-th)."""
    n = len(parent)
    children = [[] for _ in range(n)]
    roots = []
    for j in range(n):
        if parent[j] < 0:
            roots.append(j)
        else:
            children[parent[j]].append(j)
    post = []
    for r in roots:
        stack = [(r, 0)]
        while stack:
            v, ci = stack.pop()
            if ci < len(children[v]):
                stack.append((v, ci + 1))
                stack.append((children[v][ci], 0))
            else:
                post.append(v)
    return np.array(post, dtype=np.int64)


def column_structures(adj, perm, parent):
    """struct(L(:, j)) (sorted, diagonal first) for every column, by
    struct(L(:,j)) = {j} u {i > j : K(i,j) != 0} u U_{child c} struct(L(:,c))\\{c}.
    """
    n = len(adj)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    children = [[] for _ in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            children[parent[j]].append(j)
    live = {}
    structs = [None] * n
    for j in range(n):
        s = {j}
        for a in adj[perm[j]]:
            i = int(iperm[a])
            if i > j:
                s.add(i)
        for c in children[j]:
            s |= live.pop(c)
            s.discard(c)
        s.discard(-1)
        live[j] = s
        structs[j] = np.array(sorted(s), dtype=np.int64)
    return structs


# ------------------------------------------------------------ supernodes
def fundamental_supernodes(parent, cc):
    n = len(parent)
    nchild = np.zeros(n, dtype=np.int64)
    for j in range(n):
        if parent[j] >= 0:
            nchild[parent[j]] += 1
    starts = [0]
    for j in range(n - 1):
        joins = (parent[j] == j + 1 and cc[j] == cc[j + 1] + 1
                 and nchild[j + 1] == 1)
        if not joins:
            starts.append(j + 1)
    return starts + [n]


def supernode_rows(sn_ptr, lower_nbrs_of_col, parent):
    """rows(s) by the supernodal recursion of step 7.  ``lower_nbrs_of_col``
    gives, per column, the rows i > j with K(i, j) != 0."""
    ns = len(sn_ptr) - 1
    n = sn_ptr[-1]
    snode = np.empty(n, dtype=np.int64)
    for s in range(ns):
        snode[sn_ptr[s]:sn_ptr[s + 1]] = s
    rows = [None] * ns
    sparent = np.full(ns, -1, dtype=np.int64)
    kids = [[] for _ in range(ns)]
    for s in range(ns):
        f, l = sn_ptr[s], sn_ptr[s + 1] - 1
        r = set(range(f, l + 1))
        for j in range(f, l + 1):
            r |= {i for i in lower_nbrs_of_col[j] if i > l}
        for c in kids[s]:
            r |= {i for i in rows[c] if i > l}
        rows[s] = np.array(sorted(r), dtype=np.int64)
        below = rows[s][rows[s] > l]
        if len(below):
            sparent[s] = snode[below[0]]
            kids[sparent[s]].append(s)
    return rows, sparent


def relax_and_split(sn_ptr, struct_count, parent, fund_rows,
                    relax_cols, relax_zeros, max_width):
    """Apply the relaxation and width rules of step 6 to a fundamental
    partition ``sn_ptr`` whose row structures are ``fund_rows``.

    Relaxation is one backward pass: ``cur`` is the (possibly already merged)
    supernode that follows s; s merges into it when parent(last(s)) lies in
    ``cur``, the merged supernode has at most ``relax_cols`` columns and its
    panel (lower trapezoid of cols x rows, rows = cols(s) u rows(cur)) holds
    at most ``relax_zeros`` entries that are structurally zero in L."""
    ns = len(sn_ptr) - 1
    ptr = list(sn_ptr)
    if relax_cols > 0 and ns > 1:
        starts = []
        cur_f, cur_l = ptr[ns - 1], ptr[ns] - 1
        cur_rows = set(fund_rows[ns - 1].tolist())
        for s in range(ns - 2, -1, -1):
            f, l = ptr[s], ptr[s + 1] - 1
            ok = cur_f <= parent[l] <= cur_l
            if ok:
                ncol = cur_l - f + 1
                nrow = (l - f + 1) + len(cur_rows)
                slots = ncol * nrow - ncol * (ncol - 1) // 2
                true_nnz = int(sum(int(struct_count[j]) for j in range(f, cur_l + 1)))
                ok = ncol <= relax_cols and slots - true_nnz <= relax_zeros
            if ok:
                cur_f = f
                cur_rows |= set(range(f, l + 1))
            else:
                starts.append(cur_f)
                cur_f, cur_l = f, l
                cur_rows = set(fund_rows[s].tolist())
        starts.append(cur_f)
        ptr = sorted(starts) + [ptr[-1]]
    if max_width > 0:
        out = [0]
        for s in range(len(ptr) - 1):
            f, e = ptr[s], ptr[s + 1]
            c = f + max_width
            while c < e:
                out.append(c)
                c += max_width
            out.append(e)
        ptr = out
    return ptr


# ------------------------------------------------------------------ driver
@dataclass
class Symbolic:
    n: int
    perm: np.ndarray          # new -> old
    parent: np.ndarray        # etree of P K P^T (new labels)
    colcount: np.ndarray      # nnz per column of L, diagonal included
    structs: list             # struct(L(:, j)), new labels
    sn_ptr: np.ndarray        # supernode column boundaries
    sn_rows: list             # rows(s), new labels
    sn_parent: np.ndarray

    @property
    def nnz_L(self):
        return int(self.colcount.sum())

    @property
    def flops(self):
        """Multiply-adds counted as 2 flops: sum_j cc_j^2 (+ lower order)."""
        return float(np.sum(self.colcount.astype(np.float64) ** 2))


def analyse(n, W_colptr, W_rowind, J_rowptr, J_colind, leaf_size=64,
            relax_cols=0, relax_zeros=0, max_width=0):
    adj = kkt_graph(n, W_colptr, W_rowind, J_rowptr, J_colind)
    perm0 = nested_dissection(adj, leaf_size)
    parent0 = etree(adj, perm0)
    post = postorder(parent0)
    perm = perm0[post]
    parent = etree(adj, perm)
    structs = column_structures(adj, perm, parent)
    cc = np.array([len(s) for s in structs], dtype=np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    lower_nbrs = [[int(iperm[a]) for a in adj[perm[j]] if iperm[a] > j]
                  for j in range(n)]
    ptr = fundamental_supernodes(parent, cc)
    fund_rows, _ = supernode_rows(ptr, lower_nbrs, parent)
    ptr = relax_and_split(ptr, cc, parent, fund_rows, relax_cols,
                          relax_zeros, max_width)
    rows, sparent = supernode_rows(ptr, lower_nbrs, parent)
    return Symbolic(n, perm, parent, cc, structs, np.array(ptr, np.int64),
                    rows, sparent)
