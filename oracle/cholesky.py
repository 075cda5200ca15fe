"""Oracle O4: numeric sparse Cholesky and triangular solves (Sec. V-B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain left-looking column Cholesky (cmod / cdiv) of P K P^T on the column
structures of the symbolic analysis, in FP64:

    for j = 0 .. n-1:
        x = K'(j:, j)                       (scattered into a dense vector)
        for every k < j with L(j, k) != 0:  x -= L(j:, k) * L(j, k)
        if not x_j > 0 (or x_j not finite): stop, column j failed
        L(j, j) = sqrt(x_j);  L(j+1:, j) = x_{j+1:} / L(j, j)

followed by column-oriented forward and backward substitution.  The paper's
refactorisation keeps the symbolic structure fixed (Sec. V-B); so does this.

Parity: pinned by tests against a dense Cholesky of small matrices and by the
factorisation residual ||P K P^T - L L^T|| / ||K|| on every test matrix.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(Exception):
    def __init__(self, column):
        super().__init__(f"non-positive pivot in column {column}")
        self.column = column


def permuted_lower(n, K_rows, K_cols, K_vals, perm):
    """Lower-triangular entries of P K P^T grouped by column, from COO
    triplets of the FULL symmetric K (both triangles): the entries that land
    in the strict upper triangle of P K P^T are dropped, duplicates summed.
    Returns a list of {row: value} per new column."""
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    r = iperm[np.asarray(K_rows)]
    c = iperm[np.asarray(K_cols)]
    keep = r >= c
    cols = [dict() for _ in range(n)]
    for a, b, v in zip(r[keep].tolist(), c[keep].tolist(),
                       np.asarray(K_vals)[keep].tolist()):
        d = cols[b]
        d[a] = d.get(a, 0.0) + v
    return cols


def factor(n, structs, lower_cols):
    """Left-looking Cholesky.  ``structs[j]`` is struct(L(:, j)) (sorted,
    diagonal first); ``lower_cols[j]`` maps row -> value of P K P^T in
    column j (rows >= j).  Returns the list of column value arrays aligned
    with ``structs``.  Raises NotPositiveDefinite(j) on failure."""
    # rows of L: for each j, the columns k < j with L(j, k) != 0 and the
    # position of row j inside struct(L(:, k))
    row_cols = [[] for _ in range(n)]
    for k in range(n):
        for pos, i in enumerate(structs[k].tolist()):
            if i != k:
                row_cols[i].append((k, pos))
    vals = [None] * n
    work = np.zeros(n)
    for j in range(n):
        sj = structs[j]
        work[sj] = 0.0
        for i, v in lower_cols[j].items():
            work[i] += v
        for k, pos in row_cols[j]:
            sk = structs[k][pos:]          # rows >= j of column k
            lk = vals[k][pos:]
            work[sk] -= lk * lk[0]
        d = work[j]
        if not (d > 0.0) or not np.isfinite(d):
            raise NotPositiveDefinite(j)
        ljj = np.sqrt(d)
        col = work[sj] / ljj
        col[0] = ljj
        vals[j] = col
    return vals


def solve_lower(n, structs, vals, b):
    """Forward substitution L z = b (column oriented)."""
    z = np.array(b, dtype=np.float64, copy=True)
    for j in range(n):
        z[j] /= vals[j][0]
        z[structs[j][1:]] -= vals[j][1:] * z[j]
    return z


def solve_upper(n, structs, vals, z):
    """Backward substitution L^T w = z (column oriented)."""
    w = np.array(z, dtype=np.float64, copy=True)
    for j in range(n - 1, -1, -1):
        w[j] = (w[j] - np.dot(vals[j][1:], w[structs[j][1:]])) / vals[j][0]
    return w


def to_dense_L(n, structs, vals):
    L = np.zeros((n, n))
    for j in range(n):
        L[structs[j], j] = vals[j]
    return L


class SparseCholesky:
    """Symbolic structure + numeric factor of P K P^T; ``solve`` applies
    K^{-1} in the original ordering."""

    def __init__(self, sym, n, K_rows, K_cols, K_vals):
        self.sym = sym
        self.n = n
        self.perm = sym.perm
        lower = permuted_lower(n, K_rows, K_cols, K_vals, sym.perm)
        self.vals = factor(n, sym.structs, lower)

    def solve(self, b):
        bp = np.asarray(b, dtype=np.float64)[self.perm]
        z = solve_lower(self.n, self.sym.structs, self.vals, bp)
        w = solve_upper(self.n, self.sym.structs, self.vals, z)
        x = np.empty(self.n)
        x[self.perm] = w
        return x
