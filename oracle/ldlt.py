"""Oracle O2: dense symmetric indefinite LDL^T with Bunch-Kaufman pivoting.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The KKT matrix K_orig of Eq. (kkt:condensed) is symmetric and indefinite, with
inertia (n, 0, m) when the step is well defined (Eq. inertia).  Its plain
dense factorisation is P K P^T = L D L^T, L unit lower triangular and D
block diagonal with 1x1 and 2x2 blocks, by the partial-pivoting strategy of
Bunch and Kaufman ("Some stable methods for calculating inertia and solving
symmetric linear systems", Math. Comp. 31, 1977).  At step k, on the active
trailing matrix A (rows and columns k..N-1), with alpha = (1 + sqrt(17)) / 8:

    lambda = max_{i > k} |A_ik|            attained at row r
    if max(|A_kk|, lambda) = 0:            1x1 block D_k = 0 (column is zero)
    elif |A_kk| >= alpha lambda:           1x1 pivot A_kk
    else:
        sigma = max_{i >= k, i != r} |A_ir|
        if |A_kk| sigma >= alpha lambda^2: 1x1 pivot A_kk
        elif |A_rr| >= alpha sigma:        1x1 pivot A_rr (swap k and r)
        else:                              2x2 pivot on (k, r) (swap k+1 and r)

followed by the symmetric rank-1 or rank-2 elimination of the pivot columns.
Every 2x2 block so chosen has a negative determinant (|A_kk A_rr| < alpha^2
lambda^2 < lambda^2 = A_rk^2), so it holds one positive and one negative
eigenvalue; Sylvester's law of inertia then reads In(K) off D.

Solutions of K v = b follow by substitution with L, D and L^T.  The
elimination is unblocked and runs one Python-level step per column; it is
meant for the small dense systems of the tests (a few thousand unknowns at
most).

Parity: pinned by tests: the factorisation residual ||P K P^T - L D L^T||
against the unit roundoff on random indefinite and KKT matrices hitting all
four pivot cases; the determinant sign of every 2x2 block; inertia against
the eigenvalues (LAPACK ``eigvalsh``); solutions against LAPACK's LU solve;
no pivoting and D = diag(L_chol)^2 on diagonally dominant SPD matrices
(checked against a Cholesky factor); the 2x2 pivot of [[0, 1], [1, 0]].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

ALPHA = (1.0 + np.sqrt(17.0)) / 8.0

# pivot kinds recorded per step (for the tests that check every case ran)
PIV_ZERO, PIV_KK, PIV_KK_SIGMA, PIV_RR, PIV_2X2 = range(5)


@dataclass
class LDLT:
    """P K P^T = L D L^T.  ``perm[i]`` is the row of K placed at position i;
    D is stored as its diagonal ``d`` and first subdiagonal ``e`` (nonzero
    only inside 2x2 blocks); ``blocks`` lists (start, size) in order."""
    perm: np.ndarray
    L: np.ndarray
    d: np.ndarray
    e: np.ndarray
    blocks: list = field(default_factory=list)
    kinds: list = field(default_factory=list)

    def D(self):
        N = len(self.d)
        Dm = np.diag(self.d)
        idx = np.arange(N - 1)
        Dm[idx + 1, idx] = self.e
        Dm[idx, idx + 1] = self.e
        return Dm

    def inertia(self):
        """(n_plus, n_zero, n_minus) by Sylvester's law on D's blocks."""
        npos = nzero = nneg = 0
        for k, s in self.blocks:
            if s == 1:
                v = self.d[k]
                npos += v > 0
                nneg += v < 0
                nzero += v == 0
            else:
                det = self.d[k] * self.d[k + 1] - self.e[k] * self.e[k]
                tr = self.d[k] + self.d[k + 1]
                if det < 0:
                    npos += 1
                    nneg += 1
                elif det > 0:
                    npos += 2 if tr > 0 else 0
                    nneg += 2 if tr < 0 else 0
                else:
                    nzero += 1
                    npos += tr > 0
                    nneg += tr < 0
                    nzero += tr == 0
        return int(npos), int(nzero), int(nneg)

    def solve(self, b):
        """v with K v = b: L y = P b, D z = y, L^T w = z, v = P^T w."""
        y = scipy.linalg.solve_triangular(self.L, np.asarray(b, dtype=np.float64)[self.perm],
                                          lower=True, unit_diagonal=True)
        z = np.empty_like(y)
        for k, s in self.blocks:
            if s == 1:
                if self.d[k] == 0.0:
                    raise np.linalg.LinAlgError(f"singular: zero pivot at {k}")
                z[k] = y[k] / self.d[k]
            else:
                a, c, bb = self.d[k], self.d[k + 1], self.e[k]
                det = a * c - bb * bb
                z[k] = (c * y[k] - bb * y[k + 1]) / det
                z[k + 1] = (a * y[k + 1] - bb * y[k]) / det
        w = scipy.linalg.solve_triangular(self.L.T, z, lower=False, unit_diagonal=True)
        v = np.empty_like(w)
        v[self.perm] = w
        return v


def _swap(A, L, perm, i, j, k):
    """Symmetric interchange of positions i and j (both >= k) of the active
    matrix, with the rows of the finished columns of L and the permutation."""
    if i == j:
        return
    A[[i, j], :] = A[[j, i], :]
    A[:, [i, j]] = A[:, [j, i]]
    L[[i, j], :k] = L[[j, i], :k]
    perm[[i, j]] = perm[[j, i]]


def factor(K) -> LDLT:
    """Bunch-Kaufman LDL^T of the dense symmetric matrix K (both triangles
    given; only the symmetric part is meaningful)."""
    A = np.array(K.toarray() if hasattr(K, "toarray") else K, dtype=np.float64, copy=True)
    N = A.shape[0]
    assert A.shape == (N, N)
    perm = np.arange(N)
    L = np.eye(N)
    d = np.zeros(N)
    e = np.zeros(max(N - 1, 0))
    blocks, kinds = [], []
    k = 0
    while k < N:
        akk = abs(A[k, k])
        if k + 1 < N:
            col = np.abs(A[k + 1:, k])
            r = k + 1 + int(np.argmax(col))
            lam = float(col[r - k - 1])
        else:
            r, lam = k, 0.0
        if max(akk, lam) == 0.0:
            s, kind = 1, PIV_ZERO
        elif akk >= ALPHA * lam:
            s, kind = 1, PIV_KK
        else:
            colr = np.abs(A[k:, r])
            colr[r - k] = 0.0
            sigma = float(np.max(colr))
            if akk * sigma >= ALPHA * lam * lam:
                s, kind = 1, PIV_KK_SIGMA
            elif abs(A[r, r]) >= ALPHA * sigma:
                s, kind = 1, PIV_RR
                _swap(A, L, perm, k, r, k)
            else:
                s, kind = 2, PIV_2X2
                _swap(A, L, perm, k + 1, r, k)
        if s == 1:
            piv = A[k, k]
            d[k] = piv
            if kind != PIV_ZERO:
                c = A[k + 1:, k].copy()
                l = c / piv
                A[k + 1:, k + 1:] -= np.outer(l, c)
                L[k + 1:, k] = l
        else:
            E = A[k:k + 2, k:k + 2].copy()
            C = A[k + 2:, k:k + 2].copy()
            det = E[0, 0] * E[1, 1] - E[0, 1] * E[1, 0]
            Einv = np.array([[E[1, 1], -E[0, 1]], [-E[1, 0], E[0, 0]]]) / det
            Lc = C @ Einv
            A[k + 2:, k + 2:] -= Lc @ C.T
            L[k + 2:, k:k + 2] = Lc
            d[k], d[k + 1], e[k] = E[0, 0], E[1, 1], E[1, 0]
        blocks.append((k, s))
        kinds.append(kind)
        k += s
    return LDLT(perm, L, d, e, blocks, kinds)
