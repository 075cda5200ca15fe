"""Planted-mistake check of the oracle's pins (run by hand: python tests/mutants.py).

TEST INFRASTRUCTURE.  The oracle is trusted only because its pins (the
``-m "not gpu"`` tests of ``tests/test_oracle_*.py``) fail when it is wrong.
This script checks that claim: for every entry of MUTANTS it copies
``oracle/``, ``gen/`` and ``tests/`` into a temporary directory, plants one
plausible mistake in the copy (a dropped term, a flipped sign, a wrong index,
a rule's constant or comparison changed, a step skipped) and runs the pins
of that module there.  A mistake that no pin notices "survives".  The
repository's own files are never modified, and every run has a time limit
(a mistake that makes a pin loop forever counts as noticed).

Entries marked EXPECTED_SURVIVOR are rule details of the cited filter
line-search method that change the IPM's iteration counts but not its
optimum; the oracle's header and the design notes state that their parity is
pinned only through the optimum.  The script exits non-zero when any other
mistake survives.
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXPECTED_SURVIVOR = "expected"

# (file, pins, text in the file, text planted instead[, EXPECTED_SURVIVOR])
MUTANTS = [
    # oracle/ldlt.py  (pins: tests/test_oracle_ldlt.py)
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'L[[i, j], :k] = L[[j, i], :k]',
     'pass'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'Einv = np.array([[E[1, 1], -E[0, 1]]',
     'Einv = np.array([[E[1, 1], E[0, 1]]'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'colr[r - k] = 0.0',
     'pass'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     '_swap(A, L, perm, k + 1, r, k)',
     '_swap(A, L, perm, k, r, k)'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'elif abs(A[r, r]) >= ALPHA * sigma:',
     'elif abs(A[r, r]) >= ALPHA * lam:'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'npos += 1\n                    nneg += 1',
     'npos += 2'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'A[k + 2:, k + 2:] -= Lc @ C.T',
     'A[k + 2:, k + 2:] += Lc @ C.T'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'if akk * sigma >= ALPHA * lam * lam:',
     'if akk * sigma >= ALPHA * lam:'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'colr = np.abs(A[k:, r])',
     'colr = np.abs(A[k + 1:, r])'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'z[k + 1] = (a * y[k + 1] - bb * y[k]) / det',
     'z[k + 1] = (a * y[k + 1] + bb * y[k]) / det'),
    ('oracle/ldlt.py', 'tests/test_oracle_ldlt.py',
     'v[self.perm] = w',
     'v = w[self.perm]'),
    # oracle/kkt.py  (pins: tests/test_oracle_kkt.py)
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'dx = chol.solve(r1 + Jm.T @ (D * r2))',
     'dx = chol.solve(r1 - Jm.T @ (D * r2))'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'dy = D * (Jm @ dx - r2)',
     'dy = D * (Jm @ dx + r2)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'dx = chol.solve(r1 + Jm.T @ (D * r2))',
     'dx = chol.solve(r1)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'r_gamma = r1 + gamma * (Jm.T @ r2)',
     'r_gamma = r1 - gamma * (Jm.T @ r2)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'rhs = Jm @ q - r2',
     'rhs = Jm @ q + r2'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'dx = chol.solve(r_gamma - Jm.T @ dy)',
     'dx = chol.solve(r_gamma + Jm.T @ dy)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'p = r + (rr_new / rr) * p',
     'p = r + (rr / rr_new) * p'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'v = v + precond(r)',
     'v = precond(r)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'vals = np.concatenate([v, v[off], np.asarray(sigma) + delta_x])',
     'vals = np.concatenate([v, v[off], np.asarray(sigma)])'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'vals = np.concatenate([v, v[off], np.asarray(sigma) + delta_x])',
     'vals = np.concatenate([v, v, np.asarray(sigma) + delta_x])'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'Cm = sp.diags(np.zeros(m) if C is None else -np.asarray(C))',
     'Cm = sp.diags(np.zeros(m) if C is None else np.asarray(C))'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'return sp.bmat([[H, Jm.T], [Jm, Cm]], format="csr")',
     'return sp.bmat([[H, Jm], [Jm.T, Cm]], format="csr")'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'K = (H + Jm.T @ sp.diags(np.asarray(D)) @ Jm).tocoo()',
     'K = (H + Jm.T @ Jm).tocoo()'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'return float(np.max(np.abs(r)) / (kn * np.max(np.abs(v)) + np.max(np.abs(b))))',
     'return float(np.max(np.abs(r)) / (kn * np.max(np.abs(v))))'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'return float(np.max(np.asarray(abs(K).sum(axis=1)).ravel()))',
     'return float(np.max(np.asarray(abs(K).sum(axis=0)).ravel()) * 0.5)'),
    ('oracle/kkt.py', 'tests/test_oracle_kkt.py',
     'for _ in range(refine_steps):\n        v = v + solve(b - Kd @ v)',
     'for _ in range(refine_steps):\n        v = solve(b - Kd @ v)'),
    # oracle/cholesky.py  (pins: tests/test_oracle_kkt.py)
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'keep = r >= c',
     'keep = r > c'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'd[a] = d.get(a, 0.0) + v',
     'd[a] = v'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'work[sk] -= lk * lk[0]',
     'work[sk] -= lk * lk[-1]'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'work[sk] -= lk * lk[0]',
     'work[sk] += lk * lk[0]'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'if not (d > 0.0) or not np.isfinite(d):',
     'if not (d >= 0.0) or not np.isfinite(d):'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'col = work[sj] / ljj',
     'col = work[sj] / d'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'z[structs[j][1:]] -= vals[j][1:] * z[j]',
     'z[structs[j][1:]] += vals[j][1:] * z[j]'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'w[j] = (w[j] - np.dot(vals[j][1:], w[structs[j][1:]])) / vals[j][0]',
     'w[j] = (w[j] - np.dot(vals[j][1:], w[structs[j][1:]]))'),
    ('oracle/cholesky.py', 'tests/test_oracle_kkt.py',
     'sk = structs[k][pos:]',
     'sk = structs[k][pos + 1:]'),
    # oracle/tray.py  (pins: tests/test_oracle_tray.py)
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'g[:, n] = V * (y[:, 1] - x[:, 0])',
     'g[:, n] = V * (y[:, 0] - x[:, 0])'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'g[:, n] = L * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n + 1])',
     'g[:, n] = L * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n - 1])'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'g[:, n] = (p.F * p.xf + L * x[:, n - 1] - S * x[:, n]',
     'g[:, n] = (p.F + L * x[:, n - 1] - S * x[:, n]'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'g[:, n] = S * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n + 1])',
     'g[:, n] = L * (x[:, n - 1] - x[:, n]) - V * (y[:, n] - y[:, n + 1])'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'g[:, n] = S * x[:, n - 1] - (p.F - p.D) * x[:, n] - V * y[:, n]',
     'g[:, n] = S * x[:, n - 1] - p.F * x[:, n] - V * y[:, n]'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'V = L + p.D',
     'V = L'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'S = p.F + L',
     'S = L'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'return p.alpha * x / (1.0 + (p.alpha - 1.0) * x)',
     'return p.alpha * x / (1.0 + (p.alpha + 1.0) * x)'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'return -2.0 * p.alpha * (p.alpha - 1.0) / (1.0 + (p.alpha - 1.0) * x) ** 3',
     'return 2.0 * p.alpha * (p.alpha - 1.0) / (1.0 + (p.alpha - 1.0) * x) ** 3'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'liq_in = L if n <= kf else S',
     'liq_in = L if n < kf else S'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     "out.append(('u', None, D * x[:, n - 1] - D * y[:, n]))",
     "out.append(('u', None, D * x[:, n - 1] + D * y[:, n]))"),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     "return [('x', n - 1, D), ('y', n, -D)]",
     "return [('x', n - 1, D), ('y', n, D)]"),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'cb[1:, :p.k] = x[1:] - x[:-1] - (p.h / p.M) * g',
     'cb[1:, :p.k] = x[1:] - x[:-1] - p.h * g'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'gu[:] = 2.0 * p.rho * (u - p.ubar)',
     'gu[:] = 2.0 * (u - p.ubar)'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'du += obj_weight * 2.0 * p.rho',
     'du += obj_weight * 2.0'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'dx -= lamb[:, k:] * vle_d2(p, x)',
     'dx += lamb[:, k:] * vle_d2(p, x)'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'ux[1:, i] += -hm * v * ln',
     'ux[1:, i] += hm * v * ln'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     'uy[1:, i] += -hm * v * ln',
     'uy[:-1, i] += -hm * v * ln'),
    ('oracle/tray.py', 'tests/test_oracle_tray.py',
     "add(r, _col(p, 'x', t1 - 1, n), -np.ones(T))",
     "add(r, _col(p, 'x', t1, n), -np.ones(T))"),
    # oracle/symbolic.py  (pins: tests/test_oracle_symbolic.py)
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'adj[a].add(b)',
     'pass'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'v = min(last, key=lambda w: (degree_in(adj, w, comp), w))',
     'v = max(last, key=lambda w: (degree_in(adj, w, comp), w))'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'v = min(last, key=lambda w: (degree_in(adj, w, comp), w))',
     'v = min(last, key=lambda w: (degree_in(adj, w, comp), -w))'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'v = min(g, key=lambda w: (len(g[w]), w))',
     'v = min(g, key=lambda w: (len(g[w]), -w))'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'g[a] |= (nb - {a})',
     'pass'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'lv = e // 2',
     'lv = (e + 1) // 2'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'below = set(levels[lv + 1])',
     'below = set(levels[lv - 1])'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'return out + sep',
     'return sep + out'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'if e < 2:',
     'if e < 1:'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'while ancestor[r] != -1 and ancestor[r] != j:',
     'while ancestor[r] != -1 and ancestor[r] != j and False:'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'stack.append((v, ci + 1))\n                stack.append((children[v][ci], 0))',
     'stack.append((children[v][ci], 0))\n                stack.append((v, ci + 1))'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     's.discard(c)',
     'pass'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'joins = (parent[j] == j + 1 and cc[j] == cc[j + 1] + 1',
     'joins = (parent[j] == j + 1 and cc[j] >= cc[j + 1]'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'and nchild[j + 1] == 1)',
     'and nchild[j + 1] >= 1)'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'r |= {i for i in rows[c] if i > l}',
     'pass'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'sparent[s] = snode[below[0]]',
     'sparent[s] = snode[below[-1]]'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'ok = ncol <= relax_cols and slots - true_nnz <= relax_zeros',
     'ok = ncol <= relax_cols'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'slots = ncol * nrow - ncol * (ncol - 1) // 2',
     'slots = ncol * nrow'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'c = f + max_width',
     'c = f + max_width + 1'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'perm = perm0[post]',
     'perm = perm0'),
    ('oracle/symbolic.py', 'tests/test_oracle_symbolic.py',
     'for s in sorted(nodes):',
     'for s in sorted(nodes, reverse=True):'),
    # oracle/ipm.py  (pins: tests/test_oracle_ipm.py)
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'sigma = self.zl / gl + self.zu / gu',
     'sigma = self.zl / gl - self.zu / gu'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'gphi = g - mu / gl + mu / gu',
     'gphi = g - mu / gl - mu / gu'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'dzu = mu / gu - self.zu + (self.zu / gu) * dx',
     'dzu = mu / gu - self.zu - (self.zu / gu) * dx'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'tau = max(o.tau_min, 1.0 - mu)',
     'tau = o.tau_min', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'self.mu = max(o.tol / 10, min(o.kappa_mu * self.mu, self.mu ** o.theta_mu))',
     'self.mu = max(o.tol / 10, o.kappa_mu * self.mu)'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'ry = -(c - s) - (gphi_s - self.y) / sig_s',
     'ry = -(c - s) + (gphi_s - self.y) / sig_s'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'ok = pht <= ph + o.eta_phi * alpha * dphi',
     'ok = pht <= ph', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'self.zl = np.maximum(np.minimum(self.zl, k * mu / gl), mu / (k * gl))',
     'pass', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'a_du = min(_max_step_pos(self.zl, dzl, tau), _max_step_pos(self.zu, dzu, tau))',
     'a_du = _max_step_pos(self.zl, dzl, tau)', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'du = g + Jm.T @ self.y - self.zl + self.zu',
     'du = g + Jm.T @ self.y'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'if not f_type:\n                    self.filter.append',
     'if True:\n                    self.filter.append', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'ds = (dy - gphi_s + self.y) / sig_s',
     'ds = (dy + gphi_s - self.y) / sig_s'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     's_d = max(o.s_max, sum_mult / cnt_mult) / o.s_max',
     's_d = 1.0', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'if errmu > o.kappa_eps * self.mu:',
     'if errmu > self.mu:', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'self.y = self.y + alpha * dy',
     'self.y = self.y + a_du * dy', EXPECTED_SURVIVOR),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'alpha *= 0.5',
     'alpha *= 0.9'),
    ('oracle/ipm.py', 'tests/test_oracle_ipm.py',
     'return float(np.sum(np.abs(c)))',
     'return float(np.sqrt(np.sum(c * c)))', EXPECTED_SURVIVOR),
]


def run(entry, timeout=120):
    path, pins, old, new = entry[:4]
    with tempfile.TemporaryDirectory(prefix="oracle_mutant_") as tmp:
        for d in ("oracle", "gen", "tests"):
            shutil.copytree(os.path.join(ROOT, d), os.path.join(tmp, d),
                            ignore=shutil.ignore_patterns("__pycache__", "test_gpu_*", "test_zz_*"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp)
        target = os.path.join(tmp, path)
        src = open(target).read()
        if old not in src:
            return "missing"          # the oracle changed: update the table
        with open(target, "w") as f:
            f.write(src.replace(old, new, 1))
        try:
            r = subprocess.run([sys.executable, "-m", "pytest", pins, "-q", "-x", "-m", "not gpu",
                                "-p", "no:cacheprovider"], cwd=tmp, capture_output=True,
                               text=True, timeout=timeout)
        except subprocess.TimeoutExpired:
            return "noticed (pins hang)"
        return "survived" if r.returncode == 0 else "noticed"


def main():
    unexpected = 0
    for entry in MUTANTS:
        res = run(entry)
        expected = len(entry) > 4
        if res in ("survived", "missing") and not expected:
            unexpected += 1
        tag = " (expected: optimum-level pin only)" if expected else ""
        print(f"{res:22s} {entry[0]}: {entry[2][:60]!r}{tag}", flush=True)
    print(f"{len(MUTANTS)} planted mistakes, {unexpected} unexpected survivors")
    return 1 if unexpected else 0


if __name__ == "__main__":
    sys.exit(main())
