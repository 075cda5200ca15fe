"""Python binding of the KKT solver: one object per symbolic analysis.

Every numeric step runs in the CUDA library through the C ABI; this module
only converts arguments (numpy index arrays for patterns, torch CUDA FP64
tensors for values, torch's current stream).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native as nat


class KKTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{nat.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _dptr(t):
    """Device pointer of a contiguous CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_options(**kw) -> nat.Options:
    o = nat.Options()
    nat.lib().kkt_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "scheme" and isinstance(v, str):
            v = {"lifted": nat.KKT_LIFTED, "hykkt": nat.KKT_HYKKT}[v]
        setattr(o, k, v)
    return o


@dataclass
class SymbolicSizes:
    ns: int
    nnz_L: int
    panel: int
    row_entries: int
    levels: int
    flops: float


class KKTSolver:
    """Symbolic analysis once (``kkt_analyse``), then any number of
    ``factor``/``solve`` calls with new values on the same pattern."""

    def __init__(self, n, m, W_colptr, W_rowind, J_rowptr, J_colind, host_only=False, **options):
        self.n, self.m = int(n), int(m)
        self._keep = [_i32(W_colptr), _i32(W_rowind), _i32(J_rowptr), _i32(J_colind)]
        self.options = default_options(**options)
        L = nat.lib()
        ctx = ctypes.c_void_p()
        fn = L.kkt_analyse_host if host_only else L.kkt_analyse
        st = fn(self.n, self.m, *[nat.ptr_i32(a) for a in self._keep],
                ctypes.byref(self.options), ctypes.byref(ctx))
        if st != nat.KKT_OK:
            raise KKTError(st, L.kkt_last_error(None).decode())
        self._ctx = ctx
        self.info = nat.Info()

    # ------------------------------------------------------------- symbolic
    def sizes(self) -> SymbolicSizes:
        ns = ctypes.c_int()
        nnz, panel, rows = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lev = ctypes.c_int()
        fl = ctypes.c_double()
        self._check(nat.lib().kkt_symbolic_sizes(self._ctx, ctypes.byref(ns), ctypes.byref(nnz),
                                                 ctypes.byref(panel), ctypes.byref(rows),
                                                 ctypes.byref(lev), ctypes.byref(fl)))
        return SymbolicSizes(ns.value, nnz.value, panel.value, rows.value, lev.value, fl.value)

    def symbolic(self) -> dict:
        s = self.sizes()
        out = dict(perm=np.empty(self.n, np.int32), parent=np.empty(self.n, np.int32),
                   colcount=np.empty(self.n, np.int32), sn_ptr=np.empty(s.ns + 1, np.int32),
                   sn_rowptr=np.empty(s.ns + 1, np.int32),
                   sn_rows=np.empty(max(1, s.row_entries), np.int32))
        self._check(nat.lib().kkt_symbolic_export(
            self._ctx, *[nat.ptr_i32(out[k]) for k in
                         ("perm", "parent", "colcount", "sn_ptr", "sn_rowptr", "sn_rows")]))
        out["sn_rows"] = out["sn_rows"][:s.row_entries]
        return out

    # ------------------------------------------------------------- numeric
    def factor(self, Wval, Jval, sigma, D=None, delta_x=0.0, stream=None):
        """Refactorise with new values.  Returns the status code (0 or
        KKT_ERR_NOT_SPD; other errors raise)."""
        st = nat.lib().kkt_factor(self._ctx, _dptr(Wval), _dptr(Jval), _dptr(sigma), _dptr(D),
                                  float(delta_x), _stream(stream), ctypes.byref(self.info))
        if st not in (nat.KKT_OK, nat.KKT_ERR_NOT_SPD):
            self._check(st)
        return st

    def solve(self, rx, ry, dx, dy, ds=None, stream=None):
        """Solve K_orig [dx; dy] = [rx; ry] into the given tensors.  Returns
        the status code (0, KKT_ERR_MAXIT or KKT_ERR_STALL; others raise)."""
        st = nat.lib().kkt_solve(self._ctx, _dptr(rx), _dptr(ry), _dptr(dx), _dptr(dy), _dptr(ds),
                                 _stream(stream), ctypes.byref(self.info))
        if st not in (nat.KKT_OK, nat.KKT_ERR_MAXIT, nat.KKT_ERR_STALL):
            self._check(st)
        return st

    def factor_solve(self, Wval, Jval, sigma, D, delta_x, rx, ry, dx, dy, stream=None):
        """``factor`` then ``solve`` as one CUDA graph launch
        (``kkt_factor_solve``); ``delta_x`` is one value per instance (a
        float for a single system).  Returns the status (KKT_ERR_NOT_SPD
        when some instance's pivot failed, else as ``solve``)."""
        d = np.ascontiguousarray(np.atleast_1d(np.asarray(delta_x, dtype=np.float64)))
        st = nat.lib().kkt_factor_solve(self._ctx, _dptr(Wval), _dptr(Jval), _dptr(sigma), _dptr(D),
                                        nat.ptr_f64(d), _dptr(rx), _dptr(ry), _dptr(dx), _dptr(dy),
                                        _stream(stream), ctypes.byref(self.info))
        if st not in (nat.KKT_OK, nat.KKT_ERR_MAXIT, nat.KKT_ERR_STALL, nat.KKT_ERR_NOT_SPD):
            self._check(st)
        return st

    def backsolve(self, b, x, stream=None):
        """x = K^{-1} b with the current factor (condensed matrix only)."""
        self._check(nat.lib().kkt_backsolve(self._ctx, _dptr(b), _dptr(x), _stream(stream)))

    def factor_export(self):
        """Numeric factor L (permuted order) as CSC numpy arrays."""
        s = self.sizes()
        colptr = np.empty(self.n + 1, np.int64)
        rowind = np.empty(s.panel, np.int32)
        val = np.empty(s.panel, np.float64)
        self._check(nat.lib().kkt_factor_export(self._ctx, nat.ptr_i64(colptr), nat.ptr_i32(rowind),
                                                nat.ptr_f64(val)))
        return colptr, rowind, val

    def set_profiling(self, on=True):
        self._check(nat.lib().kkt_set_profiling(self._ctx, int(bool(on))))

    def stats(self) -> dict:
        st = nat.Stats()
        self._check(nat.lib().kkt_get_stats(self._ctx, ctypes.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self._check(nat.lib().kkt_reset_stats(self._ctx))

    def last_error(self):
        return nat.lib().kkt_last_error(self._ctx).decode()

    def _check(self, st):
        if st != nat.KKT_OK:
            raise KKTError(st, self.last_error())

    def close(self):
        if getattr(self, "_ctx", None):
            nat.lib().kkt_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKTBatchSolver(KKTSolver):
    """A batch of independent systems of uneven sizes, factorised and solved
    together (``kkt_analyse_batch``).  ``instances`` is a sequence of
    (n, m, W_colptr, W_rowind, J_rowptr, J_colind); value arrays and vectors
    are the instances' arrays concatenated in order (see ``layout``)."""

    def __init__(self, instances, host_only=False, **options):
        inst = [tuple(x) for x in instances]
        self.count = len(inst)
        ns = np.array([int(x[0]) for x in inst], np.int32)
        ms = np.array([int(x[1]) for x in inst], np.int32)
        self.n, self.m = int(ns.sum()), int(ms.sum())
        self._keep = [[_i32(a) for a in x[2:6]] for x in inst]
        ptrs = [(nat.I32P * self.count)(*[nat.ptr_i32(k[j]) for k in self._keep]) for j in range(4)]
        self._keep_ptrs = (ns, ms, ptrs)
        self.options = default_options(**options)
        L = nat.lib()
        ctx = ctypes.c_void_p()
        fn = L.kkt_analyse_batch_host if host_only else L.kkt_analyse_batch
        st = fn(self.count, nat.ptr_i32(ns), nat.ptr_i32(ms), *ptrs, ctypes.byref(self.options),
                ctypes.byref(ctx))
        if st != nat.KKT_OK:
            raise KKTError(st, L.kkt_last_error(None).decode())
        self._ctx = ctx
        self.info = nat.Info()

    def layout(self):
        """(x_off, y_off): instance i owns variables x_off[i]:x_off[i+1] and
        constraints y_off[i]:y_off[i+1] of the concatenated vectors."""
        xo = np.empty(self.count + 1, np.int32)
        yo = np.empty(self.count + 1, np.int32)
        self._check(nat.lib().kkt_batch_layout(self._ctx, None, nat.ptr_i32(xo), nat.ptr_i32(yo)))
        return xo, yo

    def factor_batch(self, Wval, Jval, sigma, D=None, delta_x=None, stream=None):
        """Refactorise with one delta_x per instance (default 0).  Returns
        the status (KKT_ERR_NOT_SPD when some instance failed; see results)."""
        d = np.zeros(self.count) if delta_x is None else np.ascontiguousarray(delta_x, np.float64)
        st = nat.lib().kkt_factor_batch(self._ctx, _dptr(Wval), _dptr(Jval), _dptr(sigma), _dptr(D),
                                        nat.ptr_f64(d), _stream(stream), ctypes.byref(self.info))
        if st not in (nat.KKT_OK, nat.KKT_ERR_NOT_SPD):
            self._check(st)
        return st

    def solve(self, rx, ry, dx, dy, ds=None, stream=None):
        """Solve every instance that has a factor.  Returns the status
        (KKT_ERR_NOT_SPD when some instances have none; see results)."""
        st = nat.lib().kkt_solve(self._ctx, _dptr(rx), _dptr(ry), _dptr(dx), _dptr(dy), _dptr(ds),
                                 _stream(stream), ctypes.byref(self.info))
        if st not in (nat.KKT_OK, nat.KKT_ERR_MAXIT, nat.KKT_ERR_STALL, nat.KKT_ERR_NOT_SPD):
            self._check(st)
        return st

    def results(self):
        """Per-instance status, refinement sweeps, CG iterations, backward
        error and first failing column of the last factor / solve."""
        out = dict(status=np.empty(self.count, np.int32), refine_iters=np.empty(self.count, np.int32),
                   cg_iters=np.empty(self.count, np.int32), bwd_err=np.empty(self.count),
                   failed_col=np.empty(self.count, np.int32))
        self._check(nat.lib().kkt_batch_results(
            self._ctx, nat.ptr_i32(out["status"]), nat.ptr_i32(out["refine_iters"]),
            nat.ptr_i32(out["cg_iters"]), nat.ptr_f64(out["bwd_err"]), nat.ptr_i32(out["failed_col"])))
        return out


def autotune_batch(instances, sample=32, stream=None, **options):
    """Options (relax_cols, relax_zeros, max_width, subtree_cols) whose
    batch factorisation is fastest on this GPU (``kkt_autotune_batch``);
    returns (options dict for KKTBatchSolver, median factor ms of the sample)."""
    inst = [tuple(x) for x in instances]
    cnt = len(inst)
    ns = np.array([int(x[0]) for x in inst], np.int32)
    ms = np.array([int(x[1]) for x in inst], np.int32)
    keep = [[_i32(a) for a in x[2:6]] for x in inst]
    ptrs = [(nat.I32P * cnt)(*[nat.ptr_i32(k[j]) for k in keep]) for j in range(4)]
    base = default_options(**options)
    best = nat.Options()
    t = ctypes.c_double()
    st = nat.lib().kkt_autotune_batch(cnt, nat.ptr_i32(ns), nat.ptr_i32(ms), *ptrs, ctypes.byref(base),
                                      int(sample), _stream(stream), ctypes.byref(best), ctypes.byref(t))
    if st != nat.KKT_OK:
        raise KKTError(st, nat.lib().kkt_last_error(None).decode())
    out = dict(options)
    for f in ("relax_cols", "relax_zeros", "max_width", "subtree_cols"):
        out[f] = getattr(best, f)
    return out, t.value


def eval_fn(fn, x, stream=None):
    """Evaluates one of the library's FP64 helper functions (nat.KKT_FN_*)
    elementwise on the device: y[i] = f(x[i]), or f(x[0][i], x[1][i]) for the
    binary ones (x of shape (2, n)).  x: CUDA float64 tensor; returns y."""
    import torch
    x = x.contiguous()
    n = x.shape[-1] if fn in nat.KKT_FN_BINARY else x.numel()
    if fn in nat.KKT_FN_BINARY and (x.dim() != 2 or x.shape[0] != 2):
        raise ValueError("binary helper functions take x of shape (2, n)")
    y = torch.empty(n, dtype=torch.float64, device=x.device)
    st = nat.lib().kkt_eval_fn(int(fn), int(n), _dptr(x), _dptr(y), _stream(stream))
    if st != 0:
        raise KKTError(st, "kkt_eval_fn failed")
    return y
