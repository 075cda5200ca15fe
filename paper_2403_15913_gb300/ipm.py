"""Binding of the device IPM driver (kkt_ipm_* in include/kkt.h): argument
marshalling only; every step runs in the CUDA library."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat
from .solver import KKTError, _dptr, _stream, default_options


class IPMSolver:
    """Minimal filter line-search IPM on the column model, on the device."""

    def __init__(self, params, scheme="lifted", tol=1e-8, max_iter=200, mu_init=0.1,
                 relaxed=None, tau_relax=1e-8, **kkt_options):
        self.params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        L = nat.lib()
        ko = default_options(scheme=scheme, **kkt_options)
        io = nat.IPMOptions()
        L.kkt_ipm_default_options(ctypes.byref(io))
        io.tol, io.max_iter, io.mu_init, io.tau_relax = tol, max_iter, mu_init, tau_relax
        io.relaxed = -1 if relaxed is None else int(bool(relaxed))
        self.max_iter = max_iter
        h = ctypes.c_void_p()
        st = L.kkt_ipm_create(nat.ptr_f64(self.params), ctypes.byref(ko), ctypes.byref(io),
                              ctypes.byref(h))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_create failed")
        self._h = h
        n, m = ctypes.c_int(), ctypes.c_int()
        L.kkt_tray_sizes(nat.ptr_f64(self.params), ctypes.byref(n), ctypes.byref(m), None, None)
        self.n, self.m = n.value, m.value
        self.info = nat.IPMInfo()

    def set_initial_state(self, x0=None, stream=None):
        """Pin the stage-0 compositions to x0 (k values) for the next init;
        None restores xbar_0."""
        a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        st = nat.lib().kkt_ipm_set_initial_state(self._h, None if a is None else nat.ptr_f64(a),
                                                 _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_set_initial_state failed")

    def init_shifted(self, prev, stream=None):
        """Start from a previous solution shifted by one stage."""
        st = nat.lib().kkt_ipm_init_shifted(self._h, _dptr(prev), _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_init_shifted failed")

    def init_warm(self, mu=1e-4, recenter=True, stream=None):
        """Warm start from this solver's last iterate shifted one stage
        (multipliers included, or recentred on mu), barrier parameter mu."""
        st = nat.lib().kkt_ipm_init_warm(self._h, float(mu), int(bool(recenter)), _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_init_warm failed")

    def device_bytes(self):
        b = ctypes.c_int64()
        nat.lib().kkt_ipm_device_bytes(self._h, ctypes.byref(b))
        return b.value

    def init(self, x0=None, stream=None):
        st = nat.lib().kkt_ipm_init(self._h, _dptr(x0), _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_init failed")

    def step(self, stream=None):
        """One iteration; returns the status code (0 stepped, 1 converged,
        negative: error such as a failed line search)."""
        return nat.lib().kkt_ipm_step(self._h, _stream(stream), ctypes.byref(self.info))

    def solve(self, stream=None):
        history = []
        for _ in range(self.max_iter + 1):
            st = self.step(stream)
            history.append(dict(self.info.as_dict(), status=st))
            if st != nat.KKT_OK:
                break
        return history

    def get(self, stream=None):
        import torch
        x = torch.empty(self.n, dtype=torch.float64, device="cuda")
        y = torch.empty(self.m, dtype=torch.float64, device="cuda")
        zl = torch.empty(self.n, dtype=torch.float64, device="cuda")
        zu = torch.empty(self.n, dtype=torch.float64, device="cuda")
        s = torch.zeros(self.m, dtype=torch.float64, device="cuda")
        st = nat.lib().kkt_ipm_get(self._h, _dptr(x), _dptr(y), _dptr(zl), _dptr(zu), _dptr(s),
                                   _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_get failed")
        return x, y, zl, zu, s

    def kkt_stats(self):
        ctx = nat.lib().kkt_ipm_kkt(self._h)
        out = nat.Stats()
        nat.lib().kkt_get_stats(ctx, ctypes.byref(out))
        return out.as_dict()

    def set_profiling(self, on=True):
        nat.lib().kkt_set_profiling(nat.lib().kkt_ipm_kkt(self._h), int(bool(on)))

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().kkt_ipm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Member(IPMSolver):
    """A member of an IPMBatch: the IPMSolver calls that set up or read one
    problem (init, init_shifted, init_warm, set_initial_state, get); it steps
    only with its batch and does not own its handle."""

    def __init__(self, handle, params):
        self._h = handle
        self._owned = False
        self.params = params
        L = nat.lib()
        n, m = ctypes.c_int(), ctypes.c_int()
        L.kkt_tray_sizes(nat.ptr_f64(self.params), ctypes.byref(n), ctypes.byref(m), None, None)
        self.n, self.m = n.value, m.value
        self.info = nat.IPMInfo()

    def close(self):
        self._h = None


class IPMBatch:
    """Lock-step IPMs over many column problems with one batched KKT factor
    and solve per iteration (kkt_ipm_batch_*)."""

    def __init__(self, params_list, scheme="lifted", tol=1e-8, max_iter=200, mu_init=0.1,
                 relaxed=None, tau_relax=1e-8, **kkt_options):
        self.params = np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.float64) for p in params_list]))
        self.count = len(params_list)
        L = nat.lib()
        ko = default_options(scheme=scheme, **kkt_options)
        io = nat.IPMOptions()
        L.kkt_ipm_default_options(ctypes.byref(io))
        io.tol, io.max_iter, io.mu_init, io.tau_relax = tol, max_iter, mu_init, tau_relax
        io.relaxed = -1 if relaxed is None else int(bool(relaxed))
        h = ctypes.c_void_p()
        st = L.kkt_ipm_batch_create(self.count, nat.ptr_f64(self.params), ctypes.byref(ko),
                                    ctypes.byref(io), ctypes.byref(h))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_ipm_batch_create failed")
        self._h = h
        self.members = [_Member(L.kkt_ipm_batch_member(h, i), self.params[i]) for i in range(self.count)]
        self.infos = (nat.IPMInfo * self.count)()

    def init(self, stream=None):
        for mem in self.members:
            mem.init(stream=stream)

    def step(self, stream=None):
        """One lock-step iteration: 0 while some member iterates, 1 when none
        does, negative on a batch-wide error."""
        return nat.lib().kkt_ipm_batch_step(self._h, _stream(stream), self.infos)

    def solve(self, stream=None):
        """Iterate until no member iterates; returns (statuses, iterations)
        per member (1 = converged)."""
        status = np.zeros(self.count, np.int32)
        iters = np.zeros(self.count, np.int32)
        st = nat.lib().kkt_ipm_batch_solve(self._h, _stream(stream), nat.ptr_i32(status), nat.ptr_i32(iters),
                                           self.infos)
        if st not in (nat.KKT_CONVERGED, nat.KKT_ERR_MAXIT, nat.KKT_ERR_STALL, nat.KKT_ERR_NOT_SPD):
            raise KKTError(st, nat.lib().kkt_ipm_batch_last_error(self._h).decode())
        return status, iters

    def start_member(self, i):
        """Continuous batching: member i (initialised since it last stopped)
        joins the following steps."""
        st = nat.lib().kkt_ipm_batch_start_member(self._h, int(i))
        if st != nat.KKT_OK:
            raise KKTError(st, nat.lib().kkt_ipm_batch_last_error(self._h).decode())

    def member_status(self, i):
        """(status, iterations) of member i: status 0 while it iterates."""
        s = np.zeros(1, np.int32)
        it = np.zeros(1, np.int32)
        nat.lib().kkt_ipm_batch_member_status(self._h, int(i), nat.ptr_i32(s), nat.ptr_i32(it))
        return int(s[0]), int(it[0])

    def device_bytes(self):
        b = ctypes.c_int64()
        nat.lib().kkt_ipm_batch_device_bytes(self._h, ctypes.byref(b))
        return b.value

    def info(self, i):
        return self.infos[i].as_dict()

    def kkt_stats(self):
        out = nat.Stats()
        nat.lib().kkt_get_stats(nat.lib().kkt_ipm_batch_kkt(self._h), ctypes.byref(out))
        return out.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            for mem in self.members:
                mem.close()
            nat.lib().kkt_ipm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
