"""Binding of the NMPC server (kkt_server_* in include/kkt.h): argument
marshalling only; scheduling, admission and every solve run in the native
library."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat
from .solver import KKTError


class NMPCServer:
    """Concurrent receding-horizon solves of many column-model clients
    (batch > 0: cohorts of up to `batch` clients share one batched IPM whose
    iterations factorise the union of their KKT systems once)."""

    def __init__(self, slots=8, hbm_budget_gb=40.0, scheme="lifted", precision=0, gamma=1e7, tol=1e-8,
                 max_iter=200, mu_init=0.1, warm_start=True, warm_mu=1e-4, warm_recenter=True,
                 batch=0, device=None):
        import torch
        L = nat.lib()
        o = nat.ServerOptions()
        L.kkt_server_default_options(ctypes.byref(o))
        o.slots, o.hbm_budget_gb = int(slots), float(hbm_budget_gb)
        o.scheme = {"lifted": nat.KKT_LIFTED, "hykkt": nat.KKT_HYKKT}[scheme]
        o.precision, o.gamma, o.tol = int(precision), float(gamma), float(tol)
        o.max_iter, o.mu_init, o.warm_start = int(max_iter), float(mu_init), int(bool(warm_start))
        o.warm_mu = float(warm_mu)
        o.warm_recenter = int(bool(warm_recenter))
        o.batch = int(batch)
        dev = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        st = L.kkt_server_create(ctypes.byref(o), dev, ctypes.byref(h))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_server_create failed")
        self._h = h
        self.sizes = []

    def add_client(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        c = ctypes.c_int()
        st = nat.lib().kkt_server_add_client(self._h, nat.ptr_f64(p), ctypes.byref(c))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_server_add_client failed")
        n, m = ctypes.c_int(), ctypes.c_int()
        nat.lib().kkt_tray_sizes(nat.ptr_f64(p), ctypes.byref(n), ctypes.byref(m), None, None)
        self.sizes.append((n.value, m.value))
        return c.value

    def submit(self, client, x0=None, keep_solution=False):
        a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        rid = ctypes.c_int64()
        st = nat.lib().kkt_server_submit(self._h, int(client), None if a is None else nat.ptr_f64(a),
                                         int(bool(keep_solution)), ctypes.byref(rid))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_server_submit failed")
        return rid.value, int(client)

    def wait(self, ticket, want_solution=False):
        """Result dict of a submitted request (and its x if it was kept)."""
        rid, client = ticket
        r = nat.RequestResult()
        x = np.empty(self.sizes[client][0]) if want_solution else None
        st = nat.lib().kkt_server_wait(self._h, rid, ctypes.byref(r), None if x is None else nat.ptr_f64(x))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_server_wait failed")
        d = r.as_dict()
        return (d, x) if want_solution else d

    def drain(self):
        nat.lib().kkt_server_drain(self._h)

    def stats(self):
        s = nat.ServerStats()
        nat.lib().kkt_server_get_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().kkt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
