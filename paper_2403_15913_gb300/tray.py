"""Binding of the distillation-column model kernels (Sec. VI-A): host
patterns and device evaluation through the C ABI."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat
from .solver import KKTError, _dptr, _stream


class TrayModel:
    def __init__(self, params):
        self.params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        n, m, nw, nj = (ctypes.c_int() for _ in range(4))
        st = nat.lib().kkt_tray_sizes(nat.ptr_f64(self.params), ctypes.byref(n), ctypes.byref(m),
                                      ctypes.byref(nw), ctypes.byref(nj))
        if st != nat.KKT_OK:
            raise KKTError(st, "bad tray parameters")
        self.n, self.m, self.nnzW, self.nnzJ = n.value, m.value, nw.value, nj.value

    def pattern(self):
        Wc = np.empty(self.n + 1, np.int32)
        Wr = np.empty(self.nnzW, np.int32)
        Jr = np.empty(self.m + 1, np.int32)
        Jc = np.empty(self.nnzJ, np.int32)
        st = nat.lib().kkt_tray_pattern(nat.ptr_f64(self.params), nat.ptr_i32(Wc), nat.ptr_i32(Wr),
                                        nat.ptr_i32(Jr), nat.ptr_i32(Jc))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_tray_pattern failed")
        return Wc, Wr, Jr, Jc

    def eval(self, w, lam=None, obj_weight=1.0, f=None, grad=None, c=None, Jval=None, Wval=None,
             stream=None):
        """Evaluate into the given CUDA float64 tensors (None skips)."""
        st = nat.lib().kkt_tray_eval(nat.ptr_f64(self.params), _dptr(w), _dptr(lam),
                                     float(obj_weight), _dptr(f), _dptr(grad), _dptr(c),
                                     _dptr(Jval), _dptr(Wval), _stream(stream))
        if st != nat.KKT_OK:
            raise KKTError(st, "kkt_tray_eval failed")
