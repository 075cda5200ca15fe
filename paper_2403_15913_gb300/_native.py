"""ctypes declarations of the C ABI in include/kkt.h (argument marshalling
only).  Loading fails loudly when the in-tree CUDA library is missing."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkkt_gb300.so")

KKT_CONVERGED = 1
KKT_OK = 0
KKT_ERR_ARG = -1
KKT_ERR_OOM = -2
KKT_ERR_CUDA = -3
KKT_ERR_NOT_SPD = -4
KKT_ERR_MAXIT = -5
KKT_ERR_STALL = -6
KKT_ERR_TIMEOUT = -7
KKT_ERR_STATE = -8
KKT_ERR_INTERNAL = -9
STATUS_NAMES = {1: "converged", 0: "ok", -1: "arg", -2: "oom", -3: "cuda", -4: "not_spd", -5: "maxit",
                -6: "stall", -7: "timeout", -8: "state", -9: "internal"}

KKT_STATIC_SCRATCH_DOUBLES = 1 << 21   # size of the allocation-free backsolve's scratch

KKT_LIFTED = 0
KKT_HYKKT = 1

EXPORTED = [
    "kkt_default_options", "kkt_analyse", "kkt_analyse_host", "kkt_symbolic_sizes",
    "kkt_symbolic_export", "kkt_factor", "kkt_solve", "kkt_backsolve", "kkt_backsolve_noalloc",
    "kkt_factor_export", "kkt_analyse_batch", "kkt_analyse_batch_host", "kkt_batch_layout",
    "kkt_factor_batch", "kkt_factor_solve", "kkt_batch_results", "kkt_autotune_batch", "kkt_batch_set_active",
    "kkt_set_precision",
    "kkt_last_error", "kkt_destroy", "kkt_tray_sizes", "kkt_tray_pattern",
    "kkt_tray_eval", "kkt_set_profiling", "kkt_get_stats", "kkt_reset_stats",
    "kkt_ipm_default_options", "kkt_ipm_create", "kkt_ipm_init", "kkt_ipm_step", "kkt_ipm_solve",
    "kkt_ipm_get",
    "kkt_ipm_kkt", "kkt_ipm_destroy", "kkt_ipm_set_initial_state", "kkt_ipm_init_shifted", "kkt_ipm_init_warm",
    "kkt_ipm_device_bytes", "kkt_device_bytes",
    "kkt_ipm_batch_create", "kkt_ipm_batch_member", "kkt_ipm_batch_start", "kkt_ipm_batch_step",
    "kkt_ipm_batch_solve", "kkt_ipm_batch_kkt", "kkt_ipm_batch_last_error", "kkt_ipm_batch_destroy",
    "kkt_ipm_batch_start_member", "kkt_ipm_batch_member_status", "kkt_ipm_batch_device_bytes",
    "kkt_server_default_options", "kkt_server_create", "kkt_server_add_client", "kkt_server_submit",
    "kkt_server_wait", "kkt_server_drain", "kkt_server_get_stats", "kkt_server_destroy",
    "kkt_eval_fn", "kkt_debug_corrupt_map",
]

# helper functions of kkt_eval_fn
KKT_FN_RSQRT, KKT_FN_RCP, KKT_FN_SPLIT_M, KKT_FN_SPLIT_E = 0, 1, 2, 3
KKT_FN_MAX_ABS, KKT_FN_MAX_NN, KKT_FN_MIN_NN, KKT_FN_F32_ROUNDTRIP = 4, 5, 6, 7
KKT_FN_BINARY = (KKT_FN_MAX_ABS, KKT_FN_MAX_NN, KKT_FN_MIN_NN)


class Options(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("relax_cols", ctypes.c_int), ("relax_zeros", ctypes.c_int),
                ("max_width", ctypes.c_int), ("delta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("tol_refine", ctypes.c_double),
                ("tol_cg", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("target_relaxed", ctypes.c_int),
                ("subtree_cols", ctypes.c_int), ("precision", ctypes.c_int),
                ("solver", ctypes.c_int), ("block", ctypes.c_int),
                ("staged_solve", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("refine_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("failed_col", ctypes.c_int), ("status_detail", ctypes.c_int),
                ("bwd_err", ctypes.c_double), ("delta_x", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("assemble_ms", ctypes.c_double), ("factor_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("factor_launches", ctypes.c_int64),
                ("factor_calls", ctypes.c_int64), ("kinv_calls", ctypes.c_int64),
                ("fp32_factors", ctypes.c_int64), ("fp64_fallbacks", ctypes.c_int64),
                ("graph_steps", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class IPMOptions(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mu_init", ctypes.c_double),
                ("relaxed", ctypes.c_int), ("tau_relax", ctypes.c_double)]


class IPMInfo(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int), ("ls_trials", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("mu", ctypes.c_double), ("objective", ctypes.c_double),
                ("inf_pr", ctypes.c_double), ("inf_du", ctypes.c_double),
                ("inf_compl", ctypes.c_double), ("err0", ctypes.c_double),
                ("alpha_pr", ctypes.c_double), ("alpha_du", ctypes.c_double),
                ("delta_x", ctypes.c_double), ("bwd_err", ctypes.c_double),
                ("t_eval_ms", ctypes.c_double), ("t_kkt_ms", ctypes.c_double),
                ("t_step_ms", ctypes.c_double), ("launches", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerOptions(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("hbm_budget_gb", ctypes.c_double), ("scheme", ctypes.c_int),
                ("precision", ctypes.c_int), ("gamma", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("mu_init", ctypes.c_double), ("warm_start", ctypes.c_int),
                ("warm_mu", ctypes.c_double), ("warm_recenter", ctypes.c_int), ("batch", ctypes.c_int)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("client", ctypes.c_int), ("slot", ctypes.c_int),
                ("status", ctypes.c_int), ("iters", ctypes.c_int), ("cold", ctypes.c_int),
                ("warm", ctypes.c_int), ("objective", ctypes.c_double), ("inf_pr", ctypes.c_double),
                ("inf_du", ctypes.c_double), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("contexts_created", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("resident_bytes", ctypes.c_int64), ("peak_resident_bytes", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("resident_clients", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

P = ctypes.c_void_p
I32P = ctypes.POINTER(ctypes.c_int)
I64P = ctypes.POINTER(ctypes.c_int64)
F64P = ctypes.POINTER(ctypes.c_double)


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library {LIB_PATH} is missing; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    _lib = load(LIB_PATH)
    return _lib


def load(path):
    """Open a build of the library at `path` and declare its C ABI (the
    bounds-check build is a second library with the same symbols)."""
    L = ctypes.CDLL(path)
    L.kkt_default_options.argtypes = [ctypes.POINTER(Options)]
    L.kkt_default_options.restype = None
    for name in ("kkt_analyse", "kkt_analyse_host"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int, ctypes.c_int, I32P, I32P, I32P, I32P,
                      ctypes.POINTER(Options), ctypes.POINTER(P)]
        f.restype = ctypes.c_int
    I32PP = ctypes.POINTER(I32P)
    for name in ("kkt_analyse_batch", "kkt_analyse_batch_host"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int, I32P, I32P, I32PP, I32PP, I32PP, I32PP,
                      ctypes.POINTER(Options), ctypes.POINTER(P)]
        f.restype = ctypes.c_int
    L.kkt_batch_layout.argtypes = [P, I32P, I32P, I32P]
    L.kkt_batch_layout.restype = ctypes.c_int
    L.kkt_factor_batch.argtypes = [P, P, P, P, P, F64P, P, ctypes.POINTER(Info)]
    L.kkt_factor_batch.restype = ctypes.c_int
    L.kkt_factor_solve.argtypes = [P, P, P, P, P, F64P, P, P, P, P, P, ctypes.POINTER(Info)]
    L.kkt_factor_solve.restype = ctypes.c_int
    L.kkt_autotune_batch.argtypes = [ctypes.c_int, I32P, I32P, I32PP, I32PP, I32PP, I32PP,
                                     ctypes.POINTER(Options), ctypes.c_int, P, ctypes.POINTER(Options),
                                     F64P]
    L.kkt_autotune_batch.restype = ctypes.c_int
    L.kkt_batch_results.argtypes = [P, I32P, I32P, I32P, F64P, I32P]
    L.kkt_batch_results.restype = ctypes.c_int
    L.kkt_batch_set_active.argtypes = [P, I32P]
    L.kkt_batch_set_active.restype = ctypes.c_int
    L.kkt_set_precision.argtypes = [P, ctypes.c_int]
    L.kkt_set_precision.restype = ctypes.c_int
    L.kkt_symbolic_sizes.argtypes = [P, I32P, I64P, I64P, I64P, I32P, F64P]
    L.kkt_symbolic_sizes.restype = ctypes.c_int
    L.kkt_symbolic_export.argtypes = [P, I32P, I32P, I32P, I32P, I32P, I32P]
    L.kkt_symbolic_export.restype = ctypes.c_int
    L.kkt_factor.argtypes = [P, P, P, P, P, ctypes.c_double, P, ctypes.POINTER(Info)]
    L.kkt_factor.restype = ctypes.c_int
    L.kkt_solve.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(Info)]
    L.kkt_solve.restype = ctypes.c_int
    L.kkt_backsolve.argtypes = [P, P, P, P]
    L.kkt_backsolve.restype = ctypes.c_int
    L.kkt_backsolve_noalloc.argtypes = [P, P, P, P]
    L.kkt_backsolve_noalloc.restype = ctypes.c_int
    L.kkt_factor_export.argtypes = [P, I64P, I32P, F64P]
    L.kkt_factor_export.restype = ctypes.c_int
    L.kkt_last_error.argtypes = [P]
    L.kkt_last_error.restype = ctypes.c_char_p
    L.kkt_destroy.argtypes = [P]
    L.kkt_destroy.restype = None
    L.kkt_tray_sizes.argtypes = [F64P, I32P, I32P, I32P, I32P]
    L.kkt_tray_sizes.restype = ctypes.c_int
    L.kkt_tray_pattern.argtypes = [F64P, I32P, I32P, I32P, I32P]
    L.kkt_tray_pattern.restype = ctypes.c_int
    L.kkt_tray_eval.argtypes = [F64P, P, P, ctypes.c_double, P, P, P, P, P, P]
    L.kkt_tray_eval.restype = ctypes.c_int
    L.kkt_set_profiling.argtypes = [P, ctypes.c_int]
    L.kkt_set_profiling.restype = ctypes.c_int
    L.kkt_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.kkt_get_stats.restype = ctypes.c_int
    L.kkt_reset_stats.argtypes = [P]
    L.kkt_reset_stats.restype = ctypes.c_int
    L.kkt_ipm_default_options.argtypes = [ctypes.POINTER(IPMOptions)]
    L.kkt_ipm_default_options.restype = None
    L.kkt_ipm_create.argtypes = [F64P, ctypes.POINTER(Options), ctypes.POINTER(IPMOptions),
                                 ctypes.POINTER(P)]
    L.kkt_ipm_create.restype = ctypes.c_int
    L.kkt_ipm_init.argtypes = [P, P, P]
    L.kkt_ipm_init.restype = ctypes.c_int
    L.kkt_ipm_step.argtypes = [P, P, ctypes.POINTER(IPMInfo)]
    L.kkt_ipm_step.restype = ctypes.c_int
    L.kkt_ipm_solve.argtypes = [P, P, ctypes.POINTER(IPMInfo)]
    L.kkt_ipm_solve.restype = ctypes.c_int
    L.kkt_ipm_get.argtypes = [P, P, P, P, P, P, P]
    L.kkt_ipm_get.restype = ctypes.c_int
    L.kkt_ipm_kkt.argtypes = [P]
    L.kkt_ipm_kkt.restype = P
    L.kkt_ipm_destroy.argtypes = [P]
    L.kkt_ipm_destroy.restype = None
    L.kkt_ipm_set_initial_state.argtypes = [P, F64P, P]
    L.kkt_ipm_set_initial_state.restype = ctypes.c_int
    L.kkt_ipm_init_shifted.argtypes = [P, P, P]
    L.kkt_ipm_init_shifted.restype = ctypes.c_int
    L.kkt_ipm_init_warm.argtypes = [P, ctypes.c_double, ctypes.c_int, P]
    L.kkt_ipm_init_warm.restype = ctypes.c_int
    L.kkt_ipm_device_bytes.argtypes = [P, I64P]
    L.kkt_ipm_device_bytes.restype = ctypes.c_int
    L.kkt_ipm_batch_create.argtypes = [ctypes.c_int, F64P, ctypes.POINTER(Options), ctypes.POINTER(IPMOptions),
                                       ctypes.POINTER(P)]
    L.kkt_ipm_batch_create.restype = ctypes.c_int
    L.kkt_ipm_batch_member.argtypes = [P, ctypes.c_int]
    L.kkt_ipm_batch_member.restype = P
    L.kkt_ipm_batch_start.argtypes = [P]
    L.kkt_ipm_batch_start.restype = ctypes.c_int
    L.kkt_ipm_batch_start_member.argtypes = [P, ctypes.c_int]
    L.kkt_ipm_batch_start_member.restype = ctypes.c_int
    L.kkt_ipm_batch_member_status.argtypes = [P, ctypes.c_int, I32P, I32P]
    L.kkt_ipm_batch_member_status.restype = ctypes.c_int
    L.kkt_ipm_batch_device_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.kkt_ipm_batch_device_bytes.restype = ctypes.c_int
    L.kkt_ipm_batch_step.argtypes = [P, P, ctypes.POINTER(IPMInfo)]
    L.kkt_ipm_batch_step.restype = ctypes.c_int
    L.kkt_ipm_batch_solve.argtypes = [P, P, I32P, I32P, ctypes.POINTER(IPMInfo)]
    L.kkt_ipm_batch_solve.restype = ctypes.c_int
    L.kkt_ipm_batch_kkt.argtypes = [P]
    L.kkt_ipm_batch_kkt.restype = P
    L.kkt_ipm_batch_last_error.argtypes = [P]
    L.kkt_ipm_batch_last_error.restype = ctypes.c_char_p
    L.kkt_ipm_batch_destroy.argtypes = [P]
    L.kkt_ipm_batch_destroy.restype = None
    L.kkt_device_bytes.argtypes = [P, I64P]
    L.kkt_device_bytes.restype = ctypes.c_int
    L.kkt_eval_fn.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
    L.kkt_eval_fn.restype = ctypes.c_int
    L.kkt_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
    L.kkt_server_default_options.restype = None
    L.kkt_server_create.argtypes = [ctypes.POINTER(ServerOptions), ctypes.c_int, ctypes.POINTER(P)]
    L.kkt_server_create.restype = ctypes.c_int
    L.kkt_server_add_client.argtypes = [P, F64P, I32P]
    L.kkt_server_add_client.restype = ctypes.c_int
    L.kkt_server_submit.argtypes = [P, ctypes.c_int, F64P, ctypes.c_int, I64P]
    L.kkt_server_submit.restype = ctypes.c_int
    L.kkt_server_wait.argtypes = [P, ctypes.c_int64, ctypes.POINTER(RequestResult), F64P]
    L.kkt_server_wait.restype = ctypes.c_int
    L.kkt_server_drain.argtypes = [P]
    L.kkt_server_drain.restype = ctypes.c_int
    L.kkt_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    L.kkt_server_get_stats.restype = ctypes.c_int
    L.kkt_server_destroy.argtypes = [P]
    L.kkt_server_destroy.restype = None
    L.kkt_debug_corrupt_map.argtypes = [P, ctypes.c_int]
    L.kkt_debug_corrupt_map.restype = ctypes.c_int
    return L


def ptr_i32(a):
    return a.ctypes.data_as(I32P)


def ptr_i64(a):
    return a.ctypes.data_as(I64P)


def ptr_f64(a):
    return a.ctypes.data_as(F64P)
