#!/usr/bin/env python
"""Benchmark of the hot path: time per interior-point iteration.

Workload: the distillation column of Sec. VI-A (32 trays) on T = 5000
implicit-Euler stages (n = 325,065 variables, m = 320,064 constraints),
solved by the device IPM driver from the standard start (compositions at
xbar_0, reflux at ubar) to tolerance 1e-8.

One step = one IPM iteration, all on the GPU: derivative evaluation kernels,
assembly of the condensed matrix, supernodal Cholesky (inertia correction when
a pivot fails), the Lifted-KKT (or HyKKT) solve refined to a backward error
<= 1e-10 on its target system, step recovery, fraction to boundary and the
filter line search.  When the IPM converges it is restarted (untimed).  The
symbolic analysis is done once before timing (the paper's SYM column).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--scheme lifted|hykkt]
        python bench.py --impl reference ...   (the CPU oracle, timed as it stands)

--workload kkt times one KKT step instead (assembly, factor, solve and
refinement at a seeded iterate with Sigma log-uniform on --sigma), e.g. the
mixed-precision case: --workload kkt --T 20000 --sigma 1e-8,1e8 --precision
fp32, which also runs the all-FP64 factor on the same input for comparison.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070   # SMs x DFMA/clk/SM x flops x GHz = 1258.6
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070  # SMs x FFMA lanes/SM x flops x GHz = 80,548
METRIC = "KKT solve time per IPM iteration"
PREC = {"fp64": 0, "fp32": 1, "df64": 2}
# DRAM bytes of one numeric factorisation (dram__bytes_read.sum +
# dram__bytes_write.sum of its kernels in one ncu capture of this
# benchmark), keyed by (trays, stages, solver, precision); other
# configurations report null
FACTOR_TRAFFIC = {(32, 5000, "supernodal", "fp64"): 484.5e6}
DTYPE = {"fp64": "f64", "fp32": "f32 factor + f64 refinement", "df64": "df64 (float-pair) factor + f64 refinement"}
UNIT = "ms/iter"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", default="lifted", choices=["lifted", "hykkt"])
    ap.add_argument("--T", type=int, default=5000)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--gamma", type=float, default=1e4)
    ap.add_argument("--solver", default="supernodal", choices=["supernodal", "bcr"],
                    help="K factorisation: supernodal Cholesky or block cyclic reduction of the stage blocks")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64"],
                    help="factor precision; fp32 and df64 (float pairs) refine in FP64 and fall back "
                         "to an FP64 factor")
    ap.add_argument("--workload", default="ipm", choices=["ipm", "kkt", "batch", "serve"])
    ap.add_argument("--clients", type=int, default=64, help="serve workload: controllers")
    ap.add_argument("--requests", type=int, default=400, help="serve workload: timed requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve workload: Poisson arrivals per s")
    ap.add_argument("--slots", type=int, default=8, help="serve workload: concurrent solves")
    ap.add_argument("--batch", type=int, default=256, help="batch workload: instances")
    ap.add_argument("--autotune", action="store_true",
                    help="batch workload: pick the supernode partition with kkt_autotune_batch first")
    ap.add_argument("--sigma", default="1e-6,1e6", help="kkt workload: Sigma_x range")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


def across_ranks(value, op, dist=None, device="cuda"):
    """A per-rank scalar combined over the process group: "max" for times
    (the slowest rank sets the job time), "sum" for throughputs (whole-job
    aggregate).  Without a group the value itself."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.item()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"kkt_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- oracle
def oracle_ipm_sample(k, T_sample, scheme, budget_s):
    """Oracle IPM iterations at a bounded size until the budget is spent:
    returns seconds per iteration (model, sparse factor, hybrid solve, line
    search: the oracle as it stands, single thread)."""
    import numpy as np
    from gen.tray import TrayParams, ipm_start
    from oracle import ipm as oipm, symbolic, tray as otray
    p = TrayParams(k=k, T=T_sample)
    x0 = ipm_start(p)
    W = otray.hessian_lower_csc(p, x0, np.zeros(p.m))
    J = otray.jacobian_csr(p, x0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], leaf_size=64, relax_cols=32,
                           relax_zeros=128, max_width=64)
    iters, t_total = 0, 0.0
    while t_total < budget_s or iters == 0:
        lin = oipm.KKTLinearSolver(scheme, p.n, p.m, None, None, sym=sym, gamma=1e4)
        s = oipm.IPM(oipm.TrayModel(p), lin, oipm.IPMOptions(relaxed=(scheme == "lifted")), x0)
        while not s.done and s.it < 200 and t_total < budget_s * 2:
            t0 = time.perf_counter()
            info = s.step()
            dt = time.perf_counter() - t0
            if info.status != "converged":
                iters += 1
                t_total += dt
        if s.it == 0:
            break
    return t_total / max(1, iters), iters


def cpu_baseline(args, budget_s=15.0, T_sample=50):
    per, iters = oracle_ipm_sample(args.k, T_sample, args.scheme, budget_s)
    scale = (args.T + 1) / (T_sample + 1)
    return {"value": per * scale * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{iters} oracle IPM iterations ({args.scheme}) at {args.k} trays, T={T_sample}: "
                       f"{per*1e3:.1f} ms each, scaled x{scale:.1f} to T={args.T} (work linear in T)")}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    T_sample = 50
    # warm-up iterations, then the timed ones (each step: one oracle IPM
    # iteration at T=50, scaled to the workload's horizon)
    oracle_ipm_sample(args.k, T_sample, args.scheme, budget_s=0.5 * args.warmup)
    per, iters = oracle_ipm_sample(args.k, T_sample, args.scheme, budget_s=max(2.0, 1.5 * args.steps))
    scale = (args.T + 1) / (T_sample + 1)
    ms = per * scale * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"tray column k={args.k} T={args.T} (n={(2*args.k+1)*(args.T+1)}), "
                               f"{args.scheme} IPM iteration; oracle at T={T_sample} scaled by "
                               f"(T+1)/{T_sample+1}", "scheme": args.scheme},
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{iters} oracle IPM iterations at T={T_sample}, scaled x{scale:.1f}"},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from gen.tray import TrayParams, ipm_start
    from paper_2403_15913_gb300 import IPMSolver
    from paper_2403_15913_gb300 import _native as nat
    import ctypes

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # replicas: every rank solves its own instance (horizon-shifted start)
    p = TrayParams(k=args.k, T=args.T)
    t0 = time.perf_counter()
    ipm = IPMSolver(p.as_array(), scheme=args.scheme, gamma=args.gamma, max_cg=500,
                    precision=PREC[args.precision],
                    solver=1 if args.solver == "bcr" else 0, block=2 * args.k + 1)
    t_analyse = time.perf_counter() - t0
    kctx = nat.lib().kkt_ipm_kkt(ipm._h)
    ns, nnzL, panel, rows, lev, fl = (ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(),
                                      ctypes.c_int64(), ctypes.c_int(), ctypes.c_double())
    nat.lib().kkt_symbolic_sizes(kctx, ctypes.byref(ns), ctypes.byref(nnzL), ctypes.byref(panel),
                                 ctypes.byref(rows), ctypes.byref(lev), ctypes.byref(fl))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    x0 = torch.as_tensor(ipm_start(p)).cuda()
    state = {"solves": 0, "iters_per_solve": []}
    infos = []

    def ipm_step():
        """One IPM iteration; restarts the solve (untimed) when converged."""
        st = ipm.step()
        if st == nat.KKT_CONVERGED:
            state["iters_per_solve"].append(ipm.info.iter)
            ipm.init(x0)
            state["solves"] += 1
            return None
        if st != nat.KKT_OK:
            raise RuntimeError(f"IPM step failed with status {st}")
        infos.append(ipm.info.as_dict())
        return True

    ipm.init(x0)
    done = 0
    while done < args.warmup:
        flush.zero_()
        if ipm_step():
            done += 1
    torch.cuda.synchronize()
    infos.clear()
    ipm.set_profiling(True)
    nat.lib().kkt_reset_stats(kctx)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    wall0 = time.perf_counter()
    while len(step_ms) < args.steps:
        flush.zero_()                                    # L2 flush, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ok = ipm_step()
        e1.record(stream)
        if ok:
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = statistics.mean(step_ms)
    st = nat.Stats()
    nat.lib().kkt_get_stats(kctx, ctypes.byref(st))
    st = st.as_dict()
    ms = across_ranks(ms, "max", dist)
    ipm.set_profiling(False)

    # ---- end to end through the public API: whole solves from a host x0
    h_x0 = torch.as_tensor(ipm_start(p)).pin_memory()
    d_x0 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    h_x = torch.empty(p.n, dtype=torch.float64).pin_memory()
    h_y = torch.empty(p.m, dtype=torch.float64).pin_memory()
    e2e_total, e2e_iters = 0.0, 0
    for rep in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_x0.copy_(h_x0, non_blocking=True)
        ipm.init(d_x0)
        hist = ipm.solve()
        x, y, _, _, _ = ipm.get()
        h_x.copy_(x, non_blocking=True)
        h_y.copy_(y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= 1:
            e2e_total += e0.elapsed_time(e1)
            e2e_iters += hist[-1]["iter"]
    e2e_ms = e2e_total / max(1, e2e_iters)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fcalls = max(1, st["factor_calls"])
    factor_ms = st["factor_ms"] / fcalls
    kinv_ms = st["solve_ms"] / max(1, st["kinv_calls"])
    f32 = args.precision == "fp32"
    roof = {"kernel": ("block cyclic reduction (bcr_elim/bcr_update kernels)" if args.solver == "bcr" else
                       "supernodal Cholesky (factor_subtree/level, potrf/trsm/syrk kernels)"),
            "bound": "alu", "achieved": fl.value / (factor_ms * 1e-3) / 1e9,
            "peak": FP32_PEAK_GFLOPS if f32 else FP64_PEAK_GFLOPS, "unit": "GFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = FACTOR_TRAFFIC.get((args.k, args.T, args.solver, args.precision))
    roof["peak_source"] = ("FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived, of nominal units)"
                           if f32 else
                           "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived, of nominal units)")
    n_steps = len(step_ms)
    line = {
        "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": f"tray column k={args.k} T={args.T} (n={p.n}, m={p.m}), full IPM "
                               f"iteration ({args.scheme}) from xbar_0 = {p.x0bar}, tol 1e-8",
                   "scheme": args.scheme, "gamma": args.gamma if args.scheme == "hykkt" else None,
                   "precision": args.precision, "solver": args.solver,
                   "fp32_factors": st["fp32_factors"], "fp64_fallbacks": st["fp64_fallbacks"],
                   "tau_relax": 1e-8 if args.scheme == "lifted" else None,
                   "l2": "flushed (256 MB write) between timed steps",
                   "analyse_s": round(t_analyse, 3), "supernodes": ns.value, "nnz_L": nnzL.value,
                   "panel_entries": panel.value, "tree_levels": lev.value,
                   "factor_gflop": fl.value / 1e9,
                   "ipm_iters_to_converge": state["iters_per_solve"][:4],
                   "phase_ms": {"eval": statistics.mean(i["t_eval_ms"] for i in infos),
                                "kkt_solve": statistics.mean(i["t_kkt_ms"] for i in infos),
                                "factor": factor_ms, "kinv": kinv_ms,
                                "assemble": st["assemble_ms"] / fcalls,
                                "factor_calls_per_step": st["factor_calls"] / n_steps,
                                "kinv_per_step": st["kinv_calls"] / n_steps},
                   "max_bwd_err": max(i["bwd_err"] for i in infos),
                   "refine_iters": [i["refine_iters"] for i in infos][:6],
                   "cg_iters": [i["cg_iters"] for i in infos][:6],
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": e2e_ms, "unit": UNIT,
                "h2d_bytes_per_step": p.n * 8 / max(1, e2e_iters),
                "d2h_bytes_per_step": (p.n + p.m) * 8 / max(1, e2e_iters),
                "scope": "whole solves: x0 host->device, all iterations, (x, y) device->host"},
        "gpu_launches": (int(st["launches"] / n_steps * args.steps) + sum(i["launches"] for i in infos))
                        if n_steps else 0,
        "clocks": clk,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------- one KKT step
KKT_METRIC = "KKT step time (assemble + factor + refined solve)"


def oracle_kkt_sample(k, T_sample, scheme, sig, gamma, budget_s):
    """Oracle KKT steps (condensed assembly, left-looking sparse Cholesky,
    refined solve) at a bounded size: seconds per step."""
    import numpy as np
    from gen.tray import TrayParams, kkt_point
    from oracle import kkt as okkt, symbolic, tray as otray
    p = TrayParams(k=k, T=T_sample)
    pt = kkt_point(p, 0, sig)
    W = otray.hessian_lower_csc(p, pt.w, pt.lam)
    J = otray.jacobian_csr(p, pt.w)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], leaf_size=64, relax_cols=32,
                           relax_zeros=128, max_width=64)
    n_done, t = 0, 0.0
    while t < budget_s or n_done == 0:
        t0 = time.perf_counter()
        for dx in (0.0, 1e-4, 8e-4, 6.4e-3, 5.12e-2, 0.4096, 3.2768, 26.2144):
            try:
                if scheme == "lifted":
                    okkt.lifted_solve(sym, p.n, p.m, W, J, pt.sigma, dx, np.full(p.m, 1e8), pt.rx, pt.ry)
                else:
                    okkt.hykkt_solve(sym, p.n, p.m, W, J, pt.sigma, dx, gamma, pt.rx, pt.ry)
                break
            except Exception:
                continue
        t += time.perf_counter() - t0
        n_done += 1
    return t / n_done, n_done


def run_kkt(args, ws, rank, local):
    import ctypes
    import numpy as np
    import torch
    from gen.tray import TrayParams, kkt_point
    from paper_2403_15913_gb300 import KKTSolver, TrayModel
    from paper_2403_15913_gb300 import _native as nat

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sig = tuple(float(v) for v in args.sigma.split(","))
    p = TrayParams(k=args.k, T=args.T)
    pt = kkt_point(p, args.seed + rank, sig)
    tm = TrayModel(p.as_array())
    Wc, Wr, Jr, Jc = tm.pattern()
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))
    h_in = {k: f64(v).pin_memory() for k, v in (("w", pt.w), ("lam", pt.lam), ("sigma", pt.sigma),
                                                 ("rx", pt.rx), ("ry", pt.ry))}
    d_in = {k: v.cuda() for k, v in h_in.items()}
    Wv = torch.zeros(tm.nnzW, dtype=torch.float64, device="cuda")
    Jv = torch.zeros(tm.nnzJ, dtype=torch.float64, device="cuda")
    dx = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opts = dict(scheme=args.scheme, gamma=args.gamma, max_cg=500, leaf_size=64, relax_cols=32,
                relax_zeros=128, max_width=64, solver=1 if args.solver == "bcr" else 0,
                block=2 * args.k + 1)

    def make(prec):
        t0 = time.perf_counter()
        s = KKTSolver(p.n, p.m, Wc, Wr, Jr, Jc, precision=prec, **opts)
        return s, time.perf_counter() - t0

    def step(s, d, delta_x):
        tm.eval(d["w"], d["lam"], 1.0, None, None, None, Jv, Wv)
        st = s.factor(Wv, Jv, d["sigma"], None, delta_x)
        if st != 0:
            return st
        return s.solve(d["rx"], d["ry"], dx, dy)

    def find_delta(s):
        delta_x = 0.0
        while step(s, d_in, delta_x) == nat.KKT_ERR_NOT_SPD:
            delta_x = 1e-4 if delta_x == 0 else delta_x * 8
        torch.cuda.synchronize()
        return delta_x

    def timed(s, delta_x, steps):
        for _ in range(args.warmup):
            flush.zero_()
            step(s, d_in, delta_x)
        torch.cuda.synchronize()
        s.reset_stats()
        s.set_profiling(True)
        ms, infos = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step(s, d_in, delta_x)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(dict(s.info.as_dict(), status=st))
        s.set_profiling(False)
        return ms, infos, s.stats()

    prec = PREC[args.precision]
    solver, t_analyse = make(prec)
    delta_x = find_delta(solver)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, infos, st = timed(solver, delta_x, args.steps)
    clk = clocks.stop()
    v = torch.cat([dx, dy]).cpu().numpy()
    mean_ms = across_ranks(statistics.mean(ms), "max", dist)
    fp64_cmp = None
    if prec != 0:
        s64, _ = make(0)
        ms64, infos64, st64 = timed(s64, delta_x, args.steps)
        v64 = torch.cat([dx, dy]).cpu().numpy()
        fp64_cmp = {"ms": statistics.mean(ms64), "factor_ms": st64["factor_ms"] / max(1, st64["factor_calls"]),
                    "bwd_err": max(i["bwd_err"] for i in infos64),
                    "refine_iters": [i["refine_iters"] for i in infos64][:4],
                    "rel_diff_vs_fp64_path": float(np.max(np.abs(v - v64)) / np.max(np.abs(v64)))}
        s64.close()
    # end to end: inputs host->device, step, (dx, dy) device->host
    h_out = torch.empty(p.n + p.m, dtype=torch.float64).pin_memory()
    d_e2e = {k: torch.empty_like(v) for k, v in d_in.items()}
    e2e = []
    for rep in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in d_e2e:
            d_e2e[k].copy_(h_in[k], non_blocking=True)
        step(solver, d_e2e, delta_x)
        h_out[:p.n].copy_(dx, non_blocking=True)
        h_out[p.n:].copy_(dy, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            e2e.append(e0.elapsed_time(e1))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    sym = solver.sizes()
    fcalls = max(1, st["factor_calls"])
    factor_ms = st["factor_ms"] / fcalls
    f32 = prec == 1
    roof = {"kernel": ("block cyclic reduction (bcr_elim/bcr_update kernels)" if args.solver == "bcr" else
                       "supernodal Cholesky (factor_subtree/level, potrf/trsm/syrk kernels)"),
            "bound": "alu", "achieved": sym.flops / (factor_ms * 1e-3) / 1e9,
            "peak": FP32_PEAK_GFLOPS if f32 else FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "traffic": None,
            "peak_source": ("FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived, of nominal units)"
                            if f32 else
                            "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived, of nominal units)")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    in_bytes = sum(v.numel() * 8 for v in h_in.values())
    line = {
        "metric": KKT_METRIC, "value": mean_ms, "unit": "ms/step", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": f"tray column k={args.k} T={args.T} (n={p.n}, m={p.m}), one {args.scheme} "
                               f"KKT step at a seeded iterate, Sigma log-uniform on [{sig[0]:g}, {sig[1]:g}]",
                   "scheme": args.scheme, "gamma": args.gamma if args.scheme == "hykkt" else None,
                   "delta": 1e-8 if args.scheme == "lifted" else None, "delta_x": delta_x,
                   "precision": args.precision, "solver": args.solver, "l2": "flushed (256 MB write) between timed steps",
                   "analyse_s": round(t_analyse, 3), "factor_gflop": sym.flops / 1e9,
                   "factor_ms": factor_ms, "kinv_ms": st["solve_ms"] / max(1, st["kinv_calls"]),
                   "fp32_factors": st["fp32_factors"], "fp64_fallbacks": st["fp64_fallbacks"],
                   "status_detail": [i["status_detail"] for i in infos][:4],
                   "max_bwd_err": max(i["bwd_err"] for i in infos),
                   "refine_iters": [i["refine_iters"] for i in infos][:4],
                   "cg_iters": [i["cg_iters"] for i in infos][:4],
                   "statuses": sorted(set(i["status"] for i in infos)),
                   "fp64_factor_path": fp64_cmp,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": statistics.mean(e2e), "unit": "ms/step", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": (p.n + p.m) * 8,
                "scope": "iterate, Sigma and rhs host->device, eval + factor + solve, (dx, dy) device->host"},
        "gpu_launches": int(st["launches"] / max(1, args.steps) * args.steps) + args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and ws == 1:
        T_s = 50
        per, n_s = oracle_kkt_sample(args.k, T_s, args.scheme, sig, args.gamma, 15.0)
        scale = (args.T + 1) / (T_s + 1)
        line["cpu_baseline"] = {"value": per * scale * 1e3, "unit": "ms/step", "cores": 1, "kind": "oracle",
                                "sample": f"{n_s} oracle {args.scheme} KKT steps at {args.k} trays, T={T_s}: "
                                          f"{per*1e3:.1f} ms each, scaled x{scale:.1f} to T={args.T}"}
    solver.close()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------- batched KKT
BATCH_METRIC = "batched KKT solves/s"


def batch_specs(count, seed):
    """Instance shapes of the batched workload: trays uniform in
    {16, 24, 32, 48, 64}, horizons uniform in [20, 400]."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return [(int(rng.choice([16, 24, 32, 48, 64])), int(rng.integers(20, 401))) for _ in range(count)]


def run_batch(args, ws, rank, local):
    import numpy as np
    import torch
    from gen.tray import TrayParams, kkt_point
    from paper_2403_15913_gb300 import KKTBatchSolver, KKTSolver, TrayModel, autotune_batch

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sig = tuple(float(v) for v in args.sigma.split(","))
    specs = batch_specs(args.batch, args.seed + 1000 * rank)
    params = [TrayParams(k=k, T=T) for k, T in specs]
    models = [TrayModel(p.as_array()) for p in params]
    pats = [tm.pattern() for tm in models]
    pts = [kkt_point(p, args.seed + 17 * i + 100000 * rank, sig) for i, p in enumerate(params)]
    stream = torch.cuda.current_stream()
    opts = dict(scheme=args.scheme, gamma=args.gamma, max_cg=500, leaf_size=64, relax_cols=32,
                relax_zeros=128, max_width=64)
    prec = PREC[args.precision]
    tuned = None
    if args.autotune:
        t0 = time.perf_counter()
        opts, tune_ms = autotune_batch([(p.n, p.m, *pt) for p, pt in zip(params, pats)], sample=32,
                                       precision=prec, **opts)
        opts.pop("precision", None)
        tuned = {"sample_factor_ms": tune_ms, "seconds": round(time.perf_counter() - t0, 2),
                 **{k: opts[k] for k in ("relax_cols", "relax_zeros", "max_width", "subtree_cols")}}
    t0 = time.perf_counter()
    bs = KKTBatchSolver([(p.n, p.m, *pt) for p, pt in zip(params, pats)], precision=prec, **opts)
    t_analyse = time.perf_counter() - t0
    xo, yo = bs.layout()
    wo = np.concatenate([[0], np.cumsum([tm.nnzW for tm in models])])
    jo = np.concatenate([[0], np.cumsum([tm.nnzJ for tm in models])])
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))
    # derivative values at every instance's seeded iterate, by the device kernels
    Wv = torch.zeros(int(wo[-1]), dtype=torch.float64, device="cuda")
    Jv = torch.zeros(int(jo[-1]), dtype=torch.float64, device="cuda")
    for i, (tm, pt) in enumerate(zip(models, pts)):
        w, lam = f64(pt.w).cuda(), f64(pt.lam).cuda()
        tm.eval(w, lam, 1.0, None, None, None, Jv[jo[i]:jo[i + 1]], Wv[wo[i]:wo[i + 1]])
    h_in = {"W": Wv.cpu().pin_memory(), "J": Jv.cpu().pin_memory(),
            "sigma": f64(np.concatenate([pt.sigma for pt in pts])).pin_memory(),
            "rx": f64(np.concatenate([pt.rx for pt in pts])).pin_memory(),
            "ry": f64(np.concatenate([pt.ry for pt in pts])).pin_memory()}
    d_in = {k: v.cuda() for k, v in h_in.items()}
    dx = torch.zeros(bs.n, dtype=torch.float64, device="cuda")
    dy = torch.zeros(bs.m, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # per-instance delta_x (inertia correction ladder, untimed)
    delta = np.zeros(args.batch)
    while bs.factor_batch(d_in["W"], d_in["J"], d_in["sigma"], None, delta) != 0:
        bad = bs.results()["failed_col"] >= 0
        delta[bad] = np.where(delta[bad] == 0, 1e-4, delta[bad] * 8)

    def step(d):
        bs.factor_batch(d["W"], d["J"], d["sigma"], None, delta)
        return bs.solve(d["rx"], d["ry"], dx, dy)

    for _ in range(args.warmup):
        flush.zero_()
        step(d_in)
    torch.cuda.synchronize()
    bs.reset_stats()
    bs.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, statuses, etas = [], set(), []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        statuses.add(step(d_in))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        etas.append(float(bs.results()["bwd_err"].max()))
    clk = clocks.stop()
    bs.set_profiling(False)
    st = bs.stats()
    res = bs.results()
    mean_ms = across_ranks(statistics.mean(ms), "max", dist)
    value = args.batch * ws / (mean_ms * 1e-3)

    # the plain per-instance FP64 path on the same inputs: one context per
    # instance, factor + solve one after the other
    singles = []
    for i, (p, pt) in enumerate(zip(params, pats)):
        singles.append(KKTSolver(p.n, p.m, *pt, precision=0, **opts))
    sx = [dx[xo[i]:xo[i + 1]] for i in range(args.batch)]
    sy = [dy[yo[i]:yo[i + 1]] for i in range(args.batch)]
    views = [{k: d_in[k][a:b] for k, (a, b) in (("W", (wo[i], wo[i + 1])), ("J", (jo[i], jo[i + 1])),
                                                  ("sigma", (xo[i], xo[i + 1])), ("rx", (xo[i], xo[i + 1])),
                                                  ("ry", (yo[i], yo[i + 1])))} for i in range(args.batch)]

    def serial():
        for i, s1 in enumerate(singles):
            v = views[i]
            s1.factor(v["W"], v["J"], v["sigma"], None, float(delta[i]))
            s1.solve(v["rx"], v["ry"], sx[i], sy[i])

    serial()
    torch.cuda.synchronize()
    ser_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        serial()
        e1.record(stream)
        torch.cuda.synchronize()
        ser_ms.append(e0.elapsed_time(e1))
    ser_eta = max(s1.info.bwd_err for s1 in singles)
    for s1 in singles:
        s1.close()
    # end to end: values and right-hand sides host->device, batched factor +
    # solve, (dx, dy) device->host
    h_out = torch.empty(bs.n + bs.m, dtype=torch.float64).pin_memory()
    d_e2e = {k: torch.empty_like(v) for k, v in d_in.items()}
    e2e = []
    for rep in range(4):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in d_e2e:
            d_e2e[k].copy_(h_in[k], non_blocking=True)
        step(d_e2e)
        h_out[:bs.n].copy_(dx, non_blocking=True)
        h_out[bs.n:].copy_(dy, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            e2e.append(e0.elapsed_time(e1))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    sym = bs.sizes()
    factor_ms = st["factor_ms"] / max(1, st["factor_calls"])
    f32 = prec == 1
    roof = {"kernel": "batched supernodal Cholesky (factor_subtree/level, potrf/trsm/syrk kernels)",
            "bound": "alu", "achieved": sym.flops / (factor_ms * 1e-3) / 1e9,
            "peak": FP32_PEAK_GFLOPS if f32 else FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "traffic": None,
            "peak_source": ("FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived, of nominal units)"
                            if f32 else
                            "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived, of nominal units)")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    in_bytes = sum(v.numel() * 8 for v in h_in.values())
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": f"{args.batch} independent tray-column KKT systems, trays uniform in "
                               f"{{16,24,32,48,64}}, T uniform in [20,400] (n = {bs.n}, m = {bs.m} in "
                               f"total), one {args.scheme} factor + refined solve of the whole batch per "
                               f"step, Sigma log-uniform on [{sig[0]:g}, {sig[1]:g}]",
                   "scheme": args.scheme, "precision": args.precision, "instances": args.batch,
                   "autotuned": tuned,
                   "l2": "flushed (256 MB write) between timed steps",
                   "analyse_s": round(t_analyse, 3), "factor_gflop": sym.flops / 1e9,
                   "factor_ms": factor_ms, "kinv_ms": st["solve_ms"] / max(1, st["kinv_calls"]),
                   "tree_levels": sym.levels, "statuses": sorted(statuses),
                   "max_bwd_err": max(etas), "max_refine_iters": int(res["refine_iters"].max()),
                   "fp64_fallbacks": st["fp64_fallbacks"],
                   "delta_x_nonzero": int((delta > 0).sum()),
                   "per_instance_fp64_path": {"ms_per_batch": statistics.mean(ser_ms),
                                              "solves_per_s": args.batch / (statistics.mean(ser_ms) * 1e-3),
                                              "max_bwd_err": ser_eta},
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": args.batch * ws / (statistics.mean(e2e) * 1e-3), "unit": "solves/s",
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": (bs.n + bs.m) * 8,
                "scope": "W, J, Sigma and rhs host->device, batched factor + solve, (dx, dy) device->host"},
        "gpu_launches": int(st["launches"] / max(1, args.steps) * args.steps),
        "clocks": clk,
    }
    bs.close()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------- NMPC serving
SERVE_METRIC = "NMPC serving solves/s (full IPM solves, Poisson arrivals)"


def run_serve(args, ws, rank, local):
    """Open-loop Poisson stream of receding-horizon requests against the
    native server; the same stream against one slot (serial FP64)."""
    import numpy as np
    import torch
    from gen.tray import TrayParams
    from paper_2403_15913_gb300 import NMPCServer

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rng = np.random.default_rng(args.seed + 7919 * rank)
    params = [TrayParams(k=int(rng.choice([32, 64])), T=int(rng.integers(50, 2001)))
              for _ in range(args.clients)]
    gaps = rng.exponential(1.0 / args.rate, args.requests)
    who = rng.integers(0, args.clients, args.requests)

    def serve(slots, precision, rate=None, count=None):
        gaps_, who_ = gaps, who
        if rate is not None:
            r2 = np.random.default_rng(args.seed + 31)
            gaps_ = r2.exponential(1.0 / rate, count)
            who_ = r2.integers(0, args.clients, count)
        srv = NMPCServer(slots=slots, hbm_budget_gb=40.0, scheme=args.scheme, precision=precision,
                         gamma=args.gamma)
        cl = [srv.add_client(p.as_array()) for p in params]
        t0 = time.perf_counter()
        for t in [srv.submit(c) for c in cl]:        # contexts created, first solves (untimed)
            srv.wait(t)
        prewarm = time.perf_counter() - t0
        clocks = ClockSampler(local)
        clocks.start()
        start = time.perf_counter()
        tickets, due = [], start
        for g, c in zip(gaps_, who_):
            due += g
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(cl[c]))
        res = [srv.wait(t) for t in tickets]
        clk = clocks.stop()
        st = srv.stats()
        srv.close()
        lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in res])
        span = (max(r["t_done_ms"] for r in res) - min(r["t_submit_ms"] for r in res)) * 1e-3
        return {"solves_per_s": len(res) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "iters_mean": float(np.mean([r["iters"] for r in res])),
                "converged": int(sum(r["status"] == 1 for r in res)),
                "warm": int(sum(r["warm"] for r in res)), "prewarm_s": round(prewarm, 2),
                "contexts": st["contexts_created"], "evictions": st["evictions"],
                "peak_resident_gb": st["peak_resident_bytes"] / 1e9, "clocks": clk}

    prec = PREC[args.precision]
    conc = serve(args.slots, prec)
    serial = serve(1, 0)
    # service latency below saturation: the same server at 70% of the
    # throughput it just sustained
    light_rate = 0.7 * conc["solves_per_s"]
    light = serve(args.slots, prec, rate=light_rate, count=min(args.requests, 200))
    light.pop("clocks")
    light["rate_per_s"] = light_rate
    total = across_ranks(conc["solves_per_s"], "sum", dist)
    if rank == 0:
        clk = conc.pop("clocks")
        serial.pop("clocks")
        n_total = sum(p.n for p in params)
        line = {
            "metric": SERVE_METRIC, "value": total, "unit": "solves/s", "n_gpus": ws,
            "steps": args.requests, "warmup": args.clients, "ms_per_step": conc["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": f"{args.clients} NMPC clients (trays in {{32,64}}, T uniform in [50,2000], "
                                   f"n = {n_total} in total), {args.requests} requests with Poisson arrivals at "
                                   f"{args.rate:g}/s, each a full {args.scheme} IPM solve to 1e-8 warm-started "
                                   f"from the shifted previous solution, 40 GB admission budget",
                       "slots": args.slots, "concurrent": conc, "serial_fp64_one_slot": serial,
                       "at_70pct_of_capacity": light,
                       "speedup_vs_serial": conc["solves_per_s"] / serial["solves_per_s"],
                       "step": "one request = one full IPM solve; value = requests / (last done - first "
                               "submit); latency = done - submit (queueing included)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "e2e": {"value": total, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "scope": "host submit -> device solve -> host result per request (state from the "
                             "previous solution on the device)"},
            "gpu_launches": None,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "kkt":
        run_kkt(args, ws, rank, local)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "serve":
        run_serve(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
