#!/usr/bin/env python
"""Benchmark of the KKT hot path: KKT solve time per IPM iteration.

Workload: the distillation column of Sec. VI-A (32 trays) on T = 5000
implicit-Euler stages (n = 325,065 variables, m = 320,064 constraints), the
KKT system taken at a seeded iterate (compositions U(0.05, 0.95), reflux
U(1.05, 4.95), multipliers N(0, 1), Sigma_x log-uniform on [1e-6, 1e6],
N(0, 1) right-hand side).

One step = one KKT solve of an IPM iteration, all on the GPU:
  derivative evaluation (Jacobian and Lagrangian Hessian kernels),
  assembly of the condensed matrix, supernodal Cholesky (with inertia
  correction when a pivot fails), and the Lifted-KKT (or HyKKT) solve with
  iterative refinement to a backward error <= 1e-10 on the original system.
The symbolic analysis is done once before timing (reported separately, as
the paper's SYM column).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--scheme lifted|hykkt]
        python bench.py --impl reference ...   (the CPU oracle, timed as it stands)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070   # SMs x DFMA/clk/SM x flops x GHz = 1258.6
METRIC = "KKT solve time per IPM iteration"
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

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
def oracle_step_sample(k, T_sample, seed, scheme, gamma):
    """One KKT step of the CPU oracle at a bounded size: model derivatives,
    condensed matrix, left-looking Cholesky and the hybrid solve."""
    import numpy as np
    from gen.tray import TrayParams, kkt_point
    from oracle import kkt as okkt, symbolic, tray as otray
    p = TrayParams(k=k, T=T_sample)
    pt = kkt_point(p, seed)
    W0 = otray.hessian_lower_csc(p, pt.w, pt.lam)
    J0 = otray.jacobian_csr(p, pt.w)
    sym = symbolic.analyse(p.n, W0[0], W0[1], J0[0], J0[1], leaf_size=64, relax_cols=32,
                           relax_zeros=128, max_width=64)
    t0 = time.perf_counter()
    W = otray.hessian_lower_csc(p, pt.w, pt.lam)
    J = otray.jacobian_csr(p, pt.w)
    if scheme == "lifted":
        okkt.lifted_solve(sym, p.n, p.m, W, J, pt.sigma, 0.0, np.full(p.m, 1e8), pt.rx, pt.ry)
    else:
        okkt.hykkt_solve(sym, p.n, p.m, W, J, pt.sigma, 0.0, gamma, pt.rx, pt.ry)
    return time.perf_counter() - t0


def cpu_baseline(args, budget_s=15.0, T_sample=50):
    times = []
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s or len(times) < 2:
        times.append(oracle_step_sample(args.k, T_sample, args.seed, args.scheme, args.gamma))
        if len(times) >= 20:
            break
    per = statistics.median(times)
    scale = (args.T + 1) / (T_sample + 1)
    return {"value": per * scale * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{len(times)} oracle KKT steps ({args.scheme}) at {args.k} trays, "
                       f"T={T_sample}: median {per*1e3:.1f} ms, scaled x{scale:.1f} to T={args.T} "
                       "(work linear in T)")}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_step_sample(args.k, 50, args.seed, args.scheme, args.gamma)
        if i >= args.warmup:
            times.append(t)
    scale = (args.T + 1) / 51
    ms = statistics.mean(times) * scale * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"tray column k={args.k} T={args.T} (n={(2*args.k+1)*(args.T+1)}), "
                               f"{args.scheme} KKT step, oracle on T=50 scaled by (T+1)/51",
                   "scheme": args.scheme},
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: one oracle KKT step at T=50 scaled x{scale:.1f}"},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from gen.tray import TrayParams, kkt_point
    from paper_2403_15913_gb300 import KKTSolver, TrayModel

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = TrayParams(k=args.k, T=args.T)
    pt = kkt_point(p, args.seed + rank)
    tm = TrayModel(p.as_array())
    Wc, Wr, Jr, Jc = tm.pattern()
    t0 = time.perf_counter()
    solver = KKTSolver(p.n, p.m, Wc, Wr, Jr, Jc, scheme=args.scheme, gamma=args.gamma,
                       max_cg=500)
    t_analyse = time.perf_counter() - t0
    sizes = solver.sizes()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    w, lam, sigma = dev(pt.w), dev(pt.lam), dev(pt.sigma)
    rx, ry = dev(pt.rx), dev(pt.ry)
    Wv = torch.empty(tm.nnzW, dtype=torch.float64, device="cuda")
    Jv = torch.empty(tm.nnzJ, dtype=torch.float64, device="cuda")
    dx = torch.empty(p.n, dtype=torch.float64, device="cuda")
    dy = torch.empty(p.m, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    state = {"delta_x": 0.0, "launches": 0}
    infos = []

    def kkt_step(w_, lam_, sigma_, rx_, ry_):
        tm.eval(w_, lam_, 1.0, Jval=Jv, Wval=Wv)
        state["launches"] += 1
        dxr = state["delta_x"]
        st = solver.factor(Wv, Jv, sigma_, None, dxr)
        while st == -4:                                  # inertia correction
            dxr = 1e-4 if dxr == 0.0 else dxr * 8.0
            st = solver.factor(Wv, Jv, sigma_, None, dxr)
        state["delta_x"] = dxr
        st = solver.solve(rx_, ry_, dx, dy)
        infos.append(dict(solver.info.as_dict(), status=st))
        return st

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.zero_()
        kkt_step(w, lam, sigma, rx, ry)
    torch.cuda.synchronize()
    infos.clear()
    solver.set_profiling(True)
    solver.reset_stats()
    state["launches"] = 0
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                                    # L2 flush, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kkt_step(w, lam, sigma, rx, ry)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(step_ms)
    st = solver.stats()
    launches = st["launches"] + state["launches"]
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()

    # ---- end-to-end through the public API with host buffers
    h_in = [t.cpu().pin_memory() for t in (w, lam, sigma, rx, ry)]
    h_out = [torch.empty(p.n, dtype=torch.float64).pin_memory(),
             torch.empty(p.m, dtype=torch.float64).pin_memory()]
    d_in = [torch.empty_like(t, device="cuda") for t in h_in]
    solver.set_profiling(False)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, h in zip(d_in, h_in):
            d.copy_(h, non_blocking=True)
        kkt_step(*d_in)
        h_out[0].copy_(dx, non_blocking=True)
        h_out[1].copy_(dy, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    h2d = sum(t.numel() * 8 for t in h_in)
    d2h = (p.n + p.m) * 8

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- roofline of the dominant kernel family
    fcalls = max(1, st["factor_calls"])
    kcalls = max(1, st["kinv_calls"])
    factor_ms = st["factor_ms"] / fcalls
    solve_ms = st["solve_ms"] / kcalls
    flops_factor = sizes.flops                      # sum_j cc_j^2
    flops_solve = 4.0 * sizes.nnz_L                 # forward + backward
    if st["factor_ms"] >= st["solve_ms"]:
        roof = {"kernel": "factor_level_kernel (supernodal Cholesky, all levels)",
                "bound": "alu", "achieved": flops_factor / (factor_ms * 1e-3) / 1e9,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s"}
    else:
        roof = {"kernel": "forward/backward_level_kernel (triangular solves, one K^-1)",
                "bound": "alu", "achieved": flops_solve / (solve_ms * 1e-3) / 1e9,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["peak_source"] = "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)"
    bwd = [i["bwd_err"] for i in infos]
    line = {
        "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"tray column k={args.k} T={args.T} (n={p.n}, m={p.m}), "
                               f"{args.scheme} KKT step at a seeded iterate",
                   "scheme": args.scheme, "gamma": args.gamma if args.scheme == "hykkt" else None,
                   "delta": 1e-8, "l2": "flushed (256 MB write) between timed steps",
                   "analyse_s": round(t_analyse, 3), "supernodes": sizes.ns,
                   "nnz_L": sizes.nnz_L, "panel_entries": sizes.panel, "levels": sizes.levels,
                   "factor_gflop": flops_factor / 1e9, "delta_x": state["delta_x"],
                   "max_bwd_err": max(bwd), "refine_iters": [i["refine_iters"] for i in infos][:3],
                   "cg_iters": [i["cg_iters"] for i in infos][:3],
                   "phase_ms": {"assemble": st["assemble_ms"] / fcalls, "factor": factor_ms,
                                "kinv": solve_ms, "kinv_per_step": st["kinv_calls"] / args.steps,
                                "other": st["other_ms"] / args.steps},
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": statistics.mean(e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
