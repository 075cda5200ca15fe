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

The JSON line also carries, on one GPU, "sub": the other configurations of
the metric measured in the same run at reduced step counts -- HyKKT at gamma
1e4 and 1e7 on the same column, the largest factorisation (T = 20000, Sigma
log-uniform on [1e-8, 1e8]) with the FP32 and the FP64 factor, the batch of
256 uneven systems (FP64 and FP32 factor, against one instance at a time in
FP64) and the NMPC serving stream (Poisson arrivals at 2000/s; solves/s,
p50/p99 latency, against one slot in FP64).  "e2e" is measured through the
host-buffer C ABI: whole cold solves of the same column submitted to a
one-slot server (host state in, host solution out).  "cpu_baseline" is the
oracle IPM on the same column (T = 5000, not scaled), one full iteration per
single-threaded process, several processes side by side.

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

METRIC = "KKT solve time per IPM iteration"
PREC = {"fp64": 0, "fp32": 1, "df64": 2}
# DRAM bytes of one numeric factorisation come from an ncu capture recorded
# in this file together with the SHA-256 of the kernel sources it measured;
# when the sources differ the counters are stale and roofline.traffic is null
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "factor_dram_traffic.txt")
# Supernode partition of every workload (the library's defaults; the oracle
# baselines analyse with the same ordering options)
PARTITION = dict(leaf_size=8, relax_cols=32, relax_zeros=128, max_width=32)
SUBTREE_COLS = 32

TRAFFIC_SOURCES = ("kernels.cuh", "fused_factor.cuh", "kkt.cu", "fp64_lean.cuh", "sparse_dot.cuh")


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_15913_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def stored_factor_traffic(k, T, solver, precision):
    """Bytes per factorisation from the recorded capture, or None."""
    try:
        rec = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                key, val = line.split(":", 1)
                rec[key.strip()] = val.strip()
        if rec.get("source_sha256") != kernel_source_digest():
            return None
        if rec.get("config") != f"k={k} T={T} solver={solver} precision={precision}":
            return None
        return float(rec["dram_bytes_per_factor"])
    except (OSError, KeyError, ValueError):
        return None


def max_sm_clock_mhz(gpu):
    """Maximum SM clock of the device (nvidia-smi), else the measured peaks file."""
    try:
        out = subprocess.run(["nvidia-smi", f"--id={gpu}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip().splitlines()
        return float(out[0]), "nvidia-smi clocks.max.sm"
    except Exception:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except Exception:
            return 2070.0, "nominal maximum SM clock"


def alu_peak(local, fp32=False):
    """FP64 DFMA (or FP32 FFMA) peak of the device in GFLOP/s: SM count from
    the device properties, maximum SM clock, and the per-SM issue rate of
    this chip (2 FP64 FMA lanes or 128 FP32 FMA lanes per clock)."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz, src = max_sm_clock_mhz(local)
    lanes = 128 if fp32 else 2
    peak = sms * lanes * 2 * mhz / 1e3
    what = "FP32 FFMA" if fp32 else "FP64 DFMA"
    return peak, (f"{what}: {sms} SMs (device query) x {lanes} FMA lanes/clk x 2 flop x {mhz:.0f} MHz "
                  f"({src}); derived from unit counts and clock")
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
    ap.add_argument("--cohort", type=int, default=4,
                    help="serve workload: clients per cohort of the batched server (0: not run)")
    ap.add_argument("--cohort-slots", type=int, default=8,
                    help="serve workload: cohorts the batched server runs at a time")
    ap.add_argument("--batch", type=int, default=256, help="batch workload: instances")
    ap.add_argument("--autotune", action="store_true",
                    help="batch workload: pick the supernode partition with kkt_autotune_batch first")
    ap.add_argument("--sigma", default="1e-6,1e6", help="kkt workload: Sigma_x range")
    ap.add_argument("--staged-solve", type=int, default=None,
                    help="triangular solve variant (kkt_options.staged_solve; default: the library's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="batch workload: kkt_factor_batch + kkt_solve instead of the one-graph step")
    ap.add_argument("--no-serial", action="store_true",
                    help="batch workload: skip the one-context-per-instance comparison")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: skip the sub-records of the other configurations")
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
        self.skip = 0
        self.path = os.path.join(tempfile.gettempdir(), f"kkt_bench_clocks_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return [ln for ln in f.read().split("\n") if ln.count(",") >= 8]
        except OSError:
            return []

    def start(self):
        """Start sampling every 50 ms and return once the first sample is
        written (at most 3 s), so that the samples taken after start()
        returns fall inside the caller's timed region; those are the ones
        stop() reports."""
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and not self._lines():
            time.sleep(0.01)
        self.skip = len(self._lines())

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
        lines = self._lines()
        inside = lines[self.skip:] or lines   # a region shorter than one interval: the nearest samples
        for line in inside:
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
ORACLE_WORKER_BYTES = 2.5e9   # resident set of one oracle IPM at T = 5000 is ~1.8 GB


def _host_memory_bytes():
    """Memory this process may still use: MemAvailable, capped by a cgroup limit."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            raw = open(path).read().strip()
            if raw.isdigit():
                lim = int(raw)
                used = 0
                for upath in ("/sys/fs/cgroup/memory.current",
                              "/sys/fs/cgroup/memory/memory.usage_in_bytes"):
                    try:
                        used = int(open(upath).read().strip())
                        break
                    except (OSError, ValueError):
                        continue
                free = lim - used
                avail = free if avail is None else min(avail, free)
        except OSError:
            continue
    return avail


def oracle_workers(cap):
    mem = _host_memory_bytes()
    by_mem = cap if mem is None else int(mem // ORACLE_WORKER_BYTES)
    return max(1, min(cap, os.cpu_count() or 1, by_mem))


def _oracle_ipm_worker(k, T, scheme, n_warm, n_timed, barrier, out_q):
    """One single-threaded oracle IPM on the full workload: set-up (model
    pattern, symbolic analysis), n_warm untimed iterations, a barrier, then
    n_timed timed iterations (a converged IPM restarts from the start)."""
    import numpy as np
    from gen.tray import TrayParams, ipm_start
    from oracle import ipm as oipm, symbolic, tray as otray
    p = TrayParams(k=k, T=T)
    x0 = ipm_start(p)
    W = otray.hessian_lower_csc(p, x0, np.zeros(p.m))
    J = otray.jacobian_csr(p, x0)
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **PARTITION)

    def fresh():
        lin = oipm.KKTLinearSolver(scheme, p.n, p.m, None, None, sym=sym, gamma=1e4)
        return oipm.IPM(oipm.TrayModel(p), lin, oipm.IPMOptions(relaxed=(scheme == "lifted")), x0)

    s = fresh()

    def one():
        nonlocal s
        while True:
            t0 = time.perf_counter()
            info = s.step()
            dt = time.perf_counter() - t0
            if info.status == "ok":
                return dt
            s = fresh()

    for _ in range(n_warm):
        one()
    barrier.wait()
    out_q.put([one() for _ in range(n_timed)])


def oracle_ipm_parallel(k, T, scheme, n_warm, n_timed, workers):
    """Oracle IPM iterations on the full workload, `workers` single-threaded
    processes (spawned) side by side, iterations shared round-robin.  Returns
    (wall seconds of the timed iterations, per-iteration seconds)."""
    import multiprocessing as mp
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    q = ctx.Queue()
    share = lambda tot, i: tot // workers + (1 if i < tot % workers else 0)
    procs = [ctx.Process(target=_oracle_ipm_worker,
                         args=(k, T, scheme, share(n_warm, i), share(n_timed, i), barrier, q))
             for i in range(workers)]
    for pr in procs:
        pr.start()
    barrier.wait()
    t0 = time.perf_counter()
    times = []
    for _ in procs:
        times += q.get()
    wall = time.perf_counter() - t0
    for pr in procs:
        pr.join()
    return wall, times


def ipm_workload(args, n, m):
    return (f"tray column k={args.k} T={args.T} (n={n}, m={m}), full IPM iteration ({args.scheme}) "
            f"from xbar_0 = 0.3, tol 1e-8")


def cpu_baseline(args):
    """The oracle IPM as it stands on the benchmark's own column: one
    iteration per worker process, the processes side by side."""
    workers = oracle_workers(8)
    wall, times = oracle_ipm_parallel(args.k, args.T, args.scheme, 0, workers, workers)
    return {"value": wall * 1e3 / len(times), "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": (f"{len(times)} oracle IPM iterations ({args.scheme}) on the benchmark's column "
                       f"(k={args.k}, T={args.T}, not scaled), {workers} single-threaded processes side by "
                       f"side: {wall:.1f} s wall / {len(times)} iterations; one iteration takes "
                       f"{statistics.mean(times):.1f} s on one core; set-up (model pattern, symbolic "
                       f"analysis) untimed")}


def run_reference(args, ws, rank):
    """The reference arm: the oracle IPM as it stands on the same column,
    W untimed and K timed iterations, each a full single-threaded iteration,
    run by up to 16 processes side by side (bounded by host memory) so that
    the run ends within a few minutes; ms_per_step = timed wall / K."""
    if rank != 0:
        return None
    workers = oracle_workers(16)
    wall, times = oracle_ipm_parallel(args.k, args.T, args.scheme, args.warmup, args.steps, workers)
    ms = wall * 1e3 / args.steps
    n, m = (2 * args.k + 1) * (args.T + 1), 2 * args.k * (args.T + 1)
    return {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": ipm_workload(args, n, m), "scheme": args.scheme},
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": (f"{args.steps} timed oracle IPM iterations on the benchmark's column, "
                                    f"{workers} single-threaded processes side by side ({wall:.1f} s wall); "
                                    f"one iteration takes {statistics.mean(times):.1f} s on one core")},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


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
    extra = {} if args.staged_solve is None else {"staged_solve": args.staged_solve}
    ipm = IPMSolver(p.as_array(), scheme=args.scheme, gamma=args.gamma, max_cg=500,
                    precision=PREC[args.precision],
                    solver=1 if args.solver == "bcr" else 0, block=2 * args.k + 1, **extra)
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
    # with the one-graph step (FP64 supernodal factor) the refinement loop is
    # timed as a whole inside the graph: K^{-1} itself is timed here, on the
    # factor the last iteration left, through kkt_backsolve (gather, forward
    # and backward solves, scatter), CUDA events on the launching stream
    kinv_direct = None
    if st["graph_steps"] > 0:
        bvec = torch.randn(p.n, dtype=torch.float64, device="cuda")
        xvec = torch.empty_like(bvec)
        kms = []
        for rep in range(13):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = nat.lib().kkt_backsolve(kctx, ctypes.c_void_p(bvec.data_ptr()), ctypes.c_void_p(xvec.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize()
            if rc != nat.KKT_OK:
                raise RuntimeError(f"kkt_backsolve failed with status {rc}")
            if rep >= 3:
                kms.append(e0.elapsed_time(e1))
        kinv_direct = statistics.median(kms)

    # ---- end to end through the host-buffer C ABI: whole cold solves of the
    # same column submitted to a one-slot server (kkt_server_submit with the
    # host initial state x0[k], kkt_server_wait copying the solution x[n] to
    # host memory); time per IPM iteration = wall time / iterations
    e2e_ms, e2e_iters, e2e_solves = None, 0, 0
    if args.precision == "fp64" and args.solver == "supernodal":
        from paper_2403_15913_gb300 import NMPCServer
        srv = NMPCServer(slots=1, hbm_budget_gb=200.0, scheme=args.scheme, gamma=args.gamma,
                         warm_start=False)
        cl = srv.add_client(p.as_array())
        h_state = np.full(p.k, p.x0bar)
        srv.wait(srv.submit(cl, h_state, keep_solution=True), want_solution=True)   # context set-up
        t0 = time.perf_counter()
        for _ in range(2):
            r, _x = srv.wait(srv.submit(cl, h_state, keep_solution=True), want_solution=True)
            if r["status"] != nat.KKT_CONVERGED:
                raise RuntimeError(f"end-to-end solve ended with status {r['status']}")
            e2e_iters += r["iters"]
            e2e_solves += 1
        e2e_wall = time.perf_counter() - t0
        srv.close()
        e2e_ms = e2e_wall * 1e3 / max(1, e2e_iters)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fcalls = max(1, st["factor_calls"])
    factor_ms = st["factor_ms"] / fcalls
    kinv_ms = kinv_direct if kinv_direct is not None else st["solve_ms"] / max(1, st["kinv_calls"])
    f32 = args.precision == "fp32"
    peak, peak_src = alu_peak(local, f32)
    roof = {"kernel": ("block cyclic reduction (bcr_elim/bcr_update kernels)" if args.solver == "bcr" else
                       "supernodal Cholesky (factor kernels of one kkt_factor)"),
            "bound": "alu", "achieved": fl.value / (factor_ms * 1e-3) / 1e9,
            "peak": peak, "unit": "GFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = stored_factor_traffic(args.k, args.T, args.solver, args.precision)
    roof["peak_source"] = peak_src
    n_steps = len(step_ms)
    line = {
        "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": ipm_workload(args, p.n, p.m),
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
                                "kinv_per_step": st["kinv_calls"] / n_steps,
                                "graph_steps_per_step": st["graph_steps"] / n_steps,
                                "refinement_ms": (st["solve_ms"] / n_steps) if st["graph_steps"] > 0 else None},
                   "max_bwd_err": max(i["bwd_err"] for i in infos),
                   "refine_iters": [i["refine_iters"] for i in infos][:6],
                   "cg_iters": [i["cg_iters"] for i in infos][:6],
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": ({"value": e2e_ms, "unit": UNIT,
                 "h2d_bytes_per_step": p.k * 8 * e2e_solves / max(1, e2e_iters),
                 "d2h_bytes_per_step": p.n * 8 * e2e_solves / max(1, e2e_iters),
                 "scope": (f"{e2e_solves} whole cold solves ({e2e_iters} iterations) through the host-buffer "
                           "C ABI: kkt_server_submit with the host state x0[k], kkt_server_wait copying "
                           "x[n] to host memory; wall time / iterations")}
                if e2e_ms is not None else None),
        "gpu_launches": (int(st["launches"] / n_steps * args.steps) + sum(i["launches"] for i in infos))
                        if n_steps else 0,
        "clocks": clk,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    if dist:
        dist.destroy_process_group()
    return line


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
    sym = symbolic.analyse(p.n, W[0], W[1], J[0], J[1], **PARTITION)
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
    opts = dict(scheme=args.scheme, gamma=args.gamma, max_cg=500, subtree_cols=SUBTREE_COLS,
                solver=1 if args.solver == "bcr" else 0, block=2 * args.k + 1, **PARTITION)

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
    peak, peak_src = alu_peak(local, f32)
    roof = {"kernel": ("block cyclic reduction (bcr_elim/bcr_update kernels)" if args.solver == "bcr" else
                       "supernodal Cholesky (factor kernels of one kkt_factor)"),
            "bound": "alu", "achieved": sym.flops / (factor_ms * 1e-3) / 1e9,
            "peak": peak, "unit": "GFLOP/s",
            "traffic": stored_factor_traffic(args.k, args.T, args.solver, args.precision),
            "peak_source": peak_src}
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
    if dist:
        dist.destroy_process_group()
    return line


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
    opts = dict(scheme=args.scheme, gamma=args.gamma, max_cg=500, subtree_cols=SUBTREE_COLS, **PARTITION)
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

    # FP64: the whole step as one graph launch (kkt_factor_solve); the FP32
    # factor (with its FP64 fallback) keeps the two calls
    use_graph = prec == 0 and not getattr(args, "no_graph", False)

    def step(d):
        if use_graph:
            return bs.factor_solve(d["W"], d["J"], d["sigma"], None, delta, d["rx"], d["ry"], dx, dy)
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
    do_serial = not getattr(args, "no_serial", False)
    singles = []
    for i, (p, pt) in enumerate(zip(params, pats)):
        if do_serial:
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
    for _ in range(max(1, min(args.steps, 3)) if do_serial else 0):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        serial()
        e1.record(stream)
        torch.cuda.synchronize()
        ser_ms.append(e0.elapsed_time(e1))
    ser_eta = max((s1.info.bwd_err for s1 in singles), default=None)
    for s1 in singles:
        s1.close()
    # end to end: values and right-hand sides host->device, batched factor +
    # solve, (dx, dy) device->host
    h_out = torch.empty(bs.n + bs.m, dtype=torch.float64).pin_memory()
    e2e = []
    for rep in range(4):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in d_in:   # into the buffers the graph was captured with
            d_in[k].copy_(h_in[k], non_blocking=True)
        step(d_in)
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
    peak, peak_src = alu_peak(local, f32)
    roof = {"kernel": "batched supernodal Cholesky (factor kernels of one kkt_factor_batch)",
            "bound": "alu", "achieved": sym.flops / (factor_ms * 1e-3) / 1e9,
            "peak": peak, "unit": "GFLOP/s", "traffic": None, "peak_source": peak_src}
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
                   "factor_ms": factor_ms,
                   "kinv_ms": None if use_graph else st["solve_ms"] / max(1, st["kinv_calls"]),
                   "refinement_ms": st["solve_ms"] / max(1, args.steps) if use_graph else None,
                   "tree_levels": sym.levels, "statuses": sorted(statuses),
                   "max_bwd_err": max(etas), "max_refine_iters": int(res["refine_iters"].max()),
                   "fp64_fallbacks": st["fp64_fallbacks"],
                   "step": ("one CUDA graph launch per step (kkt_factor_solve: factor, refinement "
                            "sweeps as a conditional WHILE node)" if use_graph
                            else "kkt_factor_batch + kkt_solve"),
                   "graph_launches_per_step": st["graph_steps"] / max(1, args.steps),
                   "delta_x_nonzero": int((delta > 0).sum()),
                   "per_instance_fp64_path": ({"ms_per_batch": statistics.mean(ser_ms),
                                               "solves_per_s": args.batch / (statistics.mean(ser_ms) * 1e-3),
                                               "max_bwd_err": ser_eta} if ser_ms else None),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": args.batch * ws / (statistics.mean(e2e) * 1e-3), "unit": "solves/s",
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": (bs.n + bs.m) * 8,
                "scope": "W, J, Sigma and rhs host->device, batched factor + solve, (dx, dy) device->host"},
        "gpu_launches": int(st["launches"] / max(1, args.steps) * args.steps),
        "clocks": clk,
    }
    bs.close()
    if dist:
        dist.destroy_process_group()
    return line


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

    def serve(slots, precision, rate=None, count=None, cohort=0):
        gaps_, who_ = gaps, who
        if rate is not None:
            r2 = np.random.default_rng(args.seed + 31)
            gaps_ = r2.exponential(1.0 / rate, count)
            who_ = r2.integers(0, args.clients, count)
        srv = NMPCServer(slots=slots, hbm_budget_gb=40.0, scheme=args.scheme, precision=precision,
                         gamma=args.gamma, batch=cohort)
        # a batched server groups clients into cohorts in the order they are
        # added: added by size, so a cohort's members have similar trees
        cl = [None] * len(params)
        for i in (sorted(range(len(params)), key=lambda j: params[j].n) if cohort else range(len(params))):
            cl[i] = srv.add_client(params[i].as_array())
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
        objective[(slots, precision, cohort, rate)] = {r["id"]: r["objective"] for r in res}
        return {"solves_per_s": len(res) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "iters_mean": float(np.mean([r["iters"] for r in res])),
                "converged": int(sum(r["status"] == 1 for r in res)),
                "warm": int(sum(r["warm"] for r in res)), "prewarm_s": round(prewarm, 2),
                "contexts": st["contexts_created"], "evictions": st["evictions"],
                "peak_resident_gb": st["peak_resident_bytes"] / 1e9, "clocks": clk}

    objective = {}

    def obj_diff(a, b):
        """largest relative objective difference of the same requests"""
        oa, ob = objective[a], objective[b]
        return float(max(abs(oa[i] - ob[i]) / max(abs(ob[i]), 1e-300) for i in oa))

    prec = PREC[args.precision]
    conc = serve(args.slots, prec)
    serial = serve(1, 0)
    batched = {}
    if args.cohort > 0:
        # the batched server: cohorts of clients, one union KKT factor and
        # solve per IPM iteration of a cohort, in FP64 and with the FP32
        # factor and FP64 refinement; accuracy against the serial FP64 path
        # request by request (same stream, same per-client order)
        for name, pr in (("fp64", 0), ("fp32_factor", 1)):
            r = serve(args.cohort_slots, pr, cohort=args.cohort)
            r.pop("clocks")
            r["max_rel_objective_diff_vs_serial_fp64"] = obj_diff((args.cohort_slots, pr, args.cohort, None),
                                                                  (1, 0, 0, None))
            r["speedup_vs_serial_fp64"] = r["solves_per_s"] / serial["solves_per_s"]
            batched[name] = r
        best = batched["fp32_factor"]
        light_b_rate = 0.7 * best["solves_per_s"]
        lb = serve(args.cohort_slots, 1, rate=light_b_rate, count=min(args.requests, 200), cohort=args.cohort)
        lb.pop("clocks")
        lb["rate_per_s"] = light_b_rate
        batched["fp32_factor"]["at_70pct_of_capacity"] = lb
    # service latency below saturation: the same server at 70% of the
    # throughput it just sustained
    light_rate = 0.7 * conc["solves_per_s"]
    light = serve(args.slots, prec, rate=light_rate, count=min(args.requests, 200))
    light.pop("clocks")
    light["rate_per_s"] = light_rate
    total = across_ranks(conc["solves_per_s"], "sum", dist)
    line = None
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
                       "batched": dict(batched, cohort=args.cohort, cohort_slots=args.cohort_slots),
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
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def sub_records(args, local):
    """The other configurations of the metric, measured in the same run at
    reduced step counts (one GPU): HyKKT at gamma 1e4 and 1e7 on the same
    column, the largest factorisation (T = 20000, Sigma on [1e-8, 1e8]) in
    FP32 and FP64, the 256-instance batch (FP64 and FP32 factor, against one
    instance at a time in FP64) and the NMPC serving stream."""
    import copy
    out = {}

    def sub(**kw):
        a = copy.copy(args)
        a.no_cpu_baseline, a.gpus = True, 1
        a.steps, a.warmup = kw.pop("steps", 5), kw.pop("warmup", 3)
        for key, val in kw.items():
            setattr(a, key, val)
        return a

    def safe(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:   # a failed sub-record is reported, the main line stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)

    def hykkt(g):
        ln = run_ours(sub(scheme="hykkt", gamma=g), 1, 0, local)
        c = ln["config"]
        return {"ms_per_iter": ln["value"], "e2e_ms_per_iter": ln["e2e"]["value"],
                "factor_ms": c["phase_ms"]["factor"], "kinv_ms": c["phase_ms"]["kinv"],
                "kinv_per_iter": c["phase_ms"]["kinv_per_step"], "cg_iters": c["cg_iters"],
                "max_bwd_err": c["max_bwd_err"], "steps": ln["steps"], "clocks": ln["clocks"]}

    def largest():
        ln = run_kkt(sub(workload="kkt", T=20000, sigma="1e-8,1e8", precision="fp32",
                         scheme="lifted"), 1, 0, local)
        c, f64 = ln["config"], ln["config"]["fp64_factor_path"]
        peak64, _ = alu_peak(local, False)
        return {"workload": c["workload"], "factor_gflop": c["factor_gflop"],
                "fp64": {"factor_ms": f64["factor_ms"], "step_ms": f64["ms"],
                         "frac_of_fp64_peak": c["factor_gflop"] / (f64["factor_ms"] * 1e-3) / peak64,
                         "max_bwd_err": f64["bwd_err"]},
                "fp32_factor": {"factor_ms": c["factor_ms"], "step_ms": ln["value"],
                                "frac_of_fp32_peak": ln["roofline"]["frac"],
                                "max_bwd_err": c["max_bwd_err"], "refine_iters": c["refine_iters"],
                                "fp64_fallbacks": c["fp64_fallbacks"],
                                "rel_diff_vs_fp64_path": f64["rel_diff_vs_fp64_path"]},
                "steps": ln["steps"], "clocks": ln["clocks"]}

    def batch(prec, **kw):
        ln = run_batch(sub(workload="batch", precision=prec, scheme="lifted", **kw), 1, 0, local)
        c = ln["config"]
        return {"solves_per_s": ln["value"], "ms_per_batch": ln["ms_per_step"],
                "e2e_solves_per_s": ln["e2e"]["value"], "factor_ms": c["factor_ms"],
                "factor_frac_of_peak": ln["roofline"]["frac"], "max_bwd_err": c["max_bwd_err"],
                "per_instance_fp64": c["per_instance_fp64_path"], "step": c["step"],
                "graph_launches_per_step": c["graph_launches_per_step"], "steps": ln["steps"],
                "clocks": ln["clocks"]}

    def serve():
        ln = run_serve(sub(workload="serve", scheme="lifted", precision="fp64"), 1, 0, local)
        c = ln["config"]
        return {"workload": c["workload"], "solves_per_s": ln["value"],
                "p50_ms": c["concurrent"]["p50_ms"], "p99_ms": c["concurrent"]["p99_ms"],
                "serial_fp64_one_slot": {k: c["serial_fp64_one_slot"][k]
                                         for k in ("solves_per_s", "p50_ms", "p99_ms")},
                "at_70pct_of_capacity": {k: c["at_70pct_of_capacity"][k]
                                         for k in ("rate_per_s", "solves_per_s", "p50_ms", "p99_ms")},
                "batched": {name: {k: v for k, v in r.items() if k in (
                    "solves_per_s", "p50_ms", "p99_ms", "iters_mean", "converged",
                    "max_rel_objective_diff_vs_serial_fp64", "speedup_vs_serial_fp64", "at_70pct_of_capacity")}
                    for name, r in c["batched"].items() if isinstance(r, dict)},
                "iters_mean": c["concurrent"]["iters_mean"], "clocks": ln["clocks"]}

    safe("hykkt_gamma_1e4", lambda: hykkt(1e4))
    safe("hykkt_gamma_1e7", lambda: hykkt(1e7))
    safe("largest_factor", largest)
    safe("batch_fp64", lambda: batch("fp64"))
    safe("batch_fp32", lambda: batch("fp32", no_serial=True))
    safe("serve", serve)
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
    elif args.workload == "kkt":
        line = run_kkt(args, ws, rank, local)
    elif args.workload == "batch":
        line = run_batch(args, ws, rank, local)
    elif args.workload == "serve":
        line = run_serve(args, ws, rank, local)
    else:
        line = run_ours(args, ws, rank, local)
        if line is not None and ws == 1 and not args.no_sub:
            cb = line.pop("cpu_baseline", None)
            line["sub"] = sub_records(args, local)
            if cb is not None:
                line["cpu_baseline"] = cb
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
