#!/usr/bin/env python
"""Benchmark: solves/s of the vertical-extrapolation multigrid PCG on one GB300.

Workload: the 256 x 256 x 32 extruded thin mesh (2,179,617 nodes, 12,582,912 tets) with depth
H = 1e-3 (1 + 0.5 sin 2 pi x sin 2 pi y) (aspect ratio 1e-3), interior nodes z-jittered by
+-0.3 layer thickness, all-Neumann, i.i.d. N(0, 1) nodal loads projected to zero mean, stop at
relative residual 1e-8. A step is one complete solve (every Krylov iteration with its additive
multigrid preconditioner) with the hierarchy resident on the device; the hierarchy is built once
(its time is reported as setup_s). Inputs (A: 0.39 GB, hierarchy > 1 GB) are larger than L2.

  python bench.py [--steps K] [--warmup W] [--precision fp64|fp32|bf16] [--impl vemg|reference]

Under torchrun (N > 1), every rank solves its own right-hand sides on its own GPU (independent
problems, no collective in the data path); value = solves of all ranks / max rank time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "zjit256"
RTOL = 1e-8
METRIC = "solves/s at FP64 rel-res 1e-8"


PRECONDS = {"additive": 0, "vl_sor": 1, "sa": 2}
PRECS = {"fp64": 0, "fp32": 1, "bf16": 2}
DTYPES = {"fp64": "f64", "fp32": "f64 outer + f32 preconditioner",
          "bf16": "f64 outer + f32 preconditioner with bf16 operator values"}
# ncu DRAM bytes / algorithmic bytes of the finest colour sweep (one launch, 192x192x32 mesh)
SOR_FINE_DRAM_RATIO = {"fp32": 34.63 / 32.33, "bf16": 27.33 / 25.18}
SOR_FINE_KERNEL = {"fp32": "k_sell_sor<float, float, double>", "bf16": "k_sell_sor<__nv_bfloat16, float, double>"}
CYCLES = {"persistent": 0, "launches": 1, "auto": 2, "hybrid": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vemg", choices=["vemg", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PRECS))
    ap.add_argument("--cycle", default="auto", choices=["auto", "persistent", "launches", "hybrid"],
                    help="one cooperative kernel per preconditioner application, one kernel per phase, or the "
                         "library's choice by precision")
    ap.add_argument("--precond", default="additive", choices=list(PRECONDS),
                    help="additive (the paper's preconditioner), vl_sor or sa (its two comparison forms)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other configurations (xy-jittered mesh, batched, serving) after the headline")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving workload: this many Poisson-arrival requests (512 for the full stream)")
    ap.add_argument("--rate", type=float, default=0.0, help="serving arrival rate (0: 0.8 x saturation)")
    ap.add_argument("--slots", type=int, default=8, help="serving: right-hand-side slots per engine")
    ap.add_argument("--case", default="",
                    help="profiling case NXxNYxNZ (z-jitter 0.3, eps 1e-3): two untimed solves, then exit")
    ap.add_argument("--spectrum", action="store_true",
                    help="the section 4 study: condition estimates of A and M^-1 A over eps (not a timing run)")
    ap.add_argument("--phases", action="store_true",
                    help="with --case: per-phase profile of the persistent preconditioner kernel")
    ap.add_argument("--tail-rows", type=int, default=None,
                    help="levels of at most this many rows (below the finest) run as one single-CTA kernel; "
                         "default: the library's")
    ap.add_argument("--surf-nullspace", type=int, default=None, choices=[1, 3],
                    help="near-nullspace of the surface chain: 1 (constants) or 3 ({1, x, y}); default: 3 on "
                         "xy-jittered workloads, else 1")
    ap.add_argument("--bc", default="neumann", choices=["neumann", "dirichlet_top"])
    ap.add_argument("--tail-cluster", type=int, default=None,
                    help="CTAs of the thread-block cluster that runs the coarse tail (0: one CTA); default: the "
                         "library's")
    ap.add_argument("--stream-path", action="store_true",
                    help="with --case: launch the solve's kernels on the stream, not from CUDA graphs")
    ap.add_argument("--rhs", type=int, default=0,
                    help="right-hand sides per step (0: the workload's own count); >1 uses vemg_solve_batch")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (every 200 ms) during the timed region. Each query takes driver time that
    can delay the solve's launches, so the interval is kept long."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(num(r[2]) for r in rows),
                "samples": len(rows), "reasons": reasons}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, dist, torch):
    """The slowest rank's time: every rank runs its own problems (weak scaling), so the job ends
    when the last one does. NCCL reduces a device tensor, gloo a host one."""
    if not dist:
        return ms
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, dist, torch):
    if not dist:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(ws, units_per_rank_step, steps, ms):
    """Units per second of the whole job: every rank processed units_per_rank_step units in each
    of `steps` steps, and the job took ms milliseconds (the max over ranks)."""
    return ws * units_per_rank_step * steps / (ms / 1000.0)


# --------------------------------------------------------------------------------------------
# the CPU oracle: the reference arm and the cpu_baseline leg

def time_oracle(mesh, b, sample_iters=None, openmp=False):
    """Time the oracle as it stands on this host: the plain single-threaded build, or its OpenMP
    timing build on every host core (the same bits). If sample_iters is None, one full solve;
    otherwise a solve truncated at sample_iters iterations."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    P = O.Problem(mesh, openmp=openmp)
    setup_s = time.perf_counter() - t0
    threads = int(P.L.or_threads())
    t0 = time.perf_counter()
    if sample_iters is None:
        r = P.solve(b, tol=RTOL)
        dt = time.perf_counter() - t0
        return dict(setup_s=setup_s, solve_s=dt, iters=r["iters"], relres=r["relres"], problem=P, threads=threads)
    r = P.solve(b, tol=0.0, maxit=sample_iters)
    dt = time.perf_counter() - t0
    return dict(setup_s=setup_s, sample_s=dt, iters=r["iters"], problem=P, threads=threads)


def run_reference(args):
    """The oracle as the reference arm: its OpenMP timing build on every host core. Each step is a
    full solve when (steps + warmup) full solves fit in a few minutes; otherwise each step is a
    solve truncated at 3 iterations, scaled to a full solve by preconditioner applications."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_0912_1976_gb300 import inputs as I
    mesh = I.make_workload_mesh(args.workload)
    from oracle import oracle as O
    P = O.Problem(mesh, openmp=True)
    threads = int(P.L.or_threads())
    b0 = I.normal_loads(mesh.n, 2000)
    t0 = time.perf_counter()
    full = P.solve(b0, tol=RTOL)                  # iteration count and time of a full solve (warm-up)
    full_s = time.perf_counter() - t0
    I_full = full["iters"]
    truncated = full_s * (args.steps + args.warmup) > 240.0
    sample_iters = 3
    times = []
    for k in range(args.warmup + args.steps):
        b = I.normal_loads(mesh.n, 2100 + k)
        t0 = time.perf_counter()
        if truncated:
            P.solve(b, tol=0.0, maxit=sample_iters)
        else:
            P.solve(b, tol=RTOL)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    if truncated:
        # a solve truncated at m iterations applies the preconditioner m + 1 times (the cost that
        # dominates an iteration) and a full solve of I iterations applies it I times
        solve_s = sum(times) / (len(times) * (sample_iters + 1)) * I_full
        sample = (f"{args.steps} solves of the {args.workload} workload truncated at {sample_iters} PCG "
                  f"iterations each, scaled to the {I_full} iterations of a full solve to rel-res {RTOL:g}")
    else:
        solve_s = sum(times) / len(times)
        sample = f"{args.steps} full solves of the {args.workload} workload ({I_full} iterations to rel-res {RTOL:g})"
    value = 1.0 / solve_s
    sample += f", OpenMP build of the oracle on {threads} host threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * solve_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, mesh.n),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters": I_full, "full_steps": not truncated}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, n):
    from paper_0912_1976_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    kr = args.rhs or w.get("nrhs", 1)
    return {"workload": f"{args.workload}: {w['nx']}x{w['ny']}x{w['nz']} extruded hex->6 tets, {n} nodes, "
                        f"H0 {w['depth'][1]:g}, z-jitter {w['z_jitter']}, xy-jitter {w['xy_jitter']}, "
                        f"{'all-Neumann' if args.bc == 'neumann' else 'Dirichlet top'}, N(0,1) loads"
                        f"{' mean-zero' if args.bc == 'neumann' else ''}, rtol {RTOL:g}",
            "precision": args.precision, "preconditioner": args.precond, "cycle": args.cycle, "rhs_per_step": kr,
            "tail_rows": args.tail_rows if args.tail_rows is not None else "default",
            "tail_cluster": args.tail_cluster if args.tail_cluster is not None else "default",
            "surface_nullspace": {1: "constants", 3: "{1, x, y}"}[surf_ns(args)],
            "bc": args.bc,
            "l2": "inputs larger than L2 (A alone 0.39 GB; no flush needed)",
            "parallelism": f"independent problems x{args.gpus}" if args.gpus > 1 else "single GPU"}


# --------------------------------------------------------------------------------------------
# the GPU path

def measure(args, h, B, n, ws, rank, local, dist, V, torch, probe, cycle="launches"):
    """Time args.steps solves (device-resident inputs), then the same through the host-buffer
    entry point, then (optionally) per-kernel-class probes."""
    nb = len(B)
    X = torch.empty_like(B[0])
    batched = B[0].dim() == 2
    kcols = B[0].shape[0] if batched else 1

    def step(j):
        if batched:
            _, infos = V.vemg_solve_batch(h, B[j % nb], X, rtol=RTOL, max_it=1000)
            bad = [i for i in infos if i["status"] != "OK"]
            if bad:
                raise RuntimeError(f"batched solve did not converge: {bad[0]}")
            return {"iters": max(i["iters"] for i in infos), "true_relres": max(i["true_relres"] for i in infos)}
        _, info = V.vemg_solve(h, B[j % nb], X, rtol=RTOL, max_it=1000)
        if info["status"] != "OK":
            raise RuntimeError(f"solve did not converge: {info}")
        return info

    for j in range(args.warmup):
        step(j)
    l0 = V.vemg_kernel_launches(h)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for j in range(args.steps):
        infos.append(step(args.warmup + j))
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    launches = V.vemg_kernel_launches(h) - l0
    ms = max_over_ranks(ms, dist, torch)
    iters = [i["iters"] for i in infos]
    out = {"value": whole_job_rate(ws, kcols, args.steps, ms), "ms_per_step": ms / args.steps, "iters": iters,
           "true_relres_max": max(i["true_relres"] for i in infos),
           "gdof_iter_per_s": sum_over_ranks(kcols * sum(n * it for it in iters), dist, torch) / (ms / 1000.0) / 1e9,
           "gpu_launches": launches, "clocks": clocks}
    # end to end: host buffers, host-to-device copy of the step's inputs and device-to-host copy
    # of its results inside the timed region (vemg_solve_host for one right-hand side; pinned
    # copies around vemg_solve_batch for a batch)
    bh = torch.empty(B[0].shape, dtype=torch.float64, pin_memory=True)
    xh = torch.empty(B[0].shape, dtype=torch.float64, pin_memory=True)
    bh.copy_(B[0].cpu())
    bnp, xnp = bh.numpy(), xh.numpy()
    Bd = torch.empty_like(B[0])

    def e2e_step():
        if batched:
            Bd.copy_(bh, non_blocking=True)
            V.vemg_solve_batch(h, Bd, X, rtol=RTOL, max_it=1000)
            xh.copy_(X, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        else:
            V.vemg_solve_host(h, bnp, xnp, rtol=RTOL)

    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0.record()
    for j in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    ms_e2e = max_over_ranks(ms_e2e, dist, torch)
    out["e2e"] = {"value": whole_job_rate(ws, kcols, args.steps, ms_e2e), "unit": "solves/s",
                  "h2d_bytes_per_step": 8 * n * kcols, "d2h_bytes_per_step": 8 * n * kcols}
    classes = {}
    if probe and not batched:
        # the persistent cycle (one kernel per preconditioner application), the hybrid one (its
        # finest-level colour sweeps and the cooperative kernel of the coarser levels) or, with
        # per-phase launches, its kernel classes
        if cycle == "persistent":
            kinds = {"spmv_A": V.VEMG_PROBE_SPMV_A, "vcycle": V.VEMG_PROBE_VCYCLE}
        elif cycle == "hybrid":
            kinds = {"spmv_A": V.VEMG_PROBE_SPMV_A, "sor_fine": V.VEMG_PROBE_SOR_FINE,
                     "vcycle_coarse": V.VEMG_PROBE_VCYCLE}
        else:
            kinds = {"spmv_A": V.VEMG_PROBE_SPMV_A, "sor_fine": V.VEMG_PROBE_SOR_FINE,
                     "sor_coarse": V.VEMG_PROBE_SOR_COARSE, "residual": V.VEMG_PROBE_RESIDUAL,
                     "transfer": V.VEMG_PROBE_TRANSFER, "vector": V.VEMG_PROBE_VECTOR, "dense": V.VEMG_PROBE_DENSE,
                     "tail": V.VEMG_PROBE_TAIL}
        for name, kind in kinds.items():
            V.vemg_probe(h, kind)
            for j in range(2):
                step(j)
            r = V.vemg_probe_read(h)
            V.vemg_probe(h, V.VEMG_PROBE_NONE)
            if r["launches"]:
                classes[name] = {"launches_per_solve": r["launches"] / 2, "ms_per_solve": r["ms"] / 2,
                                 "achieved_gbs": r["bytes"] / (r["ms"] / 1000.0) / 1e9,
                                 "bytes_per_launch": r["bytes"] / r["launches"],
                                 "bytes_per_solve": r["bytes"] / 2}
    out["classes"] = classes
    return out


def serve_stream(nreq, slots, precision, rate=0.0):
    """Continuous batching over the serving stream: a saturation run (all requests at t = 0) gives
    the capacity, then the Poisson run at 80% of it (or `rate`) gives the latency percentiles, each
    starting with no hierarchy resident (built on first use); `poisson_warm` replays the Poisson
    stream on the same server with its hierarchies resident (steady state). Returns the per-phase
    summaries, the Poisson rate and the clocks seen during the cold Poisson run."""
    import torch
    from paper_0912_1976_gb300 import serve as S
    fac = S.GpuFactory(slots=slots, precision=PRECS[precision])
    for i in range(len(S.SIZES)):                  # meshes are inputs: generated before the clock
        fac.mesh(i, 1.0)
    out = {}
    clocks = None
    srv = None
    for phase in (["saturation", "poisson", "poisson_warm"] if not rate else ["poisson", "poisson_warm"]):
        reqs = S.make_requests(nreq, rate=None if phase == "saturation" else rate, seed=5000)
        if phase != "poisson_warm":
            if srv is not None:
                for e in list(srv.cache.values()):
                    srv._evict(e)
            srv = S.Server(fac.build, fac.estimate, fac.free_bytes, fac.rhs, new_x=fac.new_x)
        else:
            srv.stats.update(builds=0, build_s=0.0)
        torch.cuda.synchronize()
        clk = Clocks(torch.cuda.current_device()) if phase == "poisson" else None
        t0 = time.perf_counter()
        done = srv.run(reqs)
        torch.cuda.synchronize()
        span = time.perf_counter() - t0
        if clk:
            clocks = clk.stop()
        out[phase] = dict(S.summarize(done, span), **srv.stats)
        if phase == "saturation":
            rate = 0.8 * out[phase]["requests_per_s"]
    for e in list(srv.cache.values()):
        srv._evict(e)
    return out, rate, clocks


def serve_workload(nreq, rate, slots):
    return (f"serve{nreq}: Poisson arrivals at {rate:.2f}/s over 8 meshes (44..399 squared x 24 layers, "
            "z-jitter 0.3), eps in {1e-4,1e-3,1e-2,1e-1}, Neumann/Dirichlet-top 50/50, 1-8 RHS per request, "
            f"{slots}-slot engines, rtol 1e-8")


def run_serve(args):
    out, rate, clocks = serve_stream(args.serve, args.slots, args.precision, args.rate)
    p = out["poisson"]
    line = {"metric": "serving: solves/s at FP64 rel-res 1e-8, p50/p99 latency", "value": p["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": args.serve, "warmup": 0,
            "ms_per_step": 1000.0 * p["makespan_s"] / max(p["requests"], 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": serve_workload(args.serve, rate, args.slots), "precision": args.precision},
            "p50_latency_ms": p["p50_latency_ms"], "p99_latency_ms": p["p99_latency_ms"],
            "warm_p50_latency_ms": out["poisson_warm"]["p50_latency_ms"],
            "warm_p99_latency_ms": out["poisson_warm"]["p99_latency_ms"],
            "requests_per_s": p["requests_per_s"], "clocks": clocks, "serving": out}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------------
# the other configurations, measured in the default run beside the headline

def timed_solves(h, B, steps, warmup, V, torch, batched=False):
    """Device-timed solves (CUDA events, inputs resident) with the clocks sampled meanwhile."""
    X = torch.empty_like(B)
    infos = []

    def one():
        if batched:
            _, inf = V.vemg_solve_batch(h, B, X, rtol=RTOL, max_it=2000)
            return {"iters": max(i["iters"] for i in inf), "true_relres": max(i["true_relres"] for i in inf),
                    "status": "OK" if all(i["status"] == "OK" for i in inf) else "ENOTCONV"}
        _, inf = V.vemg_solve(h, B, X, rtol=RTOL, max_it=2000)
        return inf

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        infos.append(one())
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / steps
    return {"ms_per_step": ms, "iters": infos[-1]["iters"], "status": infos[-1]["status"],
            "true_relres_max": max(i["true_relres"] for i in infos), "clocks": clocks}


def unstructured_record(V, torch, I):
    """The 192x192x48 xy-jittered mesh at eps 1e-4: Neumann (surface chain with the near-nullspace
    {1, x, y}) and Dirichlet top, mixed-precision cycles against plain FP64 PCG on the same GPU."""
    m = I.make_workload_mesh("xyjit192")
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    b = torch.from_numpy(I.normal_loads(m.n, 2000)).cuda()
    rec = {"workload": f"xyjit192: 192x192x48 extruded hex->6 tets, {m.n} nodes, H0 1e-4, z-jitter 0.3, "
                       "xy-jitter 0.2 (redrawn inverted tets), N(0,1) loads, rtol 1e-8",
           "runs": []}
    for bc, bcn in ((V.VEMG_NEUMANN, "neumann"), (V.VEMG_DIRICHLET_TOP, "dirichlet_top")):
        for prec in ("bf16", "fp64"):
            h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=PRECS[prec], surf_nullspace=3))
            r = timed_solves(h, b, 3, 1, V, torch)
            r.update(bc=bcn, precision=prec, solves_per_s=1000.0 / r["ms_per_step"],
                     gdof_iter_per_s=m.n * r["iters"] / (r["ms_per_step"] / 1000.0) / 1e9)
            rec["runs"].append(r)
            h.destroy()
        rb, r64 = rec["runs"][-2], rec["runs"][-1]
        rb["speedup_over_plain_fp64_pcg"] = r64["ms_per_step"] / rb["ms_per_step"]
    A.free()
    rec["note"] = ("at eps 1e-4 the FP64 recursive residual reaches 1e-8 while the true residual stops at the "
                   "round-off floor (section 6.2: the floor grows as eps decreases); with BF16 precision the "
                   "{1, x, y} surface chain keeps FP32 values")
    return rec


def batched_record(V, torch, I):
    """The 384x384x24 mesh with 64 right-hand sides solved together, FP32 V-cycles in FP64 flexible CG
    against the FP64 batched PCG on the same GPU."""
    m = I.make_workload_mesh("zjit384x64")
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    k = I.WORKLOADS["zjit384x64"]["nrhs"]
    B = torch.from_numpy(I.normal_loads(m.n, 4000, k=k)).cuda()
    rec = {"workload": f"zjit384x64: 384x384x24 extruded hex->6 tets, {m.n} nodes, H0 1e-3, z-jitter 0.3, "
                       f"{k} N(0,1) right-hand sides mean-zero, rtol 1e-8 per column", "runs": []}
    for prec in ("fp32", "fp64"):
        h = V.vemg_setup(A, vm, V.vemg_default_options(precision=PRECS[prec]))
        r = timed_solves(h, B, 2, 1, V, torch, batched=True)
        r.update(precision=prec, rhs_per_s=k * 1000.0 / r["ms_per_step"],
                 gdof_iter_per_s=k * m.n * r["iters"] / (r["ms_per_step"] / 1000.0) / 1e9,
                 launch_shapes=V.vemg_batch_tuning(h))
        rec["runs"].append(r)
        h.destroy()
    rec["runs"][0]["speedup_over_fp64_batched"] = rec["runs"][1]["ms_per_step"] / rec["runs"][0]["ms_per_step"]
    A.free()
    return rec


def serving_record():
    out, rate, clocks = serve_stream(512, 8, "bf16")
    p = out["poisson"]
    return {"workload": serve_workload(512, rate, 8), "precision": "bf16 (FP64 V-cycles at eps <= 1e-4)",
            "solves_per_s": p["solves_per_s"], "requests_per_s": p["requests_per_s"],
            "p50_latency_ms": p["p50_latency_ms"], "p99_latency_ms": p["p99_latency_ms"],
            "warm_p50_latency_ms": out["poisson_warm"]["p50_latency_ms"],
            "warm_p99_latency_ms": out["poisson_warm"]["p99_latency_ms"],
            "columns_converged": p["columns_converged"], "columns_at_floor": p["columns_at_floor"],
            "columns_failed": p["columns_failed"], "clocks": clocks, "phases": out}


def case_phases(args, m, h, V, torch):
    """Per-phase profile of the persistent preconditioner kernel over one solve (after one warm-up
    solve): for each (group, level, kind) the phases and their summed critical-path time."""
    from paper_0912_1976_gb300 import inputs as I
    b = torch.from_numpy(I.normal_loads(m.n, 5)).cuda()
    V.vemg_solve(h, b, rtol=RTOL)
    kind = V.VEMG_PROBE_TAIL if (args.tail_cluster or 0) > 0 else V.VEMG_PROBE_VCYCLE
    V.vemg_probe(h, kind)
    _, info = V.vemg_solve(h, b, rtol=RTOL)
    r = V.vemg_probe_read(h)
    ph = V.vemg_probe_phases(h)
    V.vemg_probe(h, V.VEMG_PROBE_NONE)
    if not ph:
        print(json.dumps({"case": args.case, "phases": None, "note": "no persistent program (cycle is launches)"}))
        return 0
    mhz = float(os.environ.get("VEMG_SM_MHZ", "2070"))
    # one persistent launch per application, or one tail launch per chain per application
    napp = max(r["launches"] // (len({p["group"] for p in ph}) if kind == V.VEMG_PROBE_TAIL else 1), 1)
    agg = {}
    for p in ph:
        k = (p["group"], p["level"], p["op"])
        a = agg.setdefault(k, [0, 0.0])
        a[0] += 1
        a[1] += p["cycles"]
    rows = [{"group": g, "level": l, "op": op, "phases": c, "us_per_application": cyc / mhz / napp}
            for (g, l, op), (c, cyc) in agg.items()]
    print(json.dumps({"case": args.case, "precision": args.precision, "iters": info["iters"],
                      "applications": napp, "ms_per_application": r["ms"] / napp,
                      "algorithmic_gb_per_s": r["bytes"] / (r["ms"] / 1e3) / 1e9, "sm_mhz_assumed": mhz,
                      "rows": rows}))
    return 0


def resolved_cycle(cycle, prec):
    """The launch structure the library runs for a requested cycle (VEMG_CYCLE_AUTO: one kernel
    per phase; BF16 values always one kernel per phase)."""
    if prec == "bf16" or cycle == "auto":
        return "launches"
    return cycle


def surf_ns(args):
    if args.surf_nullspace is not None:
        return args.surf_nullspace
    from paper_0912_1976_gb300 import inputs as I
    return 3 if I.WORKLOADS.get(args.workload, {}).get("xy_jitter", 0.0) > 0.0 else 1


def tail_opt(args):
    o = {} if args.tail_rows is None else {"tail_rows": args.tail_rows}
    if args.tail_cluster is not None:
        o["tail_cluster"] = args.tail_cluster
    o["surf_nullspace"] = surf_ns(args)
    o["bc"] = 0 if args.bc == "neumann" else 1
    return o


def run_case(args):
    """A small case for ncu captures: build the mesh, set up, run two solves."""
    import torch
    from paper_0912_1976_gb300 import inputs as I
    from paper_0912_1976_gb300 import vemg as V
    nx, ny, nz = (int(v) for v in args.case.split("x"))
    m = I.make_mesh(nx, ny, nz, I.depth_sines(1e-3), z_jitter=0.3, seed=77)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    prec = PRECS[args.precision]
    h = V.vemg_setup(A, vm, V.vemg_default_options(precision=prec, precond=PRECONDS[args.precond],
                                                   cycle=CYCLES[args.cycle], **tail_opt(args)))
    if args.phases:
        return case_phases(args, m, h, V, torch)
    kr = max(args.rhs, 1)
    if args.stream_path:
        # the same kernels launched on the stream instead of from graphs (profilers cannot see
        # into graphs with conditional nodes)
        V.vemg_probe(h, V.VEMG_PROBE_VCYCLE)
    # the second solve runs inside the NVTX range "solve" (ncu --nvtx --nvtx-include "solve/")
    if kr == 1:
        b = torch.from_numpy(I.normal_loads(m.n, 5)).cuda()
        for j in range(2):
            if j == 1:
                torch.cuda.nvtx.range_push("solve")
            _, info = V.vemg_solve(h, b, rtol=RTOL)
        torch.cuda.nvtx.range_pop()
    else:
        B = torch.from_numpy(I.normal_loads(m.n, 5, k=kr)).cuda()
        for j in range(2):
            if j == 1:
                torch.cuda.nvtx.range_push("solve")
            _, infos = V.vemg_solve_batch(h, B, rtol=RTOL)
        torch.cuda.nvtx.range_pop()
        info = infos[0]
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": m.n, "precision": args.precision, "rhs": kr, "info": info}))
    return 0


def run_spectrum(args):
    """Section 4 study: Lanczos estimates (from the CG coefficients of each solve) of the extreme
    eigenvalues and the condition number of A and of M^-1 A for the three preconditioners, over
    eps, on a layered (z-jittered) and a vertically unstructured (xy-jittered) mesh."""
    import torch
    from paper_0912_1976_gb300 import inputs as I
    from paper_0912_1976_gb300 import vemg as V
    nx, nz = 64, 16
    kinds = {"layered": dict(z_jitter=0.3, xy_jitter=0.0), "unstructured": dict(z_jitter=0.3, xy_jitter=0.2)}
    pcs = {"none": V.VEMG_PRECOND_NONE, "additive": V.VEMG_PRECOND_ADDITIVE, "vl_sor": V.VEMG_PRECOND_VL_SOR,
           "sa": V.VEMG_PRECOND_SA}
    rows = []
    for kind, jit in kinds.items():
        for eps in (1e-1, 1e-2, 1e-3, 1e-4):
            m = I.make_mesh(nx, nx, nz, I.depth_sines(eps), seed=7, **jit)
            vm = V.Mesh.from_inputs(m)
            A = V.vemg_assemble(vm)
            b = torch.from_numpy(I.normal_loads(m.n, 11)).cuda()
            for name, pc in pcs.items():
                h = V.vemg_setup(A, vm, V.vemg_default_options(precond=pc, precision=V.VEMG_PREC_FP64))
                t0 = time.perf_counter()
                _, info = V.vemg_solve(h, b, rtol=1e-8, max_it=4096)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                a, bt = V.vemg_solve_coefficients(h)
                lo, hi = V.vemg_lanczos_extremes(a, bt)
                rows.append({"mesh": kind, "eps": eps, "preconditioner": name, "iters": info["iters"],
                             "status": info["status"], "lambda_min": lo, "lambda_max": hi, "cond": hi / lo,
                             "cond_is_lower_bound": info["status"] != "OK", "solve_s": dt})
                h.destroy()
            A.free()
    print(json.dumps({"study": "spectrum (section 4): Lanczos condition estimates from CG coefficients",
                      "mesh": f"{nx}x{nx}x{nz} extruded hex->6 tets, H = eps (1 + 0.5 sin sin), seed 7",
                      "rtol": 1e-8, "max_it": 4096, "rows": rows}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.spectrum:
        return run_spectrum(args)
    if args.serve:
        return run_serve(args)
    import torch
    from paper_0912_1976_gb300 import inputs as I
    from paper_0912_1976_gb300 import vemg as V

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    mesh = I.make_workload_mesh(args.workload)
    n = mesh.n
    vm = V.Mesh.from_inputs(mesh)
    kr = args.rhs or I.WORKLOADS[args.workload].get("nrhs", 1)
    nb = min(args.steps + args.warmup, 8 if kr == 1 else 2)
    if kr == 1:
        B = [torch.from_numpy(I.normal_loads(n, 2000 + 97 * rank + j)).cuda() for j in range(nb)]
    else:
        B = [torch.from_numpy(I.normal_loads(n, 4000 + 997 * rank + 131 * j, k=kr)).cuda() for j in range(nb)]

    res = {}
    order = [args.precision] + [p for p in ("fp32", "fp64") if p != args.precision]   # comparators
    for prec in order:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A = V.vemg_assemble(vm)
        h = V.vemg_setup(A, vm, V.vemg_default_options(
            precision=PRECS[prec], precond=PRECONDS[args.precond],
            cycle=CYCLES[args.cycle], **tail_opt(args)))
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        cyc = resolved_cycle(args.cycle, prec)
        r = measure(args, h, B, n, ws, rank, local, dist, V, torch, probe=not args.no_probe, cycle=cyc)
        r["cycle"] = cyc
        r["setup_s"] = setup_s
        r["hierarchy_bytes"] = V.vemg_hierarchy_bytes(h)
        res[prec] = r
        h.destroy()
        A.free()
        del h, A

    head = res[args.precision]
    hbm, peak_kind = peaks()
    roofline = None
    classes = head["classes"]
    if classes:
        # the dominant class: the largest share of the probed (event-timed, serialised) device time
        dom = max(classes, key=lambda c: classes[c]["ms_per_solve"])
        for c in classes.values():
            c["frac"] = c["achieved_gbs"] / hbm
        c = classes[dom]
        # DRAM traffic per launch of the finest-level colour sweep, from one ncu capture on a
        # 192x192x32 mesh (colour 2, 261,577 rows): 1.07 (FP32 values) / 1.09 (BF16 values) x its
        # algorithmic bytes, scaled here by this workload's bytes per launch
        traffic = None
        if dom == "sor_coarse" and args.precision == "bf16":
            # three captured coarse launches on a 192x192x32 mesh moved 0.606-0.623 MB from DRAM each
            # (L2 hit rate 33-36%); the class mixes launches of every coarse level, so the figure is
            # the captured launches' own, not scaled to this workload's average launch
            traffic = {"bytes_per_launch": 0.6167e6,
                       "source": "ncu dram__bytes (read + write), mean of 3 k_sell_sor<__nv_bfloat16, float, float> "
                                 "launches on a 192x192x32 mesh (profiles/sor_coarse_bf16_zjit192.md); not scaled"}
        if dom == "sor_fine" and args.precision in SOR_FINE_DRAM_RATIO:
            traffic = {"bytes_per_launch": SOR_FINE_DRAM_RATIO[args.precision] * c["bytes_per_launch"],
                       "source": f"ncu dram__bytes (read + write) of one {SOR_FINE_KERNEL[args.precision]} launch "
                                 "on a 192x192x32 mesh, scaled by algorithmic bytes per launch"}
        # the whole solve: every class's algorithmic bytes over the un-probed time of a solve
        solve_bytes = sum(x["bytes_per_solve"] for x in classes.values())
        whole = solve_bytes / (head["ms_per_step"] / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": c["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": c["achieved_gbs"] / hbm, "peak_source": f"{peak_kind} hbm_gbs (copy, burst)",
                    "traffic": traffic,
                    "share_of_probed_time": c["ms_per_solve"] / sum(x["ms_per_solve"] for x in classes.values()),
                    "whole_solve": {"algorithmic_bytes_per_solve": solve_bytes, "achieved_gbs": whole,
                                    "frac": whole / hbm},
                    "classes": classes}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        bh = (B[0][0] if B[0].dim() == 2 else B[0]).cpu().numpy()
        r = time_oracle(mesh, bh)
        cpu = {"value": 1.0 / r["solve_s"], "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"one full oracle solve of the {args.workload} workload ({r['iters']} iterations, "
                         f"{r['solve_s']:.1f} s; oracle setup {r['setup_s']:.1f} s not counted)"}
        del r
        ro = time_oracle(mesh, bh, openmp=True)
        cpu["openmp"] = {"value": 1.0 / ro["solve_s"], "unit": "solves/s", "cores": ro["threads"],
                         "nproc": os.cpu_count(), "kind": "oracle (OpenMP timing build, the same bits)",
                         "sample": f"one full solve ({ro['iters']} iterations, {ro['solve_s']:.2f} s)"}
        del ro

    extra = {}
    if ws == 1 and not args.headline_only and args.workload == WORKLOAD and not args.rhs:
        torch.cuda.empty_cache()
        extra["unstructured"] = unstructured_record(V, torch, I)
        torch.cuda.empty_cache()
        extra["batched"] = batched_record(V, torch, I)
        torch.cuda.empty_cache()
        extra["serving"] = serving_record()

    if rank == 0:
        other = [p for p in res if p != args.precision]
        comparator = None
        if "fp64" in res and args.precision != "fp64":
            f = res["fp64"]
            comparator = {"name": "plain FP64 PCG (same hierarchy, FP64 V-cycles)", "value": f["value"],
                          "iters": f["iters"][0], "ms_per_step": f["ms_per_step"],
                          "e2e": f["e2e"]["value"], "true_relres_max": f["true_relres_max"],
                          "cycle": f["cycle"], "speedup_of_value": head["value"] / f["value"]}
        fp32_line = None
        if "fp32" in res and args.precision == "bf16":
            f = res["fp32"]
            fp32_line = {"name": "FP64 FCG with FP32 V-cycles and FP32 operator values", "value": f["value"],
                         "iters": f["iters"][0], "ms_per_step": f["ms_per_step"], "e2e": f["e2e"]["value"],
                         "true_relres_max": f["true_relres_max"]}
        line = {"metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES[args.precision],
                "data": "synthetic", "config": workload_config(args, n),
                "gdof_iter_per_s": head["gdof_iter_per_s"], "iters": head["iters"],
                "true_relres_max": head["true_relres_max"], "setup_s": head["setup_s"],
                "hierarchy_bytes": head["hierarchy_bytes"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
                "roofline": roofline, "cpu_baseline": cpu, "clocks": head["clocks"],
                "plain_fp64_pcg": comparator, "fp32_values": fp32_line}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
