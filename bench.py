"""Benchmark: FP64 SIPG-DG operator application throughput (GDOF/s) on the
64^3 Q3 lognormal-K workload, plus CG time to a 1e-10 residual, mixed precision
vs FP64, on 48^3 Q4.

One step = one FP64 dg_apply (both passes) of the 64^3 Q3 operator over one
synthetic input vector held in HBM.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-cg]

Under torchrun (N > 1) every rank applies its own replica of the operator
(no data-path collective); `value` is the total DOFs of all ranks per second.
`--impl reference` times the FP64 CPU oracle (element-wise, full 3D quadrature)
on a bounded sample of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"n_cells": 64, "degree": 3, "K": "lognormal", "K_seed": 2, "x_seed": 3}
CG_WORKLOAD = {"n_cells": 48, "degree": 4, "K": "lognormal", "K_seed": 4, "rtol": 1e-10}
# 256 lognormal samples on three uneven levels (multilevel Monte-Carlo shape)
BATCH_LEVELS = [(128, 16, 2), (96, 24, 3), (32, 32, 4)]   # (samples, n_cells, degree)
METRIC = "SIPG-DG apply GDOF/s (FP64)"
NOMINAL_FP64_TFLOPS = 1.25   # GB300 FP64 rate: 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz
# DRAM bytes (read + write) per DOF of one pass-2 launch (k_cell_lo<4,double>),
# from an ncu capture of the 40^3 Q3 case (462.9 MB read + 27.4 MB written for
# 4,096,000 DOFs), scaled by DOFs to the benchmark's launch; set to None when
# the kernel changes until it is captured again.
K_CELL_TRAFFIC_PER_DOF = (462.859264e6 + 27.433984e6) / 4096000


def flops_per_dof(n: int):
    """Algorithmic FLOPs per DOF per apply (FMA = 2), split by pass:
    pass 1: modal->nodal 6n + face traces (value and derivative) 24;
    pass 2: gradient and transpose 12n, nodal->modal 6n, pointwise 3,
            face test functions 24, face pointwise 36/n."""
    p1 = 6 * n + 24
    p2 = 18 * n + 3 + 24 + 36.0 / n
    return p1, p2


def bytes_per_dof_fp64(n: int):
    """Algorithmic bytes per DOF per apply: read x, read h w K, write y (8 B each)
    plus three face coefficients per cell."""
    return 24.0 + 24.0 / n ** 3


# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out)) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x.strip())
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
def run_cpu_baseline(K, x, N, k, target_s: float = 10.0):
    """Time the oracle's element-wise apply (the whole mesh, repeated until
    target_s seconds of CPU work have been timed)."""
    from oracle import SIPG
    D = SIPG(N, k)
    n3 = (k + 1) ** 3
    D.apply(K, x, cells=list(range(64)))                 # warm up BLAS
    reps, t0 = 0, time.perf_counter()
    while True:
        D.apply(K, x)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return {"value": reps * N ** 3 * n3 / dt / 1e9, "unit": "GDOF/s", "cores": cpu_threads(),
            "kind": "oracle",
            "sample": f"element-wise FP64 apply (full 3D quadrature tables) of the whole {N}^3 "
                      f"Q{k} mesh ({N ** 3 * n3} DOFs), {reps} times in {dt:.1f} s"}


def cpu_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        info = [d.get("num_threads") for d in threadpool_info() if d.get("num_threads")]
        if info:
            return int(max(info))
    except Exception:
        pass
    return len(os.sched_getaffinity(0))


def make_inputs(N, k, kseed, xseed):
    from paper_1911_01492_gb300 import inputs
    K = inputs.lognormal_coefficient(N, k, seed=kseed)
    x = inputs.uniform_vector(N, k, xseed)
    return K, x


def run_reference(args, world, rank):
    if rank != 0:
        return
    N, k = WORKLOAD["n_cells"], WORKLOAD["degree"]
    import numpy as np
    from oracle import SIPG
    K, x = make_inputs(N, k, WORKLOAD["K_seed"], WORKLOAD["x_seed"])
    D = SIPG(N, k)
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(1)
    ncell = min(N ** 3, 16384)   # one step: the oracle apply on 16384 cells of the mesh
    for _ in range(args.warmup):
        D.apply(K, x, cells=rng.choice(N ** 3, ncell, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        D.apply(K, x, cells=rng.choice(N ** 3, ncell, replace=False))
    dt = time.perf_counter() - t0
    value = args.steps * ncell * n3 / dt / 1e9
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{N}^3 Q{k} SIPG-DG apply, lognormal K (GRF corr. 0.1, "
                                   "var 1, seed 2), x~U[-1,1] (seed 3)",
                       "step": f"oracle apply on {ncell} random cells of the mesh"},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                             "sample": f"{ncell} random cells ({ncell * n3} DOFs) per step"},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def time_applies(m, x, y, steps, warmup, world):
    import torch
    for _ in range(warmup):
        m.apply(x, y)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    m.timing_enable(steps)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        m.apply(x, y)
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    napp, ms1, ms2 = m.timing_read()
    return ms, napp, ms1, ms2


def time_e2e(m, xh, yh, steps, warmup, world):
    import torch
    for _ in range(warmup):
        m.apply_host(xh, yh)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        m.apply_host(xh, yh)      # H2D x, apply, D2H y, synchronise
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    barrier(world)
    return dt


def run_cg(world):
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = CG_WORKLOAD["n_cells"], CG_WORKLOAD["degree"]
    K = inputs.lognormal_coefficient(N, k, seed=CG_WORKLOAD["K_seed"])
    m = dg.Mesh(N, k)
    Kd = torch.from_numpy(K).cuda()
    m.set_coefficient(Kd)
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    out = {"workload": f"{N}^3 Q{k} SIPG-DG, lognormal K (seed 4), f = 1, "
                       f"{m.n_dofs} DOFs, to rel. residual {CG_WORKLOAD['rtol']:g} "
                       "recomputed in FP64; Jacobi times include forming diag(A)"}
    for name, mode in (("mixed_ir", dg.DG_CG_MIXED_IR), ("fp64", dg.DG_CG_FP64),
                       ("mixed_ir_jacobi", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_JACOBI),
                       ("fp64_jacobi", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_JACOBI)):
        if mode & dg.DG_CG_PRECOND_JACOBI:
            m.set_coefficient(Kd)  # drops the cached diagonal: the solve forms it
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        barrier(world)
        _, st = m.cg_solve(b, x, rtol=CG_WORKLOAD["rtol"], maxit=200000, mode=mode,
                           raise_on_error=False)
        out[name] = {"seconds": max_over_ranks(st["seconds"], world),
                     "iterations": st["iterations"], "outer": st["outer_iterations"],
                     "rel_residual": st["rel_residual"], "status": st["status"]}
    if out["fp64"]["status"] == 0 and out["mixed_ir"]["status"] == 0:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed_ir"]["seconds"]
    if out["fp64_jacobi"]["status"] == 0 and out["mixed_ir_jacobi"]["status"] == 0:
        out["speedup_mixed_vs_fp64_jacobi"] = (out["fp64_jacobi"]["seconds"]
                                               / out["mixed_ir_jacobi"]["seconds"])
    m.close()
    return out


def _batch_meshes(levels, seed0=1000):
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    meshes, bs, xs, sizes = [], [], [], []
    s = 0
    for count, N, k in levels:
        for _ in range(count):
            m = dg.Mesh(N, k)
            m.set_coefficient(torch.from_numpy(
                inputs.lognormal_coefficient(N, k, seed=seed0 + s)).cuda())
            meshes.append(m)
            bs.append(torch.from_numpy(inputs.constant_load_vector(N, k)).cuda())
            xs.append(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
            sizes.append(m.n_dofs)
            s += 1
    return meshes, bs, xs, sizes


def _timed_batched(meshes, bs, xs, sizes, world, precond=None):
    import torch
    import paper_1911_01492_gb300 as dg
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-8, maxit=200000, raise_on_error=False,
                                precond=precond)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    work = sum(st["iterations"] * n for st, n in zip(stats, sizes))
    return {"samples": len(meshes), "seconds": dt, "gdof_per_s": world * work / dt / 1e9,
            "all_converged": all(st["status"] == 0 for st in stats),
            "max_rel_residual": max(st["rel_residual"] for st in stats),
            "iterations_min_max": [min(st["iterations"] for st in stats),
                                   max(st["iterations"] for st in stats)]}


def _timed_sequential(meshes, bs, sizes, picked):
    import torch
    t, work = 0.0, 0
    for i in picked:
        x = torch.zeros_like(bs[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = meshes[i].cg_solve(bs[i], x, rtol=1e-8, maxit=200000)
        torch.cuda.synchronize()
        t += time.perf_counter() - t0
        work += st["iterations"] * sizes[i]
    return {"samples": len(picked), "seconds": t, "gdof_per_s": work / t / 1e9}


def run_batched(world, rank, sequential_samples: int = 1, full: bool = False):
    """Batched lock-step CG (FP64, rtol 1e-8) on the 256-sample workload.

    Always: the 128 small samples (16^3 Q2) in one batched solve against 16 of
    them solved one per dg_cg_solve call, and one-per-call rates of the larger
    levels, and the small batch again with M = diag(A_s).  With full = True
    also the whole 256-sample batch, without and with M (minutes).
    """
    out = {"workload": "256 lognormal-K samples: 128 x 16^3 Q2, 96 x 24^3 Q3, 32 x 32^3 Q4 "
                       "(230,162,432 DOFs), FP64 CG to 1e-8; seeds 1000 + sample"}
    small = [BATCH_LEVELS[0]]
    meshes, bs, xs, sizes = _batch_meshes(small)
    out["small_level_batched"] = _timed_batched(meshes, bs, xs, sizes, world)
    out["small_level_one_per_call"] = _timed_sequential(
        meshes, bs, sizes, list(range(min(len(meshes), 16))))
    out["small_level_speedup"] = (out["small_level_batched"]["gdof_per_s"]
                                  / out["small_level_one_per_call"]["gdof_per_s"])
    # the same batch with M = diag(A_s); its time includes forming the diagonals
    out["small_level_batched_jacobi"] = _timed_batched(meshes, bs, xs, sizes, world,
                                                       precond="jacobi")
    for m in meshes:
        m.close()
    rates = {}
    start = 0
    for count, N, k in BATCH_LEVELS[1:]:
        ms_, bs_, xs_, sz_ = _batch_meshes([(min(count, sequential_samples), N, k)],
                                           seed0=1000 + BATCH_LEVELS[0][0] + start)
        rates[f"{N}^3 Q{k}"] = _timed_sequential(ms_, bs_, sz_, list(range(len(ms_))))
        start += count
        for m in ms_:
            m.close()
    out["one_per_call_larger_levels"] = rates
    if full:
        meshes, bs, xs, sizes = _batch_meshes(BATCH_LEVELS)
        out["full_batch"] = _timed_batched(meshes, bs, xs, sizes, world)
        out["full_batch_jacobi"] = _timed_batched(meshes, bs, xs, sizes, world,
                                                  precond="jacobi")
        for m in meshes:
            m.close()
    return out


def run_cg_probe(iters: int):
    """A fixed number of iterations of the mixed and FP64 CG on the CG
    workload (48^3 Q4), with wall times; for kernel launch lists."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = CG_WORKLOAD["n_cells"], CG_WORKLOAD["degree"]
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=CG_WORKLOAD["K_seed"])).cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    for name, mode in (("mixed_ir", dg.DG_CG_MIXED_IR), ("fp64", dg.DG_CG_FP64),
                       ("mixed_ir_jacobi", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_JACOBI),
                       ("fp64_jacobi", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_JACOBI)):
        x = torch.zeros_like(b)
        _, st = m.cg_solve(b, x, rtol=1e-12, maxit=iters, mode=mode, raise_on_error=False)
        print(json.dumps({"mode": name, "iterations": st["iterations"],
                          "ms_per_iteration": 1e3 * st["seconds"] / max(st["iterations"], 1)}),
              flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-solution part")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--batched", action="store_true",
                    help="also run the 256-sample batched CG workload")
    ap.add_argument("--batched-sequential", type=int, default=1,
                    help="samples of each larger level solved one per call for reference")
    ap.add_argument("--cg-probe", type=int, default=0, metavar="ITERS",
                    help="only run ITERS iterations of each CG mode on the CG workload "
                         "(for kernel profiles) and exit")
    ap.add_argument("--batched-full", action="store_true",
                    help="with --batched: also solve the whole 256-sample batch (minutes)")
    ap.add_argument("--n-cells", type=int, default=WORKLOAD["n_cells"],
                    help="cells per direction (default: the 64^3 workload)")
    ap.add_argument("--degree", type=int, default=WORKLOAD["degree"])
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)

    WORKLOAD["n_cells"], WORKLOAD["degree"] = args.n_cells, args.degree
    world, rank, local = dist_setup()
    if args.cg_probe:
        run_cg_probe(args.cg_probe)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_1911_01492_gb300 as dg
    N, k = WORKLOAD["n_cells"], WORKLOAD["degree"]
    n = k + 1
    K, x = make_inputs(N, k, WORKLOAD["K_seed"], WORKLOAD["x_seed"])
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    nd = m.n_dofs

    with ClockSampler(torch.cuda.current_device() if world == 1 else local) as clk:
        ms, napp, ms1, ms2 = time_applies(m, xd, yd, args.steps, args.warmup, world)
    ms = max_over_ranks(ms, world)
    ms_step = ms / args.steps
    value = world * nd / (ms_step * 1e-3) / 1e9

    # roofline of the dominant kernel (pass 2, the cell kernel): FP64 pipe
    f1, f2 = flops_per_dof(n)
    t1, t2 = ms1 / max(napp, 1), ms2 / max(napp, 1)
    dom_ms, dom_flops, dom_name = ((t2, f2 * nd, "k_cell_lo") if t2 >= t1
                                   else (t1, f1 * nd, "k_trace"))
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12
    traffic = (K_CELL_TRAFFIC_PER_DOF * nd
               if (dom_name == "k_cell_lo" and n == 4 and K_CELL_TRAFFIC_PER_DOF) else None)
    roofline = {"bound": "alu", "kernel": dom_name, "achieved": achieved,
                "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / NOMINAL_FP64_TFLOPS, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                  "pass-2 kernel on 40^3 Q3, scaled by DOFs",
                "peak_source": "nominal GB300 FP64 rate (derived: 152 SMs x 2 DFMA/clk x 2 x "
                               "2.06 GHz); a DFMA throughput probe measured 1.0 TFLOP/s",
                "pass_ms": {"k_trace": t1, "k_cell_lo": t2},
                "apply_tflops_algorithmic": (f1 + f2) * nd / (ms_step * 1e-3) / 1e12}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        e2e_steps = max(3, min(args.steps, 20))
        dt = time_e2e(m, xh, yh, e2e_steps, 2, world)
        dt = max_over_ranks(dt, world)
        e2e = {"value": world * nd * e2e_steps / dt / 1e9, "unit": "GDOF/s",
               "h2d_bytes_per_step": xh.numel() * 8, "d2h_bytes_per_step": yh.numel() * 8}

    cg = None
    if not args.no_cg:
        m.close()
        del xd, yd
        torch.cuda.empty_cache()
        cg = run_cg(world)

    batched = None
    if args.batched:
        torch.cuda.empty_cache()
        batched = run_batched(world, rank, args.batched_sequential, args.batched_full)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(K, x, N, k)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{N}^3 Q{k} SIPG-DG apply, lognormal K (GRF corr. 0.1, "
                                       "var 1, seed 2), x~U[-1,1] (seed 3)",
                           "dofs_per_gpu": nd, "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (x, h w K and y are 134 MB each)"},
                "roofline": roofline, "e2e": e2e, "gpu_launches": 2 * args.steps,
                "clocks": clk.summary(), "cpu_baseline": cpu, "cg": cg}
        if batched is not None:
            line["batched_cg"] = batched
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
