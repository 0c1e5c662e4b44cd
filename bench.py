"""Benchmark of the matrix-free SIPG-DG hot path on one GB300.

Headline (`value`): FP64 dg_apply throughput in GDOF/s on the 64^3 Q3
lognormal-K workload (16.8 M DOFs).  One step = one sweep of
APPLIES_PER_STEP FP64 applies of that operator over one synthetic input vector
held in HBM (inputs, workspaces and output each larger than L2).  The second
half of the metric, CG time to a 1e-10 residual with mixed precision against
FP64, is the `cg` object (48^3 Q4).  The other workloads of the method are
separate keys of the same line: `config1` (8^3 Q2, K = 1: one apply in us and
a manufactured-solution CG), `config2_cg` (the unpreconditioned FP64 CG on the
64^3 Q3 operator), `config4` (32^3 Q3: apply, adjoint, coefficient gradient,
differentiable apply and adjoint-CG gradient), `batched_cg` (the small level
of the 256-sample batch, one batched solve against one solve per call), `mlmc`
(one multilevel Monte-Carlo Estimate step for the mean inlet flux of the
Section 5 flow problem over the three batched levels), `affine` (the apply
and a CG on a sheared mesh, the paper's problem B), and
`oracle_legs` (the FP64 CPU oracle: one thread and all threads, CSR SpMV and
CG where the matrix fits, projected CG elsewhere).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-cg] [--no-extra] [--no-e2e] [--no-cpu-baseline]

Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank applies its
own replica of the operator (no data-path collective); `value` is the total
DOFs of all ranks per second.  `--impl reference` times the FP64 CPU oracle
(element-wise, full 3D quadrature) on a bounded sample of the same workload on
this host's cores.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"n_cells": 64, "degree": 3, "K": "lognormal", "K_seed": 2, "x_seed": 3}
APPLIES_PER_STEP = 32
CG_WORKLOAD = {"n_cells": 48, "degree": 4, "K": "lognormal", "K_seed": 4, "rtol": 1e-10}
CONFIG1 = {"n_cells": 8, "degree": 2, "x_seed": 1, "rtol": 1e-10}
CONFIG4 = {"n_cells": 32, "degree": 3, "K_seed": 5, "x_seed": 6, "K_ref_seed": 40,
           "noise_seed": 41, "rtol": 1e-10}
# 256 lognormal samples on three uneven levels (multilevel Monte-Carlo shape)
BATCH_LEVELS = [(128, 16, 2), (96, 24, 3), (32, 32, 4)]   # (samples, n_cells, degree)
METRIC = "SIPG-DG apply GDOF/s (FP64)"
NOMINAL_FP64_TFLOPS = 1.25   # GB300 FP64 rate: 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz
# Executed FP64 operations of the apply kernels at Q3 (DFMA counted 2, DADD and
# DMUL 1), from ncu's sm__sass_thread_inst_executed_op_{dfma,dadd,dmul} counters
# on 32^3 and 40^3 launches, which fit (per cell, per interior face side)
# exactly (profiles/apply_fp64_q3_executed_flops.md).  Set an entry to None
# when its kernel changes until it is counted again.
EXEC_FP64_Q3 = {"k_trace": (1792.0, 0.0), "k_cell_lo": (3440.0, 64.0),
                "k_trace_nd": (1344.0, 0.0), "k_cell_nd": (3008.0, 64.0)}
# The same counters as FP64 instructions (DFMA, DADD and DMUL one each: every
# one takes an issue slot of the FP64 pipe, whatever its flops), per cell and
# per interior face side, exact at both sizes
EXEC_FP64_INSTR_Q3 = {"k_trace": (1136.0, 0.0), "k_cell_lo": (1984.0, 48.0),
                      "k_trace_nd": (768.0, 0.0), "k_cell_nd": (1536.0, 48.0)}


def executed_fp64_per_dof(kernel: str, N: int, n: int, table=None):
    """Executed FP64 operations (or, with table=EXEC_FP64_INSTR_Q3, FP64
    instructions) per DOF of one launch on an N^3 mesh (Q3 only)."""
    e = (table or EXEC_FP64_Q3).get(kernel) if n == 4 else None
    if e is None:
        return None
    per_cell, per_face_side = e
    face_sides = 6 * N * N * (N - 1)       # interior faces, seen from both cells
    return (per_cell * N ** 3 + per_face_side * face_sides) / (N ** 3 * n ** 3)


# DRAM bytes (read + write) per DOF of one pass-2 launch (k_cell_lo<4,double>),
# from an ncu capture of the 40^3 Q3 case (462.4 MB read + 27.6 MB written for
# 4,096,000 DOFs), scaled by DOFs to the benchmark's launch; set to None when
# the kernel changes until it is captured again.
K_CELL_TRAFFIC_PER_DOF = (462.4e6 + 27.6e6) / 4096000


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
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_applies(m, x, y, steps, warmup, world, per_step=APPLIES_PER_STEP, nodal=False):
    """`steps` timed sweeps of `per_step` FP64 applies after `warmup` untimed
    sweeps; CUDA events on the launching stream, per-pass events inside the
    library (dg_timing_enable) for the roofline.  nodal: the operator in the
    scaled Gauss-point basis (dg_apply_nodal) instead of dg_apply."""
    import torch
    op = m.apply_nodal if nodal else m.apply
    for _ in range(warmup):
        for _ in range(per_step):
            op(x, y)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    m.timing_enable(steps * per_step)
    s = torch.cuda.current_stream()
    e0, e1 = _events()
    e0.record(s)
    for _ in range(steps):
        for _ in range(per_step):
            op(x, y)
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    napp, ms1, ms2 = m.timing_read()
    return ms, napp, ms1, ms2


def time_e2e(m, xh, yh, steps, warmup, world, per_step=APPLIES_PER_STEP):
    """The same sweeps through the host-buffer entry point: every apply copies
    x in from pinned host memory and y back out, inside the timed region."""
    import torch
    for _ in range(warmup):
        m.apply_host(xh, yh)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        for _ in range(per_step):
            m.apply_host(xh, yh)      # H2D x, apply, D2H y, synchronise
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    barrier(world)
    return dt


def time_setup(m, Kd, reps=3):
    """Wall time of dg_set_coefficient (coefficient kernels, line operators,
    face weights and its blocking validity check), best of reps."""
    import torch
    best = 1e300
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.set_coefficient(Kd)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best * 1e3


def time_gpu_calls(fn, reps, warmup=3):
    """Mean ms of fn() over reps calls (CUDA events on the current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = _events()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _solve_entry(st, world):
    return {"seconds": max_over_ranks(st["seconds"], world), "iterations": st["iterations"],
            "outer": st["outer_iterations"], "rel_residual": st["rel_residual"],
            "status": st["status"]}


def run_cg(world, modes=None):
    """Config 3: 48^3 Q4 lognormal K, f = 1; FP64 CG against the mixed CG to
    a 1e-10 FP64-recomputed residual, without preconditioner, with M = diag(A)
    and with the Kronecker cell blocks (setup included in the time)."""
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
    modes = modes or (("mixed_ir", dg.DG_CG_MIXED_IR), ("fp64", dg.DG_CG_FP64),
                      ("mixed_ir_jacobi", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_JACOBI),
                      ("fp64_jacobi", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_JACOBI),
                      ("mixed_ir_restart_jacobi",
                       dg.DG_CG_MIXED_IR_RESTART | dg.DG_CG_PRECOND_JACOBI),
                      ("mixed_ir_kron", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_KRON),
                      ("fp64_kron", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_KRON),
                      ("fp64_nodal", dg.DG_CG_FP64 | dg.DG_CG_NODAL),
                      ("mixed_ir_nodal", dg.DG_CG_MIXED_IR | dg.DG_CG_NODAL),
                      ("fp64_nodal_kron",
                       dg.DG_CG_FP64 | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_KRON),
                      ("mixed_ir_nodal_kron",
                       dg.DG_CG_MIXED_IR | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_KRON))
    for name, mode in modes:
        if mode & (dg.DG_CG_PRECOND_JACOBI | dg.DG_CG_PRECOND_KRON | dg.DG_CG_NODAL):
            # drops the cached preconditioner and basis data: the solve forms them
            m.set_coefficient(Kd)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        barrier(world)
        _, st = m.cg_solve(b, x, rtol=CG_WORKLOAD["rtol"], maxit=200000, mode=mode,
                           raise_on_error=False)
        out[name] = _solve_entry(st, world)
    if out["fp64"]["status"] == 0 and out["mixed_ir"]["status"] == 0:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed_ir"]["seconds"]
    if out["fp64_jacobi"]["status"] == 0 and out["mixed_ir_jacobi"]["status"] == 0:
        out["speedup_mixed_vs_fp64_jacobi"] = (out["fp64_jacobi"]["seconds"]
                                               / out["mixed_ir_jacobi"]["seconds"])
    if out.get("fp64_nodal", {}).get("status") == 0 and out["fp64"]["status"] == 0:
        out["speedup_fp64_nodal_vs_fp64"] = out["fp64"]["seconds"] / out["fp64_nodal"]["seconds"]
    if "mixed_ir_kron" in out and out["mixed_ir_kron"]["status"] == 0:
        out["speedup_mixed_kron_vs_fp64_jacobi"] = (out["fp64_jacobi"]["seconds"]
                                                    / out["mixed_ir_kron"]["seconds"])
    m.close()
    return out, K


def run_config2_cg(m, world):
    """Config 2's solve: the unpreconditioned FP64 CG (and the mixed CG) on the
    64^3 Q3 lognormal operator, f = 1, to 1e-10."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = m.n_cells, m.degree
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    out = {"workload": f"{N}^3 Q{k} SIPG-DG, lognormal K (seed 2), f = 1, {m.n_dofs} DOFs, "
                       "to rel. residual 1e-10 recomputed in FP64, M = I"}
    for name, mode in (("fp64", dg.DG_CG_FP64), ("mixed_ir", dg.DG_CG_MIXED_IR)):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        barrier(world)
        _, st = m.cg_solve(b, x, rtol=1e-10, maxit=200000, mode=mode, raise_on_error=False)
        out[name] = _solve_entry(st, world)
    if out["fp64"]["status"] == 0 and out["mixed_ir"]["status"] == 0:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed_ir"]["seconds"]
    return out


def manufactured_source(x, y, z):
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) for u = sin(pi x) sin(pi y) sin(pi z), K = 1."""
    return 3.0 * math.pi ** 2 * (np.sin(math.pi * x) * np.sin(math.pi * y)
                                 * np.sin(math.pi * z))


def run_config1(world):
    """Config 1: 8^3 Q2, K = 1.  One FP64 apply in microseconds (mean over
    many launches), and the FP64 and mixed CG to 1e-10 for the manufactured
    right-hand side (formed by dg_load_vector from f at the Gauss points)."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = CONFIG1["n_cells"], CONFIG1["degree"]
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.unit_coefficient(N, k)).cuda())
    x = torch.from_numpy(inputs.uniform_vector(N, k, CONFIG1["x_seed"])).cuda()
    y = torch.empty_like(x)
    us = 1e3 * time_gpu_calls(lambda: m.apply(x, y), 2000, warmup=20)
    f = torch.from_numpy(inputs.values_at_gauss_points(N, k, manufactured_source)).cuda()
    b = m.load_vector(f)
    out = {"workload": f"{N}^3 Q{k}, K = 1, {m.n_dofs} DOFs; x ~ U[-1,1] (seed 1); "
                       "f = 3 pi^2 sin sin sin",
           "apply_us": us, "apply_gdof_s": m.n_dofs / (us * 1e-6) / 1e9}
    for name, mode in (("fp64", dg.DG_CG_FP64), ("mixed_ir", dg.DG_CG_MIXED_IR)):
        xs = torch.zeros_like(b)
        m.cg_solve(b, xs, rtol=CONFIG1["rtol"], maxit=10000, mode=mode, raise_on_error=False)
        xs.zero_()
        torch.cuda.synchronize()
        _, st = m.cg_solve(b, xs, rtol=CONFIG1["rtol"], maxit=10000, mode=mode,
                           raise_on_error=False)
        out["cg_" + name] = _solve_entry(st, world)
    m.close()
    return out


def run_config4(world):
    """Config 4: 32^3 Q3 lognormal K.  Mean ms of dg_apply, dg_apply_adjoint,
    dg_coeff_grad, the differentiable apply (forward alone, and forward +
    backward) with the coefficient cached and with it re-derived on every call,
    one gradient of L = 0.5 ||u(K) - u_obs||^2 by the adjoint CG (forward and
    adjoint solves, FP64 with M = diag(A), to 1e-10), and the FP64 CG with
    point-Jacobi against cell-block-Jacobi preconditioning."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import autograd as dga
    from paper_1911_01492_gb300 import inputs
    c = CONFIG4
    N, k = c["n_cells"], c["degree"]
    K = inputs.lognormal_coefficient(N, k, seed=c["K_seed"])
    Kd = torch.from_numpy(K).cuda()
    m = dg.Mesh(N, k)
    out = {"workload": f"{N}^3 Q{k}, lognormal K (seed 5), {N ** 3 * (k + 1) ** 3} DOFs"}
    out["setup_ms"] = time_setup(m, Kd)
    x = torch.from_numpy(inputs.uniform_vector(N, k, c["x_seed"])).cuda()
    v = torch.from_numpy(inputs.uniform_vector(N, k, c["x_seed"] + 1)).cuda()
    y = torch.empty_like(x)
    g = torch.empty_like(x)
    reps = 50
    out["apply_ms"] = time_gpu_calls(lambda: m.apply(x, y), reps)
    out["apply_adjoint_ms"] = time_gpu_calls(lambda: m.apply_adjoint(x, y), reps)
    out["coeff_grad_ms"] = time_gpu_calls(lambda: m.coeff_grad(x, v, g), reps)
    logK = torch.log(Kd).requires_grad_()
    xg = x.clone().requires_grad_()

    def fwd_bwd(lk):
        yy = dga.apply(xg, lk, m)
        (yy * v).sum().backward()
    out["autograd_apply_fwd_bwd_ms_cached"] = time_gpu_calls(lambda: fwd_bwd(logK), 20)
    with torch.no_grad():
        out["autograd_apply_fwd_ms_cached"] = time_gpu_calls(lambda: dga.apply(xg, logK, m), 20)
    logK2 = (logK.detach() + 1e-3).requires_grad_()
    flip = [logK, logK2]
    state = {"i": 0}

    def alternating():
        state["i"] ^= 1
        fwd_bwd(flip[state["i"]])
    out["autograd_apply_fwd_bwd_ms_rederived"] = time_gpu_calls(alternating, 10)
    # the loss gradient by the adjoint CG
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    mref = dg.Mesh(N, k)
    mref.set_coefficient(torch.from_numpy(
        inputs.lognormal_coefficient(N, k, seed=c["K_ref_seed"])).cuda())
    # the reference state to 1e-11: FP64 CG stagnates near 5e-12 on this field
    uref, _ = mref.cg_solve(b, rtol=1e-11, maxit=100000,
                            mode=dg.DG_CG_FP64 | dg.DG_CG_PRECOND_JACOBI, raise_on_error=False)
    mref.close()
    rng = np.random.default_rng(c["noise_seed"])
    ur = uref.cpu().numpy()
    uobs = torch.from_numpy(ur + 0.01 * np.sqrt(np.mean(ur ** 2))
                            * rng.standard_normal(ur.shape)).cuda()
    lk = torch.log(Kd).requires_grad_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u = dga.solve(b, lk, m, rtol=c["rtol"], precond="jacobi")
    loss = 0.5 * ((u - uobs) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    out["loss_gradient_adjoint_cg_s"] = time.perf_counter() - t0
    # preconditioners on this operator (FP64 CG to 1e-10, f = 1; each time
    # includes forming the preconditioner): point Jacobi against cell blocks
    for name in ("jacobi", "block", "kron"):
        m.set_coefficient(Kd)          # drops the cached diagonal and blocks
        xs = torch.zeros_like(b)
        torch.cuda.synchronize()
        _, st = m.cg_solve(b, xs, rtol=1e-10, maxit=100000, precond=name, raise_on_error=False)
        out["cg_fp64_" + name] = _solve_entry(st, world)
    out["loss_gradient_note"] = ("forward CG + adjoint CG + dg_coeff_grad, FP64 with "
                                 "M = diag(A), rtol 1e-10, coefficient derived once")
    out["dlogK_norm"] = float(lk.grad.norm())
    m.close()
    return out


def run_resilience(world):
    """Backup and recovery of the CG (Section 2.3) on the 32^3 Q3 lognormal
    operator, FP64 PCG with M = diag(A) to 1e-10, f = 1: the fault-free solve;
    the overhead of backups every 32 iterations into pinned host memory (full
    state, x, x rounded to FP32) without a loss; and, with the DOFs of the
    first eighth of the cells (four z-planes) lost at half the fault-free
    iteration count, the iterations and seconds of each recovery."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    c = CONFIG4
    N, k = c["n_cells"], c["degree"]
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=c["K_seed"]))
                      .cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    out = {"workload": f"{N}^3 Q{k}, lognormal K (seed 5), f = 1, FP64 PCG (Jacobi) to 1e-10",
           "interval": 32, "lost_cells": [0, N ** 3 // 8]}
    m.cg_solve(b, rtol=1e-10, precond="jacobi")            # diagonal and graphs warm
    _, st0 = m.cg_solve(b, rtol=1e-10, precond="jacobi")
    out["fault_free"] = _solve_entry(st0, world)
    fault = st0["iterations"] // 2

    def entry(st):
        e = _solve_entry(st, world)
        e.update({key: st[key] for key in ("fault_injected_at", "backup_iteration",
                                            "backups_taken", "aux_iterations", "backup_bytes")})
        return e
    for backup in ("full", "x64", "x32"):
        _, st = m.cg_solve_resilient(b, rtol=1e-10, backup=backup, interval=32,
                                     precond="jacobi", raise_on_error=False)
        out["no_loss_" + backup] = entry(st)
    for backup, recovery in (("full", "global"), ("x64", "global"), ("x32", "global"),
                             ("x64", "local"), ("none", "local"), ("x64", "local_aux"),
                             ("none", "local_aux")):
        _, st = m.cg_solve_resilient(b, rtol=1e-10, backup=backup, recovery=recovery,
                                     interval=32, fault_iteration=fault,
                                     fault_cells=(0, N ** 3 // 8), aux_rtol=1e-6,
                                     precond="jacobi", raise_on_error=False)
        out[f"loss_{backup}_{recovery}"] = entry(st)
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


def _timed_batched(meshes, bs, xs, sizes, world, precond=None, nodal=False):
    import torch
    import paper_1911_01492_gb300 as dg
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-8, maxit=200000, raise_on_error=False,
                                precond=precond, nodal=nodal)
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


def run_batched(world, rank, sequential_samples: int = 1, full: bool = False,
                larger_levels: bool = True):
    """Batched lock-step CG (FP64, rtol 1e-8) on the 256-sample workload.

    Always: the 128 small samples (16^3 Q2) in one batched solve against 16 of
    them solved one per dg_cg_solve call, and the small batch again with
    M = diag(A_s).  With larger_levels: one-per-call rates of the larger
    levels.  With full = True also the whole 256-sample batch, without and
    with M (minutes).
    """
    import torch
    out = {"workload": "256 lognormal-K samples: 128 x 16^3 Q2, 96 x 24^3 Q3, 32 x 32^3 Q4 "
                       "(230,162,432 DOFs), FP64 CG to 1e-8; seeds 1000 + sample"}
    small = [BATCH_LEVELS[0]]
    meshes, bs, xs, sizes = _batch_meshes(small)
    # the first call tunes the launch shape; time the second
    _timed_batched(meshes[:8], bs[:8], xs[:8], sizes[:8], world)
    out["small_level_batched"] = _timed_batched(meshes, bs, xs, sizes, world)
    out["small_level_one_per_call"] = _timed_sequential(
        meshes, bs, sizes, list(range(min(len(meshes), 16))))
    out["small_level_speedup"] = (out["small_level_batched"]["gdof_per_s"]
                                  / out["small_level_one_per_call"]["gdof_per_s"])
    # the same batch with M = diag(A_s); its time includes forming the diagonals
    out["small_level_batched_jacobi"] = _timed_batched(meshes, bs, xs, sizes, world,
                                                       precond="jacobi")
    # the same batch in the scaled Gauss-point basis (M = I); the first call
    # forms the basis's line operators and tunes its launch shape
    _timed_batched(meshes, bs, xs, sizes, world, nodal=True)
    out["small_level_batched_nodal"] = _timed_batched(meshes, bs, xs, sizes, world, nodal=True)
    for m in meshes:
        m.close()
    if larger_levels:
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
        out["full_batch_nodal"] = _timed_batched(meshes, bs, xs, sizes, world, nodal=True)
        for m in meshes:
            m.close()
    torch.cuda.empty_cache()
    return out


SHEAR = [[1.0, 0.3, 0.1], [0.0, 1.1, -0.2], [0.05, 0.0, 0.9]]


def run_fp32_apply(m, xd, world, steps=8):
    """The FP32 apply (dg_apply with DG_FP32) of the benchmark workload, timed
    like `value` (CUDA events over `steps` sweeps after two warm-up sweeps),
    with per-pass times."""
    import torch
    x32 = xd.float()
    y32 = torch.empty_like(x32)
    ms, napp, ms1, ms2 = time_applies(m, x32, y32, steps, 2, world)
    ms = max_over_ranks(ms, world)
    nd = m.n_dofs
    return {"workload": "the benchmark workload in FP32 (x rounded from the FP64 x)",
            "apply_gdof_s": world * nd * steps * APPLIES_PER_STEP / (ms * 1e-3) / 1e9,
            "pass_ms": {"pass1": ms1 / max(napp, 1), "pass2": ms2 / max(napp, 1)}}


def run_nodal_apply(m, xd, world, peak_fp64=None, steps=8):
    """The operator of the benchmark workload in the scaled Gauss-point basis
    (dg_apply_nodal, the apply inside DG_CG_NODAL solves), timed like `value`,
    with per-pass times, executed FP64 rates from the ncu counts and its
    one-time setup (the basis's line operators)."""
    import torch
    xh = m.to_nodal(xd)
    yh = torch.empty_like(xh)
    ms, napp, ms1, ms2 = time_applies(m, xh, yh, steps, 2, world, nodal=True)
    ms = max_over_ranks(ms, world)
    nd, n = m.n_dofs, m.n
    t1, t2 = ms1 / max(napp, 1), ms2 / max(napp, 1)
    out = {"workload": "the benchmark workload, x mapped to the scaled Gauss-point basis",
           "apply_gdof_s": world * nd * steps * APPLIES_PER_STEP / (ms * 1e-3) / 1e9,
           "pass_ms": {"k_trace_nd": t1, "k_cell_nd": t2}}
    if peak_fp64:
        for name, t in (("k_trace_nd", t1), ("k_cell_nd", t2)):
            epd = executed_fp64_per_dof(name, WORKLOAD["n_cells"], n)
            ipd = executed_fp64_per_dof(name, WORKLOAD["n_cells"], n, EXEC_FP64_INSTR_Q3)
            if epd is not None and t > 0:
                a = epd * nd / (t * 1e-3) / 1e12
                rate = ipd * nd / (t * 1e-3) / 1e12
                out.setdefault("roofline", {})[name] = {
                    "executed_flops_per_dof": epd, "achieved_tflops": a, "peak": peak_fp64,
                    "frac": a / peak_fp64, "fp64_instructions_per_dof": ipd,
                    "issue_frac": rate / (peak_fp64 / 2)}
    return out


def perturbed_vertices(N, seed=7):
    """Vertices of the N^3 unit-cube mesh with every interior vertex moved by
    up to 0.2 h in each direction (uniform, seeded): a multilinear mesh."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, N + 1)
    V = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1)
    inner = np.zeros(V.shape[:3], bool)
    inner[1:-1, 1:-1, 1:-1] = True
    return V + np.where(inner[..., None], 0.2 / N * rng.uniform(-1, 1, V.shape), 0.0)


def run_geometry_probe(n_cells: int, applies: int = 4):
    """A few FP64 applies of the n_cells^3 Q3 lognormal operator on the
    sheared affine mesh and on the perturbed multilinear mesh (for kernel
    profiles), with wall times."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = n_cells, 3
    K = torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=WORKLOAD["K_seed"])).cuda()
    x = torch.from_numpy(inputs.uniform_vector(N, k, WORKLOAD["x_seed"])).cuda()
    y = torch.empty_like(x)
    for name in ("affine", "multilinear"):
        m = dg.Mesh(N, k)
        if name == "affine":
            m.set_geometry(SHEAR)
        else:
            m.set_vertices(perturbed_vertices(N))
        m.set_coefficient(K)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(applies):
            m.apply(x, y)
        torch.cuda.synchronize()
        print(json.dumps({"geometry": name, "n_cells": N,
                          "ms_per_apply": 1e3 * (time.perf_counter() - t0) / applies}),
              flush=True)
        m.close()


# Executed FP64 operations per DOF of the geometry pass-2 kernels at Q3 (ncu
# instruction counters, DFMA x2 + DADD + DMUL): k_cell_aff 11,056 per cell at
# 32^3 and 40^3 alike, k_cell_ml 12,571 per cell at 32^3
EXEC_FP64_GEOMETRY_Q3 = {"k_cell_aff": 11056 / 64, "k_cell_ml": 12571 / 64}
# and as FP64 instructions (DFMA + DADD + DMUL) per DOF: 6,528 and 7,281 per cell
EXEC_FP64_INSTR_GEOMETRY_Q3 = {"k_cell_aff": 6528 / 64, "k_cell_ml": 7281 / 64}


def _geometry_roofline(kernel, n, nd, ms, peak_fp64):
    if n != 4 or not peak_fp64:
        return None
    achieved = EXEC_FP64_GEOMETRY_Q3[kernel] * nd / (ms * 1e-3) / 1e12
    issue = EXEC_FP64_INSTR_GEOMETRY_Q3[kernel] * nd / (ms * 1e-3) / 1e12
    return {"kernel": kernel, "bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
            "peak": peak_fp64, "frac": achieved / peak_fp64,
            "executed_flops_per_dof": EXEC_FP64_GEOMETRY_Q3[kernel],
            "fp64_issue": {"fp64_instructions_per_dof": EXEC_FP64_INSTR_GEOMETRY_Q3[kernel],
                           "achieved_tinst_s": issue, "frac": issue / (peak_fp64 / 2)}}


def run_affine(world, K64, peak_fp64=None):
    """Problems B and C: the FP64 apply of the 64^3 Q3 workload on the sheared
    mesh x = A xi (A = SHEAR) and on a multilinear mesh (perturbed vertices),
    timed like `value` (8 sweeps), with per-pass times; and the FP64 CG (M = I,
    f = 1, rtol 1e-10) on 32^3 Q3 on the sheared geometry."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = WORKLOAD["n_cells"], WORKLOAD["degree"]
    m = dg.Mesh(N, k)
    m.set_geometry(SHEAR)
    m.set_coefficient(torch.from_numpy(K64).cuda())
    x = torch.from_numpy(inputs.uniform_vector(N, k, WORKLOAD["x_seed"])).cuda()
    y = torch.empty_like(x)
    steps = 8
    ms, napp, ms1, ms2 = time_applies(m, x, y, steps, 2, world)
    nd = m.n_dofs
    out = {"geometry": SHEAR, "workload": f"{N}^3 Q{k}, lognormal K (seed 2)",
           "apply_gdof_s": world * nd * steps * APPLIES_PER_STEP / (ms * 1e-3) / 1e9,
           "pass_ms": {"k_trace": ms1 / max(napp, 1), "k_cell_aff": ms2 / max(napp, 1)},
           "roofline": _geometry_roofline("k_cell_aff", k + 1, nd, ms2 / max(napp, 1),
                                          peak_fp64)}
    m.close()
    # problem C: the same workload on a multilinear mesh
    m = dg.Mesh(N, k)
    m.set_vertices(perturbed_vertices(N))
    m.set_coefficient(torch.from_numpy(K64).cuda())
    ms, napp, ms1, ms2 = time_applies(m, x, y, steps, 2, world)
    out["multilinear"] = {"perturbation": "interior vertices moved by up to 0.2 h (seed 7)",
                          "apply_gdof_s": world * nd * steps * APPLIES_PER_STEP / (ms * 1e-3) / 1e9,
                          "pass_ms": {"k_trace": ms1 / max(napp, 1),
                                      "k_cell_ml": ms2 / max(napp, 1)},
                          "roofline": _geometry_roofline("k_cell_ml", k + 1, nd,
                                                         ms2 / max(napp, 1), peak_fp64)}
    m.close()
    del x, y
    N2, k2 = 32, 3
    m = dg.Mesh(N2, k2)
    m.set_geometry(SHEAR)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N2, k2, seed=5)).cuda())
    b = m.load_vector(torch.ones(m.n_dofs, dtype=torch.float64, device="cuda"))
    xs = torch.zeros_like(b)
    torch.cuda.synchronize()
    _, st = m.cg_solve(b, xs, rtol=1e-10, maxit=200000, raise_on_error=False)
    out["cg_fp64_32cubed_q3"] = _solve_entry(st, world)
    m.close()
    torch.cuda.empty_cache()
    return out


def run_mlmc(world):
    """Section 5: one Estimate step of MLMC for the mean inlet flux of the flow
    problem (p = 1 at x = 0, p = 0 at x = 1, zero flux elsewhere; lognormal k,
    correlation length 0.1, variance 1) on the batched levels 16^3 Q2, 24^3 Q3,
    32^3 Q4 with 32 / 8 / 4 coupled samples; every solve in the batched FP64 CG
    with M = diag(A) to 1e-10, then again one mixed-precision CG per sample
    with the Kronecker cell blocks.  Reports the estimates, the level variances
    and costs, and the samples the allocation rule asks for at eps = 0.01."""
    from paper_1911_01492_gb300 import mlmc
    levels = [(N, k) for _, N, k in BATCH_LEVELS]
    t0 = time.perf_counter()
    r = mlmc.estimate(levels, eps=0.01, n_init=[32, 8, 4], max_cycles=1, seed0=9000,
                      pool=32)
    r["wall_s"] = time.perf_counter() - t0
    r.pop("Y", None)
    # the same samples, each solved by the mixed-precision CG with the
    # Kronecker cell blocks (one solve per call)
    t0 = time.perf_counter()
    rm = mlmc.estimate(levels, eps=0.01, n_init=[32, 8, 4], max_cycles=1, seed0=9000,
                       pool=32, solver="mixed")
    r["mixed_kron"] = {"estimate": rm["estimate"], "wall_s": time.perf_counter() - t0,
                       "solve_seconds": rm["solve_seconds"],
                       "seconds_per_sample": [c["seconds_per_sample"] for c in rm["cycles"]]}
    return r


# ---------------------------------------------------------------------------
# Oracle legs (FP64 CPU oracle on this host; rank 0 only)
# ---------------------------------------------------------------------------
def _oracle_apply_rate(N, k, K, x, ncell, target_s):
    """GDOF/s of the oracle's element-wise apply on `ncell` random cells of the
    mesh, repeated for about target_s seconds."""
    from oracle import SIPG
    D = SIPG(N, k)
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(1)
    cells = rng.choice(N ** 3, min(ncell, N ** 3), replace=False)
    D.apply(K, x, cells=cells[:64])
    reps, t0 = 0, time.perf_counter()
    while True:
        D.apply(K, x, cells=cells)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return reps * len(cells) * n3 / dt / 1e9


def oracle_leg_main(args):
    """Child process of the one-thread oracle leg (BLAS limited to one thread
    through the environment): apply rate on a sample of the apply workload."""
    N, k = WORKLOAD["n_cells"], WORKLOAD["degree"]
    K, x = make_inputs(N, k, WORKLOAD["K_seed"], WORKLOAD["x_seed"])
    rate = _oracle_apply_rate(N, k, K, x, 2048, 4.0)
    print(json.dumps({"gdof_per_s": rate, "cells": 2048}), flush=True)


def run_oracle_legs(cpu_all_threads, cg3, cg2, cfg1, K48=None):
    """The FP64 CPU oracle on this host, beside the GPU numbers:
    one thread vs all threads (element-wise apply of the 64^3 Q3 workload),
    config 1 with the assembled CSR matrix (SpMV rate, CG to 1e-10 in full),
    and projected CG times (apply time per iteration x the GPU's iteration
    count) where the CSR matrix would not fit."""
    from oracle import SIPG, cg
    out = {"cores_all": cpu_threads()}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg"],
                           capture_output=True, text=True, env=env, timeout=300)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["apply_64q3_one_thread_gdof_s"] = one["gdof_per_s"]
        out["apply_64q3_one_thread_sample"] = f"{one['cells']} random cells, ~4 s"
    except Exception as e:  # reported, not fatal: the GPU numbers stand alone
        out["apply_64q3_one_thread_error"] = repr(e)[:200]
    if cpu_all_threads is not None:
        out["apply_64q3_all_threads_gdof_s"] = cpu_all_threads["value"]
    # config 1: CSR assembled in full
    from paper_1911_01492_gb300 import inputs
    N, k = CONFIG1["n_cells"], CONFIG1["degree"]
    D = SIPG(N, k)
    K1 = inputs.unit_coefficient(N, k)
    t0 = time.perf_counter()
    A = D.assemble(K1)
    out["config1_csr_assembly_s"] = time.perf_counter() - t0
    out["config1_csr_nnz"] = int(A.nnz)
    x1 = inputs.uniform_vector(N, k, CONFIG1["x_seed"])
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        A @ x1
        reps += 1
    dt = time.perf_counter() - t0
    out["config1_csr_spmv_us"] = 1e6 * dt / reps
    out["config1_csr_spmv_gdof_s"] = reps * D.n_dofs / dt / 1e9
    b1 = D.load_vector(manufactured_source)
    t0 = time.perf_counter()
    _, it, rel, _ = cg(lambda v: A @ v, b1, rtol=CONFIG1["rtol"], maxit=10000)
    out["config1_csr_cg"] = {"seconds": time.perf_counter() - t0, "iterations": it,
                             "rel_residual": rel}
    # projected CG: element-wise apply per iteration x GPU iterations
    if cpu_all_threads is not None and cg2 is not None and "fp64" in cg2:
        sec_per_apply = 16777216 / (cpu_all_threads["value"] * 1e9)
        out["config2_cg_fp64_projected_s"] = sec_per_apply * cg2["fp64"]["iterations"]
    if cg3 is not None and K48 is not None:
        N3, k3 = CG_WORKLOAD["n_cells"], CG_WORKLOAD["degree"]
        x3 = inputs.uniform_vector(N3, k3, 9)
        rate = _oracle_apply_rate(N3, k3, K48, x3, 8192, 3.0)
        out["apply_48q4_all_threads_gdof_s"] = rate
        nd = N3 ** 3 * (k3 + 1) ** 3
        out["config3_cg_fp64_projected_s"] = nd / (rate * 1e9) * cg3["fp64"]["iterations"]
        out["config3_cg_fp64_jacobi_projected_s"] = (nd / (rate * 1e9)
                                                     * cg3["fp64_jacobi"]["iterations"])
    out["projection"] = ("oracle element-wise apply time of the whole mesh x the GPU "
                         "solver's iteration count (vector operations not counted)")
    return out


def run_cg_probe(iters: int, n_cells: int = 0):
    """A fixed number of iterations of the mixed and FP64 CG on the CG
    workload (48^3 Q4, or n_cells^3 Q4), with wall times; for kernel profiles."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = n_cells or CG_WORKLOAD["n_cells"], CG_WORKLOAD["degree"]
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=CG_WORKLOAD["K_seed"])).cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    for name, mode in (("mixed_ir", dg.DG_CG_MIXED_IR), ("fp64", dg.DG_CG_FP64),
                       ("mixed_ir_jacobi", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_JACOBI),
                       ("fp64_jacobi", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_JACOBI),
                       ("mixed_ir_kron", dg.DG_CG_MIXED_IR | dg.DG_CG_PRECOND_KRON),
                       ("fp64_kron", dg.DG_CG_FP64 | dg.DG_CG_PRECOND_KRON),
                       ("fp64_nodal", dg.DG_CG_FP64 | dg.DG_CG_NODAL),
                       ("fp64_nodal_jacobi",
                        dg.DG_CG_FP64 | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_JACOBI),
                       ("mixed_ir_nodal", dg.DG_CG_MIXED_IR | dg.DG_CG_NODAL),
                       ("fp64_nodal_kron",
                        dg.DG_CG_FP64 | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_KRON),
                       ("mixed_ir_nodal_kron",
                        dg.DG_CG_MIXED_IR | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_KRON)):
        x = torch.zeros_like(b)
        _, st = m.cg_solve(b, x, rtol=1e-12, maxit=iters, mode=mode, raise_on_error=False)
        print(json.dumps({"mode": name, "iterations": st["iterations"],
                          "ms_per_iteration": 1e3 * st["seconds"] / max(st["iterations"], 1)}),
              flush=True)


def run_nodal_probe(n_cells: int, applies: int = 4):
    """The N^3 Q3 operator (lognormal K seed 2) applied `applies` times in the
    scaled Gauss-point basis, then `applies` times in the Legendre basis; prints
    the per-pass times of each.  For ncu captures of the nodal kernels."""
    import torch
    import paper_1911_01492_gb300 as dg
    from paper_1911_01492_gb300 import inputs
    N, k = n_cells, 3
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=2)).cuda())
    x = torch.from_numpy(inputs.uniform_vector(N, k, 3)).cuda()
    xh = m.to_nodal(x)
    y = torch.empty_like(x)
    for nodal in (True, False):
        m.timing_enable(applies)
        for _ in range(applies):
            (m.apply_nodal if nodal else m.apply)(xh if nodal else x, y)
        torch.cuda.synchronize()
        napp, ms1, ms2 = m.timing_read()
        print(json.dumps({"basis": "nodal" if nodal else "legendre", "n_cells": N,
                          "pass1_ms": ms1 / max(napp, 1), "pass2_ms": ms2 / max(napp, 1)}),
              flush=True)
    m.close()


def roofline_entry(N, n, nd, napp, ms1, ms2, ms_step, peak_fp64):
    """Roofline of the dominant apply kernel against the FP64 pipe: executed
    FP64 operations (ncu counts per DOF) per launch over its CUDA-event
    duration, divided by the FP64 rate measured in this run."""
    f1, f2 = flops_per_dof(n)
    t1, t2 = ms1 / max(napp, 1), ms2 / max(napp, 1)
    if t2 >= t1:
        dom_ms, dom_alg, dom_name, slot = t2, f2 * nd, "k_cell_lo", "k_cell_lo"
    else:
        dom_ms, dom_alg, dom_name, slot = t1, f1 * nd, "k_trace", "k_trace"
    exec_per_dof = executed_fp64_per_dof(slot, N, n)
    other = "k_trace" if slot == "k_cell_lo" else "k_cell_lo"
    exec_other = executed_fp64_per_dof(other, N, n)
    alg_tflops = dom_alg / (dom_ms * 1e-3) / 1e12
    r = {"bound": "alu", "kernel": dom_name, "unit": "TFLOP/s",
         "pass_ms": {"k_trace": t1, "k_cell_lo": t2},
         "algorithmic_tflops": alg_tflops,
         "apply_tflops_algorithmic": (f1 + f2) * nd / (ms_step * 1e-3 / APPLIES_PER_STEP) / 1e12,
         "peak_nominal": NOMINAL_FP64_TFLOPS,
         "peak_source": "FP64 DFMA throughput measured in this run by dg_peak_probe "
                        "(best of 6 launches filling every SM); nominal 1.25"}
    if exec_per_dof is not None:
        achieved = exec_per_dof * nd / (dom_ms * 1e-3) / 1e12
        r.update({"achieved": achieved, "peak": peak_fp64, "frac": achieved / peak_fp64,
                  "executed_flops_per_dof": exec_per_dof,
                  "frac_of_nominal": achieved / NOMINAL_FP64_TFLOPS,
                  "achieved_source": "executed FP64 operations per DOF from ncu instruction "
                                     "counters (DFMA x2 + DADD + DMUL) x DOFs / live "
                                     "CUDA-event duration of the kernel"})
    else:
        r.update({"achieved": alg_tflops, "peak": peak_fp64, "frac": alg_tflops / peak_fp64,
                  "achieved_source": "algorithmic flops (no executed-operation count for "
                                     "this kernel build)"})
    # the FP64 pipe's issue rate: instructions per launch over the launch time,
    # against the DFMA instruction rate of the probe (its flops / 2)
    issue = {}
    for name, t in (("k_trace", t1), ("k_cell_lo", t2)):
        ipd = executed_fp64_per_dof(name, N, n, EXEC_FP64_INSTR_Q3)
        if ipd is not None and t > 0:
            rate = ipd * nd / (t * 1e-3) / 1e12
            issue[name] = {"fp64_instructions_per_dof": ipd, "achieved_tinst_s": rate,
                           "peak_tinst_s": peak_fp64 / 2, "frac": rate / (peak_fp64 / 2)}
    if issue:
        r["fp64_issue"] = issue
    if exec_other is not None:
        t_other = t1 if other == "k_trace" else t2
        r["other_kernel"] = {"kernel": other, "executed_flops_per_dof": exec_other,
                             "achieved": exec_other * nd / (t_other * 1e-3) / 1e12,
                             "frac": exec_other * nd / (t_other * 1e-3) / 1e12 / peak_fp64}
    traffic = (K_CELL_TRAFFIC_PER_DOF * nd
               if (dom_name == "k_cell_lo" and n == 4 and K_CELL_TRAFFIC_PER_DOF) else None)
    r["traffic"] = traffic
    r["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the pass-2 "
                           "kernel on 40^3 Q3, scaled by DOFs")
    return r


def _leg(fn, *a, **kw):
    """Run one auxiliary measurement; a failure is reported in its key instead
    of ending the benchmark (the headline numbers stand on their own)."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": repr(e)[:300]}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-solution parts")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip configs 1 and 4, the batched small level and the oracle legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--batched", action="store_true",
                    help="also run the larger batched levels one per call")
    ap.add_argument("--batched-sequential", type=int, default=1,
                    help="samples of each larger level solved one per call for reference")
    ap.add_argument("--cg-probe", type=int, default=0, metavar="ITERS",
                    help="only run ITERS iterations of each CG mode on the CG workload "
                         "(for kernel profiles) and exit")
    ap.add_argument("--cg-probe-cells", type=int, default=0, metavar="N",
                    help="with --cg-probe: run it on an N^3 Q4 mesh instead of 48^3")
    ap.add_argument("--geometry-probe", type=int, default=0, metavar="N",
                    help="only run a few applies on the affine and multilinear N^3 Q3 "
                         "meshes (for kernel profiles) and exit")
    ap.add_argument("--nodal-probe", type=int, default=0, metavar="N",
                    help="apply the N^3 Q3 operator in the scaled Gauss-point basis and in the "
                         "Legendre basis 4 times each (for kernel profiles)")
    ap.add_argument("--batched-full", action="store_true",
                    help="with --batched: also solve the whole 256-sample batch (minutes)")
    ap.add_argument("--n-cells", type=int, default=WORKLOAD["n_cells"],
                    help="cells per direction (default: the 64^3 workload)")
    ap.add_argument("--degree", type=int, default=WORKLOAD["degree"])
    ap.add_argument("--oracle-leg", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)

    WORKLOAD["n_cells"], WORKLOAD["degree"] = args.n_cells, args.degree
    if args.oracle_leg:
        oracle_leg_main(args)
        return
    world, rank, local = dist_setup()
    if args.geometry_probe:
        run_geometry_probe(args.geometry_probe)
        return
    if args.cg_probe:
        run_cg_probe(args.cg_probe, args.cg_probe_cells)
        return
    if args.nodal_probe:
        run_nodal_probe(args.nodal_probe)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_1911_01492_gb300 as dg
    N, k = WORKLOAD["n_cells"], WORKLOAD["degree"]
    n = k + 1
    t_start = time.perf_counter()
    K, x = make_inputs(N, k, WORKLOAD["K_seed"], WORKLOAD["x_seed"])
    peak_fp64 = dg.peak_probe("fp64")
    m = dg.Mesh(N, k)
    Kd = torch.from_numpy(K).cuda()
    setup_ms = time_setup(m, Kd)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    nd = m.n_dofs

    with ClockSampler(torch.cuda.current_device() if world == 1 else local) as clk:
        ms, napp, ms1, ms2 = time_applies(m, xd, yd, args.steps, args.warmup, world)
    ms = max_over_ranks(ms, world)
    ms_step = ms / args.steps
    value = world * nd * APPLIES_PER_STEP / (ms_step * 1e-3) / 1e9
    roofline = roofline_entry(N, n, nd, napp, ms1, ms2, ms_step, peak_fp64)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        e2e_steps = max(1, min(args.steps, 20)) if args.steps >= 1 else 1
        dt = time_e2e(m, xh, yh, e2e_steps, 2, world)
        dt = max_over_ranks(dt, world)
        e2e = {"value": world * nd * e2e_steps * APPLIES_PER_STEP / dt / 1e9, "unit": "GDOF/s",
               "h2d_bytes_per_step": xh.numel() * 8 * APPLIES_PER_STEP,
               "d2h_bytes_per_step": yh.numel() * 8 * APPLIES_PER_STEP,
               "steps": e2e_steps}
        del xh, yh

    fp32 = nodal = None
    if not args.no_extra:
        fp32 = _leg(run_fp32_apply, m, xd, world)
        nodal = _leg(run_nodal_apply, m, xd, world, peak_fp64)
    cg2 = cg = K48 = None
    if not args.no_cg:
        cg2 = _leg(run_config2_cg, m, world)
    m.close()
    affine = None
    if not args.no_extra:
        torch.cuda.empty_cache()
        affine = _leg(run_affine, world, K, peak_fp64)
    del xd, yd, Kd
    torch.cuda.empty_cache()
    if not args.no_cg:
        r = _leg(run_cg, world)
        cg, K48 = r if isinstance(r, tuple) else (r, None)

    cfg1 = cfg4 = batched = mlmc_r = resil = None
    if not args.no_extra:
        cfg1 = _leg(run_config1, world)
        cfg4 = _leg(run_config4, world)
        resil = _leg(run_resilience, world)
        batched = _leg(run_batched, world, rank, args.batched_sequential, args.batched_full,
                       larger_levels=args.batched)
        mlmc_r = _leg(run_mlmc, world)
    elif args.batched or args.batched_full:
        batched = _leg(run_batched, world, rank, args.batched_sequential, args.batched_full)

    cpu = legs = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(K, x, N, k)
    if rank == 0 and not args.no_extra and not args.no_cpu_baseline:
        legs = _leg(run_oracle_legs, cpu, cg, cg2, cfg1, K48)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{N}^3 Q{k} SIPG-DG apply, lognormal K (GRF corr. 0.1, "
                                       "var 1, seed 2), x~U[-1,1] (seed 3)",
                           "step": f"one sweep of {APPLIES_PER_STEP} FP64 applies",
                           "dofs_per_gpu": nd, "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (x, h w K and y are 134 MB each; "
                                 "line operators 1 GB)"},
                "roofline": roofline, "e2e": e2e,
                "gpu_launches": 2 * args.steps * APPLIES_PER_STEP,
                "setup_ms": setup_ms,
                "clocks": clk.summary(), "cpu_baseline": cpu, "cg": cg,
                "config2_cg": cg2, "config1": cfg1, "config4": cfg4,
                "batched_cg": batched, "mlmc": mlmc_r, "affine": affine, "resilience": resil,
                "fp32_apply": fp32, "nodal_apply": nodal,
                "oracle_legs": legs,
                "bench_wall_s": time.perf_counter() - t_start}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
