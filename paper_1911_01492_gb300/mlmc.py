"""Multilevel Monte-Carlo estimate of the mean inlet flux of the Section 5 flow
problem, with every solve in the batched GPU CG.

Problem (Section 5): -div(k grad p) = 0 in the unit cube, p = 1 on x = 0,
p = 0 on x = 1, zero flux on the other faces, k lognormal with exponential
covariance; quantity of interest Q = total flux through the inlet x = 0.  The
levels are discretisations of increasing resolution (mesh size and degree).
The estimator is the telescoping sum of Section 5,
    E[Q_L] = E[Q_0] + sum_{l >= 1} E[Q_l - Q_{l-1}],
with Y_l = Q_l - Q_{l-1} evaluated on one realization seen by both levels
(inputs.lognormal_on_levels) and independent realizations across levels.

Estimate-Solve cycle (Section 5): start from a prescribed number of samples
per level, estimate each level's variance V_l and cost C_l per sample, set the
number of samples per level for a target root-mean-square error eps by the
standard MLMC rule N_l = ceil(eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) (the
allocation that minimises sum N_l C_l subject to sum V_l / N_l <= eps^2 / 2,
the other half of eps^2 left to the discretisation bias), solve the missing
samples, and repeat.  All the solves of one cycle run in one batched
lock-step CG launch series over samples of every level, whose work units are
proportional to each sample's unknowns (the proportional distribution of work
over levels that Section 5 describes for processes); the cycle also reports the
paper's ideal process split p_l = N_l t_l / (sum_k N_k t_k / p_total) with the
GPU's SMs as the processes.

The solves, the right-hand sides and the fluxes run in the library's kernels;
this module only arranges samples and forms the sample means and variances of
a few hundred scalars on the host.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import DG_BC_FLOW_X, DG_CG_MIXED_IR, Mesh, cg_solve_batched
from . import inputs

G_FLOW = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # p = 1 at x = 0, p = 0 at x = 1


def allocation(V, C, eps: float):
    """Samples per level for a root-mean-square error eps:
    N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) (statistical error
    sum_l V_l / N_l <= eps^2 / 2 at minimal cost sum_l N_l C_l)."""
    V = np.maximum(np.asarray(V, float), 0.0)
    C = np.asarray(C, float)
    s = float(np.sum(np.sqrt(V * C)))
    return [int(math.ceil(2.0 / eps ** 2 * math.sqrt(v / c) * s)) if v > 0 else 1
            for v, c in zip(V, C)]


def process_split(N, t, p_total: int):
    """Section 5's ideal processes per level, p_l = N_l t_l / T_p with
    T_p = sum_k N_k t_k / p_total, and its floor."""
    N = np.asarray(N, float)
    t = np.asarray(t, float)
    Tp = float(np.sum(N * t)) / p_total
    ideal = N * t / Tp
    return ideal.tolist(), [int(math.floor(v)) for v in ideal]


class FlowLevels:
    """Pooled meshes of the flow problem for a list of levels [(n_cells, degree)]."""

    def __init__(self, levels, pool: int = 16, corr_len: float = 0.1, variance: float = 1.0,
                 rtol: float = 1e-10, precond: str | None = "jacobi", solver: str = "batched"):
        """solver: "batched" (the lock-step batched FP64 CG over the pooled
        samples, with precond None or "jacobi") or "mixed" (one mixed-precision
        CG per sample, FP32 iterations with FP64 refinement, with the
        Kronecker cell blocks)."""
        if solver not in ("batched", "mixed"):
            raise ValueError(f"unknown solver {solver!r}")
        self.levels = [tuple(l) for l in levels]
        self.pool = pool
        self.corr_len = corr_len
        self.variance = variance
        self.rtol = rtol
        self.precond = precond
        self.solver = solver
        self._meshes = {}

    def _mesh(self, level: int, slot: int) -> Mesh:
        key = (level, slot)
        if key not in self._meshes:
            N, k = self.levels[level]
            m = Mesh(N, k)
            m.set_boundary(DG_BC_FLOW_X)
            self._meshes[key] = m
        return self._meshes[key]

    def close(self):
        for m in self._meshes.values():
            m.close()
        self._meshes.clear()

    def samples(self, level: int, seeds):
        """Y = Q_l - Q_{l-1} (Q_0 for level 0) for each seed, the fluxes, and
        the cost: (Y array, Q_fine array, Q_coarse array or None, DOF-iterations,
        solve seconds, generation seconds)."""
        import torch
        Y, Qf, Qc = [], [], []
        work, t_solve, t_gen = 0.0, 0.0, 0.0
        lv = [level] if level == 0 else [level, level - 1]
        seeds = list(seeds)
        per = max(1, self.pool // len(lv))
        for c0 in range(0, len(seeds), per):
            chunk = seeds[c0:c0 + per]
            meshes, bs, xs = [], [], []
            t0 = time.perf_counter()
            for j, sd in enumerate(chunk):
                Ks = inputs.lognormal_on_levels([self.levels[l] for l in lv], sd,
                                                self.corr_len, self.variance)
                for i, (l, K) in enumerate(zip(lv, Ks)):
                    m = self._mesh(l, j)
                    m.set_coefficient(torch.from_numpy(K).cuda())
                    meshes.append(m)
                    bs.append(m.dirichlet_rhs(G_FLOW))
                    xs.append(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
            torch.cuda.synchronize()
            t_gen += time.perf_counter() - t0
            t0 = time.perf_counter()
            if self.solver == "batched":
                st = cg_solve_batched(meshes, bs, xs, rtol=self.rtol, maxit=200000,
                                      precond=self.precond)
            else:
                st = [m.cg_solve(b, x, rtol=self.rtol, maxit=200000, mode=DG_CG_MIXED_IR,
                                 precond="kron")[1] for m, b, x in zip(meshes, bs, xs)]
            q = [m.boundary_flux(x, 0, G_FLOW[0]) for m, x in zip(meshes, xs)]
            qv = torch.cat(q).cpu().numpy()
            t_solve += time.perf_counter() - t0
            work += sum(s["iterations"] * m.n_dofs for s, m in zip(st, meshes))
            for j in range(len(chunk)):
                qf = float(qv[len(lv) * j])
                qc = float(qv[len(lv) * j + 1]) if len(lv) == 2 else 0.0
                Qf.append(qf)
                Qc.append(qc)
                Y.append(qf - qc)
        return (np.array(Y), np.array(Qf), np.array(Qc) if level > 0 else None, work,
                t_solve, t_gen)


def estimate(levels, eps: float, n_init, max_cycles: int = 3, seed0: int = 5000,
             p_total: int = 152, max_samples: int = 512, **kw):
    """Estimate-Solve cycles of MLMC for the mean inlet flux.  Returns a dict
    with the estimate, its estimated statistical error, the samples, variances
    and costs per level, and timings."""
    L = len(levels)
    F = FlowLevels(levels, **kw)
    Ys = [np.zeros(0) for _ in range(L)]
    cost = [0.0] * L       # DOF-iterations per level (summed)
    secs = [0.0] * L
    gen = 0.0
    target = list(n_init)
    cycles = []
    try:
        for cyc in range(max_cycles):
            for l in range(L):
                need = min(target[l], max_samples) - len(Ys[l])
                if need <= 0:
                    continue
                seeds = [seed0 + 100000 * l + len(Ys[l]) + i for i in range(need)]
                Y, _, _, w, ts, tg = F.samples(l, seeds)
                Ys[l] = np.concatenate([Ys[l], Y])
                cost[l] += w
                secs[l] += ts
                gen += tg
            V = [float(np.var(y, ddof=1)) if len(y) > 1 else 0.0 for y in Ys]
            C = [cost[l] / max(len(Ys[l]), 1) for l in range(L)]
            new = allocation(V, C, eps)
            t_per = [secs[l] / max(len(Ys[l]), 1) for l in range(L)]
            ideal, floor = process_split([len(y) for y in Ys], t_per, p_total)
            cycles.append({"samples": [len(y) for y in Ys], "variance": V,
                           "cost_dof_iterations": C, "seconds_per_sample": t_per,
                           "next_samples": new, "process_split_ideal": ideal,
                           "process_split": floor})
            if all(len(Ys[l]) >= min(new[l], max_samples) for l in range(L)):
                break
            target = [max(len(Ys[l]), new[l]) for l in range(L)]
    finally:
        F.close()
    means = [float(np.mean(y)) for y in Ys]
    V = [float(np.var(y, ddof=1)) if len(y) > 1 else 0.0 for y in Ys]
    return {"levels": [list(l) for l in levels], "eps": eps, "estimate": float(sum(means)),
            "level_means": means, "variance": V,
            "statistical_error": math.sqrt(sum(v / len(y) for v, y in zip(V, Ys))),
            "samples": [len(y) for y in Ys], "solve_seconds": secs,
            "generation_seconds": gen, "cycles": cycles, "Y": [y.tolist() for y in Ys]}
