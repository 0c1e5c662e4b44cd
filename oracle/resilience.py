"""Backup and recovery of the CG solver: plain FP64 CPU version.

TEST INFRASTRUCTURE ONLY.  Only the tests may import this module.  The CUDA
library and its Python binding never call it, and it shares no code with them.

What it computes (Exa-Dune paper, Section 2.3, compressed in-memory
checkpointing for linear solvers; the PCG of Section 2.4 underneath):

  * the solver takes a backup every `interval` iterations counted from its
    last (re)start, after an iteration that did not converge: "full" (x, r, p,
    rho and the iteration count; a lossless checkpoint of the whole state),
    "x64" (the iterate x), "x32" (x rounded to FP32, a lossy compression to
    half the bytes) or "none" (zero recovery);
  * a data loss hits the DOFs lost = (i0, i1): x, r and p there become zero.
    It happens at the first backup point at or after `fault_iteration`, in
    place of that backup;
  * recovery "global": every DOF rolls back to the backup; with the full
    state the iteration resumes exactly where the backup was taken (same
    iterates as without the loss), otherwise CG restarts from the backup's x;
  * recovery "local": only the lost DOFs take the backup's x (zero without a
    backup) and CG restarts;
  * recovery "local_aux": as "local", then the local auxiliary problem
    A(F,F) e = (b - A x)(F) on the lost DOFs F with every other DOF held at its
    value (the Dirichlet layer of the paper's auxiliary problem), solved by CG
    from e = 0 (so the backup in x(F) is the initial guess) to aux_rtol
    relative to its initial residual or aux_maxit iterations; x(F) += e; CG
    restarts.
With no backup taken yet, every recovery restarts from the current x with the
lost DOFs zero (plus the auxiliary solve for "local_aux").

The stopping rule is the one of dg_oracle.cg: recursive ||r|| <= rtol ||b||,
then the true residual, restarting from x while it is above rtol (at most
max_restarts restarts, recovery restarts included).

Parity status: pinned by tests/test_oracle_resilience_pins.py (no loss equals the plain
PCG bit for bit; the full-state global rollback equals the fault-free solve
bit for bit and costs exactly the rolled-back iterations; the auxiliary
problem against a dense direct solve of the assembled A(F,F); the FP32 backup
within half an FP32 unit of the iterate; convergence of every strategy).
"""
from __future__ import annotations

import numpy as np

from .dg_oracle import cg


def local_auxiliary_solve(apply, b, x, lost, minv=None, aux_rtol=1e-2, aux_maxit=1000):
    """x(F) += e with A(F,F) e = (b - A x)(F), F = range(*lost), by CG on the
    restriction of the operator to F (every other DOF held fixed).  Returns
    (x, CG iterations)."""
    i0, i1 = lost
    n = b.shape[0]

    def a_ff(v):                       # A(F,F) v = (A [0; v; 0])(F)
        w = np.zeros(n)
        w[i0:i1] = v
        return apply(w)[i0:i1]

    r_f = (b - apply(x))[i0:i1]
    m_f = None if minv is None else np.asarray(minv)[i0:i1]
    e, its, _, _ = cg(a_ff, r_f, rtol=aux_rtol, maxit=aux_maxit, max_restarts=0, minv=m_f)
    x = x.copy()
    x[i0:i1] += e
    return x, its


def resilient_cg(apply, b, rtol=1e-10, maxit=100000, interval=32, backup="full",
                 recovery="global", fault_iteration=-1, lost=(0, 0), minv=None,
                 aux_rtol=1e-2, aux_maxit=1000, max_restarts=5):
    """PCG (M = I, or M^-1 = diag(minv)) with the backups, the data loss and
    the recovery described above.  Returns (x, info) with info: iterations
    (every iteration run, rolled-back ones included), restarts, rel_residual
    (true), fault_injected_at, backup_iteration, backups_taken,
    aux_iterations, converged."""
    if backup not in ("none", "full", "x64", "x32"):
        raise ValueError(backup)
    if recovery not in ("global", "local", "local_aux"):
        raise ValueError(recovery)
    b = np.asarray(b, float)
    n = b.shape[0]
    d = np.ones(n) if minv is None else np.asarray(minv, float)
    nb = float(np.linalg.norm(b))
    info = dict(iterations=0, restarts=0, rel_residual=0.0, fault_injected_at=-1,
                backup_iteration=-1, backups_taken=0, aux_iterations=0, converged=True)
    if nb == 0.0:
        return np.zeros(n), info
    tol = rtol * nb
    x = np.zeros(n)
    saved = None                       # the latest backup

    def start(x):                      # r = b - A x, p = M^-1 r, rho = <p, r>
        r = b - apply(x)
        p = d * r if minv is not None else r.copy()
        return r, p, float(p @ r)

    it = 0
    r, p, rho = start(x)
    since = 0                          # iterations since the last (re)start
    done = float(np.linalg.norm(r)) <= tol or it >= maxit
    while True:
        if not done:
            q = apply(p)
            pq = float(p @ q)
            if not pq > 0.0:
                raise FloatingPointError("CG breakdown: <p, Ap> <= 0")
            alpha = rho / pq
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            since += 1
            info["iterations"] += 1
            z = d * r if minv is not None else r
            done = float(np.linalg.norm(r)) <= tol or it >= maxit
            if not done:
                rho_new = float(z @ r)
                p = (rho_new / rho) * p + z
                rho = rho_new
            if not done and since % interval != 0:
                continue
            if not done:
                # a backup point (the iteration did not converge)
                if fault_iteration >= 0 and info["fault_injected_at"] < 0 \
                        and it >= fault_iteration:
                    i0, i1 = lost
                    x = x.copy()
                    x[i0:i1] = 0.0             # the data loss
                    r[i0:i1] = 0.0
                    p[i0:i1] = 0.0
                    info["fault_injected_at"] = it
                    if saved is not None:
                        info["backup_iteration"] = saved["it"]
                    if saved is not None and backup == "full" and recovery == "global":
                        x, r, p = saved["x"].copy(), saved["r"].copy(), saved["p"].copy()
                        rho, it = saved["rho"], saved["it"]
                        since = 0
                        continue
                    if saved is not None:
                        src = saved["x"]
                        if recovery == "global":
                            x = src.astype(float)
                        else:
                            x[i0:i1] = src[i0:i1].astype(float)
                    if recovery == "local_aux":
                        x, info["aux_iterations"] = local_auxiliary_solve(
                            apply, b, x, lost, minv, aux_rtol, aux_maxit)
                    r, p, rho = start(x)
                    since = 0
                    info["restarts"] += 1
                    done = float(np.linalg.norm(r)) <= tol or it >= maxit
                    continue
                if backup == "full":
                    saved = dict(x=x.copy(), r=r.copy(), p=p.copy(), rho=rho, it=it)
                elif backup == "x64":
                    saved = dict(x=x.copy(), it=it)
                elif backup == "x32":
                    saved = dict(x=x.astype(np.float32), it=it)
                if backup != "none":
                    info["backups_taken"] += 1
                continue
        # converged by the recursive residual, or out of iterations
        rel = float(np.linalg.norm(b - apply(x))) / nb
        info["rel_residual"] = rel
        if rel <= rtol:
            return x, info
        if it >= maxit or info["restarts"] >= max_restarts:
            info["converged"] = False
            return x, info
        info["restarts"] += 1
        r, p, rho = start(x)
        since = 0
        done = float(np.linalg.norm(r)) <= tol or it >= maxit
