"""Resilient CG (dg_cg_solve_resilient: backups, a host-injected data loss and
the recoveries of Section 2.3) on the GPU against the FP64 oracle in
oracle/resilience.py.  The loss is made on the host side of the solver loop
(a range of x, r and p set to zero between two graph replays): nothing here
faults or traps the GPU.

* no loss: bit-identical to dg_cg_solve (deterministic reductions);
* lossless global rollback: bit-identical to the fault-free solve, exactly
  `interval` more iterations;
* every strategy at fixed iteration counts (no convergence inside): the
  iterate after loss, recovery, restart and auxiliary solve matches the
  oracle element by element (1e-10, the FP64 tolerance of the first CG
  iterates: two rounding orders differ by ~1e-15 after 12 iterations here);
* every strategy converges at a larger size, with the oracle's residual."""
import numpy as np
import pytest

from oracle import SIPG
from oracle.resilience import resilient_cg
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def setup(dg, N, k, seed):
    import torch
    K = inputs.lognormal_coefficient(N, k, seed=seed, corr_len=min(0.5, 0.1 * 64 / N))
    b = inputs.uniform_vector(N, k, seed + 1)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m, K, b, torch.from_numpy(b).cuda()


@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_no_loss_is_bit_identical_to_cg_solve(dg, precond):
    m, K, b, bd = setup(dg, 6, 3, 11)
    x0, st0 = m.cg_solve(bd, rtol=1e-10, precond=precond)
    for backup in ("full", "x64", "x32", "none"):
        x, st = m.cg_solve_resilient(bd, rtol=1e-10, backup=backup, interval=16,
                                     precond=precond)
        assert np.array_equal(x.cpu().numpy(), x0.cpu().numpy()), backup
        assert st["iterations"] == st0["iterations"] and st["fault_injected_at"] == -1
        if backup != "none" and st0["outer_iterations"] == 0:
            assert st["backups_taken"] == (st0["iterations"] - 1) // 16
        if backup == "none":
            assert st["backups_taken"] == 0 and st["backup_bytes"] == 0
    assert st["status"] == 0


@pytest.mark.parametrize("interval,fault", [(8, 20), (16, 17), (5, 5)])
@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_full_global_rollback_is_bit_identical(dg, interval, fault, precond):
    m, K, b, bd = setup(dg, 5, 2, 21)
    x0, st0 = m.cg_solve(bd, rtol=1e-10, precond=precond)
    fault_at = -(-fault // interval) * interval
    if fault_at == interval:
        fault_at = 2 * interval            # the first check takes a backup only
        fault = fault_at
    x, st = m.cg_solve_resilient(bd, rtol=1e-10, backup="full", recovery="global",
                                 interval=interval, fault_iteration=fault,
                                 fault_cells=(10, 40), precond=precond)
    assert st["fault_injected_at"] == fault_at
    assert st["backup_iteration"] == fault_at - interval
    assert np.array_equal(x.cpu().numpy(), x0.cpu().numpy())
    assert st["iterations"] == st0["iterations"] + interval
    n = m.n_dofs                           # x, r, p and the solver scalars
    assert 3 * 8 * n < st["backup_bytes"] <= 3 * 8 * n + 256


CASES = [("x64", "global", None), ("x32", "global", None), ("x64", "local", None),
         ("none", "local", None), ("full", "local", "jacobi"), ("x64", "local_aux", None),
         ("none", "local_aux", None), ("x32", "local_aux", "jacobi"),
         ("full", "global", "jacobi")]


@pytest.mark.parametrize("N,k", [(3, 2), (4, 3)])
@pytest.mark.parametrize("backup,recovery,precond", CASES)
def test_recovery_matches_oracle(dg, N, k, backup, recovery, precond):
    m, K, b, bd = setup(dg, N, k, 31)
    D = SIPG(N, k)
    minv = 1.0 / D.diagonal(K) if precond else None
    lost = (4, 9) if N == 3 else (10, 30)
    kw = dict(rtol=1e-14, maxit=12, interval=3, backup=backup, recovery=recovery,
              fault_iteration=5, aux_rtol=1e-30, aux_maxit=4)
    xref, info = resilient_cg(lambda v: D.apply(K, v), b, lost=(lost[0] * D.n3, lost[1] * D.n3),
                              minv=minv, **kw)
    x, st = m.cg_solve_resilient(bd, fault_cells=lost, precond=precond, raise_on_error=False,
                                 **kw)
    assert st["status"] == dg.DG_ERR_NOT_CONVERGED
    for key in ("fault_injected_at", "backup_iteration", "aux_iterations", "backups_taken"):
        assert st[key] == info[key], key
    assert st["iterations"] == info["iterations"]
    assert st["outer_iterations"] == info["restarts"]
    assert relmax(x.cpu().numpy(), xref) <= 1e-10


@pytest.mark.parametrize("backup,recovery", [("x64", "global"), ("x32", "global"),
                                             ("x64", "local"), ("none", "local"),
                                             ("x64", "local_aux"), ("none", "local_aux")])
def test_every_strategy_converges(dg, backup, recovery):
    m, K, b, bd = setup(dg, 8, 3, 41)
    D = SIPG(8, 3)
    x0, st0 = m.cg_solve(bd, rtol=1e-9)
    x, st = m.cg_solve_resilient(bd, rtol=1e-9, backup=backup, recovery=recovery, interval=16,
                                 fault_iteration=int(0.7 * st0["iterations"]),
                                 fault_cells=(100, 260), aux_rtol=1e-6)
    assert st["fault_injected_at"] > 0 and st["status"] == 0
    xn = x.cpu().numpy()
    assert np.linalg.norm(b - D.apply(K, xn)) <= 1.0001e-9 * np.linalg.norm(b)
    if recovery == "local_aux":
        assert st["aux_iterations"] > 0


def test_auxiliary_solve_beats_zero_recovery(dg):
    m, K, b, bd = setup(dg, 8, 2, 51)
    _, st0 = m.cg_solve(bd, rtol=1e-10)
    its = {}
    for recovery in ("local", "local_aux"):
        _, st = m.cg_solve_resilient(bd, rtol=1e-10, backup="none", recovery=recovery,
                                     interval=8, fault_iteration=int(0.8 * st0["iterations"]),
                                     fault_cells=(128, 256), aux_rtol=1e-6)
        its[recovery] = st["iterations"]
    assert its["local"] > its["local_aux"]


def test_bad_options_are_rejected(dg):
    import torch
    m, K, b, bd = setup(dg, 3, 2, 61)
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.cg_solve_resilient(bd, interval=0)
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.cg_solve_resilient(bd, recovery="local_aux", aux_maxit=0)
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.cg_solve_resilient(bd, recovery="local_aux", aux_rtol=0.0)
    # mixed precision is not a mode of the resilient solver
    st = dg.CGStats()
    res = dg.Resilience(8, dg.DG_BACKUP_FULL, dg.DG_RECOVER_GLOBAL, -1, 0, 0, 1e-2, 10,
                        -1, -1, 0, 0, 0)
    x = torch.zeros_like(bd)
    import ctypes
    rc = dg.library().dg_cg_solve_resilient(m.handle, bd.data_ptr(), x.data_ptr(), 1e-8, 100,
                                            dg.DG_CG_MIXED_IR, ctypes.byref(res),
                                            ctypes.byref(st), None)
    assert rc == dg.DG_ERR_INVALID_ARG
