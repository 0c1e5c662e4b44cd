"""Pins of the CG backup and recovery oracle (Section 2.3, compressed
in-memory checkpointing; the PCG of Section 2.4) against what the method and
the mathematics fix: no loss leaves the PCG untouched; a lossless global
rollback reproduces the fault-free iterates bit for bit at the cost of exactly
the rolled-back iterations; the local auxiliary problem is the restriction of
A to the lost DOFs (checked by a dense direct solve of the assembled A(F,F));
the FP32 backup is x rounded to nearest; every strategy converges; and the
ordering of recovery costs that the section reports (an auxiliary solve
restores the convergence that a zero recovery loses)."""
import numpy as np
import pytest

from oracle import SIPG, cg
from oracle.resilience import local_auxiliary_solve, resilient_cg
from paper_1911_01492_gb300 import inputs


def problem(N, k, seed, corr=0.4):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=seed, corr_len=corr)
    b = inputs.uniform_vector(N, k, seed + 1)
    A = D.assemble(K)
    return D, K, b, A


@pytest.fixture(scope="module")
def p32():
    return problem(3, 2, 3, 0.5)


@pytest.mark.parametrize("backup", ["full", "x64", "x32", "none"])
@pytest.mark.parametrize("jacobi", [False, True])
def test_no_loss_is_the_plain_pcg(p32, backup, jacobi):
    D, K, b, A = p32
    minv = 1.0 / D.diagonal(K) if jacobi else None
    x0, it0, rel0, _ = cg(lambda v: A @ v, b, rtol=1e-10, minv=minv)
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-10, interval=4, backup=backup, minv=minv)
    assert np.array_equal(x, x0)
    assert info["iterations"] == it0 and info["rel_residual"] == rel0
    assert info["fault_injected_at"] == -1
    if backup != "none":
        assert info["backups_taken"] == (it0 - 1) // 4


@pytest.mark.parametrize("interval,fault", [(4, 10), (8, 9), (5, 31)])
def test_full_global_rollback_is_exact(p32, interval, fault):
    D, K, b, A = p32
    n3 = D.n3
    x0, it0, _, _ = cg(lambda v: A @ v, b, rtol=1e-10)
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-10, interval=interval, backup="full",
                           recovery="global", fault_iteration=fault, lost=(5 * n3, 9 * n3))
    fault_at = -(-fault // interval) * interval
    assert info["fault_injected_at"] == fault_at
    assert info["backup_iteration"] == fault_at - interval
    assert np.array_equal(x, x0)
    assert info["iterations"] == it0 + interval and info["restarts"] == 0


def test_auxiliary_problem_is_the_restricted_direct_solve(p32):
    D, K, b, A = p32
    n3 = D.n3
    rng = np.random.default_rng(7)
    x = rng.standard_normal(b.shape[0])
    lost = (4 * n3, 11 * n3)
    i0, i1 = lost
    xa, its = local_auxiliary_solve(lambda v: A @ v, b, x, lost, aux_rtol=1e-14, aux_maxit=10000)
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    e = np.linalg.solve(Ad[i0:i1, i0:i1], (b - Ad @ x)[i0:i1])
    assert np.array_equal(xa[:i0], x[:i0]) and np.array_equal(xa[i1:], x[i1:])
    assert np.abs(xa[i0:i1] - (x[i0:i1] + e)).max() <= 1e-10 * np.abs(x[i0:i1] + e).max()
    # the local residual vanishes: the lost DOFs satisfy their equations
    r = b - Ad @ xa
    assert np.linalg.norm(r[i0:i1]) <= 1e-11 * np.linalg.norm(b - Ad @ x)
    assert 0 < its <= i1 - i0


def test_fp32_backup_is_round_to_nearest(p32):
    """The FP32 backup holds x rounded to nearest (within half an FP32 unit)
    and a global x32 rollback restarts plain CG from exactly those values:
    backups at iterations 4 and 8, the loss at 8 (in place of that backup),
    then four iterations from the iteration-4 backup up to maxit = 12."""
    D, K, b, A = p32
    n3 = D.n3
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-30, maxit=12, interval=4, backup="x32",
                           recovery="global", fault_iteration=8, lost=(0, n3))
    assert info["fault_injected_at"] == 8 and info["backup_iteration"] == 4
    assert not info["converged"] and info["iterations"] == 12
    x4, _, _, _ = cg(lambda v: A @ v, b, rtol=1e-30, maxit=4, max_restarts=0)
    x4r = x4.astype(np.float32).astype(float)
    assert np.all(np.abs(x4r - x4) <= 2.0 ** -24 * np.abs(x4))
    xr, _, _, _ = cg(lambda v: A @ v, b, x0=x4r, rtol=1e-30, maxit=4, max_restarts=0)
    assert np.array_equal(x, xr)


@pytest.mark.parametrize("backup,recovery", [("x64", "global"), ("x64", "local"),
                                             ("none", "local"), ("full", "local"),
                                             ("x64", "local_aux"), ("none", "local_aux")])
def test_recovered_iterate_follows_the_definition(p32, backup, recovery):
    """Backups at 4 and 8; the loss at 8 hits the DOFs of cells 5..8.  The
    recovered x is, by the definition of each strategy, built here from plain
    CG iterates: the backup everywhere (global), the iterate at 8 with the
    lost DOFs replaced by the backup or by zero (local), plus the auxiliary
    solve on them (local_aux); CG then restarts from it up to maxit = 12."""
    D, K, b, A = p32
    n3 = D.n3
    i0, i1 = 5 * n3, 9 * n3
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-30, maxit=12, interval=4, backup=backup,
                           recovery=recovery, fault_iteration=8, lost=(i0, i1),
                           aux_rtol=1e-30, aux_maxit=5)
    x4, _, _, _ = cg(lambda v: A @ v, b, rtol=1e-30, maxit=4, max_restarts=0)
    x8, _, _, _ = cg(lambda v: A @ v, b, rtol=1e-30, maxit=8, max_restarts=0)
    if recovery == "global":
        x0 = x4.copy()
    else:
        x0 = x8.copy()
        x0[i0:i1] = 0.0 if backup == "none" else x4[i0:i1]
    if recovery == "local_aux":
        x0, its = local_auxiliary_solve(lambda v: A @ v, b, x0, (i0, i1), aux_rtol=1e-30,
                                        aux_maxit=5)
        assert its == 5 and info["aux_iterations"] == 5
    xr, _, _, _ = cg(lambda v: A @ v, b, x0=x0, rtol=1e-30, maxit=4, max_restarts=0)
    assert np.array_equal(x, xr)
    assert info["restarts"] == 1 and info["iterations"] == 12


@pytest.mark.parametrize("backup,recovery", [("x64", "global"), ("x32", "global"),
                                             ("x64", "local"), ("none", "local"),
                                             ("x64", "local_aux"), ("none", "local_aux"),
                                             ("full", "local"), ("x32", "local_aux")])
def test_every_strategy_converges(p32, backup, recovery):
    D, K, b, A = p32
    n3 = D.n3
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-10, interval=4, backup=backup,
                           recovery=recovery, fault_iteration=10, lost=(5 * n3, 9 * n3))
    assert info["converged"] and info["fault_injected_at"] == 12
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert info["restarts"] >= 1
    if recovery == "local_aux":
        assert info["aux_iterations"] > 0


def test_loss_before_any_backup_restarts_with_zeros(p32):
    D, K, b, A = p32
    n3 = D.n3
    x, info = resilient_cg(lambda v: A @ v, b, rtol=1e-10, interval=8, backup="x64",
                           recovery="local", fault_iteration=3, lost=(0, 4 * n3))
    assert info["fault_injected_at"] == 8 and info["backup_iteration"] == -1
    assert info["converged"]


def test_auxiliary_solve_restores_the_convergence_zero_recovery_loses():
    """Section 2.3: a zero recovery alone costs many extra iterations; with
    the auxiliary problem solved on the lost cells the solve needs about the
    fault-free count again, and a lossless rollback costs exactly the
    rolled-back iterations."""
    D, K, b, A = problem(4, 2, 3)
    n3 = D.n3
    _, it0, _, _ = cg(lambda v: A @ v, b, rtol=1e-10)
    kw = dict(rtol=1e-10, interval=8, fault_iteration=int(0.8 * it0),
              lost=(16 * n3, 32 * n3), aux_rtol=1e-6)
    its = {}
    for backup, recovery in [("full", "global"), ("none", "local"), ("none", "local_aux"),
                             ("x64", "local_aux")]:
        _, info = resilient_cg(lambda v: A @ v, b, backup=backup, recovery=recovery, **kw)
        assert info["converged"]
        its[backup, recovery] = info["iterations"]
    assert its["full", "global"] == it0 + 8
    assert its["none", "local"] > its["none", "local_aux"] + 0.2 * it0
    assert its["x64", "local_aux"] <= it0 + 0.1 * it0
