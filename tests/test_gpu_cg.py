"""GPU CG solves (FP64 and mixed-precision iterative refinement) checked by the
oracle: the residual b - A x of the returned x is recomputed in FP64 on the
host, and x is compared with a direct solve within the conditioning bound."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import SIPG, cg
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def u_exact(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def f_exact(x, y, z):
    return 3 * np.pi ** 2 * u_exact(x, y, z)


def oracle_rel_residual(D, K, b, x):
    return float(np.linalg.norm(b - D.apply(K, x)) / np.linalg.norm(b))


def test_cg_fp64_manufactured_8cubed_q2(dg):
    """8^3 Q2, K = 1, f from u = sin sin sin, CG to 1e-10."""
    import torch
    N, k = 8, 2
    D = SIPG(N, k)
    K = inputs.unit_coefficient(N, k)
    b = D.load_vector(f_exact)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-10)
    x = x.cpu().numpy()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert oracle_rel_residual(D, K, b, x) <= 1.05e-10
    xd = spla.spsolve(D.assemble(K).tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * 2.3e3 * 10 * np.linalg.norm(xd)
    # the discrete solution approximates u to O(h^3)
    assert D.l2_error(x, u_exact) < 2e-3


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def small_mesh_field(N, k, seed):
    """Lognormal K with the per-cell statistics of the 64^3 workload: the
    correlation length is scaled so that it spans the same number of cells
    (0.1 at N = 64).  With the unscaled length 0.1 a coarse cell spans several
    correlation lengths and the SIPG matrix can be indefinite (see
    test_cg_reports_indefinite_coarse_mesh)."""
    return inputs.lognormal_coefficient(N, k, seed=seed, corr_len=0.1 * 64 / N)


@pytest.mark.parametrize("N,k,seed", [(4, 3, 5), (5, 2, 6), (3, 4, 4)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cg_lognormal_residual_checked_by_oracle(dg, N, k, seed, mode):
    import torch
    D = SIPG(N, k)
    K = small_mesh_field(N, k, seed)
    b = inputs.constant_load_vector(N, k)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-10, mode=mode)
    x = x.cpu().numpy()
    assert st["status"] == 0
    assert oracle_rel_residual(D, K, b, x) <= 1.05e-10
    if mode == 1:
        assert st["outer_iterations"] >= 1


@pytest.mark.parametrize("mode,precond", [(0, None), (0, "jacobi"), (1, None), (1, "jacobi")])
def test_cg_nonzero_initial_guess_and_zero_rhs(dg, mode, precond):
    import torch
    N, k = 3, 3
    D = SIPG(N, k)
    K = small_mesh_field(N, k, 9)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    b = inputs.uniform_vector(N, k, 10)
    x0 = torch.from_numpy(inputs.uniform_vector(N, k, 11)).cuda()
    rtol = 1e-11 if mode == 0 else 1e-10
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), x=x0, rtol=rtol, mode=mode, precond=precond)
    assert oracle_rel_residual(D, K, b, x.cpu().numpy()) <= 1.05 * rtol
    z = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    x, st = m.cg_solve(z.clone(), x=torch.ones_like(z), rtol=1e-10, mode=mode, precond=precond)
    assert st["status"] == 0
    assert torch.count_nonzero(x).item() == 0


def test_cg_maxit_reports_not_converged(dg):
    import torch
    N, k = 4, 2
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.unit_coefficient(N, k)).cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    x, st = m.cg_solve(b, rtol=1e-12, maxit=5, raise_on_error=False)
    assert st["status"] == dg.DG_ERR_NOT_CONVERGED
    assert st["iterations"] == 5
    with pytest.raises(dg.DGError, match="NOT_CONVERGED"):
        m.cg_solve(b, rtol=1e-12, maxit=5)


def test_cg_non_finite_rhs_reports_breakdown(dg):
    import torch
    N, k = 2, 2
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.unit_coefficient(N, k)).cuda())
    b = torch.from_numpy(inputs.uniform_vector(N, k, 3)).cuda()
    b[5] = float("nan")
    x, st = m.cg_solve(b, rtol=1e-10, raise_on_error=False)
    assert st["status"] == dg.DG_ERR_BREAKDOWN


def test_invalid_coefficient_and_aliasing_are_rejected(dg):
    import torch
    N, k = 2, 2
    m = dg.Mesh(N, k)
    K = torch.from_numpy(inputs.unit_coefficient(N, k)).cuda()
    K[7] = -1.0
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.set_coefficient(K)
    x = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError, match="coefficient not set"):
        m.apply(x)
    K[7] = float("inf")
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.set_coefficient(K)
    K[7] = 1.0
    m.set_coefficient(K)
    with pytest.raises(dg.DGError, match="alias"):
        m.apply(x, x)
    with pytest.raises(TypeError):
        m.apply(x.to(torch.int64))


def test_cg_reports_indefinite_coarse_mesh(dg):
    """3^3 Q4 with correlation length 0.1: K varies by ~1000x inside a cell and
    the SIPG matrix has two negative eigenvalues (pinned in the oracle tests).
    Both solvers must report the failure instead of returning a solution."""
    import torch
    N, k = 3, 4
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=4)).cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    for mode in (0, 1):
        x, st = m.cg_solve(b, rtol=1e-10, maxit=3000, mode=mode, raise_on_error=False)
        assert st["status"] in (dg.DG_ERR_BREAKDOWN, dg.DG_ERR_NOT_CONVERGED), st


@pytest.mark.parametrize("N,k", [(1, 2), (3, 2), (2, 3), (3, 4), (4, 1), (2, 8), (7, 3), (5, 5)])
def test_diagonal_matches_oracle(dg, N, k):
    """dg_diagonal against the oracle's a(phi, phi) by full quadrature: one
    cell (boundary faces only), every block shape of the diagonal kernel
    (8 cells per block at Q1 down to 1 at Q8) and ragged last blocks."""
    import torch
    D = SIPG(N, k)
    K = small_mesh_field(N, k, 17)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    d = m.diagonal().cpu().numpy()
    dref = D.diagonal(K)
    assert np.abs(d - dref).max() <= 1e-12 * np.abs(dref).max()
    # re-set coefficient: the cached diagonal must follow it
    m.set_coefficient(torch.from_numpy(2.0 * K).cuda())
    d2 = m.diagonal().cpu().numpy()
    assert np.abs(d2 - 2.0 * dref).max() <= 2e-12 * np.abs(dref).max()


@pytest.mark.slow
def test_diagonal_full_size_sampled_cells(dg):
    """48^3 Q4 lognormal K, the CG workload: sampled cells (corners, edges,
    interior, random) against the oracle's diagonal of those cells."""
    import torch
    N, k = 48, 4
    K = inputs.lognormal_coefficient(N, k, seed=4)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    d = m.diagonal().cpu().numpy().reshape(N ** 3, -1)
    rng = np.random.default_rng(11)
    cells = np.concatenate([[0, N - 1, N * N - 1, N ** 3 - 1, N ** 3 // 2 + N // 2],
                            rng.choice(N ** 3, 59, replace=False)])
    dref = SIPG(N, k).diagonal(K, cells=cells)
    assert np.abs(d[cells] - dref).max() <= 1e-12 * np.abs(dref).max()
    m.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_jacobi_pcg_residual_checked_by_oracle(dg, mode):
    import torch
    N, k = 4, 3
    D = SIPG(N, k)
    K = small_mesh_field(N, k, 5)
    b = inputs.constant_load_vector(N, k)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    bd = torch.from_numpy(b).cuda()
    x, st = m.cg_solve(bd, rtol=1e-10, mode=mode, precond="jacobi")
    assert st["status"] == 0
    assert oracle_rel_residual(D, K, b, x.cpu().numpy()) <= 1.05e-10
    _, st0 = m.cg_solve(bd, rtol=1e-10, mode=mode)
    assert st["iterations"] < st0["iterations"]
    # the oracle's PCG with the same diagonal needs a similar number of iterations
    if mode == 0:
        _, it_ref, _, _ = __import__("oracle").cg(lambda z: D.apply(K, z), b, rtol=1e-10,
                                                   minv=1.0 / D.assemble(K).diagonal())
        assert abs(st["iterations"] - it_ref) <= max(3, it_ref // 10)


@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_cg_fp64_unaligned_solution_vector(dg, precond):
    """x as a view 8 bytes past a 16-byte boundary takes the scalar update
    kernels; 5^3 Q2 has an odd DOF count, so the vector kernels' scalar tail
    runs in the aligned case.  Both reach the same iterate."""
    import torch
    N, k = 5, 2
    D = SIPG(N, k)
    K = small_mesh_field(N, k, 6)
    b = inputs.constant_load_vector(N, k)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    bd = torch.from_numpy(b).cuda()
    xa, sta = m.cg_solve(bd, torch.zeros_like(bd), rtol=1e-10, precond=precond)
    big = torch.zeros(m.n_dofs + 1, dtype=torch.float64, device="cuda")
    xu = big[1:]
    assert xu.data_ptr() % 16 == 8
    _, stu = m.cg_solve(bd, xu, rtol=1e-10, precond=precond)
    assert stu["status"] == 0 and sta["status"] == 0
    assert oracle_rel_residual(D, K, b, xu.cpu().numpy()) <= 1.05e-10
    assert abs(stu["iterations"] - sta["iterations"]) <= 2
    assert float((xu - xa).norm() / xa.norm()) <= 1e-8


# Every degree with at least one full bulk-copy group of the mixed direction
# kernel (4 x cells-per-block cells) and a ragged last group, plus meshes
# smaller than one group (plain loads only).
@pytest.mark.parametrize("N,k", [(6, 1), (4, 2), (4, 3), (3, 4), (3, 5), (3, 6), (3, 7), (2, 8),
                                 (3, 2), (2, 6)])
@pytest.mark.parametrize("mode,precond", [(0, None), (0, "jacobi"), (1, None), (1, "jacobi")])
def test_cg_first_iterates_match_oracle_recurrence(dg, N, k, mode, precond):
    """Three CG iterations from x = 0 for a random right-hand side: x_3 is a
    polynomial of degree two in A applied to b (M^-1 A with Jacobi), so a
    wrong entry of the operator shows up element by element.  The mixed mode
    runs the fused FP32 iteration kernels (tolerance 1e-4, from FP32
    rounding); the FP64 mode the FP64 apply (1e-10)."""
    import torch
    D = SIPG(N, k)
    K = small_mesh_field(N, k, 21)
    b = inputs.uniform_vector(N, k, 22)
    minv = 1.0 / D.diagonal(K) if precond else None
    xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3, minv=minv)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, mode=mode,
                       precond=precond, raise_on_error=False)
    assert st["iterations"] == 3, st
    tol = 1e-10 if mode == 0 else 1e-4
    assert relmax(x.cpu().numpy(), xref) <= tol


def test_bulk_copy_wait_timeout_is_reported_and_gpu_stays_usable(dg, monkeypatch):
    """A test hook makes the mixed CG's direction kernel skip its first bulk
    copy, so its bounded wait on the copy barrier runs out with no copy in
    flight: the solve must return DG_ERR_TIMEOUT (no trap, no hang), and the
    next solve on the same mesh must succeed."""
    import torch
    N, k = 4, 3
    K = small_mesh_field(N, k, 5)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()
    monkeypatch.setenv("DG_TEST_BULK_STALL", "1")
    with pytest.raises(dg.DGError, match="TIMEOUT"):
        m.cg_solve(b, rtol=1e-10, mode=dg.DG_CG_MIXED_IR)
    monkeypatch.delenv("DG_TEST_BULK_STALL")
    torch.cuda.synchronize()
    x, st = m.cg_solve(b, rtol=1e-10, mode=dg.DG_CG_MIXED_IR)
    assert st["status"] == 0
    assert oracle_rel_residual(SIPG(N, k), K, inputs.constant_load_vector(N, k),
                               x.cpu().numpy()) <= 1.05e-10


@pytest.mark.slow
@pytest.mark.parametrize("mode,precond", [(0, None), (1, None), (1, "jacobi")])
def test_cg_first_iterates_full_size_48cubed_q4(dg, mode, precond):
    """The CG workload (48^3 Q4, lognormal K seed 4) in the benchmark's launch
    configuration: three iterations from x = 0 for a random right-hand side,
    every DOF against the oracle's recurrence.  The mixed mode runs the fused
    FP32 kernels (bulk-copy direction kernel, persistent grid) at full size."""
    import torch
    N, k = 48, 4
    K = inputs.lognormal_coefficient(N, k, seed=4)
    b = inputs.uniform_vector(N, k, 23)
    D = SIPG(N, k)
    minv = 1.0 / D.diagonal(K) if precond else None
    xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3, minv=minv)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, mode=mode,
                       precond=precond, raise_on_error=False)
    assert st["iterations"] == 3, st
    tol = 1e-10 if mode == 0 else 1e-4
    assert relmax(x.cpu().numpy(), xref) <= tol
    m.close()


@pytest.mark.parametrize("N,k", [(1, 1), (2, 1), (1, 2), (2, 2), (1, 4)])
@pytest.mark.parametrize("bc", ["dirichlet", "flow_x"])
@pytest.mark.parametrize("precond", [None, "jacobi", "kron"])
def test_mixed_cg_converges_on_tiny_meshes(dg, N, k, bc, precond):
    """Systems of 8 to 512 DOFs, which the FP32 iteration converges within one
    graph chunk: the FP32 kernels must stop at the refinement request (an
    iteration on FP32 noise corrupted the kept search direction, or made
    <p, Ap> <= 0), and the solve reaches 1e-11 with the oracle's residual."""
    import torch
    D = SIPG(N, k, bc=bc)
    K = inputs.lognormal_coefficient(N, k, seed=31, corr_len=0.5)
    m = dg.Mesh(N, k)
    m.set_boundary(bc)
    m.set_coefficient(torch.from_numpy(K).cuda())
    if bc == "flow_x":
        b = D.dirichlet_rhs(K, (1.0, 0.0, 0.0, 0.0, 0.0, 0.0))
    else:
        b = inputs.uniform_vector(N, k, 32)
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-11, maxit=20000, mode=1,
                       precond=precond)
    assert st["status"] == 0 and st["iterations"] < 2000, st
    assert np.linalg.norm(b - D.apply(K, x.cpu().numpy())) <= 1.05e-11 * np.linalg.norm(b)
