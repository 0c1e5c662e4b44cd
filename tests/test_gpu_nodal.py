"""The scaled Gauss-point (collocation) basis on the GPU against the oracle.

dg_to_nodal / dg_to_modal against the oracle's Q and Q^T; dg_apply_nodal
against the oracle's Q A Q^T element by element (1e-12, degrees 1-8, odd and
one-cell meshes, both boundary conditions, and sampled cells of the 64^3 Q3
benchmark mesh); the CG in that basis (DG_CG_NODAL, FP64 and mixed) by its first iterates
against the oracle's recurrence (M = I: the Legendre-basis iterates, since Q is
orthogonal; Jacobi: the oracle's PCG on Q A Q^T with its diagonal) and by
residuals that the oracle recomputes in the Legendre basis.
"""
import numpy as np
import pytest

from oracle import SIPG, cg
from oracle.dg_oracle import kron_block_inverse
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def field(N, k, seed):
    # the per-cell statistics of the 64^3 workload (correlation length in cells)
    return inputs.lognormal_coefficient(N, k, seed=seed, corr_len=0.1 * 64 / N)


def mesh(dg, N, k, K, bc="dirichlet"):
    import torch
    m = dg.Mesh(N, k)
    if bc != "dirichlet":
        m.set_boundary(bc)
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m


@pytest.mark.parametrize("N,k", [(3, 1), (3, 2), (2, 3), (3, 4), (2, 5), (1, 6), (2, 7), (1, 8)])
def test_transforms_match_oracle_and_invert(dg, N, k):
    import torch
    D = SIPG(N, k)
    x = inputs.uniform_vector(N, k, 31)
    m = dg.Mesh(N, k)
    xh = m.to_nodal(torch.from_numpy(x).cuda())
    assert relmax(xh.cpu().numpy(), D.to_collocation(x)) <= TOL64
    back = m.to_modal(xh).cpu().numpy()
    assert relmax(back, x) <= TOL64
    xh2 = inputs.uniform_vector(N, k, 32)
    got = m.to_modal(torch.from_numpy(xh2).cuda()).cpu().numpy()
    assert relmax(got, D.from_collocation(xh2)) <= TOL64


@pytest.mark.parametrize("N,k,seed,bc", [
    (1, 1, 3, "dirichlet"), (4, 1, 4, "dirichlet"), (3, 2, 5, "dirichlet"), (5, 2, 6, "flow_x"),
    (4, 3, 7, "dirichlet"), (3, 3, 8, "flow_x"), (3, 4, 9, "dirichlet"), (2, 5, 10, "dirichlet"),
    (2, 6, 11, "flow_x"), (2, 7, 12, "dirichlet"), (1, 8, 13, "dirichlet"), (2, 8, 14, "dirichlet")])
def test_apply_nodal_matches_oracle(dg, N, k, seed, bc):
    import torch
    D = SIPG(N, k, bc=bc)
    K = field(N, k, seed)
    m = mesh(dg, N, k, K, bc)
    xh = inputs.uniform_vector(N, k, 100 + seed)
    y = m.apply_nodal(torch.from_numpy(xh).cuda()).cpu().numpy()
    assert relmax(y, D.collocation_apply(K, xh)) <= TOL64
    # the same operator through the Legendre basis: Q^T (Q A Q^T) Q x = A x
    x = inputs.uniform_vector(N, k, 200 + seed)
    yx = m.to_modal(m.apply_nodal(m.to_nodal(torch.from_numpy(x).cuda()))).cpu().numpy()
    assert relmax(yx, D.apply(K, x)) <= TOL64


def test_apply_nodal_is_symmetric_and_follows_a_new_coefficient(dg):
    import torch
    N, k = 4, 3
    K = field(N, k, 15)
    m = mesh(dg, N, k, K)
    u = torch.from_numpy(inputs.uniform_vector(N, k, 16)).cuda()
    v = torch.from_numpy(inputs.uniform_vector(N, k, 17)).cuda()
    a = float(v @ m.apply_nodal(u))
    b = float(u @ m.apply_nodal(v))
    assert abs(a - b) <= 1e-12 * abs(a)
    # set_coefficient drops the basis's line operators: the next call uses the new K
    K2 = field(N, k, 18)
    m.set_coefficient(torch.from_numpy(K2).cuda())
    D = SIPG(N, k)
    y = m.apply_nodal(u).cpu().numpy()
    assert relmax(y, D.collocation_apply(K2, u.cpu().numpy())) <= TOL64


def test_apply_nodal_full_size_64cubed_q3_sampled_cells(dg):
    """The benchmark mesh (64^3 Q3, lognormal K seed 2): every DOF of 24 random
    cells (boundary, edge and interior cells included) against the oracle,
    which applies A to Q^T x_hat on those cells only."""
    import torch
    N, k = 64, 3
    K = inputs.lognormal_coefficient(N, k, seed=2)
    D = SIPG(N, k)
    m = mesh(dg, N, k, K)
    xh = inputs.uniform_vector(N, k, 33)
    y = m.apply_nodal(torch.from_numpy(xh).cuda()).cpu().numpy().reshape(N ** 3, -1)
    rng = np.random.default_rng(34)
    cells = np.concatenate([[0, N - 1, N * N * N - 1, N * N * (N // 2) + N * (N // 2)],
                            rng.choice(N ** 3, 20, replace=False)])
    x = D.from_collocation(xh)
    ya = D.apply(K, x, cells=cells)
    Q = D.collocation_matrix()
    ref = ya.reshape(len(cells), -1) @ Q.T
    assert relmax(y[cells], ref) <= TOL64


@pytest.mark.parametrize("N,k", [(4, 3), (3, 2), (3, 4), (2, 6), (3, 1), (2, 8)])
@pytest.mark.parametrize("precond", [None, "jacobi", "kron"])
@pytest.mark.parametrize("mode", [0, 1])
def test_nodal_cg_first_iterates_match_oracle_recurrence(dg, N, k, precond, mode):
    """Three CG iterations from x = 0.  M = I and the Kronecker cell blocks: Q
    is orthogonal and Q M Q^T is the point basis's preconditioner, so x_3
    equals the Legendre-basis (P)CG iterate.  Jacobi: the oracle's PCG on
    Q A Q^T with M = diag(Q A Q^T), mapped back with Q^T.  The mixed mode runs
    the FP32 point-basis kernels (tolerance 1e-4 from FP32 rounding), the FP64
    mode the FP64 ones (1e-10)."""
    import torch
    D = SIPG(N, k)
    K = field(N, k, 41)
    b = inputs.uniform_vector(N, k, 42)
    if precond is None:
        xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3)
    elif precond == "kron":
        xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3,
                           minv=kron_block_inverse(D, K))
    else:
        xh, _, _, _ = cg(lambda v: D.collocation_apply(K, v), D.to_collocation(b), rtol=1e-14,
                         maxit=3, minv=1.0 / D.collocation_diagonal(K))
        xref = D.from_collocation(xh)
    m = mesh(dg, N, k, K)
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, precond=precond,
                       mode=mode, nodal=True, raise_on_error=False)
    assert st["iterations"] == 3, st
    assert st["status"] == dg.DG_ERR_NOT_CONVERGED
    assert relmax(x.cpu().numpy(), xref) <= (1e-10 if mode == 0 else 1e-4)


@pytest.mark.parametrize("N,k,seed,bc", [(4, 3, 5, "dirichlet"), (5, 2, 6, "dirichlet"),
                                         (3, 4, 4, "dirichlet"), (4, 2, 7, "flow_x")])
@pytest.mark.parametrize("precond", [None, "jacobi", "kron"])
@pytest.mark.parametrize("mode", [0, 1])
def test_nodal_cg_residual_checked_by_oracle(dg, N, k, seed, bc, precond, mode):
    import torch
    D = SIPG(N, k, bc=bc)
    K = field(N, k, seed)
    b = inputs.constant_load_vector(N, k)
    m = mesh(dg, N, k, K, bc)
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-10, precond=precond, mode=mode,
                       nodal=True)
    x = x.cpu().numpy()
    assert st["status"] == 0
    assert st["rel_residual"] <= 1e-10
    rel = np.linalg.norm(b - D.apply(K, x)) / np.linalg.norm(b)
    assert rel <= 1.05e-10
    # same solution as the Legendre-basis solve within the conditioning bound
    xm, _ = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-12, precond=precond)
    xm = xm.cpu().numpy()
    assert np.linalg.norm(x - xm) <= 1e-5 * np.linalg.norm(xm)


def test_nodal_cg_initial_guess_zero_rhs_and_rejected_modes(dg):
    import torch
    N, k = 3, 3
    D = SIPG(N, k)
    K = field(N, k, 9)
    m = mesh(dg, N, k, K)
    b = inputs.uniform_vector(N, k, 10)
    x0 = torch.from_numpy(inputs.uniform_vector(N, k, 11)).cuda()
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), x=x0, rtol=1e-11, nodal=True)
    rel = np.linalg.norm(b - D.apply(K, x.cpu().numpy())) / np.linalg.norm(b)
    assert rel <= 1.05e-11
    z = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    x, st = m.cg_solve(z.clone(), x=torch.ones_like(z), rtol=1e-10, nodal=True)
    assert st["status"] == 0 and torch.count_nonzero(x).item() == 0
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.cg_solve(torch.from_numpy(b).cuda(), mode=dg.DG_CG_MIXED_IR_RESTART, nodal=True)
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        m.cg_solve(torch.from_numpy(b).cuda(), precond="block", nodal=True)


def test_nodal_cg_first_iterates_full_size_48cubed_q4(dg):
    """The CG workload (48^3 Q4, lognormal K seed 4) in the benchmark's
    configuration: three iterations in the point basis, FP64 and mixed (the
    FP32 point-basis kernels at full size, bulk-copy direction kernel in its
    persistent grid), every DOF against the oracle's Legendre-basis
    recurrence."""
    import torch
    N, k = 48, 4
    K = inputs.lognormal_coefficient(N, k, seed=4)
    b = inputs.uniform_vector(N, k, 23)
    D = SIPG(N, k)
    xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3)
    m = mesh(dg, N, k, K)
    for mode, tol in ((0, 1e-10), (1, 1e-4)):
        x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, mode=mode,
                           nodal=True, raise_on_error=False)
        assert st["iterations"] == 3, st
        assert relmax(x.cpu().numpy(), xref) <= tol


# uneven levels: sizes and degrees differ inside one batch
BATCH_LEVELS = [(4, 1), (4, 2), (3, 3), (3, 4), (5, 2), (2, 4)]


def make_batch(dg, levels, seed0):
    import torch
    meshes, bs, xs, Ks = [], [], [], []
    for s, (N, k) in enumerate(levels):
        K = field(N, k, seed0 + s)
        meshes.append(mesh(dg, N, k, K))
        Ks.append(K)
        bs.append(torch.from_numpy(inputs.uniform_vector(N, k, seed0 + 1000 + s)).cuda())
        xs.append(torch.zeros(meshes[-1].n_dofs, dtype=torch.float64, device="cuda"))
    return meshes, bs, xs, Ks


@pytest.mark.parametrize("levels", [BATCH_LEVELS, [(3, 2), (2, 5), (2, 7)]])
def test_batched_nodal_matches_oracle_and_single_sample_solves(dg, levels):
    """The lock-step batched CG in the point basis (both kernel widths): every
    sample's residual recomputed by the oracle in the Legendre basis, the
    iteration count of a one-sample FP64 CG (the same iterates in exact
    arithmetic) and the same solution."""
    meshes, bs, xs, Ks = make_batch(dg, levels, 3000)
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, nodal=True)
    for s, ((N, k), m, b, x, K, st) in enumerate(zip(levels, meshes, bs, xs, Ks, stats)):
        assert st["status"] == 0, (s, st)
        bn = b.cpu().numpy()
        r = np.linalg.norm(bn - SIPG(N, k).apply(K, x.cpu().numpy())) / np.linalg.norm(bn)
        assert r <= 1.05e-10, (s, r)
        xseq, sst = m.cg_solve(b, rtol=1e-10)
        assert abs(st["iterations"] - sst["iterations"]) <= max(3, sst["iterations"] // 20)
        assert float((x - xseq).norm() / xseq.norm()) <= 1e-6


def test_batched_nodal_zero_rhs_initial_guess_and_rejected_mode(dg):
    import torch
    meshes, bs, xs, Ks = make_batch(dg, [(3, 2), (2, 3)], 3100)
    bs[1].zero_()
    xs[1].fill_(1.0)
    xs[0].copy_(torch.from_numpy(inputs.uniform_vector(3, 2, 3101)).cuda())
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, nodal=True)
    assert all(st["status"] == 0 for st in stats)
    assert torch.count_nonzero(xs[1]).item() == 0
    bn = bs[0].cpu().numpy()
    r = np.linalg.norm(bn - SIPG(3, 2).apply(Ks[0], xs[0].cpu().numpy())) / np.linalg.norm(bn)
    assert r <= 1.05e-10
    with pytest.raises(dg.DGError, match="INVALID_ARG"):
        dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, nodal=True, precond="jacobi")
