"""Cell-block Jacobi PCG (DG_CG_FP64 | DG_CG_PRECOND_BLOCK) against the FP64
oracle, whose blocks are the diagonal blocks of its assembled matrix inverted
by LAPACK: on one cell the preconditioner is the exact inverse (one
iteration); on larger meshes the first iterates follow the oracle's PCG
recurrence element by element, and converged solutions have the oracle's
residual."""
import numpy as np
import pytest

from oracle import SIPG, cg
from oracle.dg_oracle import block_jacobi_inverse
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def field(N, k, seed):
    return inputs.lognormal_coefficient(N, k, seed=seed, corr_len=0.1 * 64 / N)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_block_jacobi_is_exact_on_one_cell(dg, k):
    import torch
    K = field(1, k, 40 + k)
    b = inputs.uniform_vector(1, k, 41)
    m = dg.Mesh(1, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-12, precond="block")
    assert st["iterations"] == 1, st
    D = SIPG(1, k)
    r = np.linalg.norm(b - D.apply(K, x.cpu().numpy())) / np.linalg.norm(b)
    assert r <= 1e-12


@pytest.mark.parametrize("N,k,bc", [(3, 1, "dirichlet"), (4, 2, "dirichlet"), (3, 3, "dirichlet"),
                                    (2, 4, "dirichlet"), (3, 2, "flow_x"), (5, 1, "flow_x")])
def test_block_pcg_first_iterates_match_oracle(dg, N, k, bc):
    import torch
    D = SIPG(N, k, bc=bc)
    K = field(N, k, 42)
    b = inputs.uniform_vector(N, k, 43)
    A = D.assemble(K)
    xref, _, _, _ = cg(lambda v: A @ v, b, rtol=1e-14, maxit=3, minv=block_jacobi_inverse(A, D.n3))
    m = dg.Mesh(N, k)
    m.set_boundary(bc)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, precond="block",
                       raise_on_error=False)
    assert st["iterations"] == 3, st
    assert relmax(x.cpu().numpy(), xref) <= 1e-10


def test_block_pcg_converges_in_fewer_iterations_than_point_jacobi(dg):
    import torch
    N, k = 6, 2
    D = SIPG(N, k)
    K = field(N, k, 44)
    b = inputs.constant_load_vector(N, k)
    A = D.assemble(K)
    _, it_ref, _, _ = cg(lambda v: A @ v, b, rtol=1e-10, minv=block_jacobi_inverse(A, D.n3))
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    bd = torch.from_numpy(b).cuda()
    x, st = m.cg_solve(bd, rtol=1e-10, precond="block")
    r = np.linalg.norm(b - D.apply(K, x.cpu().numpy())) / np.linalg.norm(b)
    assert r <= 1.05e-10
    assert abs(st["iterations"] - it_ref) <= 2
    _, sj = m.cg_solve(bd, rtol=1e-10, precond="jacobi")
    assert st["iterations"] < sj["iterations"]


def test_block_rejects_other_modes_and_high_degree(dg):
    import torch
    m = dg.Mesh(2, 1)
    m.set_coefficient(torch.ones(m.n_dofs, dtype=torch.float64, device="cuda"))
    b = torch.ones(m.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError, match="DG_CG_FP64 only"):
        m.cg_solve(b, mode=dg.DG_CG_MIXED_IR, precond="block")
    m5 = dg.Mesh(1, 5)
    m5.set_coefficient(torch.ones(m5.n_dofs, dtype=torch.float64, device="cuda"))
    with pytest.raises(dg.DGError, match="degree"):
        m5.cg_solve(torch.ones(m5.n_dofs, dtype=torch.float64, device="cuda"), precond="block")
