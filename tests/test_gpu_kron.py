"""Kronecker cell-block PCG (DG_CG_PRECOND_KRON, FP64 and mixed precision)
against the FP64 oracle (oracle.dg_oracle.kron_block_inverse: the cell blocks
with the cell-mean K as dense Kronecker sums, inverted by LAPACK).

* One cell with constant K: the Kronecker block is the whole operator, so
  PCG converges in one iteration at every degree (the eigen-decomposition of
  the 1D factors on the GPU reproduces the inverse).
* The first PCG iterates follow the oracle's recurrence element by element
  (FP64 at 1e-10; mixed, whose direction, operator and preconditioner run in
  FP32, at 1e-4), on ragged cell groups, both boundary conditions and high
  degrees.
* With a cell-wise constant K the Kronecker blocks are the exact cell blocks:
  the iterates equal those of DG_CG_PRECOND_BLOCK.
* Converged solves have the oracle's residual and need fewer iterations than
  point Jacobi."""
import numpy as np
import pytest

from oracle import SIPG, cg
from oracle.dg_oracle import kron_block_inverse
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


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 8])
def test_kron_is_exact_on_one_cell_with_constant_K(dg, k):
    import torch
    K = 2.5 * np.ones(inputs.unit_coefficient(1, k).shape)
    b = inputs.uniform_vector(1, k, 50 + k)
    m = dg.Mesh(1, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-11, precond="kron")
    assert st["iterations"] == 1, st
    D = SIPG(1, k)
    assert np.linalg.norm(b - D.apply(K, x.cpu().numpy())) <= 1e-11 * np.linalg.norm(b)


CASES = [(3, 1, "dirichlet"), (4, 2, "dirichlet"), (3, 3, "dirichlet"), (2, 4, "dirichlet"),
         (3, 2, "flow_x"), (5, 1, "flow_x"), (2, 5, "dirichlet"), (2, 7, "dirichlet")]


@pytest.mark.parametrize("N,k,bc", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_kron_pcg_first_iterates_match_oracle(dg, N, k, bc, mode):
    import torch
    D = SIPG(N, k, bc=bc)
    K = field(N, k, 42)
    b = inputs.uniform_vector(N, k, 43)
    xref, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-14, maxit=3,
                       minv=kron_block_inverse(D, K))
    m = dg.Mesh(N, k)
    m.set_boundary(bc)
    m.set_coefficient(torch.from_numpy(K).cuda())
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-14, maxit=3, mode=mode,
                       precond="kron", raise_on_error=False)
    assert st["iterations"] == 3, st
    assert relmax(x.cpu().numpy(), xref) <= (1e-10 if mode == 0 else 1e-4)


@pytest.mark.parametrize("N,k", [(3, 2), (2, 4), (4, 1)])
def test_kron_equals_exact_blocks_for_cellwise_constant_K(dg, N, k):
    import torch
    rng = np.random.default_rng(60 + k)
    n3 = (k + 1) ** 3
    K = np.repeat(np.exp(rng.normal(0.0, 1.0, N ** 3)), n3)
    b = torch.from_numpy(inputs.uniform_vector(N, k, 61)).cuda()
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    xk, sk = m.cg_solve(b, rtol=1e-14, maxit=6, precond="kron", raise_on_error=False)
    xb, sb = m.cg_solve(b, rtol=1e-14, maxit=6, precond="block", raise_on_error=False)
    assert sk["iterations"] == sb["iterations"]
    assert relmax(xk.cpu().numpy(), xb.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("N,k,mode", [(8, 3, 0), (8, 3, 1), (6, 4, 1), (10, 2, 0)])
def test_kron_converges_with_oracle_residual_and_beats_jacobi(dg, N, k, mode):
    import torch
    D = SIPG(N, k)
    K = field(N, k, 4)
    b = inputs.constant_load_vector(N, k)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    bd = torch.from_numpy(b).cuda()
    x, st = m.cg_solve(bd, rtol=1e-10, mode=mode, precond="kron")
    assert st["status"] == 0
    r = np.linalg.norm(b - D.apply(K, x.cpu().numpy())) / np.linalg.norm(b)
    assert r <= 1.05e-10
    _, sj = m.cg_solve(bd, rtol=1e-10, mode=mode, precond="jacobi")
    assert st["iterations"] < 0.85 * sj["iterations"], (st, sj)


def test_kron_invalid_combinations_are_rejected(dg):
    import torch
    N, k = 2, 2
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(field(N, k, 1)).cuda())
    b = torch.from_numpy(inputs.uniform_vector(N, k, 2)).cuda()
    for mode in (dg.DG_CG_PRECOND_KRON | dg.DG_CG_PRECOND_JACOBI,
                 dg.DG_CG_MIXED_IR_RESTART | dg.DG_CG_PRECOND_KRON,
                 dg.DG_CG_PRECOND_KRON | dg.DG_CG_PRECOND_BLOCK):
        with pytest.raises(dg.DGError, match="INVALID_ARG"):
            m.cg_solve(b, rtol=1e-8, mode=mode)
