"""Pins of the Kronecker cell-block preconditioner of the oracle
(oracle.dg_oracle.kron_cell_matrices / kron_block_inverse; a reading of the
factorised cell-block solves of Section 3.4).

* With a cell-wise constant K the Kronecker sum S_x (+) S_y (+) S_z of every
  cell equals that cell's diagonal block of the operator assembled from full
  3D quadrature (an independent code path): Dirichlet and flow boundaries,
  several degrees.  A wrong sign, a dropped 1/2 on interior faces or a face
  on the wrong side fails this.
* The default volume coefficient is the Gauss-weighted arithmetic mean of K
  over the cell: for K linear in x inside a cell the blocks equal those with
  the cell-constant value at the cell centre (Gauss quadrature is exact for
  linear functions).
* The blocks are symmetric positive definite for lognormal K, and PCG with
  them needs fewer iterations than with point Jacobi."""
import numpy as np
import pytest

from oracle import SIPG, cg
from oracle.dg_oracle import (cell_blocks, kron_block_inverse, kron_cell_matrices, kron_sum)
from paper_1911_01492_gb300 import inputs


@pytest.mark.parametrize("N,k,bc", [(3, 1, "dirichlet"), (3, 2, "dirichlet"), (2, 3, "dirichlet"),
                                    (3, 2, "flow_x"), (2, 4, "flow_x")])
def test_kron_blocks_are_the_assembled_blocks_of_cellwise_constant_K(N, k, bc):
    D = SIPG(N, k, bc=bc)
    rng = np.random.default_rng(N * 10 + k)
    kc = np.exp(rng.normal(0.0, 1.0, N ** 3))
    K = np.repeat(kc, D.n3)
    B = cell_blocks(D.assemble(K), D.n3)
    S = kron_cell_matrices(D, K)
    err = max(np.abs(kron_sum(S[c]) - B[c]).max() for c in range(N ** 3))
    assert err <= 1e-13 * np.abs(B).max()


def test_default_volume_coefficient_is_the_cell_mean():
    N, k = 3, 2
    D = SIPG(N, k)
    # K = 1 + x_phys inside each cell, at the volume Gauss points ([c][e][b][a], a = x)
    n = D.n
    cx = np.arange(N ** 3) % N
    xq = (cx[:, None] + D.xi[None, :]) * D.h                        # (cells, n) by a
    K = np.broadcast_to((1.0 + xq)[:, None, None, :], (N ** 3, n, n, n)).reshape(-1)
    centre = 1.0 + (cx + 0.5) * D.h
    S = kron_cell_matrices(D, K)
    Sref = kron_cell_matrices(D, K, kvol=centre)
    assert np.abs(S - Sref).max() <= 1e-14 * np.abs(Sref).max()
    # and it differs from the geometric mean Kbar used on the faces
    S_geo = kron_cell_matrices(D, K, kvol=D.kbar(K))
    assert np.abs(S - S_geo).max() > 1e-8 * np.abs(S).max()


@pytest.mark.parametrize("bc", ["dirichlet", "flow_x"])
def test_kron_blocks_are_spd(bc):
    N, k = 4, 3
    D = SIPG(N, k, bc=bc)
    K = inputs.lognormal_coefficient(N, k, seed=3, corr_len=0.3)
    S = kron_cell_matrices(D, K)
    assert np.abs(S - np.swapaxes(S, -1, -2)).max() <= 1e-14 * np.abs(S).max()
    lam = np.linalg.eigvalsh(S)
    assert lam.min() > 0.0


def test_kron_pcg_beats_point_jacobi():
    N, k = 6, 3
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=4, corr_len=0.1 * 48 / N)
    A = D.assemble(K)
    b = inputs.constant_load_vector(N, k)
    _, it_j, rel_j, _ = cg(lambda v: A @ v, b, rtol=1e-10, minv=1.0 / A.diagonal())
    _, it_k, rel_k, _ = cg(lambda v: A @ v, b, rtol=1e-10, minv=kron_block_inverse(D, K))
    assert rel_k <= 1e-10 and rel_j <= 1e-10
    assert it_k < 0.8 * it_j
