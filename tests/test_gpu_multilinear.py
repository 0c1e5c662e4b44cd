"""The operator on a multilinear mesh (the paper's problem C) against the FP64
oracle's MultilinearSIPG, which assembles the SWIPDG form from the physical
gradients, normals, areas and penalty lengths at every quadrature point."""
import numpy as np
import pytest

from oracle.dg_oracle import MultilinearSIPG, _trilinear, lattice
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
SHEAR = [[1.0, 0.3, 0.1], [0.0, 1.1, -0.2], [0.05, 0.0, 0.9]]


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def perturbed(N, eps, seed):
    rng = np.random.default_rng(seed)
    X = lattice(N)
    return X + eps / N * rng.uniform(-1.0, 1.0, X.shape)


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def ml_mesh(dg, N, k, X, K):
    import torch
    m = dg.Mesh(N, k)
    m.set_vertices(X)
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m


@pytest.mark.parametrize("N,k", [(1, 1), (2, 1), (2, 2), (3, 2), (2, 3), (3, 3), (2, 4), (2, 6)])
def test_multilinear_apply_matches_oracle(dg, N, k):
    import torch
    X = perturbed(N, 0.3, 70 + N + k)
    K = inputs.lognormal_coefficient(N, k, seed=71, corr_len=0.5)
    x = inputs.uniform_vector(N, k, 72)
    m = ml_mesh(dg, N, k, X, K)
    yref = MultilinearSIPG(N, k, X).apply(K, x)
    xd = torch.from_numpy(x).cuda()
    assert relmax(m.apply(xd).cpu().numpy(), yref) <= TOL64
    assert relmax(m.apply_adjoint(xd).cpu().numpy(), yref) <= TOL64


def test_affine_vertices_give_the_affine_geometry(dg):
    import torch
    N, k = 3, 3
    K = inputs.lognormal_coefficient(N, k, seed=73)
    x = torch.from_numpy(inputs.uniform_vector(N, k, 74)).cuda()
    m1 = ml_mesh(dg, N, k, lattice(N, SHEAR), K)
    m2 = dg.Mesh(N, k)
    m2.set_geometry(SHEAR)
    m2.set_coefficient(torch.from_numpy(K).cuda())
    y1, y2 = m1.apply(x), m2.apply(x)
    assert float((y1 - y2).abs().max() / y2.abs().max()) <= 1e-13


def test_multilinear_cg_and_load_vector_checked_by_oracle(dg):
    import torch
    import scipy.sparse.linalg as spla
    N, k = 4, 2
    X = lattice(N, perturb=lambda P: 0.08 * np.stack(
        [np.sin(np.pi * P[..., 0]) * np.sin(2 * np.pi * P[..., 1]) * np.sin(np.pi * P[..., 2]),
         np.sin(2 * np.pi * P[..., 0]) * np.sin(np.pi * P[..., 1]) * np.sin(np.pi * P[..., 2]),
         np.sin(np.pi * P[..., 0]) * np.sin(np.pi * P[..., 1]) * np.sin(2 * np.pi * P[..., 2])],
        axis=-1))
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * u(x, y, z)
    D = MultilinearSIPG(N, k, X)
    F = np.empty((N ** 3, D.n3))
    for c in range(N ** 3):
        xq, _ = _trilinear(D.corners(c), D.qxi)
        F[c] = f(xq[:, 0], xq[:, 1], xq[:, 2])
    K = np.ones(D.n_dofs)
    m = ml_mesh(dg, N, k, X, K)
    b = m.load_vector(torch.from_numpy(F.reshape(-1)).cuda()).cpu().numpy()
    bref = D.load_vector(f, nq=k + 1)
    assert relmax(b, bref) <= TOL64
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-11)
    Am = D.assemble(K)
    assert np.linalg.norm(bref - Am @ x.cpu().numpy()) / np.linalg.norm(bref) <= 1.05e-11
    e_gpu = D.l2_error(x.cpu().numpy(), u)
    e_ref = D.l2_error(spla.spsolve(Am.tocsc(), bref), u)
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref


def test_inverted_cell_is_rejected(dg):
    N = 2
    X = lattice(N)
    X[1, 1, 1] = [1.2, 1.2, 1.2]     # pushes the centre vertex through three cells
    m = dg.Mesh(N, 1)
    with pytest.raises(dg.DGError, match="Jacobian"):
        m.set_vertices(X)
