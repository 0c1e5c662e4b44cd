"""The operator on an affine geometry (the paper's problem B) against the FP64
oracle's AffineSIPG, which assembles the SWIPDG form from the physical
gradients, face normals, face areas and penalty lengths by full quadrature."""
import numpy as np
import pytest

from oracle.dg_oracle import AffineSIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
SHEAR = [[1.0, 0.3, 0.1], [0.0, 1.1, -0.2], [0.05, 0.0, 0.9]]
SHEAR2 = [[0.8, -0.25, 0.0], [0.1, 1.2, 0.3], [-0.15, 0.2, 1.05]]
STRETCH = [[0.7, 0.0, 0.0], [0.0, 1.3, 0.0], [0.0, 0.0, 2.1]]


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def affine_mesh(dg, N, k, A, K):
    import torch
    m = dg.Mesh(N, k)
    m.set_geometry(A)
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m


@pytest.mark.parametrize("N,k,A", [(1, 1, SHEAR), (2, 1, SHEAR), (3, 2, SHEAR), (2, 3, STRETCH),
                                   (3, 3, SHEAR2), (1, 4, SHEAR), (4, 2, SHEAR2), (2, 5, SHEAR),
                                   (2, 8, SHEAR2)])
def test_affine_apply_matches_oracle(dg, N, k, A):
    import torch
    K = inputs.lognormal_coefficient(N, k, seed=60, corr_len=0.5)
    x = inputs.uniform_vector(N, k, 61)
    m = affine_mesh(dg, N, k, A, K)
    yref = AffineSIPG(N, k, A).apply(K, x)
    xd = torch.from_numpy(x).cuda()
    y = m.apply(xd).cpu().numpy()
    assert relmax(y, yref) <= TOL64
    ya = m.apply_adjoint(xd).cpu().numpy()
    assert relmax(ya, yref) <= TOL64


def test_identity_geometry_is_the_cube_operator(dg):
    import torch
    N, k = 3, 3
    K = inputs.lognormal_coefficient(N, k, seed=62)
    x = torch.from_numpy(inputs.uniform_vector(N, k, 63)).cuda()
    m0 = dg.Mesh(N, k)
    m0.set_coefficient(torch.from_numpy(K).cuda())
    m1 = affine_mesh(dg, N, k, np.eye(3).tolist(), K)
    assert torch.equal(m0.apply(x), m1.apply(x))


def test_affine_cg_and_load_vector_checked_by_oracle(dg):
    """Manufactured solution on the sheared domain: the GPU load vector equals
    the oracle's, the FP64 CG reaches the oracle-recomputed residual, and the
    L2 error equals the oracle's own direct solve's."""
    import torch
    import scipy.sparse.linalg as spla
    N, k = 4, 2
    A = np.array(SHEAR)
    Ai = np.linalg.inv(A)
    Mt = Ai @ Ai.T

    def refc(x, y, z):
        X = np.stack(np.broadcast_arrays(x, y, z), axis=-1) @ Ai.T
        return X[..., 0], X[..., 1], X[..., 2]

    def u(x, y, z):
        a, b, c = refc(x, y, z)
        return np.sin(np.pi * a) * np.sin(np.pi * b) * np.sin(np.pi * c)

    def f(x, y, z):
        a, b, c = refc(x, y, z)
        s = [np.sin(np.pi * a), np.sin(np.pi * b), np.sin(np.pi * c)]
        co = [np.cos(np.pi * a), np.cos(np.pi * b), np.cos(np.pi * c)]
        out = np.pi ** 2 * np.trace(Mt) * s[0] * s[1] * s[2]
        for d in range(3):
            for e in range(3):
                if d != e:
                    out = out - np.pi ** 2 * Mt[d, e] * co[d] * co[e] * s[3 - d - e]
        return out

    D = AffineSIPG(N, k, A)
    K = np.ones(D.n_dofs)
    m = affine_mesh(dg, N, k, SHEAR, K)
    # f at the mapped Gauss points, in the layout of K
    F = inputs.values_at_gauss_points(N, k, lambda x, y, z: f(*(
        np.moveaxis(np.stack(np.broadcast_arrays(x, y, z), axis=-1) @ A.T, -1, 0))))
    b = m.load_vector(torch.from_numpy(F).cuda()).cpu().numpy()
    bref = D.load_vector(f)
    assert relmax(b, bref) <= TOL64
    x, st = m.cg_solve(torch.from_numpy(b).cuda(), rtol=1e-11)
    xn = x.cpu().numpy()
    Am = D.assemble(K)
    assert np.linalg.norm(bref - Am @ xn) / np.linalg.norm(bref) <= 1.05e-11
    e_gpu = D.l2_error(xn, u)
    e_ref = D.l2_error(spla.spsolve(Am.tocsc(), bref), u)
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref


def test_affine_rejects_the_cube_only_paths(dg):
    import torch
    N, k = 2, 2
    m = affine_mesh(dg, N, k, SHEAR, np.ones(N ** 3 * (k + 1) ** 3))
    x = torch.ones(m.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError, match="affine"):
        m.apply(x.float())
    with pytest.raises(dg.DGError, match="affine"):
        m.cg_solve(x, mode=dg.DG_CG_MIXED_IR)
    with pytest.raises(dg.DGError, match="affine"):
        m.cg_solve(x, precond="jacobi")
    with pytest.raises(dg.DGError, match="affine"):
        m.coeff_grad(x, x)
    with pytest.raises(dg.DGError, match="affine"):
        dg.cg_solve_batched([m], [x], [torch.zeros_like(x)])
    with pytest.raises(dg.DGError, match="det A"):
        m.set_geometry([[1, 0, 0], [0, -1, 0], [0, 0, 1]])
