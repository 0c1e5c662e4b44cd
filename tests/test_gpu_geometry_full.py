"""The affine and multilinear FP64 operators at the benchmark's full size
(64^3 Q3, lognormal K), in the benchmark's launch configuration, checked at
sampled cells by the oracle.  A cell's output depends only on the cell and its
six neighbours (their coefficient, input and geometry; the SWIPDG form is
written in physical quantities), so the oracle's MultilinearSIPG on the 3^3
patch of physical cells around a sampled cell (the same vertex positions,
with boundary faces exactly where the full mesh has them) gives that cell's
output.  The affine mesh is checked the same way through its vertices (the
oracle pins equate the two forms for affine vertices).  Symmetry of the full
operator is checked on random vectors."""
import numpy as np
import pytest

from oracle.dg_oracle import MultilinearSIPG, lattice
from paper_1911_01492_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL64 = 1e-12
SHEAR = [[1.0, 0.3, 0.1], [0.0, 1.1, -0.2], [0.05, 0.0, 0.9]]
N, K_DEG = 64, 3


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


@pytest.fixture(scope="module")
def data():
    K = inputs.lognormal_coefficient(N, K_DEG, seed=2)
    x = inputs.uniform_vector(N, K_DEG, 3)
    return K, x


def sampled_cells(seed):
    rng = np.random.default_rng(seed)
    corners = [0, N - 1, N * N - 1, N ** 3 - 1, N ** 3 - N * N]
    faces = [N // 2 + N * (N // 2), N // 2 * N * N + N // 2, N // 2 + N * N * (N // 2)]
    return np.unique(np.concatenate([corners, faces, rng.choice(N ** 3, 4, replace=False)]))


def patch_output(X, K, x, c):
    """The oracle's output on cell c from the 3^3 patch of physical cells
    around it (shifted inwards at the mesh boundary)."""
    n3 = (K_DEG + 1) ** 3
    cx, cy, cz = c % N, (c // N) % N, c // (N * N)
    s = [min(max(v - 1, 0), N - 3) for v in (cx, cy, cz)]
    ids = [(s[0] + px) + N * ((s[1] + py) + N * (s[2] + pz))
           for pz in range(3) for py in range(3) for px in range(3)]
    Kp = K.reshape(N ** 3, n3)[ids].reshape(-1)
    xp = x.reshape(N ** 3, n3)[ids].reshape(-1)
    Xp = X[s[0]:s[0] + 4, s[1]:s[1] + 4, s[2]:s[2] + 4]
    cp = (cx - s[0]) + 3 * ((cy - s[1]) + 3 * (cz - s[2]))
    return MultilinearSIPG(3, K_DEG, Xp).apply(Kp, xp).reshape(27, n3)[cp]


def check_mesh(m, X, K, x, seed):
    import torch
    n3 = (K_DEG + 1) ** 3
    xd = torch.from_numpy(x).cuda()
    y = m.apply(xd).cpu().numpy().reshape(N ** 3, n3)
    for c in sampled_cells(seed):
        yp = patch_output(X, K, x, int(c))
        err = float(np.abs(y[c] - yp).max() / np.abs(yp).max())
        assert err <= TOL64, (int(c), err)
    # symmetry of the whole operator: <A x, z> = <x, A z>
    z = torch.from_numpy(inputs.uniform_vector(N, K_DEG, 99)).cuda()
    yz = m.apply(z)
    a, b = float(torch.dot(m.apply(xd), z)), float(torch.dot(xd, yz))
    assert abs(a - b) <= 1e-12 * float(m.apply(xd).norm() * z.norm())


def test_affine_full_size_sampled_cells(dg, data):
    import torch
    K, x = data
    m = dg.Mesh(N, K_DEG)
    m.set_geometry(SHEAR)
    m.set_coefficient(torch.from_numpy(K).cuda())
    check_mesh(m, lattice(N, SHEAR), K, x, 5)
    m.close()


def test_multilinear_full_size_sampled_cells(dg, data):
    import torch
    K, x = data
    rng = np.random.default_rng(7)
    X = lattice(N)
    inner = np.zeros(X.shape[:3], bool)
    inner[1:-1, 1:-1, 1:-1] = True
    X = X + np.where(inner[..., None], 0.2 / N * rng.uniform(-1.0, 1.0, X.shape), 0.0)
    m = dg.Mesh(N, K_DEG)
    m.set_vertices(X)
    m.set_coefficient(torch.from_numpy(K).cuda())
    check_mesh(m, X, K, x, 6)
    m.close()
