"""The Section 5 flow problem on the GPU: zero-flux sides, weak Dirichlet data
and the inlet flux, each against the FP64 oracle (which drops the zero-flux
boundary faces from its face loop and evaluates the data and the flux by full
face quadrature), and the closed-form series flux of a layered coefficient."""
import numpy as np
import pytest

from oracle import SIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
G = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # p = 1 at x = 0, p = 0 at x = 1


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def flow_mesh(dg, N, k, K):
    import torch
    m = dg.Mesh(N, k)
    m.set_boundary("flow_x")
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m


@pytest.mark.parametrize("N,k", [(1, 1), (2, 2), (3, 3), (4, 2), (3, 4), (2, 6)])
def test_flow_operator_matches_oracle(dg, N, k):
    import torch
    K = inputs.lognormal_coefficient(N, k, seed=21)
    x = inputs.uniform_vector(N, k, 22)
    m = flow_mesh(dg, N, k, K)
    D = SIPG(N, k, bc="flow_x")
    yref = D.apply(K, x)
    y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(y, yref) <= TOL64
    x32 = x.astype(np.float32)
    y32 = m.apply(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert relmax(y32, D.apply(K, x32.astype(np.float64))) <= TOL32
    d = m.diagonal().cpu().numpy()
    assert relmax(d, D.diagonal(K)) <= TOL64
    v = inputs.uniform_vector(N, k, 23)
    g = m.coeff_grad(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    assert relmax(g, D.coeff_grad(K, x, v).reshape(-1)) <= TOL64


@pytest.mark.parametrize("bc", ["dirichlet", "flow_x"])
def test_dirichlet_rhs_and_boundary_flux_match_oracle(dg, bc):
    import torch
    N, k = 4, 3
    K = inputs.lognormal_coefficient(N, k, seed=24)
    m = dg.Mesh(N, k)
    m.set_boundary(bc)
    m.set_coefficient(torch.from_numpy(K).cuda())
    D = SIPG(N, k, bc=bc)
    g = (0.7, -1.2, 0.4, 2.0, -0.3, 1.1)
    b = m.dirichlet_rhs(g).cpu().numpy()
    assert relmax(b, D.dirichlet_rhs(K, g)) <= TOL64
    u = inputs.uniform_vector(N, k, 25)
    ud = torch.from_numpy(u).cuda()
    for side in range(6):
        if not D.dirichlet[side]:
            with pytest.raises(dg.DGError, match="zero flux"):
                m.boundary_flux(ud, side, g[side])
            continue
        q = float(m.boundary_flux(ud, side, g[side]).item())
        qref = D.boundary_flux(K, u, side, g[side])
        assert abs(q - qref) <= 1e-12 * max(1.0, abs(qref)), (side, q, qref)


@pytest.mark.parametrize("N,k,mode", [(4, 1, "fp64"), (6, 2, "fp64"), (5, 3, "mixed")])
def test_layered_coefficient_gives_the_series_flux(dg, N, k, mode):
    """k depending on x only: the discrete solution is the exact
    piecewise-linear pressure and the inlet flux is 1 / sum_i (h / k_i)."""
    import torch
    rng = np.random.default_rng(100 + N)
    kx = np.exp(rng.standard_normal(N))
    K = np.repeat(kx[np.arange(N ** 3) % N], (k + 1) ** 3)
    m = flow_mesh(dg, N, k, K)
    b = m.dirichlet_rhs(G)
    md = dg.DG_CG_FP64 if mode == "fp64" else dg.DG_CG_MIXED_IR
    u, st = m.cg_solve(b, rtol=1e-12 if mode == "fp64" else 1e-10, mode=md, precond="jacobi")
    F = 1.0 / np.sum((1.0 / N) / kx)
    q_in = float(m.boundary_flux(u, 0, 1.0).item())
    q_out = float(m.boundary_flux(u, 1, 0.0).item())
    tol = 1e-9 if mode == "fp64" else 1e-7
    assert abs(q_in - F) <= tol * F, (q_in, F)
    assert abs(q_out + F) <= tol * F, (q_out, F)


def test_lognormal_flow_solve_checked_by_oracle(dg):
    import torch
    N, k = 5, 2
    K = inputs.lognormal_coefficient(N, k, seed=26, corr_len=0.1 * 64 / N)
    m = flow_mesh(dg, N, k, K)
    D = SIPG(N, k, bc="flow_x")
    b = m.dirichlet_rhs(G)
    bn = D.dirichlet_rhs(K, G)
    assert relmax(b.cpu().numpy(), bn) <= TOL64
    u, st = m.cg_solve(b, rtol=1e-11, precond="jacobi")
    un = u.cpu().numpy()
    r = np.linalg.norm(bn - D.apply(K, un)) / np.linalg.norm(bn)
    assert r <= 1.05e-11
    q_in = float(m.boundary_flux(u, 0, 1.0).item())
    q_out = float(m.boundary_flux(u, 1, 0.0).item())
    assert abs(q_in - D.boundary_flux(K, un, 0, 1.0)) <= 1e-12 * abs(q_in)
    assert q_in > 0 and abs(q_in + q_out) <= 1e-8 * q_in


def test_flow_batched_solve_checked_by_oracle(dg):
    import torch
    levels = [(4, 2), (3, 3), (2, 4), (5, 1)]
    meshes, bs, xs, Ks = [], [], [], []
    for s, (N, k) in enumerate(levels):
        K = inputs.lognormal_coefficient(N, k, seed=30 + s, corr_len=0.1 * 64 / N)
        m = flow_mesh(dg, N, k, K)
        meshes.append(m)
        Ks.append(K)
        bs.append(m.dirichlet_rhs(G))
        xs.append(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, precond="jacobi")
    for (N, k), K, x, st in zip(levels, Ks, xs, stats):
        assert st["status"] == 0
        D = SIPG(N, k, bc="flow_x")
        bn = D.dirichlet_rhs(K, G)
        r = np.linalg.norm(bn - D.apply(K, x.cpu().numpy())) / np.linalg.norm(bn)
        assert r <= 1.05e-10


def test_set_boundary_rejects_and_requires_a_new_coefficient(dg):
    import torch
    m = dg.Mesh(2, 1)
    with pytest.raises(dg.DGError, match="at least one side"):
        m.set_boundary(0)
    with pytest.raises(dg.DGError):
        m.set_boundary(0x40)
    m.set_coefficient(torch.ones(m.n_dofs, dtype=torch.float64, device="cuda"))
    m.set_boundary("flow_x")
    with pytest.raises(dg.DGError, match="coefficient not set"):
        m.apply(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
