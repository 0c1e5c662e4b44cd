"""GPU parity of dg_apply / dg_apply_adjoint / dg_coeff_grad against the FP64 oracle.

Tolerances (relative max-norm ||y - y_ref||_inf / ||y_ref||_inf): 1e-12 for the
FP64 operator and the gradient, 1e-5 for the FP32 operator.
"""
import numpy as np
import pytest

from oracle import SIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5

# (n_cells, degree): one cell (all faces on the boundary), two and three cells
# per direction, ragged last blocks (cells not a multiple of the cells per
# block), every supported degree, and the 8^3 Q2 workload.
CASES = [(1, 1), (1, 2), (2, 1), (2, 2), (3, 2), (5, 1), (4, 3), (3, 3), (3, 4), (2, 5),
         (2, 6), (2, 7), (2, 8), (8, 2), (6, 3), (5, 4)]


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def make_problem(dg, N, k, kseed=7, xseed=8, unit=False):
    import torch
    K = inputs.unit_coefficient(N, k) if unit else inputs.lognormal_coefficient(N, k, seed=kseed)
    x = inputs.uniform_vector(N, k, xseed)
    m = dg.Mesh(N, k)
    m.set_coefficient(torch.from_numpy(K).cuda())
    return m, K, x


@pytest.mark.parametrize("N,k", CASES)
def test_apply_fp64_matches_oracle(dg, N, k):
    import torch
    m, K, x = make_problem(dg, N, k)
    y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yref = SIPG(N, k).apply(K, x)
    assert relmax(y, yref) <= TOL64


@pytest.mark.parametrize("N,k", CASES)
def test_apply_fp32_matches_oracle(dg, N, k):
    import torch
    m, K, x = make_problem(dg, N, k)
    x32 = x.astype(np.float32)
    y = m.apply(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    yref = SIPG(N, k).apply(K, x32.astype(np.float64))
    assert relmax(y, yref) <= TOL32


@pytest.mark.parametrize("N,k", [(2, 2), (3, 3), (4, 1)])
def test_unit_vectors_give_matrix_columns(dg, N, k):
    """One-hot inputs: every column of A in the first and last cell."""
    import torch
    m, K, _ = make_problem(dg, N, k)
    D = SIPG(N, k)
    A = D.assemble(K).toarray()
    n3 = D.n3
    for col in list(range(n3)) + list(range(D.n_dofs - n3, D.n_dofs)):
        e = torch.zeros(D.n_dofs, dtype=torch.float64, device="cuda")
        e[col] = 1.0
        y = m.apply(e).cpu().numpy()
        assert relmax(y, A[:, col]) <= TOL64


def test_zero_input_and_scale_extremes(dg):
    import torch
    N, k = 3, 2
    m, K, x = make_problem(dg, N, k)
    z = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(m.apply(z)).item() == 0
    # K^- K^+ in the harmonic mean must stay finite: |log10 K| <= ~150
    for scale in (1e-100, 1e100):
        Ks = K * scale
        m.set_coefficient(torch.from_numpy(Ks).cuda())
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert relmax(y, SIPG(N, k).apply(Ks, x)) <= TOL64


@pytest.mark.parametrize("N,k", [(3, 2), (4, 3), (2, 4)])
def test_adjoint_and_symmetry(dg, N, k):
    import torch
    m, K, x = make_problem(dg, N, k)
    v = torch.from_numpy(inputs.uniform_vector(N, k, 99)).cuda()
    xd = torch.from_numpy(x).cuda()
    y = m.apply(xd)
    ya = m.apply_adjoint(xd)
    assert relmax(ya.cpu().numpy(), y.cpu().numpy()) <= TOL64
    lhs = float(torch.dot(v, m.apply(xd)))
    rhs = float(torch.dot(xd, m.apply_adjoint(v)))
    assert abs(lhs - rhs) <= 1e-12 * float(torch.dot(v.abs(), m.apply(xd.abs())))


def test_apply_is_deterministic(dg):
    import torch
    m, K, x = make_problem(dg, 6, 3)
    xd = torch.from_numpy(x).cuda()
    y1 = m.apply(xd)
    y2 = m.apply(xd)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("N,k", [(2, 2), (3, 1), (3, 3), (2, 4)])
def test_coeff_grad_matches_oracle(dg, N, k):
    import torch
    m, K, u = make_problem(dg, N, k)
    v = inputs.uniform_vector(N, k, 123)
    g = m.coeff_grad(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    gref = SIPG(N, k).coeff_grad(K, u, v).reshape(-1)
    assert relmax(g, gref) <= TOL64


@pytest.mark.parametrize("N,k,dtype,pinned", [
    (4, 3, "f64", True),    # 4 slabs of one z-layer
    (9, 2, "f64", True),    # 5 slabs of 2 layers, the last one ragged (1 layer)
    (1, 2, "f64", False),   # one cell, one slab, pageable buffers
    (17, 1, "f32", True),   # 6 slabs of 3 layers, ragged, FP32
    (5, 4, "f32", False),
])
def test_host_apply_matches_device_apply(dg, N, k, dtype, pinned):
    """The slab-pipelined host-buffer apply gives the device apply bit for bit
    (the same kernels on cell ranges), twice in a row on the same buffers."""
    import torch
    m, K, x = make_problem(dg, N, k)
    xt = torch.from_numpy(x)
    if dtype == "f32":
        xt = xt.float()
    xh = xt.pin_memory() if pinned else xt.clone()
    yh = torch.empty_like(xh)
    if pinned:
        yh = yh.pin_memory()
    yd = m.apply(xh.cuda()).cpu()
    for _ in range(2):
        yh.fill_(float("nan"))
        m.apply_host(xh, yh)
        assert torch.equal(yh, yd)


@pytest.mark.slow
def test_full_size_64cubed_q3_sampled_cells(dg):
    """The 64^3 Q3 lognormal workload in the benchmark's launch configuration;
    the oracle evaluates 200 sampled cells (corners, faces, random)."""
    import torch
    N, k = 64, 3
    m, K, x = make_problem(dg, N, k, kseed=2, xseed=3)
    y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(N ** 3, -1)
    rng = np.random.default_rng(0)
    corners = [0, N - 1, N * (N - 1), N * N - 1, N ** 3 - 1, N ** 3 - N, N ** 3 - N * N]
    cells = np.unique(np.concatenate([corners, rng.choice(N ** 3, 193, replace=False)]))
    yref = SIPG(N, k).apply(K, x, cells=cells)
    assert relmax(y[cells], yref) <= TOL64


@pytest.mark.slow
def test_full_size_64cubed_q3_fp32_sampled_cells(dg):
    """The FP32 operator on the 64^3 Q3 lognormal workload (FP32 input), at
    200 sampled cells against the FP64 oracle applied to the same FP32 input."""
    import torch
    N, k = 64, 3
    m, K, x = make_problem(dg, N, k, kseed=2, xseed=3)
    x32 = x.astype(np.float32)
    y = m.apply(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64).reshape(N ** 3, -1)
    rng = np.random.default_rng(1)
    corners = [0, N - 1, N * (N - 1), N * N - 1, N ** 3 - 1, N ** 3 - N, N ** 3 - N * N]
    cells = np.unique(np.concatenate([corners, rng.choice(N ** 3, 193, replace=False)]))
    yref = SIPG(N, k).apply(K, x32.astype(np.float64), cells=cells)
    assert relmax(y[cells], yref) <= TOL32


@pytest.mark.parametrize("N,k", [(1, 1), (3, 2), (5, 4), (2, 8), (7, 3)])
def test_load_vector_matches_oracle(dg, N, k):
    import torch
    f = lambda x, y, z: np.sin(np.pi * x) * np.cos(2.0 * y) + z * z * x + 0.5
    F = inputs.values_at_gauss_points(N, k, f)
    m = dg.Mesh(N, k)       # no coefficient needed
    b = m.load_vector(torch.from_numpy(F).cuda()).cpu().numpy()
    bref = SIPG(N, k).load_vector(f)
    assert relmax(b, bref) <= TOL64
