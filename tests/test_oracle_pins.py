"""Pins of the FP64 oracle against mathematics, not against itself.

Each test checks a fact fixed independently of the oracle's code path:
closed-form 1D Legendre data, the Kronecker-sum structure of the K = 1
operator, symmetry, positive definiteness and the continuum eigenvalue,
consistency on harmonic polynomials, L2 convergence rates, Euler homogeneity
of the coefficient gradient, finite differences, and CG against a direct solve.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import SIPG, cg, gauss_points, legendre, legendre_deriv
from paper_1911_01492_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# 1D ingredients
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 9])
def test_gauss_rule_exact_to_degree_2n_minus_1(n):
    t, w = gauss_points(n)
    assert abs(w.sum() - 1.0) < 1e-15
    for p in range(2 * n):
        assert abs((w * t ** p).sum() - 1.0 / (p + 1)) < 1e-14
    # and not beyond: t^(2n) is integrated inexactly
    assert abs((w * t ** (2 * n)).sum() - 1.0 / (2 * n + 1)) > 1e-13


@pytest.mark.parametrize("i", range(8))
def test_legendre_end_values_closed_form(i):
    a = math.sqrt(2 * i + 1)
    assert abs(legendre(i, 1.0) - a) < 1e-13
    assert abs(legendre(i, 0.0) - (-1) ** i * a) < 1e-13
    assert abs(legendre_deriv(i, 1.0) - a * i * (i + 1)) < 1e-11
    assert abs(legendre_deriv(i, 0.0) - (-1) ** (i + 1) * a * i * (i + 1)) < 1e-11


def test_legendre_orthonormal_and_stiffness_closed_form():
    t, w = gauss_points(12)
    for i in range(8):
        for j in range(8):
            m = (w * legendre(i, t) * legendre(j, t)).sum()
            assert abs(m - (i == j)) < 1e-13
            s = (w * legendre_deriv(i, t) * legendre_deriv(j, t)).sum()
            mm = min(i, j)
            ref = 2 * math.sqrt(2 * i + 1) * math.sqrt(2 * j + 1) * mm * (mm + 1) if (i + j) % 2 == 0 else 0.0
            assert abs(s - ref) < 1e-10 * max(1.0, abs(ref))


# --------------------------------------------------------------------------
# P1: the one-cell matrix in closed form
# --------------------------------------------------------------------------

def closed_form_T(k):
    n = k + 1
    sigma = 2.0 * n * n
    a = np.array([math.sqrt(2 * i + 1) for i in range(n)])
    d = a * np.array([i * (i + 1) for i in range(n)])
    T = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            S = 2 * a[i] * a[j] * min(i, j) * (min(i, j) + 1) if (i + j) % 2 == 0 else 0.0
            T[i, j] = S + (1 + (-1) ** (i + j)) * (sigma * a[i] * a[j] - a[i] * d[j] - a[j] * d[i])
    return T


def kron_sum(T):
    n = T.shape[0]
    I = np.eye(n)
    # m = i + n(j + n l): i is the fastest index
    return np.kron(I, np.kron(I, T)) + np.kron(I, np.kron(T, I)) + np.kron(T, np.kron(I, I))


def read_golden_T():
    out = {}
    cur = None
    for line in open(os.path.join(GOLDEN, "one_cell_T.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("k="):
            cur = int(line[2:])
            out[cur] = {"rows": []}
        elif "=" in line:
            key, val = line.split("=")
            out[cur][key] = float(val)
        else:
            out[cur]["rows"].append([eval(e, {"sqrt": math.sqrt}) for e in line.split(",")])
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_one_cell_matrix_is_closed_form_kronecker_sum(k):
    D = SIPG(1, k)
    A = D.assemble(np.ones(D.n_dofs)).toarray()
    ref = kron_sum(closed_form_T(k))
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()
    # the matrix-free form gives the same columns
    for col in (0, 1, D.n3 - 1):
        e = np.zeros(D.n_dofs)
        e[col] = 1.0
        y = D.apply(np.ones(D.n_dofs), e)
        assert np.abs(y - ref[:, col]).max() <= 1e-12 * np.abs(ref).max()


def test_one_cell_golden_values():
    g = read_golden_T()
    for k, rec in g.items():
        T = np.array(rec["rows"])
        assert np.abs(T - closed_form_T(k)).max() < 1e-12 * np.abs(T).max()
        D = SIPG(1, k)
        A = D.assemble(np.ones(D.n_dofs)).toarray()
        ev = np.linalg.eigvalsh(A)
        assert abs(A[0, 0] - rec["A00"]) < 1e-12 * rec["A00"]
        assert abs(ev[-1] - rec["lmax"]) < 1e-8 * rec["lmax"]
        if "lmin" in rec:
            assert abs(ev[0] - rec["lmin"]) < 1e-7


# --------------------------------------------------------------------------
# P2: K = 1 operator is h^2 times a Kronecker sum of the 1D SIPG matrix
# --------------------------------------------------------------------------

def sipg_1d(N, k):
    """1D SIPG matrix on N cells of [0,1] from closed-form trace data."""
    n = k + 1
    h = 1.0 / N
    sigma = 2.0 * n * n
    a1 = np.array([math.sqrt(2 * i + 1) for i in range(n)])   # L_i(1)
    d1 = a1 * np.array([i * (i + 1) for i in range(n)])       # L_i'(1)
    a0 = a1 * np.array([(-1) ** i for i in range(n)])          # L_i(0)
    d0 = -d1 * np.array([(-1) ** i for i in range(n)])         # L_i'(0)
    S = np.array([[2 * a1[i] * a1[j] * min(i, j) * (min(i, j) + 1) if (i + j) % 2 == 0 else 0.0
                   for j in range(n)] for i in range(n)])
    A = np.zeros((N * n, N * n))
    for e in range(N):
        A[e * n:(e + 1) * n, e * n:(e + 1) * n] += S / h
    # interior points: [w] = w_e(1) - w_{e+1}(0), {w'} = (w_e'(1) + w_{e+1}'(0)) / (2h)
    for e in range(N - 1):
        J = np.zeros(N * n)
        G = np.zeros(N * n)
        J[e * n:(e + 1) * n] = a1
        J[(e + 1) * n:(e + 2) * n] = -a0
        G[e * n:(e + 1) * n] = 0.5 * d1 / h
        G[(e + 1) * n:(e + 2) * n] = 0.5 * d0 / h
        A += -np.outer(J, G) - np.outer(G, J) + sigma / h * np.outer(J, J)
    # boundary points with outward normals
    for (e, val, der) in ((N - 1, a1, d1 / h), (0, a0, -d0 / h)):
        J = np.zeros(N * n)
        G = np.zeros(N * n)
        J[e * n:(e + 1) * n] = val
        G[e * n:(e + 1) * n] = der
        A += -np.outer(J, G) - np.outer(G, J) + sigma / h * np.outer(J, J)
    return A


@pytest.mark.parametrize("N,k", [(2, 1), (2, 2), (3, 2), (3, 1), (2, 3)])
def test_unit_coefficient_operator_is_kronecker_sum(N, k):
    n = k + 1
    h = 1.0 / N
    A1 = sipg_1d(N, k)
    I = np.eye(N * n)
    A3 = h * h * (np.kron(I, np.kron(I, A1)) + np.kron(I, np.kron(A1, I)) + np.kron(A1, np.kron(I, I)))
    D = SIPG(N, k)
    A = D.assemble(np.ones(D.n_dofs)).toarray()
    # oracle index (cz, cy, cx, l, j, i) -> tensor index (Z, Y, X), X = cx n + i
    g = np.arange(D.n_dofs)
    m, c = g % D.n3, g // D.n3
    i, j, l = m % n, (m // n) % n, m // (n * n)
    cx, cy, cz = c % N, (c // N) % N, c // (N * N)
    M = N * n
    t = (cx * n + i) + M * ((cy * n + j) + M * (cz * n + l))
    assert np.abs(A - A3[np.ix_(t, t)]).max() <= 1e-12 * np.abs(A3).max()


# --------------------------------------------------------------------------
# P3 / P4: symmetry and positive definiteness
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,k", [(3, 2), (2, 3), (2, 4)])
def test_symmetry_matrix_free(N, k):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=7)
    x = inputs.uniform_vector(N, k, 8)
    y = inputs.uniform_vector(N, k, 9)
    lhs = x @ D.apply(K, y)
    rhs = y @ D.apply(K, x)
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(x) @ np.abs(D.assemble(K)) @ np.abs(y))


@pytest.mark.parametrize("N,k,seed", [(2, 2, 2), (2, 3, 5), (3, 2, 4), (2, 4, 4)])
def test_positive_definite_under_lognormal_coefficient(N, k, seed):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=seed)
    A = D.assemble(K).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    np.linalg.cholesky(A)                  # raises if not SPD
    assert np.linalg.eigvalsh(A)[0] > 0


def test_coarse_cells_with_strong_coefficient_variation_can_be_indefinite():
    """A limitation of the per-cell face coefficient: on 3^3 Q4 with correlation
    length 0.1 (a cell spans ~3 correlation lengths, K varies ~1000x inside it)
    the face terms outweigh the local volume term and A has negative
    eigenvalues.  With the workload's per-cell statistics it is SPD."""
    D = SIPG(3, 4)
    ev = np.linalg.eigvalsh(D.assemble(inputs.lognormal_coefficient(3, 4, seed=4)).toarray())
    assert (ev < 0).sum() == 2
    K = inputs.lognormal_coefficient(3, 4, seed=4, corr_len=0.1 * 64 / 3)
    assert np.linalg.eigvalsh(D.assemble(K).toarray())[0] > 0


def test_smallest_eigenvalue_approaches_continuum():
    # lambda_min(M^-1 A) -> 3 pi^2 for -Laplace on the unit cube, M = h^3 I
    D = SIPG(8, 2)
    A = D.assemble(np.ones(D.n_dofs))
    lam = spla.eigsh(A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    lam /= D.h ** 3
    assert abs(lam - 3 * math.pi ** 2) < 2e-3 * 3 * math.pi ** 2


# --------------------------------------------------------------------------
# P5: consistency on harmonic polynomials
# --------------------------------------------------------------------------

HARMONIC = [
    lambda x, y, z: 1.0 + 0 * x,
    lambda x, y, z: x + 0 * y,
    lambda x, y, z: z - 2 * y + 0 * x,
    lambda x, y, z: x * y + 0 * z,
    lambda x, y, z: x * x - y * y + 0 * z,
    lambda x, y, z: x * y * z,
    lambda x, y, z: x * x - z * z + 3 * x * y,
]


def interior_cells(D):
    c = np.arange(D.n_cells_total)
    cx, cy, cz = D.cell_coords(c)
    N = D.N
    return c[(cx > 0) & (cx < N - 1) & (cy > 0) & (cy < N - 1) & (cz > 0) & (cz < N - 1)]


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("pi", range(len(HARMONIC)))
def test_consistency_on_harmonic_polynomials(k, pi):
    p = HARMONIC[pi]
    D = SIPG(4, k)
    Kc = 2.5
    K = np.full(D.n_dofs, Kc)
    x = D.project(p)
    y = D.apply(K, x).reshape(D.n_cells_total, D.n3)
    inner = interior_cells(D)
    scale = np.abs(D.assemble(K)).max() * np.abs(x).max()
    assert np.abs(y[inner]).max() <= 1e-12 * scale
    # and the boundary-adjacent cells see the Dirichlet condition
    if pi == 0:
        assert np.abs(y).max() > 1e-3 * scale


def test_constants_in_kernel_for_any_coefficient():
    D = SIPG(4, 2)
    K = inputs.lognormal_coefficient(4, 2, seed=3)
    x = D.project(lambda x, y, z: 1.0 + 0 * x)
    y = D.apply(K, x).reshape(D.n_cells_total, D.n3)
    inner = interior_cells(D)
    assert np.abs(y[inner]).max() <= 1e-12 * np.abs(y).max()


def test_consistency_separates_the_printed_plus_sign():
    """With the consistency terms' sign flipped, a linear function is no longer
    in the kernel on interior cells (the reason for the minus-sign reading).

    A(sigma) = Vol + C + sigma P is affine in sigma, so the consistency part is
    C = A(0) - Vol and the flipped operator is A - 2 C."""
    D = SIPG(4, 2)
    K = np.ones(D.n_dofs)
    x = D.project(lambda x, y, z: x + 0 * y)
    A = D.assemble(K)
    A0 = SIPG(4, 2, sigma=0.0).assemble(K)
    G = D.grad
    vol = sp.kron(sp.identity(D.n_cells_total), np.einsum("qmd,q,qnd->mn", G, D.h * D.wq, G))
    A_plus = A - 2 * (A0 - vol)
    inner = interior_cells(D)
    y_minus = (A @ x).reshape(-1, D.n3)[inner]
    y_plus = (A_plus @ x).reshape(-1, D.n3)[inner]
    assert np.abs(y_minus).max() < 1e-12 * np.abs(A @ x).max()
    assert np.abs(y_plus).max() > 1e-2 * np.abs(A @ x).max()


# --------------------------------------------------------------------------
# P6: L2 convergence O(h^(k+1))
# --------------------------------------------------------------------------

def u_exact(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def f_exact(x, y, z):
    return 3 * np.pi ** 2 * u_exact(x, y, z)


@pytest.mark.slow
@pytest.mark.parametrize("k,Ns", [(1, (4, 8)), (2, (4, 8)), (3, (2, 4))])
def test_l2_convergence_rate(k, Ns):
    errs = []
    for N in Ns:
        D = SIPG(N, k)
        A = D.assemble(np.ones(D.n_dofs)).tocsc()
        b = D.load_vector(f_exact, nq=k + 4)
        x = spla.spsolve(A, b)
        errs.append(D.l2_error(x, u_exact))
    rate = math.log(errs[0] / errs[1]) / math.log(Ns[1] / Ns[0])
    assert abs(rate - (k + 1)) < 0.25, (errs, rate)


# --------------------------------------------------------------------------
# P7 / P8: coefficient gradient
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,k", [(2, 2), (3, 1), (2, 3)])
def test_gradient_euler_homogeneity_and_symmetry(N, k):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=11)
    u = inputs.uniform_vector(N, k, 12)
    v = inputs.uniform_vector(N, k, 13)
    g = D.coeff_grad(K, u, v)
    total = v @ D.apply(K, u)
    assert abs(g.sum() - total) <= 1e-12 * np.abs(g).sum()
    g2 = D.coeff_grad(K, v, u)
    assert np.abs(g - g2).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("N,k", [(2, 2), (3, 1)])
def test_gradient_matches_central_differences(N, k):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=21)
    u = inputs.uniform_vector(N, k, 22)
    v = inputs.uniform_vector(N, k, 23)
    g = D.coeff_grad(K, u, v).reshape(-1)
    rng = np.random.default_rng(24)
    eps = 1e-5
    for idx in rng.choice(D.n_dofs, 12, replace=False):
        Kp = K.copy()
        Km = K.copy()
        Kp[idx] *= math.exp(eps)
        Km[idx] *= math.exp(-eps)
        fd = (v @ D.apply(Kp, u) - v @ D.apply(Km, u)) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, np.abs(g).max())
    # directional derivative along a random direction
    dlog = rng.standard_normal(D.n_dofs)
    fd = (v @ D.apply(K * np.exp(eps * dlog), u) - v @ D.apply(K * np.exp(-eps * dlog), u)) / (2 * eps)
    assert abs(fd - g @ dlog) <= 1e-7 * np.abs(g).sum()


# --------------------------------------------------------------------------
# The matrix-free and assembled forms, sampled cells, load vectors
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,k", [(3, 2), (2, 4), (4, 1)])
def test_matrix_free_equals_assembled_and_sampled(N, k):
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=31)
    x = inputs.uniform_vector(N, k, 32)
    y = D.apply(K, x)
    yA = D.assemble(K) @ x
    assert np.abs(y - yA).max() <= 1e-13 * np.abs(yA).max()
    cells = np.array([0, D.n_cells_total - 1, D.n_cells_total // 2])
    ys = D.apply(K, x, cells=cells)
    # same formula per cell; BLAS may block the products differently by row count
    assert np.abs(ys - y.reshape(-1, D.n3)[cells]).max() <= 1e-14 * np.abs(y).max()


def test_constant_load_vector_matches_quadrature():
    D = SIPG(3, 3)
    b = D.load_vector(lambda x, y, z: 1.0 + 0 * x)
    assert np.abs(b - inputs.constant_load_vector(3, 3)).max() < 1e-16


# --------------------------------------------------------------------------
# CG (Section 2.4, PCG with M = I)
# --------------------------------------------------------------------------

def test_cg_matches_direct_solve():
    D = SIPG(2, 2)
    K = inputs.lognormal_coefficient(2, 2, seed=41)
    A = D.assemble(K).toarray()
    b = inputs.uniform_vector(2, 2, 42)
    x, it, rel, hist = cg(lambda z: A @ z, b, rtol=1e-12)
    xd = np.linalg.solve(A, b)
    assert rel <= 1e-12
    assert np.abs(x - xd).max() <= 1e-12 * np.linalg.cond(A) * np.abs(xd).max()
    # CG terminates in at most n steps in exact arithmetic; allow rounding slack
    assert it <= 2 * len(b)
    assert hist[-1] <= 1e-12


def test_pcg_with_diagonal_matches_direct_solve_in_fewer_iterations():
    D = SIPG(3, 3)
    K = inputs.lognormal_coefficient(3, 3, seed=43, corr_len=0.1 * 64 / 3)
    A = D.assemble(K).toarray()
    b = inputs.constant_load_vector(3, 3)
    x0, it0, _, _ = cg(lambda z: A @ z, b, rtol=1e-11)
    x1, it1, rel, _ = cg(lambda z: A @ z, b, rtol=1e-11, minv=1.0 / np.diag(A))
    xd = np.linalg.solve(A, b)
    assert rel <= 1e-11
    assert np.abs(x1 - xd).max() <= 1e-11 * np.linalg.cond(A) * np.abs(xd).max()
    assert it1 < it0


@pytest.mark.parametrize("N,k,seed", [(1, 3, 1), (2, 2, 2), (3, 1, 3), (2, 4, 4)])
def test_diagonal_equals_assembled_diagonal(N, k, seed):
    """The oracle's diag(A) (one function on its own side of each face) equals
    the diagonal of the CSR matrix assembled from the two-sided face blocks."""
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=seed, corr_len=0.1 * 64 / N)
    dref = D.assemble(K).diagonal()
    d = D.diagonal(K)
    assert np.abs(d - dref).max() <= 1e-13 * np.abs(dref).max()
    cells = np.array([0, N ** 3 - 1, (N ** 3) // 2])
    # same formula on a subset of cells (BLAS blocking may change the rounding)
    assert np.abs(D.diagonal(K, cells=cells) - d.reshape(N ** 3, -1)[cells]).max() <= 1e-14 * np.abs(d).max()


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_diagonal_one_cell_unit_coefficient_closed_form(k):
    """One unit cube, K = 1, all six faces on the boundary.  Along each axis
    the orthonormal Legendre L_t has int_0^1 (L_t')^2 = 2 (2t+1) t (t+1),
    L_t(s)^2 = 2t+1 and L_t(s) dL_t/dn_out(s) = (2t+1) t (t+1) at both ends, so
    a(phi, phi) = sum over t in (i, j, l) of 2 (2t+1) (sigma - t (t+1))."""
    D = SIPG(1, k)
    n = k + 1
    d = D.diagonal(np.ones(n ** 3))
    sigma = 2.0 * n * n
    for m in range(n ** 3):
        t = (m % n, (m // n) % n, m // (n * n))
        exact = sum(2.0 * (2 * a + 1) * (sigma - a * (a + 1)) for a in t)
        assert abs(d[m] - exact) <= 1e-12 * exact, (m, d[m], exact)


def test_cg_zero_rhs_and_breakdown():
    x, it, rel, _ = cg(lambda z: z, np.zeros(5))
    assert it == 0 and np.all(x == 0)
    with pytest.raises(FloatingPointError):
        cg(lambda z: -z, np.ones(5))


# --------------------------------------------------------------------------
# Face weights: on piecewise constants SWIPDG is two-point-flux finite volumes
# (Section 3.4), whose transmissibility is the series conductance of the two
# half cells -- i.e. the harmonic mean of the cell coefficients.
# --------------------------------------------------------------------------

def test_constant_modes_couple_with_two_point_flux_transmissibility():
    N, k = 3, 2
    D = SIPG(N, k)
    rng = np.random.default_rng(5)
    Kc = np.exp(rng.standard_normal(D.n_cells_total))
    K = np.repeat(Kc, D.n3)                   # constant inside every cell
    A = D.assemble(K)
    h = D.h
    for c in range(D.n_cells_total):
        for d in range(3):
            if D.cell_coords(c)[d] < N - 1:
                c2 = c + D.stride(d)
                # two half cells of length h/2 in series, face area h^2
                T = h * h / (0.5 * h / Kc[c] + 0.5 * h / Kc[c2])
                assert abs(A[c * D.n3, c2 * D.n3] + D.sigma * T) <= 1e-12 * D.sigma * T
    # and the per-cell face coefficient of a cell-constant K is that constant
    assert np.abs(D.kbar(K) - Kc).max() <= 1e-14 * Kc.max()


# --------------------------------------------------------------------------
# Per-cell face coefficient Kbar_c = exp(sum_q w_q log K_{c,q}) with log K
# varying inside the cells.  For log K = alpha + beta x^2 + delta y^2 + eps z^2
# + mu y the Gauss-weighted mean over cell c (side h, corner h (cx, cy, cz)) is
# exact (the n >= 2 point rule integrates quadratics); the cell averages of
# (x/h)^2 and y/h are cx^2 + cx + 1/3 and cy + 1/2.  With n = 3 the Gauss
# weights differ (4/9 vs 5/18), so an unweighted mean of log K along any axis
# (which gives cx^2 + cx + 0.35), an arithmetic mean of K, or a mean over the
# wrong array axis all miss these values.  The face weights are then fixed in
# closed form: the constant modes of two neighbours couple only through the
# penalty term, A[(c,0),(c',0)] = -sigma h gamma_F with
# gamma_F = 2 Kbar Kbar' / (Kbar + Kbar'), and the constant mode's diagonal
# entry is sigma h times the sum of gamma_F over its six faces (gamma_F = Kbar_c
# on a boundary face).
# --------------------------------------------------------------------------

def _quadratic_log_coefficient(N, k, alpha, quad, mu):
    """log K = alpha + quad[0] x^2 + quad[1] y^2 + quad[2] z^2 + mu y at the
    Gauss points, in the [cell][e][b][a] layout."""
    n = k + 1
    t, _ = np.polynomial.legendre.leggauss(n)
    xi = 0.5 * (t + 1.0)
    h = 1.0 / N
    logK = np.empty((N, N, N, n, n, n))        # [cz, cy, cx, e, b, a]
    for cz in range(N):
        for cy in range(N):
            for cx in range(N):
                X = h * (cx + xi)[None, None, :]
                Y = h * (cy + xi)[None, :, None]
                Z = h * (cz + xi)[:, None, None]
                logK[cz, cy, cx] = (alpha + quad[0] * X ** 2 + quad[1] * Y ** 2
                                    + quad[2] * Z ** 2 + mu * Y)
    return logK.reshape(-1)


def _closed_form_kbar(D, alpha, quad, mu):
    h = D.h
    out = {}
    for c in range(D.n_cells_total):
        crd = [int(v) for v in D.cell_coords(c)]
        mean_sq = [h * h * (v * v + v + 1.0 / 3.0) for v in crd]
        out[c] = math.exp(alpha + sum(a * m for a, m in zip(quad, mean_sq))
                          + mu * h * (crd[1] + 0.5))
    return out


def test_kbar_is_the_gauss_weighted_geometric_mean_in_closed_form():
    N, k = 2, 2
    alpha, quad, mu = 0.3, (2.0, -1.1, 0.7), -1.5
    D = SIPG(N, k)
    K = np.exp(_quadratic_log_coefficient(N, k, alpha, quad, mu))
    kb = D.kbar(K)
    ref = _closed_form_kbar(D, alpha, quad, mu)
    for c in range(D.n_cells_total):
        assert abs(kb[c] - ref[c]) <= 1e-14 * ref[c], (c, kb[c], ref[c])


def test_face_weights_of_a_varying_coefficient_in_closed_form():
    N, k = 2, 2
    alpha, quad, mu = -0.2, (1.7, 0.8, -1.3), 0.9
    D = SIPG(N, k)
    h, s = D.h, D.sigma
    K = np.exp(_quadratic_log_coefficient(N, k, alpha, quad, mu))
    kb = _closed_form_kbar(D, alpha, quad, mu)
    A = D.assemble(K).tocsr()
    n3 = D.n3
    for c in range(D.n_cells_total):
        coords = [int(v) for v in D.cell_coords(c)]
        gsum = 0.0
        for d in range(3):
            for upper in (False, True):
                inside = coords[d] < N - 1 if upper else coords[d] > 0
                if inside:
                    c2 = c + D.stride(d) if upper else c - D.stride(d)
                    g = 2.0 * kb[c] * kb[c2] / (kb[c] + kb[c2])
                    ref = -s * h * g
                    assert abs(A[c * n3, c2 * n3] - ref) <= 1e-12 * abs(ref), (c, c2)
                else:
                    g = kb[c]
                gsum += g
        ref = s * h * gsum
        assert abs(A[c * n3, c * n3] - ref) <= 1e-12 * ref, c
    # the matrix-free apply uses the same face weights as the assembly
    x = inputs.uniform_vector(N, k, 3)
    assert np.abs(D.apply(K, x) - A @ x).max() <= 1e-12 * np.abs(A @ x).max()


# --------------------------------------------------------------------------
# The Section 5 flow problem: -div(k grad p) = 0, p = 1 on x = 0, p = 0 on
# x = 1, zero flux on the other faces; quantity of interest = total flux
# through the inlet.  For k depending on x only (constant in each layer of
# cells) the exact solution is piecewise linear in x, lies in the DG space, and
# satisfies the SWIPDG face terms exactly (the harmonic-mean face weight times
# the average derivative equals the continuous flux), so the discrete solution
# equals it and the inlet flux is the series conductance 1 / sum_i (h / k_i).
# --------------------------------------------------------------------------

def _layered(N, k, kx):
    n3 = (k + 1) ** 3
    c = np.arange(N ** 3)
    return np.repeat(np.asarray(kx)[c % N], n3)


@pytest.mark.parametrize("N,k", [(1, 1), (4, 1), (4, 2), (3, 3)])
def test_flow_layered_coefficient_has_the_series_flux(N, k):
    rng = np.random.default_rng(N * 10 + k)
    kx = np.exp(rng.standard_normal(N))
    K = _layered(N, k, kx)
    D = SIPG(N, k, bc="flow_x")
    g = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    A = D.assemble(K).tocsc()
    u = spla.spsolve(A, D.dirichlet_rhs(K, g))
    h = D.h
    F = 1.0 / np.sum(h / kx)
    q_in = D.boundary_flux(K, u, 0, 1.0)
    q_out = D.boundary_flux(K, u, 1, 0.0)
    assert abs(q_in - F) <= 1e-10 * F
    assert abs(q_out + F) <= 1e-10 * F
    # the discrete solution is the exact piecewise-linear pressure
    p_left = 1.0 - np.concatenate(([0.0], np.cumsum(F * h / kx)))[:-1]
    t, _ = np.polynomial.legendre.leggauss(k + 1)
    xi = 0.5 * (t + 1.0)
    n = k + 1
    L = np.array([[legendre(i, s) for i in range(n)] for s in xi])
    uc = u.reshape(N ** 3, n, n, n)                    # [c][l][j][i]
    vals = np.einsum("clji,ai,bj,el->ceba", uc, L, L, L)   # [c][e][b][a]
    c = np.arange(N ** 3)
    cx = c % N
    exact = p_left[cx][:, None] - (F / kx[cx])[:, None] * h * xi[None, :]
    assert np.abs(vals - exact[:, None, None, :]).max() <= 1e-10


def test_flow_inlet_and_outlet_flux_balance_for_any_coefficient():
    N, k = 3, 2
    D = SIPG(N, k, bc="flow_x")
    K = inputs.lognormal_coefficient(N, k, seed=11, corr_len=0.1 * 64 / N)
    g = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    u = spla.spsolve(D.assemble(K).tocsc(), D.dirichlet_rhs(K, g))
    q_in = D.boundary_flux(K, u, 0, 1.0)
    q_out = D.boundary_flux(K, u, 1, 0.0)
    assert q_in > 0.0
    assert abs(q_in + q_out) <= 1e-10 * q_in


def test_zero_flux_sides_carry_no_face_terms():
    N, k = 4, 2
    K = inputs.lognormal_coefficient(N, k, seed=12, corr_len=0.1 * 64 / N)
    ones = np.zeros((N ** 3, (k + 1) ** 3))
    ones[:, 0] = 1.0                              # the constant function
    c = np.arange(N ** 3)
    cx = c % N
    for bc, inner in (("flow_x", (cx > 0) & (cx < N - 1)),):
        y = SIPG(N, k, bc=bc).apply(K, ones.reshape(-1)).reshape(N ** 3, -1)
        assert np.abs(y[inner]).max() <= 1e-12 * np.abs(y).max()
        assert np.abs(y[~inner]).max() > 0.0
    # with Dirichlet data on every side the y/z boundary cells do see the constant
    yd = SIPG(N, k).apply(K, ones.reshape(-1)).reshape(N ** 3, -1)
    assert np.abs(yd[(cx > 0) & (cx < N - 1)]).max() > 0.0


@pytest.mark.parametrize("k", [1, 2, 4])
def test_dirichlet_rhs_closed_form(k):
    """Only the modes (i, 0, 0) of the cells on a Dirichlet x-side see constant
    data g (orthonormal tangential modes integrate to delta_{j0} delta_{l0}):
    b = h Kbar g (sigma L_i(s) - o_s L_i'(s)), o_s = -1 at x = 0, +1 at x = 1,
    with L_i(1) = sqrt(2i+1), L_i(0) = (-1)^i sqrt(2i+1), L_i'(1) = sqrt(2i+1) i(i+1),
    L_i'(0) = (-1)^(i+1) sqrt(2i+1) i(i+1)."""
    N = 3
    D = SIPG(N, k, bc="flow_x")
    K = inputs.lognormal_coefficient(N, k, seed=13, corr_len=0.1 * 64 / N)
    kb = D.kbar(K)
    gl, gr = 0.7, -1.3
    b = D.dirichlet_rhs(K, (gl, gr, 5.0, 5.0, 5.0, 5.0)).reshape(N ** 3, k + 1, k + 1, k + 1)
    sigma, h = 2.0 * (k + 1) ** 2, 1.0 / N
    ref = np.zeros_like(b)
    for c in range(N ** 3):
        cx = c % N
        for i in range(k + 1):
            a = math.sqrt(2 * i + 1)
            if cx == 0:
                Li, dLi = (-1) ** i * a, (-1) ** (i + 1) * a * i * (i + 1)
                ref[c, 0, 0, i] += h * kb[c] * gl * (sigma * Li + dLi)
            if cx == N - 1:
                Li, dLi = a, a * i * (i + 1)
                ref[c, 0, 0, i] += h * kb[c] * gr * (sigma * Li - dLi)
    assert np.abs(b - ref).max() <= 1e-12 * np.abs(ref).max()


# --------------------------------------------------------------------------
# Cell-block Jacobi: with one cell the block diagonal is A itself, so PCG
# converges in one iteration; on a larger mesh the blocks are the diagonal
# blocks of A (the cell's own volume and own-side face terms), SPD, and PCG
# with them reaches the direct solution.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
def test_block_jacobi_is_exact_on_one_cell(k):
    from oracle.dg_oracle import block_jacobi_inverse
    D = SIPG(1, k)
    K = np.exp(np.random.default_rng(k).standard_normal(D.n3))
    A = D.assemble(K)
    b = np.random.default_rng(10 + k).standard_normal(D.n_dofs)
    x, it, rel, _ = cg(lambda v: A @ v, b, rtol=1e-12, minv=block_jacobi_inverse(A, D.n3))
    assert it == 1 and rel <= 1e-12


def test_block_jacobi_blocks_are_spd_and_pcg_reaches_the_direct_solution():
    from oracle.dg_oracle import block_jacobi_inverse, cell_blocks
    N, k = 3, 2
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=14, corr_len=0.1 * 64 / N)
    A = D.assemble(K)
    blocks = cell_blocks(A, D.n3)
    assert np.abs(blocks - blocks.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(blocks).max()
    assert np.linalg.eigvalsh(blocks).min() > 0
    # a block's off-diagonal structure: the cell's own terms only (no neighbour
    # couplings), equal to the one-cell operator's volume part plus face terms
    b = inputs.uniform_vector(N, k, 15)
    x, it_b, rel, _ = cg(lambda v: A @ v, b, rtol=1e-12, minv=block_jacobi_inverse(A, D.n3))
    xd = spla.spsolve(A.tocsc(), b)
    assert rel <= 1e-12 and np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
    _, it_p, _, _ = cg(lambda v: A @ v, b, rtol=1e-12, minv=1.0 / D.diagonal(K))
    assert it_b < it_p


# --------------------------------------------------------------------------
# Affine geometry (problem B): x = A xi.  A = I is the cube operator; a
# diagonal A = diag(al, be, ga) stretches the axes, and the one-cell K = 1
# operator is the Kronecker sum of the 1D closed form T with the factors
# be ga / al, al ga / be, al be / ga (volume, face area over normal length and
# penalty length scale alike); a sheared A keeps symmetry and definiteness,
# reproduces harmonic polynomials with mixed derivatives on interior cells,
# and converges at rate k + 1.
# --------------------------------------------------------------------------

SHEAR = [[1.0, 0.3, 0.1], [0.0, 1.1, -0.2], [0.05, 0.0, 0.9]]


def test_affine_identity_is_the_cube_operator():
    from oracle.dg_oracle import AffineSIPG
    for N, k in ((2, 2), (3, 1)):
        K = inputs.lognormal_coefficient(N, k, seed=50, corr_len=0.5)
        A1 = SIPG(N, k).assemble(K)
        A2 = AffineSIPG(N, k, np.eye(3)).assemble(K)
        assert abs(A1 - A2).max() <= 1e-14 * abs(A1).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_affine_stretched_one_cell_is_a_scaled_kronecker_sum(k):
    from oracle.dg_oracle import AffineSIPG
    al, be, ga = 0.7, 1.3, 2.1
    D = AffineSIPG(1, k, np.diag([al, be, ga]))
    A = D.assemble(np.ones(D.n_dofs)).toarray()
    T = closed_form_T(k)
    I = np.eye(k + 1)
    ref = (be * ga / al * np.kron(I, np.kron(I, T)) + al * ga / be * np.kron(I, np.kron(T, I))
           + al * be / ga * np.kron(T, np.kron(I, I)))
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


def test_affine_sheared_operator_is_symmetric_positive_definite():
    from oracle.dg_oracle import AffineSIPG
    N, k = 3, 2
    D = AffineSIPG(N, k, SHEAR)
    K = inputs.lognormal_coefficient(N, k, seed=51, corr_len=0.1 * 64 / N)
    A = D.assemble(K).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("pname", ["x", "xy", "x2-y2", "yz+2xz"])
def test_affine_consistency_on_harmonic_polynomials(pname):
    from oracle.dg_oracle import AffineSIPG
    p = {"x": lambda x, y, z: 1.0 + 2.0 * x - y + 0.5 * z,
         "xy": lambda x, y, z: x * y,
         "x2-y2": lambda x, y, z: x * x - y * y,
         "yz+2xz": lambda x, y, z: y * z + 2.0 * x * z}[pname]
    N, k = 4, 2
    D = AffineSIPG(N, k, SHEAR)
    K = np.full(D.n_dofs, 1.7)
    xp = D.load_vector(p, nq=k + 2) / D.detJ          # mass matrix |det J| I
    y = D.apply(K, xp).reshape(N ** 3, -1)
    c = np.arange(N ** 3)
    cx, cy, cz = c % N, (c // N) % N, c // (N * N)
    inner = (cx > 0) & (cx < N - 1) & (cy > 0) & (cy < N - 1) & (cz > 0) & (cz < N - 1)
    assert np.abs(y[inner]).max() <= 1e-11 * np.abs(y).max()


@pytest.mark.parametrize("k", [1, 2])
def test_affine_convergence_rate(k):
    from oracle.dg_oracle import AffineSIPG
    A = np.array(SHEAR)
    Ai = np.linalg.inv(A)
    M = Ai @ Ai.T

    def ref_coords(x, y, z):
        X = np.stack(np.broadcast_arrays(x, y, z), axis=-1) @ Ai.T
        return X[..., 0], X[..., 1], X[..., 2]

    def u(x, y, z):
        a, b, c = ref_coords(x, y, z)
        return np.sin(np.pi * a) * np.sin(np.pi * b) * np.sin(np.pi * c)

    def f(x, y, z):
        a, b, c = ref_coords(x, y, z)
        s = [np.sin(np.pi * a), np.sin(np.pi * b), np.sin(np.pi * c)]
        co = [np.cos(np.pi * a), np.cos(np.pi * b), np.cos(np.pi * c)]
        out = np.pi ** 2 * (M[0, 0] + M[1, 1] + M[2, 2]) * s[0] * s[1] * s[2]
        for d in range(3):
            for e in range(3):
                if d != e:
                    other = 3 - d - e
                    out = out - np.pi ** 2 * M[d, e] * co[d] * co[e] * s[other]
        return out

    errs = []
    for N in (2, 4):
        D = AffineSIPG(N, k, A)
        Am = D.assemble(np.ones(D.n_dofs)).tocsc()
        x = spla.spsolve(Am, D.load_vector(f, nq=k + 3))
        errs.append(D.l2_error(x, u))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - (k + 1)) <= 0.35, (errs, rate)


# --------------------------------------------------------------------------
# Multilinear geometry (problem C): trilinear cells from perturbed vertices.
# Affine vertices give the affine operator; on a perturbed mesh the operator
# stays symmetric positive definite, reproduces linear functions on interior
# cells exactly (a linear function of x is trilinear in xi, and every integrand
# of the consistency identity is then a polynomial the Gauss rule integrates
# exactly), and converges at rate k + 1 on a mesh of the unit cube whose
# boundary vertices stay on the faces.
# --------------------------------------------------------------------------

def _perturbed(N, eps, seed, keep_boundary=True):
    from oracle.dg_oracle import lattice
    rng = np.random.default_rng(seed)
    X = lattice(N)
    D = eps / N * rng.uniform(-1.0, 1.0, X.shape)
    if keep_boundary:
        for ax in range(3):
            on = (np.isclose(X[..., ax], 0.0)) | (np.isclose(X[..., ax], 1.0))
            D[..., ax] = np.where(on, 0.0, D[..., ax])
    return X + D


def test_multilinear_affine_vertices_give_the_affine_operator():
    from oracle.dg_oracle import AffineSIPG, MultilinearSIPG, lattice
    for N, k in ((2, 2), (3, 1)):
        K = inputs.lognormal_coefficient(N, k, seed=52, corr_len=0.5)
        A1 = AffineSIPG(N, k, SHEAR).assemble(K)
        A2 = MultilinearSIPG(N, k, lattice(N, SHEAR)).assemble(K)
        assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()


def test_multilinear_perturbed_operator_is_symmetric_positive_definite():
    from oracle.dg_oracle import MultilinearSIPG
    N, k = 3, 2
    D = MultilinearSIPG(N, k, _perturbed(N, 0.25, 53))
    K = inputs.lognormal_coefficient(N, k, seed=54, corr_len=0.1 * 64 / N)
    A = D.assemble(K).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("k", [1, 2])
def test_multilinear_consistency_on_linear_functions(k):
    from oracle.dg_oracle import MultilinearSIPG
    N = 4
    D = MultilinearSIPG(N, k, _perturbed(N, 0.3, 55))
    p = lambda x, y, z: 0.5 + 1.5 * x - 2.0 * y + 0.75 * z
    xp = D.interpolate_reference(p)
    y = D.apply(np.full(D.n_dofs, 2.3), xp).reshape(N ** 3, -1)
    c = np.arange(N ** 3)
    cx, cy, cz = c % N, (c // N) % N, c // (N * N)
    inner = (cx > 0) & (cx < N - 1) & (cy > 0) & (cy < N - 1) & (cz > 0) & (cz < N - 1)
    assert np.abs(y[inner]).max() <= 1e-11 * np.abs(y).max()


@pytest.mark.parametrize("k", [1, 2])
def test_multilinear_convergence_rate(k):
    from oracle.dg_oracle import MultilinearSIPG, lattice

    def mesh(N):   # a smooth displacement that keeps every face of the cube in place
        return lattice(N, perturb=lambda X: 0.08 * np.stack(
            [np.sin(np.pi * X[..., 0]) * np.sin(2 * np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2]),
             np.sin(2 * np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2]),
             np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(2 * np.pi * X[..., 2])],
            axis=-1))

    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * u(x, y, z)
    errs = []
    for N in (4, 6):     # N = 2 is pre-asymptotic (its vertices barely move)
        D = MultilinearSIPG(N, k, mesh(N))
        Am = D.assemble(np.ones(D.n_dofs)).tocsc()
        x = spla.spsolve(Am, D.load_vector(f, nq=k + 3))
        errs.append(D.l2_error(x, u))
    rate = math.log(errs[0] / errs[1]) / math.log(6 / 4)
    assert abs(rate - (k + 1)) <= 0.35, (errs, rate)
