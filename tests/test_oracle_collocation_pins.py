"""Pins of the oracle's scaled Gauss-point (collocation) basis.

Q = W^{1/2} Phi maps a cell's Legendre coefficients to its Gauss-point values
scaled by sqrt(w_q).  The facts checked here do not come from the oracle's
code: the n-point Gauss rule integrates L_i L_j exactly, so Q is orthogonal;
a single Legendre mode has closed-form point values; for one cell with K = 1
the operator is the closed-form Kronecker sum T (+) T (+) T, so Q A Q^T is the
Kronecker sum of q T q^T with the 1D map q = diag(sqrt(w)) B; and CG (Section
2.4) is invariant under an orthogonal change of basis.
"""
import math

import numpy as np
import pytest

from oracle import SIPG, cg, gauss_points, legendre
from paper_1911_01492_gb300 import inputs

from test_oracle_pins import closed_form_T, kron_sum


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8])
def test_collocation_map_is_orthogonal(k):
    D = SIPG(1, k)
    Q = D.collocation_matrix()
    eye = np.eye(D.n3)
    assert np.abs(Q.T @ Q - eye).max() <= 1e-13
    assert np.abs(Q @ Q.T - eye).max() <= 1e-13


@pytest.mark.parametrize("k", [1, 2, 4])
def test_single_modes_have_closed_form_point_values(k):
    """L_0 = 1 gives sqrt(w_a w_b w_e); the mode L_1 along x (index i = 1)
    gives sqrt(3) (2 xi_a - 1) sqrt(w_a w_b w_e), the same along z (l = 1)
    varies with e only: a transposed axis or a missing square root fails."""
    D = SIPG(1, k)
    n = k + 1
    xi, w = gauss_points(n)
    for mode, axis in ((0, None), (1, 0), (n * n, 2), (n, 1)):
        e = np.zeros(D.n3)
        e[mode] = 1.0
        got = D.to_collocation(e)
        for q in range(D.n3):
            a, b, c = q % n, (q // n) % n, q // (n * n)
            ref = math.sqrt(w[a] * w[b] * w[c])
            if axis is not None:
                ref *= math.sqrt(3.0) * (2.0 * xi[(a, b, c)[axis]] - 1.0)
            assert abs(got[q] - ref) <= 1e-14, (mode, q, got[q], ref)


def test_round_trip_on_a_mesh():
    D = SIPG(3, 3)
    x = inputs.uniform_vector(3, 3, 11)
    xh = D.to_collocation(x)
    assert np.abs(D.from_collocation(xh) - x).max() <= 1e-14
    # norms are preserved
    assert abs(np.linalg.norm(xh) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_one_cell_operator_is_the_transformed_kronecker_sum(k):
    D = SIPG(1, k)
    n = k + 1
    xi, w = gauss_points(n)
    B = np.array([[legendre(i, t) for i in range(n)] for t in xi])   # [a, i]
    q1 = np.sqrt(w)[:, None] * B
    ref = kron_sum(q1 @ closed_form_T(k) @ q1.T)
    ones = np.ones(D.n3)
    cols = np.stack([D.collocation_apply(ones, np.eye(D.n3)[j]) for j in range(D.n3)], axis=1)
    assert np.abs(cols - ref).max() <= 1e-12 * np.abs(ref).max()
    # its diagonal (the Jacobi diagonal in this basis)
    d = D.collocation_diagonal(ones)
    assert np.abs(d - np.diag(ref)).max() <= 1e-12 * np.abs(ref).max()


def test_cg_iterates_are_invariant_under_the_change_of_basis():
    N, k = 3, 2
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=5)
    b = inputs.uniform_vector(N, k, 6)
    for it in (1, 2, 3, 7):
        x, _, _, _ = cg(lambda v: D.apply(K, v), b, rtol=1e-30, maxit=it, max_restarts=0)
        xh, _, _, _ = cg(lambda v: D.collocation_apply(K, v), D.to_collocation(b), rtol=1e-30,
                         maxit=it, max_restarts=0)
        assert np.abs(D.from_collocation(xh) - x).max() <= 1e-11 * np.abs(x).max(), it
