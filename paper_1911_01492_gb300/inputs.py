"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the discretisation itself.  It draws random
vectors and the random permeability field that the problem statement takes as
given (Section 5: a lognormal field with exponential covariance, sampled by
circulant embedding and FFT), and lays them out in the library's
[cell][e][b][a] quadrature-point order.

Layout conventions (shared by every producer and consumer):
  * cell c = cx + N*(cy + N*cz) for an N^3 mesh of the unit cube;
  * per-cell DOF m = i + n*(j + n*l) (i = x-mode fastest), n = degree + 1;
  * per-cell quadrature point q = a + n*(b + n*e) (a = x point fastest).
"""
from __future__ import annotations

import numpy as np

try:  # scipy's FFT has a thread pool; numpy's is the fallback
    import scipy.fft as _fft
    _FFT_KW = {"workers": -1}
except ImportError:  # pragma: no cover - scipy is present on both machines
    import numpy.fft as _fft
    _FFT_KW = {}


def n_dofs(n_cells: int, degree: int) -> int:
    """Total number of DOFs of a Q_degree DG space on n_cells^3 cubes."""
    return n_cells ** 3 * (degree + 1) ** 3


def uniform_vector(n_cells: int, degree: int, seed: int) -> np.ndarray:
    """x ~ U[-1, 1] per DOF, float64, drawn with numpy's PCG64 from `seed`."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n_dofs(n_cells, degree))


def unit_coefficient(n_cells: int, degree: int) -> np.ndarray:
    """K = 1 at every volume quadrature point."""
    return np.ones(n_dofs(n_cells, degree))


def constant_load_vector(n_cells: int, degree: int) -> np.ndarray:
    """Load vector of f = 1: b_{c,m} = h^3 * delta_{m,0}.

    With the orthonormal Legendre basis on [0,1] every mode except the constant
    one integrates to zero and the constant mode integrates to one, so the
    integral of f*phi_{c,m} over a cube of side h is h^3 for m = 0 only.
    """
    n3 = (degree + 1) ** 3
    b = np.zeros((n_cells ** 3, n3))
    b[:, 0] = (1.0 / n_cells) ** 3
    return b.reshape(-1)


_EIG_CACHE: dict = {}


def _embedding_eigenvalues(M: int, corr_len: float, variance: float):
    """Eigenvalues of the periodic (period 2M) embedding of the covariance
    C(r) = variance * exp(-r / corr_len) on a uniform grid of spacing 1/M.

    Returns (eigenvalues clipped at zero, relative mass of the clipped part).
    """
    key = (M, corr_len, variance)
    if key in _EIG_CACHE:
        return _EIG_CACHE[key]
    P = 2 * M
    d = 1.0 / M
    k = np.arange(P)
    k = np.minimum(k, P - k) * d
    r = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    c = variance * np.exp(-r / corr_len)
    lam = _fft.fftn(c, **_FFT_KW).real
    neg = lam < 0
    clipped = float(-lam[neg].sum() / lam.sum()) if neg.any() else 0.0
    lam = np.where(neg, 0.0, lam)
    _EIG_CACHE.clear()  # keep one embedding resident at most (they can be GBs)
    _EIG_CACHE[key] = (lam, clipped)
    return lam, clipped


def gaussian_random_field(M: int, seed: int, corr_len: float = 0.1,
                          variance: float = 1.0):
    """Zero-mean Gaussian field on an M^3 grid of spacing 1/M with covariance
    variance*exp(-||x-y||_2/corr_len), by circulant embedding (period 2M) and FFT.

    Draws one complex standard-normal array on the (2M)^3 torus from `seed`;
    the real part of FFT(sqrt(lambda/P^3) * xi) restricted to the first M^3
    slots has exactly the embedded covariance.  Eigenvalues below zero are
    clipped to zero; the clipped relative mass is returned with the field.
    Returns (field[ix, iy, iz] as float64 with shape (M, M, M), clipped_mass).
    """
    lam, clipped = _embedding_eigenvalues(M, corr_len, variance)
    P = 2 * M
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((P, P, P)) + 1j * rng.standard_normal((P, P, P))
    xi *= np.sqrt(lam / P ** 3)
    y = _fft.fftn(xi, overwrite_x=True, **_FFT_KW)
    return np.ascontiguousarray(y.real[:M, :M, :M]), clipped


def lognormal_coefficient(n_cells: int, degree: int, seed: int,
                          corr_len: float = 0.1, variance: float = 1.0) -> np.ndarray:
    """K = exp(G) at every volume Gauss point, G a Gaussian random field.

    G is sampled on the uniform (N*n)^3 grid of spacing h/n; the value at grid
    slot (cx*n + a, cy*n + b, cz*n + e) is assigned to Gauss point (a, b, e) of
    cell (cx, cy, cz).  Returns a flat float64 array in [c][e][b][a] order.
    """
    N, n = n_cells, degree + 1
    M = N * n
    g, _ = gaussian_random_field(M, seed, corr_len, variance)
    # g[ix, iy, iz] with ix = cx*n + a  ->  K[cz, cy, cx, e, b, a]
    g = g.reshape(N, n, N, n, N, n)            # (cx, a, cy, b, cz, e)
    g = g.transpose(4, 2, 0, 5, 3, 1)          # (cz, cy, cx, e, b, a)
    return np.exp(np.ascontiguousarray(g).reshape(-1))


def values_at_gauss_points(n_cells: int, degree: int, func) -> np.ndarray:
    """func(x, y, z) evaluated at every volume Gauss point of the mesh (the
    n = degree + 1 point Gauss-Legendre rule per direction, mapped to each
    cell), in the [c][e][b][a] layout of K.  Used for given data such as a
    source term f or a prescribed coefficient."""
    N, n = n_cells, degree + 1
    t, _ = np.polynomial.legendre.leggauss(n)
    xi = 0.5 * (t + 1.0)
    h = 1.0 / N
    pos = (np.arange(N)[:, None] + xi[None, :]).reshape(-1) * h     # slot cx*n + a
    X = pos[None, None, :]
    Y = pos[None, :, None]
    Z = pos[:, None, None]
    v = np.broadcast_to(func(X, Y, Z), (N * n, N * n, N * n))      # [iz, iy, ix]
    v = v.reshape(N, n, N, n, N, n)                                  # (cz, e, cy, b, cx, a)
    v = v.transpose(0, 2, 4, 1, 3, 5)                                # (cz, cy, cx, e, b, a)
    return np.ascontiguousarray(v, dtype=np.float64).reshape(-1)


def lognormal_on_levels(levels, seed: int, corr_len: float = 0.1,
                        variance: float = 1.0):
    """One lognormal realization K = exp(G) seen by several meshes (the coupled
    samples of a multilevel Monte-Carlo difference Q_l - Q_{l-1}).

    levels: list of (n_cells, degree).  G is sampled once, on the uniform
    M^3 grid of the finest level (M = max n_cells * (degree + 1)), and every
    level's Gauss point takes the value of the grid slot that contains it.
    Returns one flat float64 array per level in the [c][e][b][a] layout.
    """
    M = max(N * (k + 1) for N, k in levels)
    g, _ = gaussian_random_field(M, seed, corr_len, variance)    # g[ix, iy, iz]
    out = []
    for N, k in levels:
        n = k + 1
        t, _ = np.polynomial.legendre.leggauss(n)
        xi = 0.5 * (t + 1.0)
        pos = (np.arange(N)[:, None] + xi[None, :]).reshape(-1) / N   # cx*n + a
        slot = np.minimum((pos * M).astype(np.int64), M - 1)
        v = g[np.ix_(slot, slot, slot)]                  # [ix, iy, iz] over (cx,a),(cy,b),(cz,e)
        v = v.reshape(N, n, N, n, N, n).transpose(4, 2, 0, 5, 3, 1)   # (cz, cy, cx, e, b, a)
        out.append(np.exp(np.ascontiguousarray(v).reshape(-1)))
    return out
