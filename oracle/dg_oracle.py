"""FP64 CPU oracle for the symmetric weighted interior-penalty DG operator.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  The CUDA library and its Python
binding never call it, and it shares no code with them.

What it computes (Exa-Dune paper, Section 4.1, the SWIPDG bilinear form b_h;
Section 3.3, matrix-free application of that operator; Section 2.4, the PCG
algorithm), for -div(K grad u) = f on the unit cube with u = 0 on the boundary:

  a(u, v) = sum_cells  sum_q h^3 w_q K_q  grad u . grad v
          + sum_faces  sum_p h^2 w_p gamma_F [ -{d_n u}[v] - {d_n v}[u] + (sigma/h)[u][v] ]

on N^3 cubes of side h = 1/N with the tensor-product orthonormal Legendre basis
L_i(t) = sqrt(2i+1) P_i(2t-1) of degree k per direction, n = k+1 Gauss points
per direction, sigma = 2(k+1)^2, and:
  * interior faces: n points from the lower-index cell (-) to the upper one (+),
    [w] = w- - w+, {w} = (w- + w+)/2;
  * boundary faces: outward n, [w] = w, {w} = w (one-sided);
  * per-cell face coefficient Kbar_c = exp(sum_q w_q log K_{c,q}) (Gauss-weighted
    geometric mean); gamma_F = 2 Kbar- Kbar+ / (Kbar- + Kbar+) on interior faces
    (weighted averages of the SWIPDG method with per-face-constant K) and
    gamma_F = Kbar_c on boundary faces.
Consistency terms carry a MINUS sign (standard symmetric interior penalty; the
printed plus sign yields an inconsistent scheme, see the convergence pins).

Every basis function and gradient is evaluated at every 3D quadrature point
from full 3D tables: there is no sum-factorisation here.  Dense matrix products
(numpy / BLAS) are used as plain library steps.

Parity status: every public function is pinned by tests/test_oracle_pins.py
(closed-form one-cell matrices, the Kronecker-sum identity, symmetry,
positive definiteness and the continuum eigenvalue, consistency on harmonic
polynomials, L2 convergence rates, Euler homogeneity and finite differences of
the gradient, CG against a direct solve, and the per-cell face coefficient and
face weights in closed form for a log K quadratic inside the cells), and by
tests/test_oracle_kron_pins.py (the Kronecker cell blocks against the
assembled blocks of cell-wise constant fields and their volume coefficient in
closed form), and by tests/test_oracle_collocation_pins.py (the scaled
Gauss-point basis: orthogonality, single modes in closed form, the one-cell
K = 1 operator and its diagonal as transformed closed-form Kronecker sums, and
CG's invariance under the change of basis).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# 1D ingredients: Gauss points on [0,1] and the orthonormal Legendre basis.
# ----------------------------------------------------------------------------

def gauss_points(n: int):
    """n-point Gauss-Legendre rule mapped to [0, 1]; weights sum to 1."""
    t, w = npleg.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def legendre(i: int, t):
    """L_i(t) = sqrt(2i+1) P_i(2t - 1), orthonormal on [0, 1]."""
    c = np.zeros(i + 1)
    c[i] = 1.0
    return math.sqrt(2 * i + 1) * npleg.legval(2.0 * np.asarray(t, float) - 1.0, c)


def legendre_deriv(i: int, t):
    """d/dt L_i(t) = 2 sqrt(2i+1) P_i'(2t - 1)."""
    c = np.zeros(i + 1)
    c[i] = 1.0
    return 2.0 * math.sqrt(2 * i + 1) * npleg.legval(
        2.0 * np.asarray(t, float) - 1.0, npleg.legder(c))


# ----------------------------------------------------------------------------
# The discretisation: full 3D tables and face tables.
# ----------------------------------------------------------------------------

class SIPG:
    """SIPG discretisation of -div(K grad u) on N^3 cubes, Q_k Legendre basis.

    Index conventions: cell c = cx + N(cy + N cz); mode m = i + n(j + n l);
    volume point q = a + n(b + n e).  Vectors are arrays of shape (N^3, n^3)
    or their flattening.
    """

    # Boundary conditions.  "dirichlet": u = g on every boundary face (g = 0 in
    # the operator; the weak Dirichlet terms of the SIPG form).  "flow_x": the
    # Section 5 flow problem -- Dirichlet data on the faces x = 0 and x = 1,
    # zero flux (homogeneous Neumann: no boundary face term at all) on the
    # faces y = 0, y = 1, z = 0, z = 1.  Boundary sides in the order
    # (x-, x+, y-, y+, z-, z+).
    BOUNDARY = {"dirichlet": (True,) * 6,
                "flow_x": (True, True, False, False, False, False)}

    def __init__(self, n_cells: int, degree: int, sigma: float | None = None,
                 bc: str = "dirichlet"):
        if n_cells < 1 or degree < 1:
            raise ValueError("need n_cells >= 1 and degree >= 1")
        if bc not in self.BOUNDARY:
            raise ValueError(f"unknown boundary condition {bc!r}")
        self.bc = bc
        self.dirichlet = self.BOUNDARY[bc]
        self.N = n_cells
        self.k = degree
        self.n = n = degree + 1
        self.n3 = n ** 3
        self.h = 1.0 / n_cells
        self.sigma = 2.0 * (degree + 1) ** 2 if sigma is None else float(sigma)
        self.xi, self.w = gauss_points(n)

        # 1D values at the Gauss points and at the two ends of [0, 1]
        L = np.array([[legendre(i, t) for i in range(n)] for t in self.xi])       # [a, i]
        dL = np.array([[legendre_deriv(i, t) for i in range(n)] for t in self.xi])
        ends = {s: (np.array([legendre(i, float(s)) for i in range(n)]),
                    np.array([legendre_deriv(i, float(s)) for i in range(n)])) for s in (0, 1)}

        # Full 3D tables over (q, m): value and reference gradient (d/dxi).
        idx = np.arange(n)
        qa, qb, qe = np.meshgrid(idx, idx, idx, indexing="ij")   # a,b,e
        ma, mb, me = qa, qb, qe
        # flatten with first index fastest: q = a + n(b + n e)
        def flat(A):
            return A.transpose(2, 1, 0).reshape(-1)
        a_, b_, e_ = flat(qa), flat(qb), flat(qe)
        i_, j_, l_ = flat(ma), flat(mb), flat(me)
        self.phi = L[a_][:, i_] * L[b_][:, j_] * L[e_][:, l_]                  # (q, m)
        self.grad = np.stack([dL[a_][:, i_] * L[b_][:, j_] * L[e_][:, l_],
                              L[a_][:, i_] * dL[b_][:, j_] * L[e_][:, l_],
                              L[a_][:, i_] * L[b_][:, j_] * dL[e_][:, l_]], axis=-1)  # (q, m, 3)
        self.wq = self.w[a_] * self.w[b_] * self.w[e_]                           # (q,)

        # Face tables for each axis d and face side s (xi_d = s): value and
        # reference derivative along axis d at the n^2 face points p = s1 + n s2,
        # (s1, s2) = Gauss indices along the two other axes in increasing order.
        self.face_val = {}
        self.face_der = {}
        self.face_w = {}
        P1, P2 = np.meshgrid(idx, idx, indexing="ij")
        p1 = P1.T.reshape(-1)
        p2 = P2.T.reshape(-1)
        for d in range(3):
            t1, t2 = [ax for ax in range(3) if ax != d]
            self.face_w[d] = self.w[p1] * self.w[p2]
            for s in (0, 1):
                Ls, dLs = ends[s]
                val = np.empty((n * n, self.n3))
                der = np.empty((n * n, self.n3))
                for m in range(self.n3):
                    mi = (m % n, (m // n) % n, m // (n * n))
                    # factor along the normal axis d, Gauss factors along t1, t2
                    tang = L[p1, mi[t1]] * L[p2, mi[t2]]
                    val[:, m] = Ls[mi[d]] * tang
                    der[:, m] = dLs[mi[d]] * tang
                self.face_val[(d, s)] = val
                self.face_der[(d, s)] = der

    # -- geometry helpers ------------------------------------------------------
    def cell_coords(self, c):
        N = self.N
        c = np.asarray(c)
        return c % N, (c // N) % N, c // (N * N)

    def stride(self, d: int) -> int:
        return self.N ** d

    @property
    def n_cells_total(self) -> int:
        return self.N ** 3

    @property
    def n_dofs(self) -> int:
        return self.N ** 3 * self.n3

    # -- coefficient -----------------------------------------------------------
    def kbar(self, K):
        """Per-cell face coefficient Kbar_c = exp(sum_q w_q log K_{c,q})."""
        K = np.asarray(K, float).reshape(self.n_cells_total, self.n3)
        return np.exp(np.log(K) @ self.wq)

    def face_gamma(self, Kbar, c, d, upper: bool):
        """gamma on face (c, d, side): harmonic mean with the neighbour across an
        interior face, Kbar_c on a boundary face.  Returns (gamma, interior mask,
        neighbour index)."""
        c = np.asarray(c)
        coord = self.cell_coords(c)[d]
        if upper:
            interior = coord < self.N - 1
            nb = np.where(interior, c + self.stride(d), c)
        else:
            interior = coord > 0
            nb = np.where(interior, c - self.stride(d), c)
        km, kp = Kbar[c], Kbar[nb]
        gamma = np.where(interior, 2.0 * km * kp / (km + kp), km)
        return gamma, interior, nb

    # -- matrix-free application (mode E) -------------------------------------
    def apply(self, K, x, cells=None, chunk: int = 16384):
        """y = A(K) x on the requested cells (all cells by default).

        Element-by-element with the full 3D tables; each face contribution is
        evaluated from the face form with the requested cell as the test side.
        Cells are processed in chunks only to bound memory; every cell's result
        is computed by the same formula.  Returns an array of shape
        (len(cells), n^3) (flattened when cells=None).
        """
        Nc, n3 = self.n_cells_total, self.n3
        K = np.asarray(K, float).reshape(Nc, n3)
        x = np.asarray(x, float).reshape(Nc, n3)
        full = cells is None
        cells = np.arange(Nc) if full else np.asarray(cells, dtype=np.int64)
        Kbar = self.kbar(K)
        y = np.empty((len(cells), n3))
        for s in range(0, len(cells), chunk):
            y[s:s + chunk] = self._apply_cells(K, Kbar, x, cells[s:s + chunk])
        return y.reshape(-1) if full else y

    def _apply_cells(self, K, Kbar, x, cells):
        n3, h, sigma = self.n3, self.h, self.sigma
        # volume: sum_q h w_q K grad^u . grad^phi  (the 1/h^2 of the physical
        # gradients and the h^3 of the volume element leave one factor h)
        Gm = self.grad.transpose(1, 0, 2).reshape(n3, n3 * 3)   # [m, (q, d)]
        gu = (x[cells] @ Gm).reshape(len(cells), n3, 3)         # grad^u at q
        kt = h * self.wq[None, :] * K[cells]
        y = (gu * kt[:, :, None]).reshape(len(cells), n3 * 3) @ Gm.T

        for d in range(3):
            wf = h * self.face_w[d]          # h^2 w_p from the face element times 1/h
            V0, V1 = self.face_val[(d, 0)], self.face_val[(d, 1)]
            D0, D1 = self.face_der[(d, 0)], self.face_der[(d, 1)]
            for upper in (True, False):
                gamma, interior, nb = self.face_gamma(Kbar, cells, d, upper)
                W = gamma[:, None] * wf[None, :]
                xc, xn = x[cells], x[nb]
                if upper:    # this cell is the (-) side; its neighbour the (+) side
                    um, gm = xc @ V1.T, xc @ D1.T
                    up, gp = xn @ V0.T, xn @ D0.T
                    # interior: [phi] = phi-, {d phi} = d phi- / 2
                    Jphi, Aphi = V1, 0.5 * D1
                    # boundary (outward n = +e_d): [u] = u, {d_n u} = d u
                    jump_b, dn_b, Jphi_b, Aphi_b = um, gm, V1, D1
                else:        # this cell is the (+) side
                    um, gm = xn @ V1.T, xn @ D1.T
                    up, gp = xc @ V0.T, xc @ D0.T
                    # interior: [phi] = -phi+, {d phi} = d phi+ / 2
                    Jphi, Aphi = -V0, 0.5 * D0
                    # boundary (outward n = -e_d): [u] = u, {d_n u} = -d u
                    jump_b, dn_b, Jphi_b, Aphi_b = up, -gp, V0, -D0
                jump = um - up
                avg = 0.5 * (gm + gp)
                # -{d_n u}[phi] - {d_n phi}[u] + sigma [u][phi], weighted by W
                y_int = (W * (-avg + sigma * jump)) @ Jphi - (W * jump) @ Aphi
                y_bnd = (W * (-dn_b + sigma * jump_b)) @ Jphi_b - (W * jump_b) @ Aphi_b
                if not self.dirichlet[2 * d + int(upper)]:
                    y_bnd = np.zeros_like(y_bnd)      # zero-flux boundary: no face term
                y += np.where(interior[:, None], y_int, y_bnd)
        return y

    # -- assembled matrix (mode A) ---------------------------------------------
    def assemble(self, K) -> sp.csr_matrix:
        """Assemble A(K) as a CSR matrix from the same volume and face forms."""
        Nc, n3, h, sigma = self.n_cells_total, self.n3, self.h, self.sigma
        K = np.asarray(K, float).reshape(Nc, n3)
        rows, cols, vals = [], [], []
        loc = np.arange(n3)
        R, C = np.meshgrid(loc, loc, indexing="ij")

        def add_block(tc, sc, B):
            rows.append((tc * n3 + R).reshape(-1))
            cols.append((sc * n3 + C).reshape(-1))
            vals.append(B.reshape(-1))

        kt = h * self.wq[None, :] * K
        G = self.grad
        for c in range(Nc):
            B = np.einsum("qmd,q,qnd->mn", G, kt[c], G)
            add_block(c, c, B)

        Kbar = self.kbar(K)
        for d in range(3):
            wf = h * self.face_w[d]
            V0, V1 = self.face_val[(d, 0)], self.face_val[(d, 1)]
            D0, D1 = self.face_der[(d, 0)], self.face_der[(d, 1)]
            # [w] and {d_n w} as linear maps of each side's coefficients
            side = {"m": (V1, 0.5 * D1), "p": (-V0, 0.5 * D0)}
            for c in range(Nc):
                coord = self.cell_coords(c)[d]
                if coord < self.N - 1:
                    cp = c + self.stride(d)
                    km, kp = Kbar[c], Kbar[cp]
                    W = 2.0 * km * kp / (km + kp) * wf
                    for tname, tc in (("m", c), ("p", cp)):
                        Jt, At = side[tname]
                        for sname, sc in (("m", c), ("p", cp)):
                            Js, As = side[sname]
                            B = Jt.T @ (W[:, None] * (-As + sigma * Js)) - At.T @ (W[:, None] * Js)
                            add_block(tc, sc, B)
                if coord == self.N - 1 and self.dirichlet[2 * d + 1]:  # upper boundary, outward +e_d
                    W = Kbar[c] * wf
                    Jt, At = V1, D1
                    add_block(c, c, Jt.T @ (W[:, None] * (-At + sigma * Jt)) - At.T @ (W[:, None] * Jt))
                if coord == 0 and self.dirichlet[2 * d]:               # lower boundary, outward -e_d
                    W = Kbar[c] * wf
                    Jt, At = V0, -D0
                    add_block(c, c, Jt.T @ (W[:, None] * (-At + sigma * Jt)) - At.T @ (W[:, None] * Jt))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(Nc * n3, Nc * n3))
        return A.tocsr()

    # -- diagonal (Jacobi preconditioner, Section 2.4's PCG with M = diag(A)) ---
    def diagonal(self, K, cells=None):
        """diag(A(K)) on the requested cells (all by default): a(phi_m, phi_m)
        from the full 3D volume tables and the full face quadrature, with both
        functions on the cell's own side of every face.  Shape (len(cells), n^3),
        flattened when cells=None."""
        Nc, n3, h, sigma = self.n_cells_total, self.n3, self.h, self.sigma
        K = np.asarray(K, float).reshape(Nc, n3)
        full = cells is None
        cells = np.arange(Nc) if full else np.asarray(cells, dtype=np.int64)
        kt = h * self.wq[None, :] * K[cells]
        g2 = (self.grad ** 2).sum(axis=-1)                  # (q, m): |grad^ phi_m|^2
        dg = kt @ g2
        Kbar = self.kbar(K)
        for d in range(3):
            wf = h * self.face_w[d]
            V0, V1 = self.face_val[(d, 0)], self.face_val[(d, 1)]
            D0, D1 = self.face_der[(d, 0)], self.face_der[(d, 1)]
            for upper in (True, False):
                gamma, interior, _ = self.face_gamma(Kbar, cells, d, upper)
                # own trace J and own share A of {d_n phi} (the whole d_n phi
                # on the boundary); the face form gives sigma J^2 - 2 J A
                if upper:
                    J, A_int, A_bnd = V1, 0.5 * D1, D1
                else:
                    J, A_int, A_bnd = -V0, 0.5 * D0, D0
                f_int = wf @ (sigma * J * J - 2.0 * J * A_int)
                f_bnd = wf @ (sigma * J * J - 2.0 * J * A_bnd)
                if not self.dirichlet[2 * d + int(upper)]:
                    f_bnd = np.zeros_like(f_bnd)
                dg += gamma[:, None] * np.where(interior[:, None], f_int[None, :], f_bnd[None, :])
        return dg.reshape(-1) if full else dg

    # -- scaled Gauss-point (collocation) basis ----------------------------------
    # The per-cell map Q = W^{1/2} Phi, (Q x)_q = sqrt(w_q) u_h(xi_q), takes the
    # Legendre coefficients of a cell to its Gauss-point values scaled by the
    # square roots of the 3D Gauss weights.  The n-point Gauss rule integrates
    # L_i L_j exactly (degree 2n - 2), so Phi^T W Phi = I and Q is orthogonal:
    # the operator Q A Q^T has the spectrum of A, and CG on
    # (Q A Q^T) (Q x) = Q b produces Q times the iterates of CG on A x = b
    # (Section 2.4's PCG with M = I is invariant under orthogonal changes of
    # basis).  Not a construction of the paper: a reformulation of its
    # Section 4.1 operator in another orthonormal basis of the same space.
    def collocation_matrix(self):
        """Q of one cell, shape (n^3 points, n^3 modes)."""
        return np.sqrt(self.wq)[:, None] * self.phi

    def to_collocation(self, x):
        """x_hat = Q x on every cell (Legendre coefficients -> scaled point values)."""
        X = np.asarray(x, float).reshape(self.n_cells_total, self.n3)
        return (X @ self.collocation_matrix().T).reshape(-1)

    def from_collocation(self, xh):
        """x = Q^T x_hat on every cell (the inverse map)."""
        Xh = np.asarray(xh, float).reshape(self.n_cells_total, self.n3)
        return (Xh @ self.collocation_matrix()).reshape(-1)

    def collocation_apply(self, K, xh):
        """(Q A Q^T) x_hat: the operator in the scaled Gauss-point basis."""
        return self.to_collocation(self.apply(K, self.from_collocation(xh)))

    def collocation_diagonal(self, K):
        """diag(Q A Q^T) from the assembled diagonal cell blocks A_cc (small
        meshes only): the Jacobi diagonal of the operator in that basis."""
        Q = self.collocation_matrix()
        blocks = cell_blocks(self.assemble(K), self.n3)
        return np.einsum("qm,cmk,qk->cq", Q, blocks, Q).reshape(-1)

    # -- coefficient gradient ---------------------------------------------------
    def face_form_unit(self, u, v):
        """b_F^{gamma=1}(u, v) for every face side: array (Nc, 6) in the order
        (x-, x+, y-, y+, z-, z+); an interior face appears in both of its cells."""
        Nc, n3, h, sigma = self.n_cells_total, self.n3, self.h, self.sigma
        u = np.asarray(u, float).reshape(Nc, n3)
        v = np.asarray(v, float).reshape(Nc, n3)
        out = np.zeros((Nc, 6))
        cells = np.arange(Nc)
        for d in range(3):
            wf = h * self.face_w[d]
            V0, V1 = self.face_val[(d, 0)], self.face_val[(d, 1)]
            D0, D1 = self.face_der[(d, 0)], self.face_der[(d, 1)]
            for upper in (False, True):
                coord = self.cell_coords(cells)[d]
                if upper:
                    interior = coord < self.N - 1
                    nb = np.where(interior, cells + self.stride(d), cells)
                    mcell, pcell = cells, nb
                else:
                    interior = coord > 0
                    nb = np.where(interior, cells - self.stride(d), cells)
                    mcell, pcell = nb, cells

                def traces(z):
                    zm, dzm = z[mcell] @ V1.T, z[mcell] @ D1.T
                    zp, dzp = z[pcell] @ V0.T, z[pcell] @ D0.T
                    jump, avg = zm - zp, 0.5 * (dzm + dzp)
                    if upper:
                        jb, db = zm, dzm
                    else:
                        jb, db = zp, -dzp
                    I = interior[:, None]
                    return np.where(I, jump, jb), np.where(I, avg, db)

                ju, au = traces(u)
                jv, av = traces(v)
                form = ((-au * jv - av * ju + sigma * ju * jv) * wf[None, :]).sum(1)
                if not self.dirichlet[2 * d + int(upper)]:
                    form = np.where(interior, form, 0.0)   # zero-flux boundary face
                out[:, 2 * d + int(upper)] = form
        return out

    def coeff_grad(self, K, u, v):
        """g[c, q] = d(v^T A(K) u) / d log K_{c,q}.

        Volume: h w_q K_{c,q} grad^u(q) . grad^v(q).  Faces: gamma_F depends on
        K only through Kbar of its cells; d gamma/d log Kbar_c equals
        gamma * Kbar_other / (Kbar_c + Kbar_other) on an interior face and gamma
        on a boundary face, and d log Kbar_c / d log K_{c,q} = w_q.
        """
        Nc, n3, h = self.n_cells_total, self.n3, self.h
        K = np.asarray(K, float).reshape(Nc, n3)
        u = np.asarray(u, float).reshape(Nc, n3)
        v = np.asarray(v, float).reshape(Nc, n3)
        Gm = self.grad.transpose(1, 0, 2).reshape(n3, n3 * 3)
        gu = (u @ Gm).reshape(Nc, n3, 3)
        gv = (v @ Gm).reshape(Nc, n3, 3)
        g = h * self.wq[None, :] * K * (gu * gv).sum(-1)

        Kbar = self.kbar(K)
        bf = self.face_form_unit(u, v)
        cells = np.arange(Nc)
        dface = np.zeros(Nc)
        for d in range(3):
            for upper in (False, True):
                gamma, interior, nb = self.face_gamma(Kbar, cells, d, upper)
                dgam = np.where(interior, gamma * Kbar[nb] / (Kbar + Kbar[nb]), gamma)
                dface += dgam * bf[:, 2 * d + int(upper)]
        return g + dface[:, None] * self.wq[None, :]

    # -- right-hand side and errors --------------------------------------------
    # -- Dirichlet data and the boundary flux (Section 5 flow problem) --------
    def _boundary_cells(self, side: int):
        d, upper = side // 2, bool(side % 2)
        c = np.arange(self.n_cells_total)
        coord = self.cell_coords(c)[d]
        return c[coord == (self.N - 1 if upper else 0)], d, upper

    def dirichlet_rhs(self, K, g):
        """Right-hand side of the weak Dirichlet condition u = g_s on each
        Dirichlet boundary side s (g: six constants, sides x-, x+, y-, y+, z-, z+):
        b_{c,m} = sum over the Dirichlet faces of cell c of
        int_F gamma_F g [ -(d_n phi_m) + (sigma/h) phi_m ] dA,
        by the face Gauss rule (dA = h^2 w_p, d_n = outward derivative / h)."""
        Nc, n3, h, sigma = self.n_cells_total, self.n3, self.h, self.sigma
        Kbar = self.kbar(K)
        b = np.zeros((Nc, n3))
        for side in range(6):
            if not self.dirichlet[side] or g[side] == 0.0:
                continue
            cells, d, upper = self._boundary_cells(side)
            V = self.face_val[(d, int(upper))]             # (p, m)
            Dn = self.face_der[(d, int(upper))] * (1.0 if upper else -1.0)   # outward
            wa = h * h * self.face_w[d]                      # h^2 w_p
            per_m = wa @ (-Dn / h + (sigma / h) * V)         # (m,)
            b[cells] += (Kbar[cells] * g[side])[:, None] * per_m[None, :]
        return b.reshape(-1)

    def boundary_flux(self, K, u, side: int, g: float):
        """Total flux through one Dirichlet boundary side, the quantity of interest
        of Section 5: Q = int_side [ gamma_F d_n u - gamma_F (sigma/h)(u - g) ] dA
        (the boundary flux the SIPG form conserves; n outward).  Summed by the
        face Gauss rule over the side's cells."""
        if not self.dirichlet[side]:
            raise ValueError("the flux is defined on a Dirichlet side")
        h, sigma = self.h, self.sigma
        u = np.asarray(u, float).reshape(self.n_cells_total, self.n3)
        Kbar = self.kbar(K)
        cells, d, upper = self._boundary_cells(side)
        V = self.face_val[(d, int(upper))]
        Dn = self.face_der[(d, int(upper))] * (1.0 if upper else -1.0)
        wa = h * h * self.face_w[d]
        uf = u[cells] @ V.T                                  # (cells, p)
        dnu = (u[cells] @ Dn.T) / h
        q = (Kbar[cells][:, None] * (dnu - (sigma / h) * (uf - g)) * wa[None, :]).sum()
        return float(q)

    def load_vector(self, f, nq: int | None = None):
        """b_{c,m} = int_T f phi_m by an nq-point Gauss rule per direction
        (default nq = n)."""
        nq = self.n if nq is None else nq
        tq, wq1 = gauss_points(nq)
        n, N, h = self.n, self.N, self.h
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])         # [a, i]
        c = np.arange(N ** 3)
        cx, cy, cz = self.cell_coords(c)
        X = (cx[:, None] + tq[None, :]) * h
        Y = (cy[:, None] + tq[None, :]) * h
        Z = (cz[:, None] + tq[None, :]) * h
        F = f(X[:, :, None, None], Y[:, None, :, None], Z[:, None, None, :])   # (c, a, b, e)
        Fw = F * (wq1[:, None, None] * wq1[None, :, None] * wq1[None, None, :])
        # b[c, i, j, l] = h^3 sum_abe Fw L_i(a) L_j(b) L_l(e)
        b = h ** 3 * np.einsum("cabe,ai,bj,el->clji", Fw, Lq, Lq, Lq)
        return b.reshape(-1)

    def l2_error(self, x, u, nq: int | None = None):
        """||u_h - u||_{L2(Omega)} with an nq-point Gauss rule per direction
        (default k + 3)."""
        nq = self.k + 3 if nq is None else nq
        tq, wq1 = gauss_points(nq)
        n, N, h = self.n, self.N, self.h
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        x = np.asarray(x, float).reshape(N ** 3, n, n, n)                      # [c, l, j, i]
        uh = np.einsum("clji,ai,bj,el->cabe", x, Lq, Lq, Lq)
        c = np.arange(N ** 3)
        cx, cy, cz = self.cell_coords(c)
        X = (cx[:, None] + tq[None, :]) * h
        Y = (cy[:, None] + tq[None, :]) * h
        Z = (cz[:, None] + tq[None, :]) * h
        U = u(X[:, :, None, None], Y[:, None, :, None], Z[:, None, None, :])
        W = wq1[:, None, None] * wq1[None, :, None] * wq1[None, None, :]
        return math.sqrt(h ** 3 * float(((uh - U) ** 2 * W[None]).sum()))

    def project(self, p, nq: int | None = None):
        """L2 projection onto the DG space: coefficients x_{c,m} = b_{c,m} / h^3
        (the mass matrix is h^3 I for the orthonormal basis)."""
        return self.load_vector(p, nq) / self.h ** 3


# ----------------------------------------------------------------------------
# Cell-block Jacobi (Section 3.4: block solves on the cells' subspaces V_T,
# factorised): M = the block diagonal of A, one n^3 x n^3 block per cell.
# ----------------------------------------------------------------------------

def cell_blocks(A, n3: int):
    """The diagonal cell blocks of an assembled matrix: array (cells, n3, n3)."""
    A = A.tocsr()
    nc = A.shape[0] // n3
    out = np.empty((nc, n3, n3))
    for c in range(nc):
        out[c] = A[c * n3:(c + 1) * n3, c * n3:(c + 1) * n3].toarray()
    return out


def block_jacobi_inverse(A, n3: int):
    """r -> M^-1 r for M = blockdiag(A_cc), each block inverted (LAPACK)."""
    inv = np.linalg.inv(cell_blocks(A, n3))
    return lambda r: np.einsum("cij,cj->ci", inv, np.asarray(r).reshape(-1, n3)).reshape(-1)


# ----------------------------------------------------------------------------
# Kronecker cell blocks (a reading of Section 3.4's factorised block solves):
# the cell block of A with K replaced by one number per cell, kvol (by default
# the Gauss-weighted arithmetic mean of K over the cell).  For a cell-wise
# constant K the volume part of a cell block is, in the orthonormal basis
# (mass matrix h^3 I), h K (S1 (+) S1 (+) S1) with the 1D stiffness
# S1[i][j] = int_0^1 L_i' L_j', and the own-side part of each face is a 1D
# matrix in the face's normal direction:
#   lower face (xi = 0): h gamma (sigma a0 a0^T + e (d0 a0^T + a0 d0^T)),
#   upper face (xi = 1): h gamma (sigma a1 a1^T - e (d1 a1^T + a1 d1^T)),
# a_s = L(s), d_s = L'(s), e = 1/2 on interior faces (the average) and 1 on
# Dirichlet boundary faces; zero-flux sides contribute nothing.  So the block
# is the Kronecker sum S_x (+) S_y (+) S_z of three n x n matrices.
# ----------------------------------------------------------------------------

def kron_cell_matrices(D, K, kvol=None):
    """Per cell and direction the 1D matrix S_d (array (cells, 3, n, n)) of the
    Kronecker cell block; kvol: one volume coefficient per cell (default: the
    Gauss-weighted arithmetic mean of K over the cell)."""
    n, h, sigma = D.n, D.h, D.sigma
    nc = D.n_cells_total
    dL = np.array([[legendre_deriv(i, t) for i in range(n)] for t in D.xi])   # [a, i]
    S1 = dL.T @ (D.w[:, None] * dL)
    a = {s: np.array([legendre(i, float(s)) for i in range(n)]) for s in (0, 1)}
    d = {s: np.array([legendre_deriv(i, float(s)) for i in range(n)]) for s in (0, 1)}
    Kc = np.asarray(K, float).reshape(nc, D.n3)
    kv = Kc @ D.wq if kvol is None else np.asarray(kvol, float)
    kb = D.kbar(K)
    cells = np.arange(nc)
    S = np.empty((nc, 3, n, n))
    for ax in range(3):
        S[:, ax] = h * kv[:, None, None] * S1[None]
        for upper in (False, True):
            s = 1 if upper else 0
            gamma, interior, _ = D.face_gamma(kb, cells, ax, upper)
            active = interior | D.dirichlet[2 * ax + s]
            e = np.where(interior, 0.5, 1.0)
            sign = -1.0 if upper else 1.0
            sym = np.outer(d[s], a[s]) + np.outer(a[s], d[s])
            F = (sigma * np.outer(a[s], a[s]))[None] + (sign * e)[:, None, None] * sym[None]
            S[:, ax] += np.where(active, h * gamma, 0.0)[:, None, None] * F
    return S


def kron_sum(Sc):
    """The n^3 x n^3 Kronecker sum S_x (+) S_y (+) S_z of one cell (x index
    fastest, as the DOFs)."""
    n = Sc.shape[-1]
    eye = np.eye(n)
    return (np.kron(eye, np.kron(eye, Sc[0])) + np.kron(eye, np.kron(Sc[1], eye))
            + np.kron(Sc[2], np.kron(eye, eye)))


def kron_block_inverse(D, K, kvol=None):
    """r -> M^-1 r for M = the Kronecker cell blocks, each inverted densely."""
    S = kron_cell_matrices(D, K, kvol)
    inv = np.linalg.inv(np.array([kron_sum(S[c]) for c in range(S.shape[0])]))
    n3 = D.n3
    return lambda r: np.einsum("cij,cj->ci", inv, np.asarray(r).reshape(-1, n3)).reshape(-1)


# ----------------------------------------------------------------------------
# Conjugate gradients (Section 2.4, Algorithm PCG, with M = I).
# ----------------------------------------------------------------------------

def cg(apply, b, x0=None, rtol=1e-10, maxit=100000, max_restarts=5, minv=None):
    """CG following the PCG algorithm of Section 2.4.

    minv: None (M = I), an array d with M^-1 r = d * r (a diagonal M), or a
    function r -> M^-1 r (e.g. block_jacobi_inverse below).
    Stops when the recursively updated ||r|| <= rtol ||b||; then recomputes
    b - A x and restarts from x while that true residual is still above rtol.
    Returns (x, total iterations, true relative residual, residual history).
    """
    b = np.asarray(b, float)
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    if minv is None:
        precond = lambda r: r                                   # noqa: E731
    elif callable(minv):
        precond = minv
    else:
        precond = lambda r: np.asarray(minv) * r                # noqa: E731
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0, []
    it = 0
    hist = []
    for _ in range(max_restarts + 1):
        r = b - apply(x)
        p = precond(r)                     # p_1 = M r_0 (M^-1 in the usual notation)
        rho = float(p @ r)                 # rho_1 = <p_1, r_0>
        while it < maxit:
            q = apply(p)                   # q_i = A p_i
            alpha = float(p @ q)           # alpha_i = <p_i, q_i>
            if not alpha > 0.0:
                raise FloatingPointError("CG breakdown: <p, Ap> <= 0")
            x = x + (rho / alpha) * p
            r = r - (rho / alpha) * q
            it += 1
            z = precond(r)                 # z_{i+1} = M r_i
            rnorm = float(np.linalg.norm(r))
            hist.append(rnorm / nb)
            if rnorm <= rtol * nb:
                break
            rho_new = float(z @ r)
            p = (rho_new / rho) * p + z
            rho = rho_new
        true_rel = float(np.linalg.norm(b - apply(x))) / nb
        if true_rel <= rtol or it >= maxit:
            return x, it, true_rel, hist
    return x, it, true_rel, hist


# ----------------------------------------------------------------------------
# Affine geometry (the paper's problem B, Section 3.3): the domain is the image
# of the unit cube under x = A xi for a constant matrix A (det A > 0); cell c
# is the image of its reference cube, x = h A (c + xi_loc), Jacobian J = h A.
# Everything is written with physical quantities, evaluated at the same Gauss
# points: grad = J^-T grad_ref, volume weight |det J| w_q; a face with
# reference axis d has unit normal n = A^-T e_d / |A^-T e_d| (from the
# lower-index cell to the upper one), area element |det J| |J^-T e_d| w_p, and
# penalty length h_F = |T| / |F| = 1 / |J^-T e_d|.  The face form is the same
# SWIPDG form as above with n . grad (all three reference derivatives at the
# face points).  For A = I this is SIPG exactly.
# ----------------------------------------------------------------------------

class AffineSIPG:
    """SIPG on the affine image A [0,1]^3 of the N^3 cube mesh (assembled)."""

    def __init__(self, n_cells: int, degree: int, A, sigma: float | None = None):
        self.base = SIPG(n_cells, degree, sigma=sigma)      # 1D tables, indices, K-bar
        self.N, self.k, self.n, self.n3 = n_cells, degree, degree + 1, (degree + 1) ** 3
        self.h = 1.0 / n_cells
        self.sigma = self.base.sigma
        self.A = np.asarray(A, float).reshape(3, 3)
        if not np.linalg.det(self.A) > 0:
            raise ValueError("the geometry needs det A > 0")
        self.J = self.h * self.A
        self.Jinv = np.linalg.inv(self.J)
        self.detJ = float(np.linalg.det(self.J))
        n = self.n
        xi, w = self.base.xi, self.base.w
        L = np.array([[legendre(i, t) for i in range(n)] for t in xi])
        dL = np.array([[legendre_deriv(i, t) for i in range(n)] for t in xi])
        ends = {s: (np.array([legendre(i, float(s)) for i in range(n)]),
                    np.array([legendre_deriv(i, float(s)) for i in range(n)])) for s in (0, 1)}
        idx = np.arange(n)
        P1, P2 = np.meshgrid(idx, idx, indexing="ij")
        p1, p2 = P1.T.reshape(-1), P2.T.reshape(-1)
        # full reference gradients of every basis function at the face points
        self.face_grad = {}
        for d in range(3):
            t1, t2 = [ax for ax in range(3) if ax != d]
            for s in (0, 1):
                Ls, dLs = ends[s]
                G = np.empty((n * n, self.n3, 3))
                for m in range(self.n3):
                    mi = (m % n, (m // n) % n, m // (n * n))
                    f = {d: (Ls[mi[d]], dLs[mi[d]]),
                         t1: (L[p1, mi[t1]], dL[p1, mi[t1]]),
                         t2: (L[p2, mi[t2]], dL[p2, mi[t2]])}
                    for g in range(3):
                        prod = 1.0
                        for ax in range(3):
                            prod = prod * (f[ax][1] if ax == g else f[ax][0])
                        G[:, m, g] = prod
                self.face_grad[(d, s)] = G

    @property
    def n_dofs(self):
        return self.N ** 3 * self.n3

    def assemble(self, K) -> sp.csr_matrix:
        B = self.base
        Nc, n3, sigma = self.N ** 3, self.n3, self.sigma
        K = np.asarray(K, float).reshape(Nc, n3)
        Jit = self.Jinv.T
        rows, cols, vals = [], [], []
        loc = np.arange(n3)
        R, C = np.meshgrid(loc, loc, indexing="ij")

        def add(tc, sc, M):
            rows.append((tc * n3 + R).reshape(-1))
            cols.append((sc * n3 + C).reshape(-1))
            vals.append(M.reshape(-1))

        Gp = B.grad @ Jit.T                                   # physical gradients (q, m, 3)
        for c in range(Nc):
            wk = self.detJ * B.wq * K[c]
            add(c, c, np.einsum("qmd,q,qnd->mn", Gp, wk, Gp))
        Kbar = B.kbar(K)
        for d in range(3):
            ed = np.zeros(3)
            ed[d] = 1.0
            nrm = Jit @ ed
            area = self.detJ * float(np.linalg.norm(nrm))      # |det J| |J^-T e_d|
            nvec = nrm / np.linalg.norm(nrm)
            hF = 1.0 / float(np.linalg.norm(nrm))
            wa = area * B.face_w[d]
            V0, V1 = B.face_val[(d, 0)], B.face_val[(d, 1)]
            # n . grad at the face points of each side (physical)
            D0 = self.face_grad[(d, 0)] @ (Jit.T @ nvec)
            D1 = self.face_grad[(d, 1)] @ (Jit.T @ nvec)
            side = {"m": (V1, 0.5 * D1), "p": (-V0, 0.5 * D0)}
            for c in range(Nc):
                coord = B.cell_coords(c)[d]
                if coord < self.N - 1:
                    cp = c + B.stride(d)
                    g = 2.0 * Kbar[c] * Kbar[cp] / (Kbar[c] + Kbar[cp])
                    W = g * wa
                    for tn, tc in (("m", c), ("p", cp)):
                        Jt, At = side[tn]
                        for sn, sc in (("m", c), ("p", cp)):
                            Js, As = side[sn]
                            add(tc, sc, Jt.T @ (W[:, None] * (-As + (sigma / hF) * Js))
                                - At.T @ (W[:, None] * Js))
                if coord == self.N - 1 and B.dirichlet[2 * d + 1]:     # outward +n
                    W = Kbar[c] * wa
                    add(c, c, V1.T @ (W[:, None] * (-D1 + (sigma / hF) * V1)) - D1.T @ (W[:, None] * V1))
                if coord == 0 and B.dirichlet[2 * d]:                  # outward -n
                    W = Kbar[c] * wa
                    add(c, c, V0.T @ (W[:, None] * (D0 + (sigma / hF) * V0)) + D0.T @ (W[:, None] * V0))
        Am = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(Nc * n3, Nc * n3))
        return Am.tocsr()

    def apply(self, K, x):
        return self.assemble(K) @ np.asarray(x, float)

    def points(self, nq: int):
        """Physical coordinates of an nq-point Gauss rule in every cell:
        arrays X, Y, Z of shape (cells, nq, nq, nq) over (a, b, e)."""
        tq, _ = gauss_points(nq)
        N, h = self.N, self.h
        c = np.arange(N ** 3)
        cx, cy, cz = self.base.cell_coords(c)
        xi = np.stack(np.broadcast_arrays((cx[:, None, None, None] + tq[None, :, None, None]) * h,
                                          (cy[:, None, None, None] + tq[None, None, :, None]) * h,
                                          (cz[:, None, None, None] + tq[None, None, None, :]) * h),
                      axis=-1)                                   # global reference coords
        x = xi @ self.A.T
        return x[..., 0], x[..., 1], x[..., 2]

    def load_vector(self, f, nq: int | None = None):
        """b_{c,m} = int_T f phi_m dx by an nq-point Gauss rule per direction."""
        nq = self.n if nq is None else nq
        tq, wq1 = gauss_points(nq)
        n = self.n
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        X, Y, Z = self.points(nq)
        Fw = f(X, Y, Z) * (wq1[:, None, None] * wq1[None, :, None] * wq1[None, None, :])
        b = self.detJ * np.einsum("cabe,ai,bj,el->clji", Fw, Lq, Lq, Lq)
        return b.reshape(-1)

    def l2_error(self, x, u, nq: int | None = None):
        nq = self.k + 3 if nq is None else nq
        tq, wq1 = gauss_points(nq)
        n, N = self.n, self.N
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        xc = np.asarray(x, float).reshape(N ** 3, n, n, n)
        uh = np.einsum("clji,ai,bj,el->cabe", xc, Lq, Lq, Lq)
        X, Y, Z = self.points(nq)
        W = wq1[:, None, None] * wq1[None, :, None] * wq1[None, None, :]
        return math.sqrt(self.detJ * float(((uh - u(X, Y, Z)) ** 2 * W[None]).sum()))


# ----------------------------------------------------------------------------
# Multilinear geometry (the paper's problem C): the N^3 mesh with vertices at
# given positions X[i, j, k] (i, j, k = 0..N along x, y, z); each cell is the
# trilinear image of its reference cube, so the Jacobian J(xi) varies from
# point to point.  Volume: sum_q w_q |det J_q| K_q (J_q^-T grad_ref u) .
# (J_q^-T grad_ref v).  A face of reference axis d: at each face point the unit
# normal n = J^-T e_d / |J^-T e_d| and the area element |det J| |J^-T e_d| w_p
# are properties of the shared surface (the same from both cells); the normal
# derivative of each side uses that side's own Jacobian, n . J_side^-T
# grad_ref u_side.  Penalty length h_F = (|T-| + |T+|) / (2 |F|) inside and
# |T| / |F| on the boundary (|T| the cell volume, |F| the face area).  Vertices
# of an affine map give AffineSIPG exactly.
# ----------------------------------------------------------------------------

def _trilinear(Xc, xi):
    """Position and Jacobian of the trilinear map of one cell.  Xc: corner
    positions [dz][dy][dx][3]; xi: points (P, 3).  Returns x (P, 3), J (P, 3, 3)
    with J[p, i, j] = d x_i / d xi_j."""
    xi = np.asarray(xi, float)
    s = [np.stack([1.0 - xi[:, a], xi[:, a]], axis=-1) for a in range(3)]   # (P, 2)
    ds = np.array([-1.0, 1.0])
    x = np.einsum("zyxi,pz,py,px->pi", Xc, s[2], s[1], s[0])
    J = np.stack([np.einsum("zyxi,pz,py,x->pi", Xc, s[2], s[1], ds),
                  np.einsum("zyxi,pz,y,px->pi", Xc, s[2], ds, s[0]),
                  np.einsum("zyxi,z,py,px->pi", Xc, ds, s[1], s[0])], axis=-1)
    return x, J


class MultilinearSIPG:
    """SIPG on the trilinear mesh with vertex positions X (N+1, N+1, N+1, 3),
    indexed [i, j, k] along x, y, z (assembled)."""

    def __init__(self, n_cells: int, degree: int, X, sigma: float | None = None):
        self.base = SIPG(n_cells, degree, sigma=sigma)
        self.N, self.k, self.n, self.n3 = n_cells, degree, degree + 1, (degree + 1) ** 3
        self.sigma = self.base.sigma
        self.X = np.asarray(X, float).reshape(n_cells + 1, n_cells + 1, n_cells + 1, 3)
        n = self.n
        xi, w = self.base.xi, self.base.w
        idx = np.arange(n)
        A, B, E = np.meshgrid(idx, idx, idx, indexing="ij")
        flat = lambda T: T.transpose(2, 1, 0).reshape(-1)          # q = a + n(b + n e)
        self.qxi = np.stack([xi[flat(A)], xi[flat(B)], xi[flat(E)]], axis=-1)
        P1, P2 = np.meshgrid(idx, idx, indexing="ij")
        p1, p2 = P1.T.reshape(-1), P2.T.reshape(-1)
        self.fxi = {}
        for d in range(3):
            t1, t2 = [ax for ax in range(3) if ax != d]
            for s in (0, 1):
                pts = np.zeros((n * n, 3))
                pts[:, d] = float(s)
                pts[:, t1] = xi[p1]
                pts[:, t2] = xi[p2]
                self.fxi[(d, s)] = pts
        self.aff = AffineSIPG(n_cells, degree, np.eye(3), sigma=sigma)   # face gradient tables

    @property
    def n_dofs(self):
        return self.N ** 3 * self.n3

    def corners(self, c):
        cx, cy, cz = (int(v) for v in self.base.cell_coords(c))
        Xc = np.empty((2, 2, 2, 3))
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    Xc[dz, dy, dx] = self.X[cx + dx, cy + dy, cz + dz]
        return Xc

    def cell_volume(self, c):
        _, J = _trilinear(self.corners(c), self.qxi)
        return float(np.sum(self.base.wq * np.abs(np.linalg.det(J))))

    def _face(self, c, d, s):
        """Face data of cell c on its side s of axis d: area element (P,),
        unit normal (P, 3) (along +e_d), and the operator of the normal
        derivative on the cell's own side (P, n3)."""
        _, J = _trilinear(self.corners(c), self.fxi[(d, s)])
        Jinv = np.linalg.inv(J)
        ed = np.zeros(3)
        ed[d] = 1.0
        nrm = np.einsum("pji,j->pi", Jinv, ed)                   # J^-T e_d
        lens = np.linalg.norm(nrm, axis=1)
        area = np.abs(np.linalg.det(J)) * lens * self.base.face_w[d]
        nvec = nrm / lens[:, None]
        m = np.einsum("pij,pj->pi", Jinv, nvec)                  # J^-1 n
        Dn = np.einsum("pmg,pg->pm", self.aff.face_grad[(d, s)], m)
        return area, nvec, Dn

    def assemble(self, K) -> sp.csr_matrix:
        B = self.base
        Nc, n3, sigma = self.N ** 3, self.n3, self.sigma
        K = np.asarray(K, float).reshape(Nc, n3)
        rows, cols, vals = [], [], []
        loc = np.arange(n3)
        R, C = np.meshgrid(loc, loc, indexing="ij")

        def add(tc, sc, M):
            rows.append((tc * n3 + R).reshape(-1))
            cols.append((sc * n3 + C).reshape(-1))
            vals.append(M.reshape(-1))

        vol = np.empty(Nc)
        for c in range(Nc):
            _, J = _trilinear(self.corners(c), self.qxi)
            Jinv = np.linalg.inv(J)
            detJ = np.abs(np.linalg.det(J))
            vol[c] = float(np.sum(B.wq * detJ))
            Gp = np.einsum("qmg,qgi->qmi", B.grad, Jinv)          # (J^-T grad)_i = sum_g grad_g Jinv[g, i]
            wk = detJ * B.wq * K[c]
            add(c, c, np.einsum("qmd,q,qnd->mn", Gp, wk, Gp))
        Kbar = B.kbar(K)
        for d in range(3):
            V0, V1 = B.face_val[(d, 0)], B.face_val[(d, 1)]
            for c in range(Nc):
                coord = B.cell_coords(c)[d]
                if coord < self.N - 1:
                    cp = c + B.stride(d)
                    area, _, Dm = self._face(c, d, 1)
                    _, _, Dp = self._face(cp, d, 0)
                    hF = 0.5 * (vol[c] + vol[cp]) / area.sum()
                    g = 2.0 * Kbar[c] * Kbar[cp] / (Kbar[c] + Kbar[cp])
                    W = g * area
                    side = {"m": (V1, 0.5 * Dm), "p": (-V0, 0.5 * Dp)}
                    for tn, tc in (("m", c), ("p", cp)):
                        Jt, At = side[tn]
                        for sn, sc in (("m", c), ("p", cp)):
                            Js, As = side[sn]
                            add(tc, sc, Jt.T @ (W[:, None] * (-As + (sigma / hF) * Js))
                                - At.T @ (W[:, None] * Js))
                if coord == self.N - 1 and B.dirichlet[2 * d + 1]:
                    area, _, D1 = self._face(c, d, 1)
                    hF = vol[c] / area.sum()
                    W = Kbar[c] * area
                    add(c, c, V1.T @ (W[:, None] * (-D1 + (sigma / hF) * V1)) - D1.T @ (W[:, None] * V1))
                if coord == 0 and B.dirichlet[2 * d]:
                    area, _, D0 = self._face(c, d, 0)
                    hF = vol[c] / area.sum()
                    W = Kbar[c] * area
                    add(c, c, V0.T @ (W[:, None] * (D0 + (sigma / hF) * V0)) + D0.T @ (W[:, None] * V0))
        Am = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(Nc * n3, Nc * n3))
        return Am.tocsr()

    def apply(self, K, x):
        return self.assemble(K) @ np.asarray(x, float)

    def _cell_points(self, nq):
        tq, wq1 = gauss_points(nq)
        P = np.stack(np.meshgrid(tq, tq, tq, indexing="ij"), axis=-1)   # [a, b, e] -> (xi1, xi2, xi3)
        P = P.transpose(0, 1, 2, 3).reshape(-1, 3)
        W = (wq1[:, None, None] * wq1[None, :, None] * wq1[None, None, :]).reshape(-1)
        return tq, P, W

    def load_vector(self, f, nq: int | None = None):
        """b_{c,m} = int_T f phi_m dx (nq-point Gauss rule per direction)."""
        nq = self.n + 1 if nq is None else nq
        tq, P, W = self._cell_points(nq)
        n = self.n
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        out = np.empty((self.N ** 3, self.n3))
        for c in range(self.N ** 3):
            x, J = _trilinear(self.corners(c), P)
            fw = (f(x[:, 0], x[:, 1], x[:, 2]) * W * np.abs(np.linalg.det(J))).reshape(nq, nq, nq)
            out[c] = np.einsum("abe,ai,bj,el->lji", fw, Lq, Lq, Lq).reshape(-1)
        return out.reshape(-1)

    def interpolate_reference(self, p, nq: int | None = None):
        """Coefficients of (p o x)(xi) by the L2 projection in reference
        coordinates (exact when p o x lies in Q_k, e.g. p linear in x)."""
        nq = self.n + 2 if nq is None else nq
        tq, P, W = self._cell_points(nq)
        n = self.n
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        out = np.empty((self.N ** 3, self.n3))
        for c in range(self.N ** 3):
            x, _ = _trilinear(self.corners(c), P)
            pw = (p(x[:, 0], x[:, 1], x[:, 2]) * W).reshape(nq, nq, nq)
            out[c] = np.einsum("abe,ai,bj,el->lji", pw, Lq, Lq, Lq).reshape(-1)
        return out.reshape(-1)

    def l2_error(self, xc, u, nq: int | None = None):
        nq = self.k + 3 if nq is None else nq
        tq, P, W = self._cell_points(nq)
        n = self.n
        Lq = np.array([[legendre(i, t) for i in range(n)] for t in tq])
        xc = np.asarray(xc, float).reshape(self.N ** 3, n, n, n)
        tot = 0.0
        for c in range(self.N ** 3):
            x, J = _trilinear(self.corners(c), P)
            uh = np.einsum("lji,ai,bj,el->abe", xc[c], Lq, Lq, Lq).reshape(-1)
            tot += float(np.sum((uh - u(x[:, 0], x[:, 1], x[:, 2])) ** 2 * W * np.abs(np.linalg.det(J))))
        return math.sqrt(tot)


def lattice(n_cells: int, A=None, perturb=None):
    """Vertex positions (N+1, N+1, N+1, 3) of the uniform lattice on [0,1]^3,
    mapped by x -> A x and then displaced by perturb(x) (a function of the
    positions returning displacements)."""
    t = np.linspace(0.0, 1.0, n_cells + 1)
    X = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1)
    if A is not None:
        X = X @ np.asarray(A, float).T
    if perturb is not None:
        X = X + perturb(X)
    return X
