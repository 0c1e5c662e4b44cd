/*
 * dg.h -- C ABI of the GB300 matrix-free SIPG-DG library.
 *
 * Operator: the symmetric weighted interior-penalty DG form of the Exa-Dune
 * paper, Section 4.1 (bilinear form b_h with face coupling terms), for
 * -div(K grad u) = f on the unit cube, u = 0 on the boundary, discretised on
 * n_cells^3 axis-aligned cubes of side h = 1/n_cells with the tensor-product
 * orthonormal Legendre basis L_i(t) = sqrt(2i+1) P_i(2t-1) of degree k in each
 * direction (Section 3.3: matrix-free application by sum factorisation).
 * Readings of the paper used here: consistency terms with a minus sign;
 * penalty sigma/h with sigma = 2(k+1)^2; per-cell face coefficient
 * Kbar_c = exp(sum_q w_q log K_{c,q}); face weight gamma_F = harmonic mean of
 * the two cells' Kbar on interior faces, Kbar_c on boundary faces.
 *
 * Layouts (all vectors are dense, unpadded, contiguous):
 *   cell      c = cx + N*(cy + N*cz),                    N = n_cells
 *   DOF       m = i + n*(j + n*l)  (x-mode i fastest),   n = k + 1
 *   vector    v[c*n^3 + m]          (a cell's DOFs are contiguous)
 *   quad pt   q = a + n*(b + n*e)  (x-point a fastest), n Gauss points per direction
 *   K, g      K[c*n^3 + q]
 *
 * Conventions.  Every function returns DG_OK (0) or a DG_ERR_* code and, on
 * error, sets a thread-local message readable with dg_last_error().  Device
 * pointers are raw CUDA device addresses owned by the caller; the library owns
 * only the opaque mesh handle and the device workspaces it allocates.  `stream`
 * is a cudaStream_t passed as void* (NULL = the legacy default stream); work is
 * enqueued on it asynchronously unless a function says it blocks.  Calls that
 * share a mesh must not run concurrently on different streams: they share the
 * mesh's workspaces.
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DG_OK = 0,
  DG_ERR_INVALID_ARG = 1,   /* bad pointer, size, mode, aliasing, or invalid K  */
  DG_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details) */
  DG_ERR_NOT_CONVERGED = 3, /* CG reached maxit before the tolerance            */
  DG_ERR_BREAKDOWN = 4,     /* CG saw <p, Ap> <= 0 or a non-finite scalar        */
  DG_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                */
  DG_ERR_OOM = 6            /* a device allocation failed                        */
};

enum { DG_FP64 = 0, DG_FP32 = 1 };            /* operator precision            */
enum { DG_CG_FP64 = 0, DG_CG_MIXED_IR = 1, DG_CG_MIXED_IR_RESTART = 2 };  /* dg_cg_solve modes */
enum { DG_CG_PRECOND_JACOBI = 256 };  /* OR into a mode: PCG with M = diag(A) */
enum { DG_CG_PRECOND_BLOCK = 512 };   /* OR into DG_CG_FP64: PCG with M = the cell blocks of A */
enum { DG_CG_PRECOND_KRON = 1024 };   /* OR into DG_CG_FP64 or DG_CG_MIXED_IR: Kronecker cell blocks */
enum { DG_CG_NODAL = 2048 };          /* OR into DG_CG_FP64 or DG_CG_MIXED_IR: iterate in the scaled Gauss-point basis */
/* Boundary conditions (dg_set_boundary): bit f set = boundary side f is Dirichlet,
 * sides in the order x-, x+, y-, y+, z-, z+; the other sides carry zero flux. */
enum { DG_BC_DIRICHLET = 0x3F, DG_BC_FLOW_X = 0x03 };

typedef struct dg_mesh dg_mesh;

/* Per-solve statistics (written by the solvers). */
typedef struct {
  int iterations;          /* CG iterations (inner iterations for MIXED_IR)         */
  int outer_iterations;    /* refinement steps (MIXED_IR), restarts (FP64)          */
  double rel_residual;     /* ||b - A x||_2 / ||b||_2 recomputed in FP64 at the end */
  double rel_residual_rec; /* last recursively updated residual norm / ||b||        */
  double seconds;          /* wall time of the solve on the host                    */
  int status;              /* DG_OK or the error code the solve returned            */
} dg_cg_stats;

/* Last error message of the calling thread ("" if none).  The pointer stays
 * valid until the next failing call on this thread.  (Library bookkeeping; the
 * paper has no counterpart.) */
const char* dg_last_error(void);

/* Create a mesh of n_cells^3 cubes of the unit cube with Q_degree elements,
 * 1 <= n_cells <= 1024, 1 <= degree <= 8, on the current CUDA device.
 * Section 4.1 (continuous problem and discretization): the fine partition of
 * the domain and the broken polynomial space V on it on which the SWIPDG form
 * is posed; here the partition is n_cells^3 axis-aligned cubes and V is the
 * tensor-product Q_degree space of each cube (Section 3.3 uses the same
 * tensor-product structure for sum factorisation).
 * Allocates the device workspaces (coefficient data, traces).  K is unset
 * until dg_set_coefficient.  Errors: INVALID_ARG, OOM, CUDA. */
int dg_create_mesh(int n_cells, int degree, dg_mesh** out);

/* Free the mesh and its workspaces (NULL is accepted). Synchronises the device.
 * (Library bookkeeping; the paper has no counterpart.) */
int dg_destroy_mesh(dg_mesh* mesh);

/* Sizes: DOFs (= n_cells^3 (degree+1)^3), cells, n = degree+1, sigma (the
 * penalty factor sigma_e of the Section 4.1 face form).  Any output pointer
 * may be NULL. */
int dg_mesh_info(const dg_mesh* mesh, long long* n_dofs, long long* n_cells_total,
                 int* n_points_1d, double* sigma);

/* Boundary conditions of the mesh: bit f of dirichlet_mask set = boundary side f
 * (x-, x+, y-, y+, z-, z+) carries a weak Dirichlet condition (the SIPG boundary
 * face terms; the data enter only the right-hand side, dg_dirichlet_rhs); a
 * clear bit = zero flux (homogeneous Neumann: no boundary face term).
 * DG_BC_DIRICHLET (default, every side) is the Section 4.1 problem in H^1_0;
 * DG_BC_FLOW_X is the Section 5 flow problem (p given on x = 0 and x = 1, zero
 * flux on the other four sides).  Drops the coefficient (and the Jacobi
 * diagonal): call dg_set_coefficient again afterwards.  Errors: INVALID_ARG
 * (NULL mesh, mask outside 1..0x3f: at least one side must be Dirichlet). */
int dg_set_boundary(dg_mesh* mesh, int dirichlet_mask);

/* Affine geometry (the paper's problem B, Section 3.3: affine cells): the mesh
 * becomes the image of the unit-cube mesh under x = A xi, A a 3x3 matrix (host
 * array, row-major) with det A > 0; every cell is then a parallelepiped with
 * Jacobian h A.  The operator is the same SWIPDG form written with the
 * physical gradients, face normals, face areas and penalty length |T| / |F|.
 * A = I (the default) is the unit cube (and ends a multilinear geometry set
 * by dg_set_vertices).  On a non-identity geometry the FP64
 * dg_apply / dg_apply_adjoint, dg_load_vector (f at the mapped Gauss points)
 * and dg_cg_solve with DG_CG_FP64 (no preconditioner) are available; the
 * other calls return INVALID_ARG.  Drops the coefficient: call
 * dg_set_coefficient again afterwards.  Errors: INVALID_ARG (NULL pointer,
 * non-finite entry, det A <= 0), CUDA. */
int dg_set_geometry(dg_mesh* mesh, const double* A);

/* Multilinear geometry (the paper's problem C, Section 3.3: multilinear
 * geometries): the vertices of the structured mesh moved to the positions X
 * (host array of (n_cells+1)^3 points x 3 doubles; vertex (i, j, k) along x, y,
 * z at ((k (N+1) + j) (N+1) + i) * 3); every cell is the trilinear image of its
 * reference cube.  The operator is the SWIPDG form with the physical gradients
 * at every quadrature point, the surface normal and area element at every face
 * point, each side's own Jacobian in its normal derivative, and penalty length
 * h_F = (|T-| + |T+|) / (2 |F|) (|T| / |F| on the boundary).  Forms the
 * per-point geometry once (about 8 doubles per DOF).  The same calls as on an
 * affine geometry are available; dg_set_geometry returns to an affine one.
 * Drops the coefficient.  Errors: INVALID_ARG (NULL pointer, non-finite
 * coordinate, a cell with non-positive Jacobian determinant), OOM, CUDA. */
int dg_set_vertices(dg_mesh* mesh, const double* X);

/* Set the diffusion coefficient K (device pointer, FP64, layout K[c*n^3 + q],
 * values at the volume Gauss points).  K is the coefficient A = lambda kappa of
 * the Section 4.1 problem -div(A grad p) = f (here a scalar field); Section 5
 * draws it as a lognormal random field, the workload this library targets.
 * Derives the weighted volume factors
 * h w_q K (FP64 and FP32 copies), Kbar per cell and gamma per face side.
 * Blocks until done: K <= 0 or non-finite anywhere returns INVALID_ARG and
 * leaves the mesh without a coefficient. */
int dg_set_coefficient(dg_mesh* mesh, const double* K, void* stream);

/* y = A(K) x (Section 3.3 matrix-free application of the Section 4.1 form).
 * x, y: device pointers to n_dofs values of type double (prec = DG_FP64) or
 * float (prec = DG_FP32); y is overwritten; x == y returns INVALID_ARG
 * (overlapping ranges are not detected).  The FP32 operator computes and
 * accumulates in FP32 from FP32-rounded tables and coefficients. */
int dg_apply(const dg_mesh* mesh, const void* x, void* y, int prec, void* stream);

/* xbar = A(K)^T ybar.  The paper has no counterpart: this is the adjoint that
 * differentiation through dg_apply needs.  The Section 4.1 SWIPDG form is
 * symmetric (b(v,w) = b(w,v)), so the transposed data flow (test functions <->
 * trial functions) is the same sequence of contractions; arguments as
 * dg_apply. */
int dg_apply_adjoint(const dg_mesh* mesh, const void* ybar, void* xbar, int prec, void* stream);

/* Same as dg_apply but x and y are HOST buffers (pinned or pageable): the
 * Section 3.3 operator application with the host<->device copies inside the
 * call (the paper has no counterpart; it runs on host memory throughout).  The
 * mesh is cut into at most 16 slabs of z-layers: x is copied in slab by slab
 * on a copy stream, pass 1 of each slab runs on an internal stream as soon as
 * its x has arrived, pass 2 of slab s runs on `stream` once pass 1 has covered
 * slab s+1, and y is copied back slab by slab on a second copy stream, so that
 * with pinned buffers both copies overlap the kernels.  Blocks until y is
 * written.  Not recorded by dg_timing_enable. */
int dg_apply_host(const dg_mesh* mesh, const void* x_host, void* y_host, int prec, void* stream);

/* g[c*n^3 + q] = d(v^T A(K) u) / d log K_{c,q}  (FP64 device pointers, g
 * overwritten).  The paper has no counterpart: this differentiates the
 * Section 4.1 form b(u, v) with respect to the log of its coefficient A at the
 * volume Gauss points (the gradient that a loss on the Section 5 lognormal
 * field needs).  Volume part h w_q K_q grad u . grad v at the point; face part
 * w_q * sum over the cell's faces of d gamma_F / d log Kbar_c times the face
 * form with gamma = 1.  g must not alias u or v. */
int dg_coeff_grad(const dg_mesh* mesh, const double* u, const double* v, double* g, void* stream);

/* Solve A(K) x = b by CG (Section 2.4's PCG; M = I unless the mode adds
 * DG_CG_PRECOND_JACOBI).  b, x: FP64 device
 * pointers; x holds the initial guess on entry and the solution on exit.
 * mode DG_CG_FP64: FP64 operator and vectors.
 * mode DG_CG_MIXED_IR: mixed-precision CG with iterative refinement of the
 *   residual: the CG recurrence runs on the FP32 operator with FP32 vectors and
 *   FP64-accurate inner products; each time its residual has dropped by 5x
 *   the FP32 correction is added to x in FP64 and r = b - A x is recomputed
 *   with the FP64 operator and replaces the FP32 residual (the search
 *   direction is kept).
 * mode DG_CG_MIXED_IR_RESTART: classical iterative refinement: FP64 outer
 *   residual and update, each correction solved from zero by FP32 CG to a 10x
 *   residual reduction.
 * mode | DG_CG_PRECOND_JACOBI: any of the above as PCG with M = diag(A)
 *   (Section 2.4's PCG algorithm); the diagonal is formed on the first such
 *   solve after dg_set_coefficient (one kernel, see dg_diagonal).
 * DG_CG_FP64 | DG_CG_PRECOND_BLOCK: PCG with M = the block diagonal of A, one
 *   n^3 x n^3 block per cell (its own volume and own-side face terms), stored
 *   inverted in FP64 (the factorised block solves on the cell subspaces of
 *   Section 3.4); formed on the first such solve after dg_set_coefficient
 *   (degree 1..4; n^6 doubles per cell, e.g. 125 KB per cell at degree 4);
 *   BREAKDOWN if a block is not positive definite.
 * DG_CG_FP64 or DG_CG_MIXED_IR | DG_CG_PRECOND_KRON: PCG with M = the
 *   Kronecker cell blocks: each cell block of the operator with K replaced by
 *   its Gauss-weighted mean over the cell, which in the orthonormal basis is
 *   the Kronecker sum S_x (+) S_y (+) S_z of three n x n matrices (1D
 *   stiffness times h Kmean plus the own-side terms of the two faces of that
 *   direction, Section 4.1); applied by fast diagonalisation (per cell three
 *   eigenbases and eigenvalues, 3n^2 + 3n values; 12n flops per DOF), in FP32
 *   inside the mixed mode.  A reading of the factorised cell-block solves of
 *   Section 3.4 that costs O(n) per DOF instead of O(n^3).  Formed on the
 *   first such solve after dg_set_coefficient (any degree); BREAKDOWN if a 1D
 *   factor has a negative eigenvalue (a direction with only zero-flux faces,
 *   one cell across, has a singular factor, which is allowed).
 * DG_CG_FP64 or DG_CG_MIXED_IR | DG_CG_NODAL (M = I, DG_CG_PRECOND_JACOBI or
 *   DG_CG_PRECOND_KRON): the same CG run on (Q A Q^T) x_hat = Q b in the
 *   scaled Gauss-point basis of dg_to_nodal, the FP32 operator of the mixed
 *   mode and its FP64 refinements included.  Q is orthogonal, so with M = I
 *   the iterates are Q times those of the Legendre-basis CG (in exact
 *   arithmetic), and so they are with the Kronecker cell blocks, whose
 *   eigenbases are rotated into the basis (Q M Q^T); each operator
 *   application skips the six 1D basis transforms per cell.  With
 *   DG_CG_PRECOND_JACOBI the diagonal is that of Q A Q^T (a different, and
 *   measured weaker, preconditioner than diag(A)).  b and x are mapped once
 *   into the basis and x back once; the returned residual is recomputed in
 *   the Legendre basis, and if the mapping's rounding left it above rtol, the
 *   same solver (precision and preconditioner) continues from x in the
 *   Legendre basis (its iterations counted in iterations, one more outer
 *   iteration).  Formed on the first such solve after dg_set_coefficient: the
 *   line operators of Q A Q^T (as many values as dg_set_coefficient's, ~7.5
 *   doubles per DOF at degree 3), two solve vectors, for the mixed mode h K at
 *   the points in FP32, for the Kronecker blocks the rotated factors.  Cube
 *   meshes only.
 * Stops when ||b - A x|| <= rtol ||b|| recomputed in FP64.  Blocking.
 * Returns NOT_CONVERGED at maxit (x holds the last iterate), BREAKDOWN on
 * <p, Ap> <= 0 or non-finite scalars, TIMEOUT if a bounded wait of the mixed
 * mode's FP32 direction kernel on its bulk copies ran out (the kernel stops
 * cleanly; the context stays usable).  st may be NULL. */
int dg_cg_solve(const dg_mesh* mesh, const double* b, double* x, double rtol, int maxit,
                int mode, dg_cg_stats* st, void* stream);

/* Backup and recovery of the CG (Section 2.3, compressed in-memory
 * checkpointing, on one GPU).  The solver copies a backup into pinned host
 * memory every backup_interval iterations: DG_BACKUP_FULL (x, r, p and the CG
 * scalars; lossless), DG_BACKUP_X64 (x), DG_BACKUP_X32 (x rounded to FP32, a
 * lossy compression to half the bytes) or DG_BACKUP_NONE (zero recovery).  A
 * data loss is injected on the host at the first backup check at or after
 * fault_iteration: x, r and p of the cells [fault_cell_begin, fault_cell_end)
 * (lexicographic cell index, x fastest) are set to zero, as if the rank
 * holding them had failed; -1: no loss.  Recovery:
 *   DG_RECOVER_GLOBAL     every DOF rolls back to the backup.  With the full
 *                         state the iteration resumes exactly, so the solution
 *                         is bit-identical to the fault-free one; with an x
 *                         backup CG restarts from it.
 *   DG_RECOVER_LOCAL      only the lost cells take the backup's x (zero
 *                         without a backup); CG restarts.
 *   DG_RECOVER_LOCAL_AUX  as LOCAL, then the local auxiliary problem
 *                         A(F,F) e = (b - A x)(F) on the lost DOFs F, every
 *                         other DOF held fixed (the Dirichlet layer), solved
 *                         by CG to aux_rtol (relative to its initial residual)
 *                         or aux_maxit iterations; x(F) += e; CG restarts.
 * With no backup yet at the loss, every recovery restarts from the current x
 * with the lost cells zero (plus the auxiliary solve for LOCAL_AUX). */
enum { DG_BACKUP_NONE = 0, DG_BACKUP_FULL = 1, DG_BACKUP_X64 = 2, DG_BACKUP_X32 = 3 };
enum { DG_RECOVER_GLOBAL = 0, DG_RECOVER_LOCAL = 1, DG_RECOVER_LOCAL_AUX = 2 };
typedef struct {
  int backup_interval;         /* in: iterations between backups (>= 1)                  */
  int backup;                  /* in: DG_BACKUP_*                                        */
  int recovery;                /* in: DG_RECOVER_*                                       */
  int fault_iteration;         /* in: inject the loss at this iteration or later; -1 none */
  long long fault_cell_begin;  /* in: first lost cell                                    */
  long long fault_cell_end;    /* in: one past the last lost cell                        */
  double aux_rtol;             /* in: LOCAL_AUX tolerance (> 0)                          */
  int aux_maxit;               /* in: LOCAL_AUX iteration cap (>= 1)                     */
  int fault_injected_at;       /* out: iteration of the loss (-1: none)                  */
  int backup_iteration;        /* out: iteration of the backup used (-1: none)           */
  int backups_taken;           /* out                                                    */
  int aux_iterations;          /* out: iterations of the auxiliary solve                 */
  long long backup_bytes;      /* out: bytes of one backup                               */
} dg_resilience;

/* Solve A(K) x = b by FP64 CG (mode DG_CG_FP64, optionally | DG_CG_PRECOND_JACOBI)
 * with the backups, the injected loss and the recovery of *res (the paper's
 * Section 2.3).  b, x: caller-owned FP64 device arrays of n_dofs values (x in:
 * initial guess, out: solution), as for dg_cg_solve; res: caller-owned host
 * struct, in and out fields as above.  The pinned host backup (backup_bytes)
 * is allocated by the call and freed before it returns.  st->iterations
 * counts every iteration run, the rolled-back ones included;
 * st->outer_iterations the restarts (recoveries included).  Blocking; ordered
 * after the work already on `stream`.  Errors as dg_cg_solve; INVALID_ARG for
 * a NULL res, bad options, another mode or a non-cube mesh; DG_ERR_CUDA if
 * the pinned backup cannot be allocated. */
int dg_cg_solve_resilient(const dg_mesh* mesh, const double* b, double* x, double rtol,
                          int maxit, int mode, dg_resilience* res, dg_cg_stats* st,
                          void* stream);

/* d = diag(A(K)) (FP64 device pointer, n_dofs values in the layout of x,
 * overwritten): the diagonal the Jacobi preconditioner uses (Section 2.4's
 * PCG with M = diag(A)).  Entry (c, m) is a(phi_{c,m}, phi_{c,m}) of the
 * bilinear form of Section 4.1: the volume term by sum factorisation with
 * squared 1D tables, the face terms in closed form (orthonormal basis, exact
 * Gauss rule on the face).  Cached until the next dg_set_coefficient.
 * Blocking.  Errors: INVALID_ARG (NULL mesh or d, no coefficient), OOM, CUDA,
 * BREAKDOWN (a diagonal entry <= 0 or non-finite). */
int dg_diagonal(const dg_mesh* mesh, double* d, void* stream);

/* Solve count independent systems A_s x_s = b_s (meshes may differ in size and
 * degree; FP64) with CG run in lock-step.  Section 3.5 runs k independent
 * Krylov solvers in lock-step (horizontal vectorisation); Section 5 needs many
 * independent solves on levels of different size (multilevel Monte Carlo).
 * Every iteration of all unfinished
 * samples is one persistent launch, and the iteration loop is captured in a
 * CUDA graph.  b[s], x[s]: device pointers (arrays of count pointers on the
 * host).  st: count entries (may be NULL).  Returns the first non-OK sample
 * status, or OK; TIMEOUT if a bounded grid-barrier wait of the persistent
 * kernel ran out (the kernel stops cleanly).  Blocking. */
int dg_cg_solve_batched(const dg_mesh* const* meshes, int count, const double* const* b,
                        double* const* x, double rtol, int maxit, dg_cg_stats* st, void* stream);

/* dg_cg_solve_batched with a mode: DG_CG_FP64 (the same as
 * dg_cg_solve_batched) or DG_CG_FP64 | DG_CG_PRECOND_JACOBI, every sample then
 * running Section 2.4's PCG with M = diag(A_s) (formed per mesh as by
 * dg_diagonal, cached until its next dg_set_coefficient), or
 * DG_CG_FP64 | DG_CG_NODAL: every sample's CG (M = I) in the scaled
 * Gauss-point basis of dg_to_nodal (b and x mapped per sample, the persistent
 * kernel on the transform-free passes, x mapped back, the residual recomputed
 * in the Legendre basis and a sample left above rtol by the mapping's
 * rounding finished by dg_cg_solve).  Other modes: INVALID_ARG.  Everything
 * else as dg_cg_solve_batched. */
int dg_cg_solve_batched_mode(const dg_mesh* const* meshes, int count, const double* const* b,
                             double* const* x, double rtol, int maxit, int mode,
                             dg_cg_stats* st, void* stream);

/* b = the load vector of f (Section 4.1 right-hand side l(v) = sum over cells of
 * the integral of f v): b[c*n^3 + m] = h^3 sum_q w_q f[c*n^3 + q] phi_m(xi_q),
 * with f given at the volume Gauss points (FP64 device pointer, layout as K)
 * and the mesh's n-point Gauss rule per direction; b (FP64 device pointer,
 * n_dofs values) is overwritten.  Needs no coefficient.  Asynchronous on
 * `stream`.  Errors: INVALID_ARG (NULL mesh or vector, f == b), CUDA. */
int dg_load_vector(const dg_mesh* mesh, const double* f, double* b, void* stream);

/* Kernel timing for measurement tools (no paper counterpart).  While enabled,
 * each dg_apply / dg_apply_adjoint on this mesh records CUDA
 * events on its stream before pass 1 (traces), between the passes and after
 * pass 2 (cell kernel), for at most max_applies applications.  dg_timing_read
 * waits for those events, returns the number of recorded applications and the
 * summed durations of each pass in milliseconds, and disables timing.
 * Errors: INVALID_ARG (NULL mesh, max_applies < 1 or > 65536), OOM, CUDA. */
int dg_timing_enable(dg_mesh* mesh, int max_applies);
int dg_timing_read(dg_mesh* mesh, int* n_applies, double* ms_pass1, double* ms_pass2);

/* b = the right-hand side of constant Dirichlet data g[f] on each Dirichlet
 * boundary side f (host array of six doubles, sides x-, x+, y-, y+, z-, z+;
 * entries of zero-flux sides are ignored): b_{c,m} = sum over the cell's
 * Dirichlet faces of int_F gamma_F g [ -(d_n phi_m) + (sigma/h) phi_m ] dA, the
 * weak Dirichlet terms of the SIPG form (Section 4.1 face form on the boundary;
 * the Section 5 flow problem has p = 1 on x = 0, p = 0 on x = 1).  b (FP64
 * device pointer, n_dofs values) is overwritten; add a load vector for a source
 * term.  Needs the coefficient.  Asynchronous.  Errors: INVALID_ARG (NULL
 * pointer, no coefficient, non-finite g), CUDA. */
int dg_dirichlet_rhs(const dg_mesh* mesh, const double* g, double* b, void* stream);

/* *q = the total flux through Dirichlet boundary side `side` (0..5) of the
 * discrete solution u with data g on that side (Section 5's quantity of
 * interest, the flux through the inlet x = 0 for side 0):
 *   Q = sum over the side's faces of int_F gamma_F [ d_n u - (sigma/h)(u - g) ] dA,
 * n outward: the boundary flux that the SIPG form conserves (for the solution
 * of the flow problem the inlet and outlet fluxes cancel).  u, q: FP64 device
 * pointers (q: one double, overwritten).  Asynchronous; fixed summation order.
 * Errors: INVALID_ARG (NULL pointer, no coefficient, side outside 0..5 or a
 * zero-flux side, non-finite g), CUDA. */
int dg_boundary_flux(const dg_mesh* mesh, const double* u, int side, double g, double* q,
                     void* stream);

/* Arithmetic-throughput probe for measurement tools (no paper counterpart):
 * the best of several timed launches of a kernel that keeps the FP64 (kind 0),
 * FP32 (kind 1) or packed FP32x2 (kind 2) fused multiply-add pipe busy on every
 * SM of the current device, in TFLOP/s (an FMA counts 2 flops per lane).
 * Benchmarks divide the executed operation rate of the operator kernels by it.
 * Blocks; allocates and frees 64 bytes.  Errors: INVALID_ARG, CUDA. */
int dg_peak_probe(int kind, double* tflops, void* stream);

/* The scaled Gauss-point (collocation) basis.  No counterpart in the paper: a
 * change to another orthonormal basis of the Section 4.1 discrete space, in
 * which the Section 3.3 sum-factorised operator needs no basis transforms.
 * Per cell, x_hat = Q x with Q = W^{1/2} (B (x) B (x) B): x_hat(a,b,e) =
 * sqrt(w_a w_b w_e) u_h(xi_a, xi_b, xi_e) at the n^3 Gauss points, point
 * index a + n(b + n e) (a along x), the layout of the coefficients.  Q is
 * orthogonal (the Gauss rule integrates L_i L_j exactly), so dg_to_modal
 * (x = Q^T x_hat) is its inverse and both preserve inner products.  FP64
 * device vectors of n_dofs values, caller-owned, not aliased; asynchronous on
 * `stream`; INVALID_ARG on NULL, aliased vectors or an affine or multilinear
 * mesh.  dg_apply_nodal: y_hat = (Q A(K) Q^T) x_hat in FP64 (two kernels:
 * face traces by Lagrange end values, then per-line operators and neighbour
 * face terms); its first call after dg_set_coefficient forms the line
 * operators of Q A Q^T (allocated once per mesh). */
int dg_to_nodal(const dg_mesh* mesh, const double* x, double* xhat, void* stream);
int dg_to_modal(const dg_mesh* mesh, const double* xhat, double* x, void* stream);
int dg_apply_nodal(const dg_mesh* mesh, const double* xhat, double* yhat, void* stream);

/* y = A(K) x in FP64, for callers that cannot allocate device memory.  The
 * paper has no counterpart; this is a deployment variant of dg_apply (Section
 * 3.3 application of the Section 4.1 form).  Some callers may not call
 * cudaMalloc: allocator-free embedded or real-time runtimes that reserve all
 * device memory when they start, and host frameworks that own every device
 * allocation and forbid libraries to make their own.  dg_create_mesh allocates
 * its workspaces, so these callers pass K (FP64 at the volume Gauss points,
 * layout as dg_set_coefficient), x and y (FP64, n_cells^3 (degree+1)^3 values,
 * device pointers owned by the caller) and get y without any allocation: the
 * call makes no cudaMalloc, cudaFree or allocating library call.  Temporaries
 * live in a 64 MiB file-scope device array that every GPU loading the library
 * holds until exit; sizes whose temporaries do not fit (about 75 bytes per DOF,
 * e.g. more than 24^3 cells at degree 3) return INVALID_ARG with the needed
 * size.  The first call on a device looks up the array's device address, so it
 * should come before any stream capture.  The array is shared by all calls and
 * keeps the last call's contents: calls that overlap on the GPU race and must
 * be serialised by the caller.  Blocks until y is written (it copies the K
 * validity flag back to the host and synchronises `stream`); K <= 0 or
 * non-finite returns INVALID_ARG. */
int dg_apply_static(int n_cells, int degree, const double* K, const double* x, double* y,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DG_GB300_H */
