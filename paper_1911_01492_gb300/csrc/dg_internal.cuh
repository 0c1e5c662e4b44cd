// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/dg.h"

#define DG_MAXN 9  // points (= modes) per direction, degree <= 8

// 1D tables on the reference interval [0,1] for n = degree + 1 Gauss points.
// Passed to kernels by value (kernel parameters live in constant memory, so
// every table entry is a uniform constant operand).
template <typename T>
struct DGTab {
  T B[DG_MAXN][DG_MAXN];   // B[a][i]  = L_i(xi_a)      modal -> nodal values
  T Bd[DG_MAXN][DG_MAXN];  // Bd[a][i] = L_i'(xi_a)     modal -> nodal derivative
  T D[DG_MAXN][DG_MAXN];   // D[a][b]  = l_b'(xi_a)     nodal collocation derivative
  T w[DG_MAXN];            // Gauss weights on [0,1] (sum 1)
  T a0[DG_MAXN], a1[DG_MAXN];    // L_i(0), L_i(1)
  T d0[DG_MAXN], d1[DG_MAXN];    // L_i'(0), L_i'(1)
  T l0[DG_MAXN], l1[DG_MAXN];    // l_a(0), l_a(1)     (Lagrange basis on the Gauss points)
  T dl0[DG_MAXN], dl1[DG_MAXN];  // l_a'(0), l_a'(1)
  T sigma;                        // penalty factor 2(k+1)^2 (dimensionless)
};

// 1D data of the scaled Gauss-point basis (dg_nodal.cu): a cell's values
// u_hat(a,b,e) = sqrt(w_a w_b w_e) u_h(xi_a, xi_b, xi_e).  Face traces of u_h
// and the test functions' face values in that basis carry 1 / sqrt(w) per
// point along the line; the tangential factors cancel against the face weight.
template <typename T>
struct DGTabN {
  T sw[DG_MAXN];                  // sqrt(w_a)
  T isw[DG_MAXN];                 // 1 / sqrt(w_a)
  T l0[DG_MAXN], l1[DG_MAXN];     // l_a(0) / sqrt(w_a), l_a(1) / sqrt(w_a)
  T dl0[DG_MAXN], dl1[DG_MAXN];   // l_a'(0) / sqrt(w_a), l_a'(1) / sqrt(w_a)
  T hdl0[DG_MAXN], hdl1[DG_MAXN]; // the same halved
  T Dh[DG_MAXN][DG_MAXN];         // sqrt(w_f) D[f][i] / sqrt(w_i)
};

// Host-side construction of the FP64 tables (dg_tables.cpp) and rounding to FP32.
void dg_build_tables(int n, double sigma, DGTab<double>* t64, DGTab<float>* t32);
// the n Gauss-Legendre points and weights on [0,1] of those tables
void dg_gauss_points(int n, double* xi, double* w);

// CG scalar state kept on the device (one per solve / per batched sample).
struct DGCGState {
  double rho;       // <z, r> of the current residual (z = M^-1 r; = <r, r> without M)
  double rr;        // <r, r> of the current residual (the convergence norm)
  double pq;        // <p, A p>
  double alpha;     // rho / pq
  double beta;      // rho_new / rho
  double tol2;      // (stopping tolerance)^2 for <r, r>
  double bnorm2;    // <b, b>
  double res2;      // ||b - A x||^2 of the last true-residual check
  double b2;        // ||b||^2 of the last true-residual check
  double rho_new;   // <r, r> after the current update (mixed mode)
  double rmax2;     // ||r||^2 at the last FP64 residual refinement (mixed mode)
  double delta2;    // refine when <r,r> drops below delta2 * rmax2 (mixed mode)
  int done;         // 1 once converged, broken down or out of iterations
  int breakdown;    // 1 if pq <= 0 or a scalar became non-finite
  int iters;        // iterations performed
  int maxit;        // iteration cap
  unsigned int ticket;  // completion counter of the last-block reductions
  int ru_skip;      // 0 when this iteration ends with an FP64 refinement (mixed mode)
  int n_refine;     // FP64 residual refinements performed (mixed mode)
  int restart;      // 1: the next direction update restarts with p = r (mixed mode)
  int stall;        // consecutive refinements that fell short of a 2x reduction
  int timeout;      // 1 if a kernel gave up a bounded wait (bulk-copy barrier)
};

// z-slabs of the pipelined host-buffer apply (at most)
#define DG_HOST_SLABS 16

struct dg_mesh {
  int N;            // cells per direction
  int k;            // degree
  int n;            // points per direction = k + 1
  long long ncells; // N^3
  long long ndofs;  // N^3 n^3
  double h;
  double sigma;
  int dirichlet_mask;  // bit f: boundary side f (x-, x+, y-, y+, z-, z+) is Dirichlet
  // affine geometry x = A xi (dg_set_geometry): metric det A A^-1 A^-T, face
  // penalty factors det A |A^-T e_d|^2, det A; affine = false for A = I
  bool affine;
  double geomG[3][3];
  double geomKappa[3];
  double geomDet;
  // multilinear geometry (dg_set_vertices): per volume point the metric
  // |det J| J^-1 J^-T / h (6 values: xx, yy, zz, xy, xz, yz) [c][6][n^3] and
  // |det J| [c][n^3]; per face point of every cell face the area element / h
  // and the own-side vector J^-1 n [c][6][4][n^2]; per cell face sigma / h_F [c][6]
  bool multilinear;
  double *geo_vol, *geo_det, *geo_face, *geo_pen;
  int device;
  int sm_count;
  DGTab<double> tab64;
  DGTab<float> tab32;

  // coefficient data (dg_set_coefficient)
  bool has_coef;
  double* kt64;     // h w_q K_{c,q}                  [c][q]
  float* kt32;
  double* gh64;     // h gamma_F per face side        [c][6] (x-, x+, y-, y+, z-, z+)
  float* gh32;
  double* dgam;     // d gamma_F / d log Kbar_c       [c][6]
  double* fw64;     // face-point weights W/2 and derivative weight  [c][6][2][n^2]
  double* lineop64; // per-line volume operators (FP64)  [c][3][n^2][n(n+1)/2]
  float* fw32;
  // Jacobi preconditioner: 1 / diag(A), formed on the first preconditioned solve
  double* diag64;
  double* dinv64;
  float* dinv32;
  bool has_diag;
  // cell-block Jacobi: the inverted diagonal cell blocks [c][n^3][n^3] (FP64)
  double* binv64;
  bool has_block;
  // Kronecker cell blocks: per cell Q_x, Q_y, Q_z (n x n) and their eigenvalues
  // [c][3n^2 + 3n], FP64 and FP32
  double* kron64;
  float* kron32;
  bool has_kron;
  // scaled Gauss-point basis (DG_CG_NODAL, dg_nodal.cu): its 1D tables, the
  // line operators and Jacobi diagonal of Q A Q^T (formed on first use after
  // the coefficient is set) and the solve's b and x in that basis
  DGTabN<double> tabN64;
  DGTabN<float> tabN32;
  bool has_nodal, has_nodal_diag;
  bool nodal_op;      // set while a solve runs in that basis: the internal
                      // FP64 apply launcher then applies Q A Q^T
  double* lineopN64;  // [c][3][n^2][n(n+1)/2]
  double* dinvN64;
  float* dinvN32;
  double *bN64, *xN64;
  float* hk32;        // h K at the volume points (FP32 operator in that basis) [c][q]
  bool has_nodal32;
  // the Kronecker cell blocks in that basis: eigenbases rotated by
  // q = diag(sqrt(w)) B per direction, same layout as kron64 / kron32
  double* kronN64;
  float* kronN32;
  bool has_kron_nodal;
  double* kbar;     // Kbar_c                          [c]
  int* dflag;       // device-side error flag of the setup kernels

  // apply workspaces: nodal values, x-modal/yz-nodal values, face traces
  double *U64, *X64, *TR64;
  float *U32, *X32, *TR32;
  // second set for the coefficient gradient (traces of v), lazily allocated
  double *U64b, *X64b, *TR64b;
  // host staging for dg_apply_host: device copies of x and y, copy-in,
  // copy-out and pass-1 streams and per-slab events of the pipeline
  void *hx_dev, *hy_dev;
  cudaStream_t hstream[3];
  cudaEvent_t hev[3 * DG_HOST_SLABS + 1];

  // solver workspaces, lazily allocated
  double *r64, *p64, *q64, *t64, *s64;  // t64, s64: u = M^-1 r and s = A p of the batched solver
  float *d32, *r32, *p32, *q32;
  double* partials;       // reduction partials (DG_RED_BLOCKS doubles x DG_RED_SUMS)
  double* partials_cells; // one partial per cell block (fused FP32 mixed kernels)
  DGCGState* state;       // device CG state
  DGCGState* state_host;  // pinned mirror
  cudaStream_t solve_stream;
  cudaEvent_t ev;
  int dir_bulk_grid[2];   // persistent grid of the bulk-copy direction kernel (M = I, Jacobi)

  // optional per-pass kernel timing (dg_timing_enable / dg_timing_read)
  cudaEvent_t* tev;       // 3 events per recorded application
  int tev_cap;            // applications the event array holds
  int tev_used;           // applications recorded so far
  bool timing;
};

// record the timing event `slot` (0 before pass 1, 1 between passes, 2 after
// pass 2) of the current application when timing is enabled (dg_mesh.cu)
void dg_timing_mark(const dg_mesh* m, int slot, cudaStream_t s);

// Deterministic two-level reductions use this fixed grid.
#define DG_RED_BLOCKS 1216  // 8 x 152 SMs
#define DG_RED_THREADS 256
#define DG_RED_SUMS 4     // most sums one reduction kernel may form (partials size)

// coefficient setup kernels (dg_mesh.cu), shared with the allocation-free
// apply: h w_q K and Kbar per cell (FP32 copy skipped when kt32 is NULL); h gamma
// and d gamma / d log Kbar per face side (gh32 / dgam skipped when NULL)
__global__ void k_coef_cells(const double* __restrict__ K, double* __restrict__ kt64,
                             float* __restrict__ kt32, double* __restrict__ kbar,
                             long long ncells, int n, double h, int* flag,
                             const __grid_constant__ DGTab<double> tab);
// (dmask: bit f set when boundary side f is Dirichlet; the boundary faces of
// the other sides carry zero flux, gamma = 0)
__global__ void k_coef_faces(const double* __restrict__ kbar, double* __restrict__ gh64,
                             float* __restrict__ gh32, double* __restrict__ dgam, int Nc,
                             double h, int dmask);

// error reporting (dg_mesh.cu)
int dg_fail(int code, const char* fmt, ...);
int dg_cuda_fail(cudaError_t e, const char* what);
#define DG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return dg_cuda_fail(e__, #call); \
  } while (0)

// launchers (dg_apply_f64.cu / dg_apply_f32.cu)
// one pass (1: traces, 2: cell terms) over the cells [cbeg, cend)
int dg_launch_pass_f64(const dg_mesh* m, int pass, const double* x, double* y, long long cbeg,
                       long long cend, cudaStream_t s);
int dg_launch_pass_f32(const dg_mesh* m, int pass, const float* x, float* y, long long cbeg,
                       long long cend, cudaStream_t s);
int dg_launch_apply_f64(const dg_mesh* m, const double* x, double* y, const int* skip,
                        cudaStream_t s);
int dg_launch_apply_f32(const dg_mesh* m, const float* x, float* y, const int* skip,
                        cudaStream_t s);
// FP64 apply on an affine mesh (dg_affine.cu) and its kernel attributes
int dg_launch_apply_affine(const dg_mesh* m, const double* x, double* y, const int* skip,
                           cudaStream_t s);
int dg_prepare_affine(int n);
int dg_launch_apply_multilinear(const dg_mesh* m, const double* x, double* y, const int* skip,
                                cudaStream_t s);
// INVALID_ARG if the mesh is affine (for the paths that assume cube faces)
int dg_require_cube(const dg_mesh* m, const char* who);
// traces only (used by the coefficient gradient): U, X, TR of x into the given buffers
int dg_launch_trace_f64(const dg_mesh* m, const double* x, double* U, double* X, double* TR,
                        cudaStream_t s);
int dg_launch_coeff_grad(const dg_mesh* m, double* g, cudaStream_t s);
// fused FP32 kernels of the mixed CG iteration (dg_mixed32.cu)
// rin: r32 (z = r, or z = dinv r with dinv), or z = M^-1 r already formed
int dg_launch_mixed32_dir_cell(const dg_mesh* m, const float* rin, const float* dinv,
                               cudaStream_t s);
long long dg_mixed32_blocks(int n, long long ncells);
// attributes and persistent grid of the mixed kernels (before any capture)
int dg_prepare_mixed32(dg_mesh* m);
// one-time kernel attributes (dynamic shared memory) for points-per-direction n
int dg_prepare_apply_f64(int n);
int dg_prepare_apply_f32(int n);
int dg_prepare_grad(int n);

// scaled Gauss-point basis (dg_nodal.cu): tables (at mesh creation), the
// line operators of Q A Q^T and solve vectors (formed if needed), its Jacobi
// diagonal, the FP64 apply of Q A Q^T, and x_hat = Q x / x = Q^T x_hat
void dg_build_nodal_tables(const DGTab<double>& t, int n, DGTabN<double>* d, DGTabN<float>* f);
int dg_ensure_nodal(dg_mesh* m, cudaStream_t s);
int dg_ensure_nodal_diag(dg_mesh* m, cudaStream_t s);
int dg_ensure_nodal32(dg_mesh* m, cudaStream_t s);  // h K in FP32 for the mixed CG
int dg_launch_apply_nodal_f64(const dg_mesh* m, const double* x, double* y, const int* skip,
                              cudaStream_t s);
int dg_launch_collocation(const dg_mesh* m, const double* in, double* out, bool to_nodal,
                          cudaStream_t s);

// 1 / diag(A) for the Jacobi preconditioner (dg_precond.cu); forms it if needed
int dg_ensure_diagonal(dg_mesh* m, cudaStream_t s);
// cell-block Jacobi (dg_block.cu): the inverted blocks (formed if needed), and
// z = M^-1 r with <z, r> into the CG state (init: rho and p = z; else beta, rho)
int dg_ensure_block(dg_mesh* m, cudaStream_t s);
// Kronecker cell-block preconditioner (dg_kron.cu): factors formed once per
// coefficient; z = M^-1 r with <z, r> into the CG state (mode: FP64 iteration,
// FP64 initialisation with p = z, FP32 mixed iteration)
enum { DG_KRON_FP64 = 0, DG_KRON_FP64_INIT = 1, DG_KRON_FP32 = 2 };
int dg_ensure_kron(dg_mesh* m, cudaStream_t s);
int dg_ensure_kron_nodal(dg_mesh* m, cudaStream_t s);  // the same in the point basis
int dg_launch_kron_apply(const dg_mesh* m, const void* r, void* z, void* p, int mode,
                         cudaStream_t s);
int dg_launch_block_apply(const dg_mesh* m, const double* r, double* z, double* p, bool init,
                          cudaStream_t s);
// workspace helpers (dg_mesh.cu)
int dg_ensure_solver_ws(dg_mesh* m);
int dg_ensure_grad_ws(dg_mesh* m);
