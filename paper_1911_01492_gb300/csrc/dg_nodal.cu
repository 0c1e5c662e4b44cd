// The operator in the scaled Gauss-point (collocation) basis, for CG.
//
// Per cell, Q = W^{1/2} (B (x) B (x) B) maps the Legendre coefficients x to the
// values of u_h at the n^3 Gauss points scaled by sqrt(w_a w_b w_e).  The
// n-point Gauss rule integrates L_i L_j exactly, so B^T diag(w) B = I and Q is
// orthogonal.  The operator of the Section 4.1 form is A = T^T A_pt T, with T
// the modal-to-point map and A_pt acting on point values (collocation
// derivatives, the coefficient at the points, face traces by Lagrange end
// values); hence Q A Q^T = W^{-1/2} A_pt W^{-1/2}.  CG (Section 2.4, M = I) on
// (Q A Q^T) x_hat = Q b produces exactly Q times the iterates of CG on
// A x = b, since Q preserves every inner product.
//
// Why: in the Legendre basis every application of A spends its FP64
// instructions on six 1D basis transforms per cell (three forward, three
// back), about a quarter of the FP64 work at Q3.  In the scaled point basis
// those transforms vanish: pass 1 only forms face traces (Lagrange end values
// of each line), pass 2 only applies the per-line operators (the volume term
// and the own-side face terms) and the neighbours' face terms.  A solve maps b
// and x into the basis once and x back once.
//
// In that basis the scaling is folded into the data: the line operators of
// Q A Q^T are those of A_pt times isw_i isw_j / (w_s w_t) (k_line_ops<N,
// true>); the Lagrange end values carry isw_a = 1/sqrt(w_a); the face weight
// h gamma w_s w_t / 2 of a face point loses its tangential weights against
// the two isw factors of the traces, so every point of a face has the weight
// h gamma / 2 and no per-point face-weight array is read.
#include "dg_nodal_impl.cuh"

namespace dgk {

// ---------------------------------------------------------------------------
// x_hat = Q x (TO_NODAL) or x = Q^T x_hat, per cell by three 1D contractions
// (the parity-split B and B^T of the operator kernels) and the point scaling.
// One thread per line of each of the block's CPB cells, lines exchanged
// through shared memory.
// ---------------------------------------------------------------------------
template <int N, bool TO_NODAL>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_collocation(const double* __restrict__ in, double* __restrict__ out, long long ncells,
              const __grid_constant__ DGTab<double> tab,
              const __grid_constant__ DGTabN<double> tn) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s = reinterpret_cast<double*>(smem_raw);
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  const long long c = c0 + lc;
  double* sc = s + lc * N3;
  const double* src = in + c * N3;
  double* dst = out + c * N3;
  if (TO_NODAL) {
    if (active) {  // z-lines (i = p, j = q): modes along z -> points
      double v[N], u[N];
#pragma unroll
      for (int l = 0; l < N; ++l) v[l] = src[l * N2 + q * N + p];
      b_fwd<N>(tab, v, u);
#pragma unroll
      for (int e = 0; e < N; ++e) sc[e * N2 + q * N + p] = u[e];
    }
    __syncthreads();
    if (active) {  // y-lines (i = p, e = q)
      double v[N], u[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = sc[q * N2 + j * N + p];
      b_fwd<N>(tab, v, u);
#pragma unroll
      for (int b = 0; b < N; ++b) sc[q * N2 + b * N + p] = u[b];
    }
    __syncthreads();
    if (active) {  // x-lines (b = p, e = q), then the scaling sqrt(w_a w_b w_e)
      double v[N], u[N];
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = sc[q * N2 + p * N + i];
      b_fwd<N>(tab, v, u);
      const double f = tn.sw[p] * tn.sw[q];
#pragma unroll
      for (int a = 0; a < N; ++a) dst[q * N2 + p * N + a] = u[a] * (tn.sw[a] * f);
    }
  } else {
    if (active) {  // x-lines (b = p, e = q): the scaling, then B^T along x
      double v[N], R[N];
      const double f = tn.sw[p] * tn.sw[q];
#pragma unroll
      for (int a = 0; a < N; ++a) v[a] = src[q * N2 + p * N + a] * (tn.sw[a] * f);
      b_bwd<N>(tab, v, R);
#pragma unroll
      for (int i = 0; i < N; ++i) sc[q * N2 + p * N + i] = R[i];
    }
    __syncthreads();
    if (active) {  // y-lines (i = p, e = q)
      double v[N], R[N];
#pragma unroll
      for (int b = 0; b < N; ++b) v[b] = sc[q * N2 + b * N + p];
      b_bwd<N>(tab, v, R);
#pragma unroll
      for (int j = 0; j < N; ++j) sc[q * N2 + j * N + p] = R[j];
    }
    __syncthreads();
    if (active) {  // z-lines (i = p, j = q): points along z -> modes
      double v[N], R[N];
#pragma unroll
      for (int e = 0; e < N; ++e) v[e] = sc[e * N2 + q * N + p];
      b_bwd<N>(tab, v, R);
#pragma unroll
      for (int l = 0; l < N; ++l) dst[l * N2 + q * N + p] = R[l];
    }
  }
}

// The two passes (dg_nodal_impl.cuh) as stand-alone kernels over blocks of CPB
// cells.
template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_trace_nd(const T* __restrict__ x, T* __restrict__ TR, long long ncells, const int* skip,
           const __grid_constant__ DGTabN<T> tn) {
  constexpr int C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  trace_cells_nd<N, T>(x, TR, c0, nblk, tn, reinterpret_cast<T*>(smem_raw));
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_cell_nd(const double* __restrict__ x, const double* __restrict__ TR,
          const double* __restrict__ lineop, const double* __restrict__ gh,
          double* __restrict__ y, long long ncells, int Nc, const int* skip,
          const __grid_constant__ DGTabN<double> tn) {
  constexpr int C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  cell_cells_nd<N>(x, TR, lineop, gh, y, c0, nblk, Nc, tn, reinterpret_cast<double*>(smem_raw));
}

// 1 / diag(Q A Q^T): at point (a, b, e) the sum of the diagonal entries of the
// x-, y- and z-line operators through it (the neighbour terms couple other
// cells only).  One thread per DOF.
template <int N>
__global__ void k_diag_nd(const double* __restrict__ lineop, double* __restrict__ dinv64,
                          float* __restrict__ dinv32, long long ndofs) {
  constexpr int N2 = N * N, N3 = N * N * N, NP = N * (N + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ndofs) return;
  const long long c = t / N3;
  const int qi = (int)(t - c * N3);
  const int a = qi % N, b = (qi / N) % N, e = qi / N2;
  const double* L = lineop + c * 3 * N2 * NP;
  const double d = L[(0 * N2 + b + N * e) * NP + packed<N>(a, a)] +
                   L[(1 * N2 + a + N * e) * NP + packed<N>(b, b)] +
                   L[(2 * N2 + a + N * b) * NP + packed<N>(e, e)];
  const double di = 1.0 / d;
  dinv64[t] = di;
  dinv32[t] = (float)di;
}

// h K at the volume points in FP32 from h w_q K (the FP32 cell kernel of the
// point basis scales its collocation derivatives by sqrt(w) instead).
__global__ void k_hk32(const double* __restrict__ kt, float* __restrict__ hk, long long ndofs,
                       int n, const __grid_constant__ DGTab<double> tab) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ndofs) return;
  const int qi = (int)(t % ((long long)n * n * n));
  const int a = qi % n, b = (qi / n) % n, e = qi / (n * n);
  hk[t] = (float)(kt[t] / (tab.w[a] * tab.w[b] * tab.w[e]));
}

template <int N>
struct NodalF {
  template <typename T>
  static cudaError_t apply(const dg_mesh* m, const double* x, double* y, const int* skip,
                           cudaStream_t s) {
    const unsigned blocks = (unsigned)((m->ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
    const size_t s1 = sizeof(double) * Cfg<N>::CPB * N * N * N;
    dg_timing_mark(m, 0, s);
    k_trace_nd<N, double><<<blocks, Cfg<N>::THREADS, s1, s>>>(x, m->TR64, m->ncells, skip,
                                                             m->tabN64);
    dg_timing_mark(m, 1, s);
    k_cell_nd<N><<<blocks, Cfg<N>::THREADS, 2 * s1, s>>>(x, m->TR64, m->lineopN64, m->gh64, y,
                                                        m->ncells, m->N, skip, m->tabN64);
    dg_timing_mark(m, 2, s);
    return cudaGetLastError();
  }
  template <typename T>
  static cudaError_t run(int what, const dg_mesh* m, const double* x, double* y,
                         const int* skip, cudaStream_t s) {
    const unsigned blocks = (unsigned)((m->ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
    const size_t s1 = sizeof(double) * Cfg<N>::CPB * N * N * N;
    switch (what) {
      case 0: return apply<T>(m, x, y, skip, s);
      case 1:
        k_collocation<N, true><<<blocks, Cfg<N>::THREADS, s1, s>>>(x, y, m->ncells, m->tab64,
                                                                   m->tabN64);
        return cudaGetLastError();
      case 2:
        k_collocation<N, false><<<blocks, Cfg<N>::THREADS, s1, s>>>(x, y, m->ncells, m->tab64,
                                                                    m->tabN64);
        return cudaGetLastError();
      case 3: {
        const long long threads = m->ncells * 3 * N * N;
        k_line_ops<N, true><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            m->kt64, m->gh64, m->lineopN64, m->ncells, m->N, m->tab64, m->tabN64);
        return cudaGetLastError();
      }
      case 4:
        k_diag_nd<N><<<(unsigned)((m->ndofs + 255) / 256), 256, 0, s>>>(
            m->lineopN64, m->dinvN64, m->dinvN32, m->ndofs);
        return cudaGetLastError();
      default: return cudaErrorInvalidValue;
    }
  }
};

}  // namespace dgk

void dg_build_nodal_tables(const DGTab<double>& t, int n, DGTabN<double>* d, DGTabN<float>* f) {
  *d = DGTabN<double>{};
  *f = DGTabN<float>{};
  for (int a = 0; a < n; ++a) {
    const double sw = std::sqrt(t.w[a]), isw = 1.0 / sw;
    d->sw[a] = sw;
    d->isw[a] = isw;
    d->l0[a] = t.l0[a] * isw;
    d->l1[a] = t.l1[a] * isw;
    d->dl0[a] = t.dl0[a] * isw;
    d->dl1[a] = t.dl1[a] * isw;
    d->hdl0[a] = 0.5 * t.dl0[a] * isw;
    d->hdl1[a] = 0.5 * t.dl1[a] * isw;
  }
  for (int fq = 0; fq < n; ++fq)
    for (int i = 0; i < n; ++i) d->Dh[fq][i] = d->sw[fq] * t.D[fq][i] * d->isw[i];
  for (int a = 0; a < n; ++a) {
    f->sw[a] = (float)d->sw[a];
    f->isw[a] = (float)d->isw[a];
    f->l0[a] = (float)d->l0[a];
    f->l1[a] = (float)d->l1[a];
    f->dl0[a] = (float)d->dl0[a];
    f->dl1[a] = (float)d->dl1[a];
    f->hdl0[a] = (float)d->hdl0[a];
    f->hdl1[a] = (float)d->hdl1[a];
    for (int i = 0; i < n; ++i) f->Dh[a][i] = (float)d->Dh[a][i];
  }
}

namespace {
int run_nodal(int what, const dg_mesh* m, const double* x, double* y, const int* skip,
              cudaStream_t s, const char* who) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (m->n) {
    case 2: e = dgk::NodalF<2>::run<double>(what, m, x, y, skip, s); break;
    case 3: e = dgk::NodalF<3>::run<double>(what, m, x, y, skip, s); break;
    case 4: e = dgk::NodalF<4>::run<double>(what, m, x, y, skip, s); break;
    case 5: e = dgk::NodalF<5>::run<double>(what, m, x, y, skip, s); break;
    case 6: e = dgk::NodalF<6>::run<double>(what, m, x, y, skip, s); break;
    case 7: e = dgk::NodalF<7>::run<double>(what, m, x, y, skip, s); break;
    case 8: e = dgk::NodalF<8>::run<double>(what, m, x, y, skip, s); break;
    case 9: e = dgk::NodalF<9>::run<double>(what, m, x, y, skip, s); break;
    default: break;
  }
  if (e != cudaSuccess) return dg_cuda_fail(e, who);
  return DG_OK;
}
}  // namespace

int dg_ensure_nodal(dg_mesh* m, cudaStream_t s) {
  if (m->has_nodal) return DG_OK;
  if (int rc = dg_require_cube(m, "the scaled Gauss-point basis")) return rc;
  const size_t nd = (size_t)m->ndofs;
  const size_t nlo = (size_t)3 * m->n * m->n * (size_t)(m->n * (m->n + 1) / 2) * (size_t)m->ncells;
  if (m->lineopN64 == nullptr) DG_CUDA(cudaMalloc((void**)&m->lineopN64, nlo * sizeof(double)));
  if (m->bN64 == nullptr) DG_CUDA(cudaMalloc((void**)&m->bN64, nd * sizeof(double)));
  if (m->xN64 == nullptr) DG_CUDA(cudaMalloc((void**)&m->xN64, nd * sizeof(double)));
  int rc = run_nodal(3, m, nullptr, nullptr, nullptr, s, "nodal line operators");
  if (rc) return rc;
  m->has_nodal = true;
  return DG_OK;
}

int dg_ensure_nodal_diag(dg_mesh* m, cudaStream_t s) {
  int rc = dg_ensure_nodal(m, s);
  if (rc || m->has_nodal_diag) return rc;
  const size_t nd = (size_t)m->ndofs;
  if (m->dinvN64 == nullptr) DG_CUDA(cudaMalloc((void**)&m->dinvN64, nd * sizeof(double)));
  if (m->dinvN32 == nullptr) DG_CUDA(cudaMalloc((void**)&m->dinvN32, nd * sizeof(float)));
  rc = run_nodal(4, m, nullptr, nullptr, nullptr, s, "nodal Jacobi diagonal");
  if (rc) return rc;
  m->has_nodal_diag = true;
  return DG_OK;
}

int dg_ensure_nodal32(dg_mesh* m, cudaStream_t s) {
  int rc = dg_ensure_nodal(m, s);
  if (rc || m->has_nodal32) return rc;
  if (m->hk32 == nullptr) DG_CUDA(cudaMalloc((void**)&m->hk32, (size_t)m->ndofs * sizeof(float)));
  dgk::k_hk32<<<(unsigned)((m->ndofs + 255) / 256), 256, 0, s>>>(m->kt64, m->hk32, m->ndofs, m->n,
                                                                 m->tab64);
  DG_CUDA(cudaGetLastError());
  m->has_nodal32 = true;
  return DG_OK;
}

int dg_launch_apply_nodal_f64(const dg_mesh* m, const double* x, double* y, const int* skip,
                              cudaStream_t s) {
  return run_nodal(0, m, x, y, skip, s, "apply in the point basis (fp64) launch");
}

int dg_launch_collocation(const dg_mesh* m, const double* in, double* out, bool to_nodal,
                          cudaStream_t s) {
  return run_nodal(to_nodal ? 1 : 2, m, in, out, nullptr, s, "basis transform launch");
}

static int check_nodal_args(const dg_mesh* m, const void* a, const void* b, const char* who) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "%s: mesh is NULL", who);
  if (a == nullptr || b == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "%s: NULL vector", who);
  if (a == b) return dg_fail(DG_ERR_INVALID_ARG, "%s: input and output alias", who);
  return dg_require_cube(m, who);
}

extern "C" int dg_to_nodal(const dg_mesh* m, const double* x, double* xhat, void* stream) {
  if (int rc = check_nodal_args(m, x, xhat, "dg_to_nodal")) return rc;
  return dg_launch_collocation(m, x, xhat, true, (cudaStream_t)stream);
}

extern "C" int dg_to_modal(const dg_mesh* m, const double* xhat, double* x, void* stream) {
  if (int rc = check_nodal_args(m, xhat, x, "dg_to_modal")) return rc;
  return dg_launch_collocation(m, xhat, x, false, (cudaStream_t)stream);
}

extern "C" int dg_apply_nodal(const dg_mesh* mc, const double* xhat, double* yhat, void* stream) {
  if (int rc = check_nodal_args(mc, xhat, yhat, "dg_apply_nodal")) return rc;
  if (!mc->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_nodal: coefficient not set");
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = dg_ensure_nodal(m, s)) return rc;
  return dg_launch_apply_nodal_f64(m, xhat, yhat, nullptr, s);
}
