// Right-hand side of the discrete problem (Section 4.1: l(v) = sum over cells
// of the integral of f v), from f given at the volume Gauss points:
//   b_{c,m} = h^3 sum_q w_q f_{c,q} phi_m(xi_q)
// with the same n-point Gauss rule per direction as the operator.  The
// orthonormal tensor basis phi_m = L_i L_j L_l makes this three 1D
// contractions with B[a][i] = L_i(xi_a) (nodal -> modal, transposed), after
// the pointwise weights w_a w_b w_e: sum factorisation as in Section 3.3.
// Thread layout as the operator kernels: n^2 threads per cell, each owning one
// 1D line per stage; a block holds CPB cells.
#include <cmath>

#include "dg_apply_impl.cuh"

namespace dgk {

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_load_vector(const double* __restrict__ f, double* __restrict__ b, long long ncells, double h3,
              const double* __restrict__ pw, const __grid_constant__ DGTab<double> tab) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N;
  __shared__ double s[C * N3];
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  double* sc = s + lc * N3;
  // x-lines: thread owns (b = p, e = q); weighted values -> x-modes
  if (active) {
    const double* fc = f + (c0 + lc) * N3;
    const double wbe = h3 * tab.w[p] * tab.w[q];
    double v[N], R[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int idx = q * N2 + p * N + a;
      // |det J| per point on a multilinear mesh, the constant h^3 det A otherwise
      v[a] = (pw != nullptr ? wbe * pw[(c0 + lc) * N3 + idx] : wbe) * tab.w[a] * fc[idx];
    }
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int i = 0; i < N; ++i) sc[q * N2 + p * N + i] = R[i];
  }
  __syncthreads();
  // y-lines: thread owns (i = p, e = q)
  if (active) {
    double v[N], R[N];
#pragma unroll
    for (int bb = 0; bb < N; ++bb) v[bb] = sc[q * N2 + bb * N + p];
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int j = 0; j < N; ++j) sc[q * N2 + j * N + p] = R[j];
  }
  __syncthreads();
  // z-lines: thread owns (i = p, j = q); result in the vector layout
  if (active) {
    double v[N], R[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sc[e * N2 + q * N + p];
    b_bwd<N>(tab, v, R);
    double* bc = b + (c0 + lc) * N3;
#pragma unroll
    for (int l = 0; l < N; ++l) bc[l * N2 + q * N + p] = R[l];
  }
}

template <int N>
struct LoadVectorF {
  template <typename T>
  static cudaError_t run(const double* f, double* b, long long ncells, double h3,
                         const double* pw, const DGTab<double>* tab, cudaStream_t s) {
    const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
    k_load_vector<N><<<blocks, Cfg<N>::THREADS, 0, s>>>(f, b, ncells, h3, pw, *tab);
    return cudaGetLastError();
  }
};

}  // namespace dgk

extern "C" int dg_load_vector(const dg_mesh* m, const double* f, double* b, void* stream) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_load_vector: mesh is NULL");
  if (f == nullptr || b == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_load_vector: NULL vector");
  if ((const void*)f == (const void*)b)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_load_vector: f and b alias");
  // |det J| = h^3 det A (cube, affine) or per point (multilinear)
  const double h3 = m->multilinear ? 1.0 : m->h * m->h * m->h * m->geomDet;
  const double* pw = m->multilinear ? m->geo_det : nullptr;
  cudaError_t e = dgk::dispatch_n<double, dgk::LoadVectorF>(m->n, f, b, m->ncells, h3, pw,
                                                            (const DGTab<double>*)&m->tab64,
                                                            (cudaStream_t)stream);
  if (e != cudaSuccess) return dg_cuda_fail(e, "dg_load_vector: launch");
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Weak Dirichlet data and the boundary flux (the Section 5 flow problem:
// p = 1 on x = 0, p = 0 on x = 1, zero flux elsewhere; quantity of interest =
// total flux through the inlet).
//
// On a boundary face of side s (axis d, outward sign o = -1 on the lower and
// +1 on the upper side) with constant data g, the SIPG right-hand side is
//   b_{c,m} = int_F gamma_F g [ -(d_n phi_m) + (sigma/h) phi_m ] dA.
// With the orthonormal basis and the exact face Gauss rule the tangential
// factors integrate to delta_{j0} delta_{l0}, so only the modes t e_d (t along
// d, the other two mode indices 0) see the face:
//   b_{c, t e_d} += h gamma_F g ( sigma L_t(s) - o L_t'(s) ).
// The boundary flux the SIPG form conserves,
//   Q = sum over the side's faces of int_F gamma_F [ d_n u - (sigma/h)(u - g) ] dA,
// reduces in the same way to
//   Q = sum_c h gamma_F ( o sum_t u_{c, t e_d} L_t'(s) - sigma (sum_t u_{c, t e_d} L_t(s) - g) ).
// ---------------------------------------------------------------------------

struct DirichletData {
  double g[6];  // data per side (x-, x+, y-, y+, z-, z+)
};

// One thread per cell: b = 0, plus the contributions of its Dirichlet boundary faces.
__global__ void k_dirichlet_rhs(const double* __restrict__ gh, double* __restrict__ b, int Nc,
                                int n, int dmask, const __grid_constant__ DirichletData data,
                                const __grid_constant__ DGTab<double> tab) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)Nc * Nc * Nc;
  if (c >= nc) return;
  const int n3 = n * n * n;
  double* bc = b + c * n3;
  for (int m = 0; m < n3; ++m) bc[m] = 0.0;
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  const int stride[3] = {1, n, n * n};
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1;
    const bool upper = f & 1;
    if (!((dmask >> f) & 1) || data.g[f] == 0.0) continue;
    if (crd[d] != (upper ? Nc - 1 : 0)) continue;
    const double w = gh[c * 6 + f] * data.g[f];
    for (int t = 0; t < n; ++t) {
      const double v = upper ? tab.a1[t] : tab.a0[t];
      const double dv = upper ? tab.d1[t] : -tab.d0[t];  // outward derivative
      bc[t * stride[d]] += w * (tab.sigma * v - dv);
    }
  }
}

// One block: the flux through boundary side `side`, summed over its cells in
// a fixed order.
__global__ void __launch_bounds__(256)
k_boundary_flux(const double* __restrict__ u, const double* __restrict__ gh, int Nc, int n,
                int side, double g, double* __restrict__ q, const __grid_constant__ DGTab<double> tab) {
  __shared__ double sred[8];
  const int d = side >> 1;
  const bool upper = side & 1;
  const int n3 = n * n * n;
  const int stride[3] = {1, n, n * n};
  const long long cstride[3] = {1, Nc, (long long)Nc * Nc};
  const long long cfix = (upper ? Nc - 1 : 0) * cstride[d];
  const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;  // the two tangential axes
  double acc = 0.0;
  for (long long k = threadIdx.x; k < (long long)Nc * Nc; k += blockDim.x) {
    const long long c = cfix + (k % Nc) * cstride[d1] + (k / Nc) * cstride[d2];
    const double* uc = u + c * n3;
    double val = 0.0, der = 0.0;
    for (int t = 0; t < n; ++t) {
      const double ut = uc[t * stride[d]];
      val = fma(upper ? tab.a1[t] : tab.a0[t], ut, val);
      der = fma(upper ? tab.d1[t] : -tab.d0[t], ut, der);
    }
    acc += gh[c * 6 + side] * (der - tab.sigma * (val - g));
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < 8; ++i) tot += sred[i];
    *q = tot;
  }
}

extern "C" int dg_dirichlet_rhs(const dg_mesh* m, const double* g, double* b, void* stream) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_dirichlet_rhs: mesh is NULL");
  if (!m->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_dirichlet_rhs: coefficient not set");
  if (g == nullptr || b == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_dirichlet_rhs: NULL g or b");
  if (int rc = dg_require_cube(m, "dg_dirichlet_rhs")) return rc;
  DirichletData data;
  for (int f = 0; f < 6; ++f) {
    if (!std::isfinite(g[f]))
      return dg_fail(DG_ERR_INVALID_ARG, "dg_dirichlet_rhs: g[%d] is not finite", f);
    data.g[f] = g[f];
  }
  const unsigned blocks = (unsigned)((m->ncells + 127) / 128);
  k_dirichlet_rhs<<<blocks, 128, 0, (cudaStream_t)stream>>>(m->gh64, b, m->N, m->n,
                                                          m->dirichlet_mask, data, m->tab64);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

extern "C" int dg_boundary_flux(const dg_mesh* m, const double* u, int side, double g, double* q,
                                void* stream) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_boundary_flux: mesh is NULL");
  if (!m->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_boundary_flux: coefficient not set");
  if (u == nullptr || q == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_boundary_flux: NULL u or q");
  if (int rc = dg_require_cube(m, "dg_boundary_flux")) return rc;
  if (side < 0 || side > 5)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_boundary_flux: side %d outside 0..5", side);
  if (!((m->dirichlet_mask >> side) & 1))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_boundary_flux: side %d carries zero flux (not a Dirichlet side)", side);
  if (!std::isfinite(g)) return dg_fail(DG_ERR_INVALID_ARG, "dg_boundary_flux: g not finite");
  k_boundary_flux<<<1, 256, 0, (cudaStream_t)stream>>>(u, m->gh64, m->N, m->n, side, g, q,
                                                       m->tab64);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}
