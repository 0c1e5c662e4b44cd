// Jacobi preconditioner: diag(A(K)), formed directly by sum factorisation.
//
// Entry (c, m), m = i + n (j + n l), of the diagonal is a(phi_{c,m}, phi_{c,m}).
// The volume part is
//   sum_{a,b,e} Kt[a,b,e] ( L_i'(a)^2 L_j(b)^2 L_l(e)^2 + L_i(a)^2 L_j'(b)^2 L_l(e)^2
//                         + L_i(a)^2 L_j(b)^2 L_l'(e)^2 ),   Kt = h w K,
// i.e. the volume operator with every 1D table squared: three contractions
// per cell (z, then y, then x).  On a face the test and trial function both
// live on the cell's own side, so the jump is the own trace and the average
// of the normal derivative is half the own one (all of it on the boundary).
// The Gauss rule with n = k + 1 points integrates L_j^2 exactly and the
// Legendre basis is orthonormal, so the tangential sums give 1 and a face
// with axis d contributes
//   h gamma_F ( sigma L_t(s)^2 - c_F L_t(s) dL_t/dn_out(s) ),
// t the mode index along d, s = 0 or 1 the face side, c_F = 1 inside and 2
// on the boundary (the one-sided form -2 (d_n phi) phi + sigma phi^2).
// One warp per cell; the whole diagonal costs about one operator application.
#include "dg_internal.cuh"

namespace {

constexpr int kDiagSmemDoubles = 6144;  // 48 KB per block

// Cells per block so that five n^3 FP64 arrays per cell fit in 48 KB.
int diag_cells_per_block(int n) {
  const int per = 5 * n * n * n;
  int w = kDiagSmemDoubles / per;
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

__global__ void k_diag(const double* __restrict__ kt, const double* __restrict__ gh,
                       double* __restrict__ diag, double* __restrict__ dinv,
                       float* __restrict__ dinv32, long long ncells, int Nc, int n, int* flag,
                       const __grid_constant__ DGTab<double> tab) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= ncells) return;
  const int n2 = n * n, n3 = n2 * n;
  double* sk = sm + (size_t)warp * 5 * n3;  // Kt of the cell, [e][b][a]
  double* t1 = sk + n3;                     // sum_e Kt L_l(e)^2      [l][b][a]
  double* t2 = t1 + n3;                     // sum_e Kt L_l'(e)^2     [l][b][a]
  double* s1 = t2 + n3;                     // sum_b t1 L_j(b)^2      [l][j][a]
  double* s2 = s1 + n3;                     // sum_b (t1 L_j'(b)^2 + t2 L_j(b)^2)
  for (int q = lane; q < n3; q += 32) sk[q] = kt[c * n3 + q];
  __syncwarp();
  for (int o = lane; o < n3; o += 32) {  // o = a + n (b + n l)
    const int a = o % n, b = (o / n) % n, l = o / n2;
    double u = 0.0, v = 0.0;
    for (int e = 0; e < n; ++e) {
      const double k = sk[a + n * (b + n * e)];
      const double B = tab.B[e][l], Bd = tab.Bd[e][l];
      u = fma(k, B * B, u);
      v = fma(k, Bd * Bd, v);
    }
    t1[o] = u;
    t2[o] = v;
  }
  __syncwarp();
  for (int o = lane; o < n3; o += 32) {  // o = a + n (j + n l)
    const int a = o % n, j = (o / n) % n, l = o / n2;
    double u = 0.0, v = 0.0;
    for (int b = 0; b < n; ++b) {
      const int src = a + n * (b + n * l);
      const double B = tab.B[b][j], Bd = tab.Bd[b][j];
      u = fma(t1[src], B * B, u);
      v = fma(t1[src], Bd * Bd, fma(t2[src], B * B, v));
    }
    s1[o] = u;
    s2[o] = v;
  }
  __syncwarp();
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  const double sig = tab.sigma;
  for (int o = lane; o < n3; o += 32) {  // o = i + n (j + n l)
    const int i = o % n, j = (o / n) % n, l = o / n2;
    double d = 0.0;
    for (int a = 0; a < n; ++a) {
      const double B = tab.B[a][i], Bd = tab.Bd[a][i];
      const int src = a + n * (j + n * l);
      d = fma(Bd * Bd, s1[src], fma(B * B, s2[src], d));
    }
    const int t[3] = {i, j, l};
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      const int md = t[dir];
      const double cl = crd[dir] > 0 ? 1.0 : 2.0;       // lower face, outward normal -e_dir
      const double cu = crd[dir] < Nc - 1 ? 1.0 : 2.0;  // upper face, outward normal +e_dir
      d += gh[c * 6 + 2 * dir] * (sig * tab.a0[md] * tab.a0[md] + cl * tab.a0[md] * tab.d0[md]);
      d += gh[c * 6 + 2 * dir + 1] * (sig * tab.a1[md] * tab.a1[md] - cu * tab.a1[md] * tab.d1[md]);
    }
    if (!(d > 0.0) || !isfinite(d)) atomicOr(flag, 1);
    const double inv = 1.0 / d;
    diag[c * n3 + o] = d;
    dinv[c * n3 + o] = inv;
    dinv32[c * n3 + o] = (float)inv;
  }
}

}  // namespace

int dg_ensure_diagonal(dg_mesh* m, cudaStream_t s) {
  if (m->has_diag) return DG_OK;
  const size_t nd = (size_t)m->ndofs;
  if (m->diag64 == nullptr) {
    DG_CUDA(cudaMalloc((void**)&m->diag64, nd * sizeof(double)));
    DG_CUDA(cudaMalloc((void**)&m->dinv64, nd * sizeof(double)));
    DG_CUDA(cudaMalloc((void**)&m->dinv32, nd * sizeof(float)));
  }
  const int cpb = diag_cells_per_block(m->n);
  const size_t smem = sizeof(double) * 5 * (size_t)(m->n * m->n * m->n) * cpb;
  const unsigned blocks = (unsigned)((m->ncells + cpb - 1) / cpb);
  DG_CUDA(cudaMemsetAsync(m->dflag, 0, sizeof(int), s));
  k_diag<<<blocks, 32 * cpb, smem, s>>>(m->kt64, m->gh64, m->diag64, m->dinv64, m->dinv32,
                                        m->ncells, m->N, m->n, m->dflag, m->tab64);
  DG_CUDA(cudaGetLastError());
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, m->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (flag)
    return dg_fail(DG_ERR_BREAKDOWN,
                   "Jacobi preconditioner: diag(A) has an entry <= 0 or non-finite");
  m->has_diag = true;
  return DG_OK;
}

extern "C" int dg_diagonal(const dg_mesh* mc, double* d, void* stream) {
  if (mc == nullptr || d == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_diagonal: NULL mesh or output");
  if (!mc->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_diagonal: coefficient not set");
  if (int rc0 = dg_require_cube(mc, "dg_diagonal")) return rc0;
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = dg_ensure_diagonal(m, s);
  if (rc) return rc;
  DG_CUDA(cudaMemcpyAsync(d, m->diag64, sizeof(double) * (size_t)m->ndofs,
                          cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}
