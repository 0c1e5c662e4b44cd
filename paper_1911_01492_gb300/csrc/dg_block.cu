// Cell-block Jacobi preconditioner for the FP64 CG: M = the block diagonal of
// A, one n^3 x n^3 block per cell (its own volume term and the parts of its six
// face terms in which trial and test function both live on the cell), stored
// inverted.  This is the factorised ("partially matrix-free") form of the
// block solves on the cell subspaces V_T of Section 3.4; Section 2.4's PCG
// applies it as z = M^-1 r.
//
// Block of cell c in the modal basis m = (i, j, l), m' = (i', j', l'):
//   volume: sum_q Kt_q grad phi_m . grad phi_m' by a partial sum factorisation:
//     Px[i,i'][b,e] = sum_a Kt[a,b,e] L_i'(a) L_i''(a)   (and Py, Pz alike),
//     then entry = sum_{b,e} Px[i,i'][b,e] L_j(b) L_j'(b) L_l(e) L_l'(e) + (y, z);
//   faces: with the orthonormal basis and the exact face Gauss rule the
//     tangential factors give delta_{jj'} delta_{ll'} (x-faces), so face f
//     (axis d, mode index t along d) adds
//       (h gamma_F / 2) (2 sigma v_t v_t' -+ c (v_t d_t' + d_t v_t'))
//     with v, d the values and derivatives L_t(s), L_t'(s) at the face, "-" on
//     the upper face, c = 1 inside and 2 on a Dirichlet boundary (gamma_F = 0
//     on a zero-flux side).
// The inverse is formed in shared memory by Gauss-Jordan elimination without
// pivoting (the block is symmetric positive definite), one thread block per
// cell.  Degrees 1..4 (n^3 <= 125: a block of 125 KB).
#include <cmath>

#include "dg_apply_impl.cuh"

namespace {

constexpr int BLK_THREADS = 256;

template <int N>
__global__ void __launch_bounds__(BLK_THREADS)
k_block_inverse(const double* __restrict__ kt, const double* __restrict__ gh,
                double* __restrict__ binv, long long ncells, int Nc, int dmask, int* flag,
                const __grid_constant__ DGTab<double> tab) {
  constexpr int N2 = N * N, N3 = N * N * N, M = N3;
  extern __shared__ __align__(16) double sm[];
  double* A = sm;                 // M x M
  double* P = A + M * M;          // 3 x N^4: Px, Py, Pz
  double* ks = P + 3 * N2 * N2;   // N^3: h w K of the cell
  const long long c = blockIdx.x;
  if (c >= ncells) return;
  for (int t = threadIdx.x; t < N3; t += blockDim.x) ks[t] = kt[c * N3 + t];
  __syncthreads();
  // partial contractions: P_d[t,t'][u,v] over the derivative direction
  for (int t = threadIdx.x; t < 3 * N2 * N2; t += blockDim.x) {
    const int d = t / (N2 * N2), r = t - d * N2 * N2;
    const int tt = r / N2, uv = r - tt * N2;
    const int t1 = tt / N, t2 = tt % N, u = uv / N, v = uv % N;
    double acc = 0.0;
    for (int a = 0; a < N; ++a) {
      // point (x, y, z) indices with `a` along d and (u, v) along the other two
      const int qa = d == 0 ? a : u, qb = d == 1 ? a : (d == 0 ? u : v), qe = d == 2 ? a : v;
      acc = fma(ks[qa + N * (qb + N * qe)] * tab.Bd[a][t1], tab.Bd[a][t2], acc);
    }
    P[t] = acc;
  }
  __syncthreads();
  const double S2 = 4.0 * N * N;  // 2 sigma
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
    const int m = t / M, mp = t - m * M;
    const int i = m % N, j = (m / N) % N, l = m / N2;
    const int ip = mp % N, jp = (mp / N) % N, lp = mp / N2;
    double acc = 0.0;
    const double* Px = P + (i * N + ip) * N2;
    const double* Py = P + N2 * N2 + (j * N + jp) * N2;
    const double* Pz = P + 2 * N2 * N2 + (l * N + lp) * N2;
    for (int u = 0; u < N; ++u) {
      for (int v = 0; v < N; ++v) {
        // Px over (y = u, z = v), Py over (x = u, z = v), Pz over (x = u, y = v)
        acc = fma(Px[u * N + v], tab.B[u][j] * tab.B[u][jp] * tab.B[v][l] * tab.B[v][lp], acc);
        acc = fma(Py[u * N + v], tab.B[u][i] * tab.B[u][ip] * tab.B[v][l] * tab.B[v][lp], acc);
        acc = fma(Pz[u * N + v], tab.B[u][i] * tab.B[u][ip] * tab.B[v][j] * tab.B[v][jp], acc);
      }
    }
    // own-side face terms
    const int mi[3] = {i, j, l}, mpi[3] = {ip, jp, lp};
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1;
      const bool upper = f & 1;
      const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
      if (mi[o1] != mpi[o1] || mi[o2] != mpi[o2]) continue;
      const bool interior = upper ? (crd[d] < Nc - 1) : (crd[d] > 0);
      const double cf = interior ? 1.0 : 2.0;
      const double w = 0.5 * gh[c * 6 + f];
      const int a1 = mi[d], a2 = mpi[d];
      const double v1 = upper ? tab.a1[a1] : tab.a0[a1], v2 = upper ? tab.a1[a2] : tab.a0[a2];
      const double d1 = upper ? tab.d1[a1] : tab.d0[a1], d2 = upper ? tab.d1[a2] : tab.d0[a2];
      const double sgn = upper ? -1.0 : 1.0;
      acc += w * (S2 * v1 * v2 + sgn * cf * (v1 * d2 + d1 * v2));
    }
    A[t] = acc;
  }
  (void)dmask;
  __syncthreads();
  // Gauss-Jordan inverse in place
  __shared__ double piv;
  for (int k = 0; k < M; ++k) {
    if (threadIdx.x == 0) {
      const double a = A[k * M + k];
      if (!(a > 0.0) || !isfinite(a)) atomicOr(flag, 1);
      piv = 1.0 / a;
    }
    __syncthreads();
    const double p = piv;
    for (int j = threadIdx.x; j < M; j += blockDim.x)
      if (j != k) A[k * M + j] *= p;
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      const int i = t / M, j = t - i * M;
      if (i != k && j != k) A[t] = fma(-A[i * M + k], A[k * M + j], A[t]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x)
      if (i != k) A[i * M + k] = -A[i * M + k] * p;
    if (threadIdx.x == 0) A[k * M + k] = p;
    __syncthreads();
  }
  double* out = binv + c * (long long)M * M;
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) out[t] = A[t];
}

template <int N>
size_t block_inverse_smem() {
  constexpr int N2 = N * N, N3 = N * N * N;
  return sizeof(double) * ((size_t)N3 * N3 + 3 * N2 * N2 + N3);
}

// z_c = Binv_c r_c for every cell; with init: also p = z.  Partial sums of
// <z, r> per block; the last block adds them in a fixed order and sets
// rho = <z, r> (init) or beta = <z, r> / rho, rho = <z, r>.
template <int N, bool INIT>
__global__ void __launch_bounds__(128)
k_block_apply(const double* __restrict__ binv, const double* __restrict__ r,
              double* __restrict__ z, double* __restrict__ p, long long ncells,
              double* partials, DGCGState* st) {
  constexpr int N3 = N * N * N;
  if (!INIT && st->done) return;
  __shared__ double sr[N3];
  __shared__ double sw[4];
  __shared__ bool last;
  double acc = 0.0;
  for (long long c = blockIdx.x; c < ncells; c += gridDim.x) {
    __syncthreads();
    for (int t = threadIdx.x; t < N3; t += blockDim.x) sr[t] = r[c * N3 + t];
    __syncthreads();
    const double* B = binv + c * (long long)N3 * N3;  // symmetric: read column m (coalesced)
    for (int m = threadIdx.x; m < N3; m += blockDim.x) {
      double v = 0.0;
      for (int mp = 0; mp < N3; ++mp) v = fma(B[mp * N3 + m], sr[mp], v);
      z[c * N3 + m] = v;
      if (INIT) p[c * N3 + m] = v;
      acc = fma(v, sr[m], acc);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = sw[0] + sw[1] + sw[2] + sw[3];
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double rd[128];
  const double tot = dgk::last_block_total<128>(partials, (int)gridDim.x, rd);
  if (threadIdx.x == 0) {
    if (!isfinite(tot)) {
      st->breakdown = 1;
      st->done = 1;
    } else if (INIT) {
      st->rho = tot;
    } else {
      st->beta = tot / st->rho;
      st->rho = tot;
    }
    st->ticket = 0u;
  }
}

template <int N>
struct BlockBuildF {
  template <typename T>
  static cudaError_t run(dg_mesh* m, cudaStream_t s) {
    const size_t smem = block_inverse_smem<N>();
    cudaError_t e = cudaFuncSetAttribute(k_block_inverse<N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_block_inverse<N><<<(unsigned)m->ncells, BLK_THREADS, smem, s>>>(
        m->kt64, m->gh64, m->binv64, m->ncells, m->N, m->dirichlet_mask, m->dflag, m->tab64);
    return cudaGetLastError();
  }
};

template <int N>
struct BlockApplyF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const double* r, double* z, double* p, bool init,
                         cudaStream_t s) {
    const unsigned blocks = (unsigned)(m->ncells < DG_RED_BLOCKS ? m->ncells : DG_RED_BLOCKS);
    if (init)
      k_block_apply<N, true><<<blocks, 128, 0, s>>>(m->binv64, r, z, p, m->ncells, m->partials,
                                                    m->state);
    else
      k_block_apply<N, false><<<blocks, 128, 0, s>>>(m->binv64, r, z, p, m->ncells,
                                                     m->partials, m->state);
    return cudaGetLastError();
  }
};

template <template <int> class F, typename... Args>
cudaError_t dispatch_block(int n, Args... args) {
  switch (n) {
    case 2: return F<2>::template run<double>(args...);
    case 3: return F<3>::template run<double>(args...);
    case 4: return F<4>::template run<double>(args...);
    case 5: return F<5>::template run<double>(args...);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int dg_ensure_block(dg_mesh* m, cudaStream_t s) {
  if (m->has_block) return DG_OK;
  if (m->n > 5)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "cell-block Jacobi: degree %d; the blocks are formed for degree 1..4", m->k);
  if (m->binv64 == nullptr) {
    const size_t n3 = (size_t)m->n * m->n * m->n;
    cudaError_t e = cudaMalloc((void**)&m->binv64, sizeof(double) * n3 * n3 * (size_t)m->ncells);
    if (e != cudaSuccess) return dg_cuda_fail(e, "cell-block Jacobi: block storage");
  }
  DG_CUDA(cudaMemsetAsync(m->dflag, 0, sizeof(int), s));
  cudaError_t e = dispatch_block<BlockBuildF>(m->n, m, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "cell-block Jacobi: block inverse");
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, m->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (flag) return dg_fail(DG_ERR_BREAKDOWN, "cell-block Jacobi: a block is not positive definite");
  m->has_block = true;
  return DG_OK;
}

int dg_launch_block_apply(const dg_mesh* m, const double* r, double* z, double* p, bool init,
                          cudaStream_t s) {
  cudaError_t e = dispatch_block<BlockApplyF>(m->n, m, r, z, p, init, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "cell-block Jacobi: apply");
  return DG_OK;
}
