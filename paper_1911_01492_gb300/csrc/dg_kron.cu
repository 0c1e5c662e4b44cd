// Kronecker cell-block preconditioner (DG_CG_PRECOND_KRON): a reading of the
// paper's factorised cell-block solves (Section 3.4, block preconditioners on
// the cells' subspaces V_T).  Each cell block of A is replaced by the block of
// the operator with K set to its Gauss-weighted mean over the cell.  In the
// orthonormal Legendre basis (mass matrix h^3 I) that block is the Kronecker
// sum S_x (+) S_y (+) S_z of three n x n matrices,
//   S_d = h Kmean S1 + lower-face and upper-face own-side terms (Section 4.1),
// S1 the 1D stiffness matrix.  It is inverted by fast diagonalisation: with
// S_d = Q_d diag(lambda_d) Q_d^T,
//   M^-1 = (Q_z x Q_y x Q_x) diag(1 / (lx_i + ly_j + lz_l)) (Q_z x Q_y x Q_x)^T,
// six line contractions and a pointwise scaling per cell: 12n flops and
// (3n^2 + 3n) / n^3 stored values per DOF, against 2n^3 flops and n^3 values
// for the exact cell blocks.
//
// k_kron_setup: one thread per (cell, direction) forms S_d in FP64 and its
//   eigen-decomposition by cyclic Jacobi rotations; stores Q_d and lambda_d in
//   FP64 and FP32 ([c][ Q_x Q_y Q_z (row-major [i][j], column j the j-th
//   eigenvector) | l_x l_y l_z ]).
// k_kron_apply: z = M^-1 r for a group of cells per block (one thread per
//   plane of lines, the 1D factor in registers, in place in shared memory),
//   <z, r> formed in the scaling phase and reduced by the last block.
#include "dg_internal.cuh"

#include "dg_apply_impl.cuh"

namespace dgk {
namespace {

template <int N>
__global__ void __launch_bounds__(128)
k_kron_setup(const double* __restrict__ kt, const double* __restrict__ gh,
             double* __restrict__ K64, float* __restrict__ K32, long long ncells, int Nc,
             int* flag, const __grid_constant__ DGTab<double> tab) {
  constexpr int N2 = N * N, N3 = N * N * N, KS = 3 * N2 + 3 * N;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * ncells) return;
  const long long c = t / 3;
  const int d = (int)(t - 3 * c);
  const long long coord = d == 0 ? c % Nc : d == 1 ? (c / Nc) % Nc : c / ((long long)Nc * Nc);
  // h Kmean = sum_q h w_q K_q
  double hk = 0.0;
  for (int q = 0; q < N3; ++q) hk += kt[c * N3 + q];
  const double glo = gh[c * 6 + 2 * d], ghi = gh[c * 6 + 2 * d + 1];  // h gamma (0: zero flux)
  const double elo = coord > 0 ? 0.5 : 1.0, ehi = coord < Nc - 1 ? 0.5 : 1.0;
  const double sg = tab.sigma;
  double A[N][N], V[N][N];
  double scale = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s1 = 0.0;
      for (int a = 0; a < N; ++a) s1 += tab.w[a] * tab.Bd[a][i] * tab.Bd[a][j];
      const double lo =
          sg * tab.a0[i] * tab.a0[j] + elo * (tab.d0[i] * tab.a0[j] + tab.a0[i] * tab.d0[j]);
      const double hi =
          sg * tab.a1[i] * tab.a1[j] - ehi * (tab.d1[i] * tab.a1[j] + tab.a1[i] * tab.d1[j]);
      A[i][j] = hk * s1 + glo * lo + ghi * hi;
      V[i][j] = i == j ? 1.0 : 0.0;
      scale += A[i][j] * A[i][j];
    }
  }
  // cyclic Jacobi: A <- J^T A J zeroes A[p][q] with the rotation in the (p, q)
  // plane, t = tan of the angle the smaller root of t^2 + 2 theta t - 1 = 0;
  // V <- V J accumulates the eigenvectors
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0;
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) off += A[p][q] * A[p][q];
    if (off <= 1e-32 * scale) break;
#pragma unroll
    for (int p = 0; p < N; ++p) {
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        const double apq = A[p][q];
        if (fabs(apq) <= 1e-300) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cs;
#pragma unroll
        for (int k = 0; k < N; ++k) {  // columns p, q of A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = cs * akp - sn * akq;
          A[k][q] = sn * akp + cs * akq;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {  // rows p, q of J^T (A J)
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = cs * apk - sn * aqk;
          A[q][k] = sn * apk + cs * aqk;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = cs * vkp - sn * vkq;
          V[k][q] = sn * vkp + cs * vkq;
        }
      }
    }
  }
  double* o64 = K64 + c * KS;
  float* o32 = K32 + c * KS;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      o64[d * N2 + i * N + j] = V[i][j];
      o32[d * N2 + i * N + j] = (float)V[i][j];
    }
    // a direction whose two faces are both zero-flux boundary faces (one cell
    // across) has the singular factor h Kmean S1: its zero eigenvalue, up to
    // rounding, is kept at zero (the sum over the three directions stays
    // positive as long as another direction has a face with gamma > 0)
    double lam = A[i][i];
    if (lam < 0.0 && lam > -1e-12 * sqrt(scale)) lam = 0.0;
    ok = ok && lam >= 0.0 && isfinite(lam);
    o64[3 * N2 + d * N + i] = lam;
    o32[3 * N2 + d * N + i] = (float)lam;
  }
  if (!ok) atomicExch(flag, 1);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// Cells per block of the apply: one thread per plane of lines (N threads per
// cell, ~128 threads), shared memory for the work array and the factors
// within 40 KB (48 KB with the reduction arrays); at least Cfg<N>::CPB so the
// block count fits the mesh's per-block partials.
template <int N, typename T>
struct KronCfg {
  static constexpr int KS = 3 * N * N + 3 * N;
  static constexpr int PER_CELL = (N * N * N + KS) * (int)sizeof(T);
  static constexpr int BY_THREADS = 128 / N, BY_SMEM = 40960 / PER_CELL;
  static constexpr int C = BY_THREADS < BY_SMEM ? BY_THREADS : BY_SMEM;  // cells per block
  static constexpr int THREADS = C * N;
  static_assert(C >= Cfg<N>::CPB, "more blocks than the mesh's partials");
};

// The grid reduction of <z, r>: each block publishes its partial, the last
// block sums them in a fixed order and sets the CG scalars by MODE.
template <int NT, int MODE>
__device__ __forceinline__ void kron_finish(double part, double* __restrict__ partials,
                                            DGCGState* st, double* rd) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double tot = last_block_total<NT>(partials, (int)gridDim.x, rd);
  if (threadIdx.x == 0) {
    if (!isfinite(tot)) {
      st->breakdown = 1;
      st->done = 1;
      st->ru_skip = 1;
    } else if (MODE == 1) {
      st->rho = tot;
    } else if (MODE == 0) {
      st->beta = tot / st->rho;
      st->rho = tot;
    } else {
      st->rho_new = tot;
      st->beta = st->restart ? 0.0 : tot / st->rho;
    }
    st->ticket = 0u;
  }
}

// z = M^-1 r on the block's cells, in place in sw (the cells' values in their
// own order; sq holds their factors): thread (cell lc, plane t) contracts the
// N lines of plane t in each phase with the cell's 1D factor in registers.
// Returns the thread's part of <z, r> = sum over the transformed values t of
// t^2 / (lx + ly + lz), formed where the scaling is applied; the terms are
// positive, so per-thread sums (FP32 in the FP32 kernels) stay within n u
// relative, and threads and blocks are added in FP64.  In FP32 the scaling
// uses a fast reciprocal (two ulps: the preconditioner only needs to be a
// fixed symmetric positive definite operator).  Every thread of the block
// calls it; it synchronises before returning.
template <int N, typename T>
__device__ __forceinline__ T kron_solve_cells(T* sw, const T* sq, int nblk) {
  constexpr int N2 = N * N, N3 = N * N * N, KS = 3 * N2 + 3 * N;
  const int lc = threadIdx.x / N;
  const int t = threadIdx.x - lc * N;
  const bool active = lc < nblk;
  T* w = sw + lc * N3;
  const T* Qx = sq + lc * KS;
  const T* Qy = Qx + N2;
  const T* Qz = Qy + N2;
  const T* lam = Qx + 3 * N2;
  T q[N][N];
  auto load_q = [&](const T* Q) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int k = 0; k < N; ++k) q[i][k] = Q[i * N + k];
  };
  // one line of w (first element f, stride sd): w <- Q^T w (TR) or Q w
  auto line = [&](int f, int sd, bool tr) {
    T v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = w[f + i * sd];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      T a = (tr ? q[0][k] : q[k][0]) * v[0];
#pragma unroll
      for (int i = 1; i < N; ++i) a = fma(tr ? q[i][k] : q[k][i], v[i], a);
      w[f + k * sd] = a;
    }
  };
  if (active) {  // (Q_x)^T along the x-lines (j, l = t)
    load_q(Qx);
#pragma unroll
    for (int j = 0; j < N; ++j) line(t * N2 + j * N, 1, true);
  }
  __syncthreads();
  if (active) {  // (Q_y)^T along the y-lines (i, l = t)
    load_q(Qy);
#pragma unroll
    for (int i = 0; i < N; ++i) line(t * N2 + i, N, true);
  }
  __syncthreads();
  T acc = T(0);
  if (active) {  // z-lines (i, j = t): (Q_z)^T, the scaling, Q_z
    load_q(Qz);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T v[N], u[N];
#pragma unroll
      for (int l = 0; l < N; ++l) v[l] = w[l * N2 + t * N + i];
      const T lxy = lam[i] + lam[N + t];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        T a = q[0][k] * v[0];
#pragma unroll
        for (int l = 1; l < N; ++l) a = fma(q[l][k], v[l], a);
        if constexpr (sizeof(T) == 4)
          u[k] = a * __fdividef(1.0f, lxy + lam[2 * N + k]);
        else
          u[k] = a / (lxy + lam[2 * N + k]);
        acc = fma(a, u[k], acc);
      }
#pragma unroll
      for (int l = 0; l < N; ++l) {
        T a = q[l][0] * u[0];
#pragma unroll
        for (int k = 1; k < N; ++k) a = fma(q[l][k], u[k], a);
        w[l * N2 + t * N + i] = a;
      }
    }
  }
  __syncthreads();
  if (active) {  // Q_y along the y-lines
    load_q(Qy);
#pragma unroll
    for (int i = 0; i < N; ++i) line(t * N2 + i, N, false);
  }
  __syncthreads();
  if (active) {  // Q_x along the x-lines
    load_q(Qx);
#pragma unroll
    for (int j = 0; j < N; ++j) line(t * N2 + j * N, 1, false);
  }
  __syncthreads();
  return acc;
}

// Sum of one double per thread over the block, fixed order; valid in warp 0.
template <int NT>
__device__ __forceinline__ double block_total(double v, double* rd) {
  rd[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < NT; i += 32) s += rd[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  }
  __syncthreads();
  return s;
}

// MODE: 0 FP64 PCG iteration (beta = <z,r> / rho, rho = <z,r>); 1 FP64
// initialisation (rho = <z,r>, p = z, runs even when done); 2 FP32 mixed
// iteration (rho_new = <z,r>, beta = 0 on a restart, else <z,r> / rho).
template <int N, typename T, int MODE>
__global__ void __launch_bounds__(KronCfg<N, T>::THREADS)
k_kron_apply(const T* __restrict__ KD, const T* __restrict__ r, T* __restrict__ z,
             T* __restrict__ p, long long ncells, double* __restrict__ partials, DGCGState* st) {
  using KC = KronCfg<N, T>;
  constexpr int C = KC::C, N3 = N * N * N, NT = KC::THREADS, KS = KC::KS;
  if (MODE != 1 && st->done) return;
  if (MODE == 2 && st->ru_skip == 0) return;  // an FP64 refinement is pending
  __shared__ T sw[C * N3], sq[C * KS];
  __shared__ double rd[NT];
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  for (int i = threadIdx.x; i < nblk * N3; i += NT) sw[i] = r[c0 * N3 + i];
  for (int i = threadIdx.x; i < nblk * KS; i += NT) sq[i] = KD[c0 * KS + i];
  __syncthreads();
  const T acc = kron_solve_cells<N, T>(sw, sq, nblk);
  for (int i = threadIdx.x; i < nblk * N3; i += NT) {
    const T zv = sw[i];
    z[c0 * N3 + i] = zv;
    if (MODE == 1) p[c0 * N3 + i] = zv;
  }
  const double part = block_total<NT>((double)acc, rd);
  kron_finish<NT, MODE>(part, partials, st, rd);
}

// The factors in the scaled Gauss-point basis: per cell and direction
// Qhat = q Q with q[a][i] = sqrt(w_a) L_i(xi_a) (orthogonal), the eigenvalues
// unchanged: Q M Q^T is again a Kronecker sum with these eigenbases.  One
// thread per (cell, direction).
template <int N>
__global__ void k_kron_rotate(const double* __restrict__ K64, double* __restrict__ KN64,
                              float* __restrict__ KN32, long long ncells,
                              const __grid_constant__ DGTab<double> tab) {
  constexpr int N2 = N * N, KS = 3 * N2 + 3 * N;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * ncells) return;
  const long long c = t / 3;
  const int d = (int)(t - 3 * c);
  const double* Q = K64 + c * KS + d * N2;
  double* Q64 = KN64 + c * KS + d * N2;
  float* Q32 = KN32 + c * KS + d * N2;
  for (int a = 0; a < N; ++a) {
    const double sw = sqrt(tab.w[a]);
    for (int j = 0; j < N; ++j) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) acc = fma(tab.B[a][i], Q[i * N + j], acc);
      Q64[a * N + j] = sw * acc;
      Q32[a * N + j] = (float)(sw * acc);
    }
  }
  const double* L = K64 + c * KS + 3 * N2 + d * N;
  for (int j = 0; j < N; ++j) {
    KN64[c * KS + 3 * N2 + d * N + j] = L[j];
    KN32[c * KS + 3 * N2 + d * N + j] = (float)L[j];
  }
}

template <int N>
struct KronRotateF {
  template <typename T>
  static cudaError_t run(dg_mesh* m, cudaStream_t s) {
    const long long threads = 3 * m->ncells;
    k_kron_rotate<N><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        m->kron64, m->kronN64, m->kronN32, m->ncells, m->tab64);
    return cudaGetLastError();
  }
};

template <int N>
struct KronSetupF {
  template <typename T>
  static cudaError_t run(dg_mesh* m, cudaStream_t s) {
    const long long threads = 3 * m->ncells;
    k_kron_setup<N><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        m->kt64, m->gh64, m->kron64, m->kron32, m->ncells, m->N, m->dflag, m->tab64);
    return cudaGetLastError();
  }
};

template <int N>
struct KronApplyF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const void* r, void* z, void* p, int mode,
                         cudaStream_t s) {
    using K64 = KronCfg<N, double>;
    using K32 = KronCfg<N, float>;
    // inside a solve in the scaled Gauss-point basis: the rotated factors
    const double* f64 = m->nodal_op ? m->kronN64 : m->kron64;
    const float* f32 = m->nodal_op ? m->kronN32 : m->kron32;
    const unsigned b64 = (unsigned)((m->ncells + K64::C - 1) / K64::C);
    const unsigned b32 = (unsigned)((m->ncells + K32::C - 1) / K32::C);
    switch (mode) {
      case DG_KRON_FP64:
        k_kron_apply<N, double, 0><<<b64, K64::THREADS, 0, s>>>(
            f64, (const double*)r, (double*)z, nullptr, m->ncells, m->partials_cells,
            m->state);
        break;
      case DG_KRON_FP64_INIT:
        k_kron_apply<N, double, 1><<<b64, K64::THREADS, 0, s>>>(
            f64, (const double*)r, (double*)z, (double*)p, m->ncells, m->partials_cells,
            m->state);
        break;
      default:
        k_kron_apply<N, float, 2><<<b32, K32::THREADS, 0, s>>>(
            f32, (const float*)r, (float*)z, nullptr, m->ncells, m->partials_cells,
            m->state);
        break;
    }
    return cudaGetLastError();
  }
};

}  // namespace
}  // namespace dgk

int dg_ensure_kron(dg_mesh* m, cudaStream_t s) {
  if (m->has_kron) return DG_OK;
  const size_t KS = (size_t)(3 * m->n * m->n + 3 * m->n);
  if (m->kron64 == nullptr) {
    cudaError_t e = cudaMalloc((void**)&m->kron64, sizeof(double) * KS * (size_t)m->ncells);
    if (e == cudaSuccess)
      e = cudaMalloc((void**)&m->kron32, sizeof(float) * KS * (size_t)m->ncells);
    if (e != cudaSuccess) return dg_cuda_fail(e, "Kronecker cell blocks: storage");
  }
  DG_CUDA(cudaMemsetAsync(m->dflag, 0, sizeof(int), s));
  cudaError_t e = dgk::dispatch_n<double, dgk::KronSetupF>(m->n, m, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "Kronecker cell blocks: setup");
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, m->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (flag)
    return dg_fail(DG_ERR_BREAKDOWN,
                   "Kronecker cell blocks: a 1D factor has a negative eigenvalue");
  m->has_kron = true;
  return DG_OK;
}

int dg_ensure_kron_nodal(dg_mesh* m, cudaStream_t s) {
  int rc = dg_ensure_kron(m, s);
  if (rc || m->has_kron_nodal) return rc;
  const size_t KS = (size_t)(3 * m->n * m->n + 3 * m->n);
  if (m->kronN64 == nullptr) {
    cudaError_t e = cudaMalloc((void**)&m->kronN64, sizeof(double) * KS * (size_t)m->ncells);
    if (e == cudaSuccess)
      e = cudaMalloc((void**)&m->kronN32, sizeof(float) * KS * (size_t)m->ncells);
    if (e != cudaSuccess) return dg_cuda_fail(e, "Kronecker cell blocks (point basis): storage");
  }
  cudaError_t e = dgk::dispatch_n<double, dgk::KronRotateF>(m->n, m, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "Kronecker cell blocks (point basis): rotation");
  m->has_kron_nodal = true;
  return DG_OK;
}

int dg_launch_kron_apply(const dg_mesh* m, const void* r, void* z, void* p, int mode,
                         cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, dgk::KronApplyF>(m->n, m, r, z, p, mode, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "Kronecker cell blocks: apply");
  return DG_OK;
}
