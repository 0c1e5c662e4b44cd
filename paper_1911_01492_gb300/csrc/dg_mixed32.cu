// FP32 kernels of the mixed-precision CG iteration (DG_CG_MIXED_IR).
//
// FP32 arithmetic is ~75x cheaper than FP64 on GB300, so the FP32 operator is
// bound by memory traffic, not arithmetic.  These kernels trade arithmetic for
// bytes and fold the CG vector work into the operator passes:
//   k_dir32:  p = r + beta p (beta from the device CG state, 0 on a restart;
//             formed once by k_update_xr / k_refine_r, not per thread),
//             then pass 1 of p writing only the face traces (no U, X);
//   k_cell32: reloads p, recomputes its nodal values, x-modal values and own
//             face traces in shared memory, reads the neighbours' traces,
//             forms the face weights from h*gamma on the fly, computes
//             q = A p, and folds <p, q> (FP64-accurate: exact products summed
//             in compensated float-float) into its epilogue; the last block to
//             finish commits rho = rho_new (formed with beta by the kernel
//             that updated r) and sets alpha = rho / <p, q>.
// Per DOF this moves ~35 B for the operator (instead of ~66 B in the generic
// two-pass FP32 path) and removes the separate direction and dot kernels.
// Measured at 48^3 Q4 (13.8 M DOFs): k_dir32 63 us + k_cell32 191 us per
// iteration; the same fusion built on stored U and X (generic pass 2) took
// 86 + 185 us, so recomputing in shared memory is kept.  Both are bound by
// instruction issue (~8 warp instructions per DOF), not by FP32 arithmetic or
// bytes.
#include "dg_apply_impl.cuh"

namespace dgk {

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

template <int N, bool PC>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_dir32(const float* __restrict__ r, float* __restrict__ p, float* __restrict__ TR,
        const float* __restrict__ dinv, long long ncells, const DGCGState* __restrict__ st,
        const __grid_constant__ DGTab<float> tab) {
  constexpr int C = Cfg<N>::CPB, N3 = N * N * N;
  if (st->done || st->iters >= st->maxit) return;
  const float beta = (float)st->beta;  // set once by the kernel that formed rho_new
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* s = reinterpret_cast<float*>(smem_raw);
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) {
    const long long i = c0 * N3 + t;
    float z = r[i];
    if constexpr (PC) z = dinv[i] * z;  // z = M^-1 r
    const float v = fmaf(beta, p[i], z);  // p = z + beta p
    p[i] = v;
    s[t] = v;
  }
  __syncthreads();
  trace_core<N, float, 2>(nullptr, nullptr, TR, c0, nblk, tab, s, nullptr, nullptr);
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_cell32(const float* __restrict__ p, const float* __restrict__ TR, const float* __restrict__ kt,
         const float* __restrict__ gh, float* __restrict__ q, long long ncells, int Nc,
         double* __restrict__ partials, DGCGState* st, const __grid_constant__ DGTab<float> tab) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N, NT = Cfg<N>::THREADS;
  if (st->done || st->iters >= st->maxit) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* su = reinterpret_cast<float*>(smem_raw);
  float* sx = su + C * N3;
  float* sr = sx + C * N3;
  float* sk = sr + C * N3;
  float* str = sk + C * N3;  // C * 12 * N2 own face traces
  __shared__ float rh[NT], rl[NT];
  __shared__ bool is_last;
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  // NT = C n^2 threads cover the block's C n^3 values in N strides; each
  // thread keeps its p values in registers for the <p, q> epilogue
  float preg[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;
    preg[k] = 0.0f;
    if (t < nblk * N3) {
      preg[k] = p[c0 * N3 + t];
      su[t] = preg[k];
      sk[t] = kt[c0 * N3 + t];
    }
  }
  __syncthreads();
  trace_core<N, float, 1>(nullptr, nullptr, nullptr, c0, nblk, tab, su, sx, str);
  __syncthreads();
  const FaceLocal<float> fs{TR, str, gh, &tab};
  cell_core<N, float>(fs, q, c0, nblk, Nc, tab, su, sx, sr, sk);
  // <p, q> over the block's cells; q is still in sx after cell_core
  float hi = 0.0f, lo = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;
    if (t >= nblk * N3) break;
    const float a = preg[k], b = sx[t];
    const float pr = a * b;
    const float e = fmaf(a, b, -pr);
    float s1, t1;
    two_sum_f(hi, pr, s1, t1);
    hi = s1;
    lo += t1 + e;
  }
  rh[threadIdx.x] = hi;
  rl[threadIdx.x] = lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    float h = 0.0f, l = 0.0f;
    for (int i = 0; i < NT; ++i) {
      float s1, t1;
      two_sum_f(h, rh[i], s1, t1);
      h = s1;
      l += t1 + rl[i];
    }
    partials[blockIdx.x] = (double)h + (double)l;
    __threadfence();
    is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // last block: fixed-order sum of all block partials in FP64
  __shared__ double rd[NT];
  double a = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) a += ((volatile double*)partials)[b];
  rd[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < NT; ++i) tot += rd[i];
    st->pq = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      st->breakdown = 1;
      st->done = 1;
      st->ru_skip = 1;
    } else {
      const double rho = st->rho_new;  // k_dir32 has used beta; commit the new rho
      st->rho = rho;
      st->restart = 0;
      st->alpha = rho / tot;
    }
    st->ticket = 0u;
  }
  (void)N2;
}



template <int N>
struct Mixed32F {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const float* dinv, cudaStream_t s) {
    constexpr int C = Cfg<N>::CPB, N3 = N * N * N;
    const unsigned blocks = (unsigned)((m->ncells + C - 1) / C);
    if (dinv)
      k_dir32<N, true><<<blocks, Cfg<N>::THREADS, sizeof(float) * C * N3, s>>>(
          m->r32, m->p32, m->TR32, dinv, m->ncells, m->state, m->tab32);
    else
      k_dir32<N, false><<<blocks, Cfg<N>::THREADS, sizeof(float) * C * N3, s>>>(
          m->r32, m->p32, m->TR32, dinv, m->ncells, m->state, m->tab32);
    const size_t sm2 = sizeof(float) * (4 * C * N3 + C * 12 * N * N);
    k_cell32<N><<<blocks, Cfg<N>::THREADS, sm2, s>>>(m->p32, m->TR32, m->kt32, m->gh32, m->q32,
                                                     m->ncells, m->N, m->partials_cells,
                                                     m->state, m->tab32);
    return cudaGetLastError();
  }
};

}  // namespace dgk

int dg_launch_mixed32_dir_cell(const dg_mesh* m, const float* dinv, cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<float, dgk::Mixed32F>(m->n, m, dinv, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "mixed-precision FP32 kernels launch");
  return DG_OK;
}

long long dg_mixed32_blocks(int n, long long ncells) {
  int cpb = 2;
  switch (n) {
    case 2: cpb = dgk::Cfg<2>::CPB; break;
    case 3: cpb = dgk::Cfg<3>::CPB; break;
    case 4: cpb = dgk::Cfg<4>::CPB; break;
    case 5: cpb = dgk::Cfg<5>::CPB; break;
    case 6: cpb = dgk::Cfg<6>::CPB; break;
    case 7: cpb = dgk::Cfg<7>::CPB; break;
    case 8: cpb = dgk::Cfg<8>::CPB; break;
    default: cpb = dgk::Cfg<9>::CPB; break;
  }
  return (ncells + cpb - 1) / cpb;
}
