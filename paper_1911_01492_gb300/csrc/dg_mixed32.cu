// FP32 kernels of the mixed-precision CG iteration (DG_CG_MIXED_IR).
//
// FP32 arithmetic is ~75x cheaper than FP64 on GB300, so the FP32 operator is
// bound by memory traffic and instruction issue, not arithmetic.  These
// kernels trade arithmetic for bytes and fold the CG vector work into the
// operator passes:
//   k_dir32_bulk: p = z + beta p (z = M^-1 r; beta from the device CG state,
//             0 on a restart, formed once by k_update_xr / k_refine_r), then
//             pass 1 of p writing only the face traces (no U, X).  Its inputs
//             are staged in shared memory by bulk copies (TMA engine),
//             double-buffered over groups of cells in a persistent grid.
//   k_cell32: reloads p, recomputes its nodal and x-modal values in shared
//             memory (each line-thread forms its own face traces from its
//             line's values), reads the neighbours' traces,
//             forms the face weights from h*gamma, computes q = A p, and folds
//             <p, q> (FP64-accurate: exact products summed in compensated
//             float-float) into its epilogue; the last block to finish commits
//             rho = rho_new (formed with beta by the kernel that updated r) and
//             sets alpha = rho / <p, q>.
// Per DOF this moves ~38 B for the operator (instead of ~66 B in the generic
// two-pass FP32 path) and removes the separate direction and dot kernels.
// Measured at 48^3 Q4 (13.8 M DOFs): k_dir32_bulk 53 us + k_cell32 123 us per
// iteration.  The same fusion built on stored U and X (generic pass 2) was
// slower, so recomputing in shared memory is kept.  k_cell32 is bound by
// instruction issue and block barriers (~9 warp instructions per DOF).
#include <cstdlib>

#include "dg_apply_impl.cuh"

namespace dgk {

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// ---------------------------------------------------------------------------
// Bulk copies (TMA engine, cp.async.bulk) completing on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
  return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// make the barrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this CTA's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  (void)state;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned); completion is signalled on bar as transaction bytes
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete, at most `limit`
// polls; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

// z-line loaders for trace_core (see ZFromShared): the thread that owns a
// z-line produces its values itself, with no barrier before the contraction.
// ZDirUpdate: p = z + beta p (z = M^-1 r) from the staged group buffers,
// written to global p (the operator pass reads it) and returned for the
// contraction.
template <bool PC>
struct ZDirUpdate {
  const float* sr;  // staged r of the group
  const float* sd;  // staged 1/diag(A) (PC)
  float* pg;        // global p of the group
  float beta;
  template <int N, typename T>
  __device__ __forceinline__ void operator()(const T* sc, int lc, int pp, int qq,
                                             T (&v)[N]) const {
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const int idx = l * N * N + qq * N + pp;
      const int off = lc * N * N * N + idx;
      float z = sr[off];
      if constexpr (PC) z = sd[off] * z;
      const float val = fmaf(beta, sc[idx], z);
      pg[off] = val;
      v[l] = val;
    }
  }
};

// ZLoadKeep: the z-line of p from global memory, also kept in `keep` for the
// <p, q> epilogue (each element of the block is on exactly one z-line).
template <int NK>
struct ZLoadKeep {
  const float* pg;  // global p of the block's first cell
  float (&keep)[NK];
  template <int N, typename T>
  __device__ __forceinline__ void operator()(const T* sc, int lc, int pp, int qq,
                                             T (&v)[N]) const {
    (void)sc;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      v[l] = pg[lc * N * N * N + l * N * N + qq * N + pp];
      keep[l] = v[l];
    }
  }
};

// Direction kernel with the block's inputs staged by bulk copies,
// double-buffered.  The cells are cut into groups of G = 4 CPB cells: G n^3
// floats are a multiple of 16 bytes for every n, so each group of r, p (and
// 1/diag) starts on a 16-byte boundary and is one bulk copy.  A block has one
// thread per line of every cell of a group (G n^2 threads) and walks its
// groups in a persistent grid: while it computes group g (p = z + beta p into
// shared and global memory, then the face traces), one thread has already
// started the copies of the block's next group into the other buffer.  With
// CPB-cell blocks and two buffers each the residency fell to 5 blocks of 4
// warps per SM and the kernel was no faster than plain loads; whole-group
// blocks keep the SM full.  A ragged last group is loaded with plain loads.  Waits on the copy barriers
// are bounded: on expiry the kernel sets st->timeout and st->done, waits
// (bounded again) for its copies still in flight and returns.
// stall_test != 0 (test hook) skips the first copy, so that the first wait
// runs out with no copy in flight.
template <int N, bool PC>
struct Dir32Bulk {
  static constexpr int C = Cfg<N>::CPB, N3 = N * N * N, G = 4 * C;
  static constexpr int NARR = PC ? 3 : 2;  // r, p (and 1/diag(A))
  static constexpr int THREADS = G * N * N;  // one thread per line of every cell of a group
  static constexpr unsigned GROUP_BYTES = (unsigned)(G * N3 * sizeof(float));
  // 2 barriers, then NARR arrays x 2 buffers
  static constexpr size_t SMEM = 16 + 2 * NARR * (size_t)GROUP_BYTES;
  static_assert(GROUP_BYTES % 16 == 0, "bulk copies need 16-byte multiples");
};

template <int N, bool PC>
__global__ void __launch_bounds__(Dir32Bulk<N, PC>::THREADS)
k_dir32_bulk(const float* __restrict__ r, float* __restrict__ p, float* __restrict__ TR,
             const float* __restrict__ dinv, long long ncells, DGCGState* st,
             long long limit, int stall_test, const __grid_constant__ DGTab<float> tab) {
  using B = Dir32Bulk<N, PC>;
  constexpr int N3 = B::N3, G = B::G, NT = B::THREADS;
  if (st->done || st->iters >= st->maxit) return;
  const float beta = (float)st->beta;  // set once by the kernel that formed rho_new
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
  float* buf = reinterpret_cast<float*>(smem_raw + 16);
  // buffer b (0, 1) of r, p and 1/diag: pointer arithmetic, not arrays
  // indexed at run time (which would live in local memory)
  auto br = [&](int b) { return buf + b * G * N3; };
  auto bp = [&](int b) { return buf + (2 + b) * G * N3; };
  auto bd = [&](int b) { return buf + (4 + b) * G * N3; };  // PC only
  const long long ngroups = (ncells + G - 1) / G;
  const long long nfull = ncells / G;  // groups moved by bulk copies
  auto issue = [&](long long g, int b) {  // thread 0 only
    mbar_arrive_expect_tx(&bar[b], B::NARR * B::GROUP_BYTES);
    bulk_g2s(br(b), r + g * G * N3, B::GROUP_BYTES, &bar[b]);
    bulk_g2s(bp(b), p + g * G * N3, B::GROUP_BYTES, &bar[b]);
    if constexpr (PC) bulk_g2s(bd(b), dinv + g * G * N3, B::GROUP_BYTES, &bar[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long g = blockIdx.x;
  // a copy into buffer 0 / 1 is in flight (thread 0's view)
  bool issued0 = false, issued1 = false;
  auto set_issued = [&](int b, bool v) {
    if (b) issued1 = v;
    else issued0 = v;
  };
  if (threadIdx.x == 0 && g < nfull && !stall_test) {
    issue(g, 0);
    issued0 = true;
  }
  bool failed = false;
  int it = 0;
  for (; g < ngroups; g += gridDim.x, ++it) {
    const int b = it & 1;
    const long long gn = g + gridDim.x;
    if (threadIdx.x == 0 && gn < nfull) {
      fence_proxy_async();  // the previous group's generic accesses to buffer b^1
      issue(gn, b ^ 1);
      set_issued(b ^ 1, true);
    }
    const long long cg0 = g * G;
    if (g < nfull) {
      const bool ok = mbar_wait_bounded(&bar[b], (unsigned)((it >> 1) & 1), limit);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (threadIdx.x == 0) set_issued(b, false);
    } else {  // ragged last group
      const int n = (int)(ncells - cg0) * N3;
      for (int t = threadIdx.x; t < n; t += NT) {
        br(b)[t] = r[cg0 * N3 + t];
        bp(b)[t] = p[cg0 * N3 + t];
        if constexpr (PC) bd(b)[t] = dinv[cg0 * N3 + t];
      }
      __syncthreads();
    }
    {
      const int nblk = (int)((ncells - cg0) < G ? (ncells - cg0) : G);
      // p = z + beta p by the z-line threads, then pass 1 of p (traces only)
      const ZDirUpdate<PC> zl{br(b), bd(b), p + cg0 * N3, beta};
      trace_core<N, float, 2>(nullptr, nullptr, TR, cg0, nblk, tab, bp(b), nullptr, zl);
      __syncthreads();
    }
  }
  if (failed && threadIdx.x == 0) {
    st->timeout = 1;
    st->done = 1;
    st->ru_skip = 1;
    // copies of this block still in flight: wait for them, bounded again
    for (int bb = 0; bb < 2; ++bb)
      if (bb ? issued1 : issued0)
        mbar_wait_bounded(&bar[bb], (unsigned)(((it + (bb != (it & 1))) >> 1) & 1), limit);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_inval(&bar[0]);
    mbar_inval(&bar[1]);
  }
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
  __shared__ float rh[NT], rl[NT];
  __shared__ bool is_last;
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  // h w K of the block's cells: loaded into registers now, stored to shared
  // memory after pass 1 (the cell phase reads it), so that these loads and
  // the z-line loads of p below are in flight together
  float kreg[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;
    kreg[k] = t < nblk * N3 ? kt[c0 * N3 + t] : 0.0f;
  }
  // pass 1 in shared memory; each z-line thread loads its line of p from
  // global memory and keeps it for the <p, q> epilogue
  float preg[N];
#pragma unroll
  for (int l = 0; l < N; ++l) preg[l] = 0.0f;
  const ZLoadKeep<N> zl{p + c0 * N3, preg};
  trace_core<N, float, 3>(nullptr, nullptr, nullptr, c0, nblk, tab, su, sx, zl);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;
    if (t < nblk * N3) sk[t] = kreg[k];
  }
  __syncthreads();
  const FaceLocal<float> fs{TR, gh, &tab};
  cell_core<N, float>(fs, q, c0, nblk, Nc, tab, su, sx, sr, sk);
  // <p, q> over the block's cells on the z-lines of p kept above; q is
  // still in sx after cell_core (same layout as p)
  float hi = 0.0f, lo = 0.0f;
  const int zlc = threadIdx.x / N2, zt2 = threadIdx.x - zlc * N2;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    if (zlc >= nblk) break;
    const float a = preg[l], b = sx[zlc * N3 + l * N2 + zt2];
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
  // Fixed-order compensated block sum: lane l of warp 0 folds entries
  // l, l + 32, ... (NT >= 32 for every degree, so warp 0 is full), then a
  // butterfly over the warp.  A serial sum by one thread kept the whole block
  // resident for ~NT dependent TwoSums.
  if (threadIdx.x < 32) {
    float h = rh[threadIdx.x], l = rl[threadIdx.x];
    for (int i = threadIdx.x + 32; i < NT; i += 32) {
      float s1, t1;
      two_sum_f(h, rh[i], s1, t1);
      h = s1;
      l += t1 + rl[i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, off);
      const float ol = __shfl_xor_sync(0xffffffffu, l, off);
      float s1, t1;
      two_sum_f(h, oh, s1, t1);
      h = s1;
      l += ol + t1;
    }
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = (double)h + (double)l;
      __threadfence();
      is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
    }
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
      const double rho = st->rho_new;  // k_dir32_bulk has used beta; commit the new rho
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
    // test hook (read when the iteration is captured): the direction kernel
    // skips its first bulk copy and gives up its wait after a few polls
    const char* env = getenv("DG_TEST_BULK_STALL");
    const bool stall_now = env != nullptr && env[0] == '1';
    const long long limit = stall_now ? (1LL << 12) : (1LL << 22);
    const int pc = dinv != nullptr;
    const unsigned gb = (unsigned)m->dir_bulk_grid[pc];
    if (pc)
      k_dir32_bulk<N, true><<<gb, Dir32Bulk<N, true>::THREADS, Dir32Bulk<N, true>::SMEM, s>>>(
          m->r32, m->p32, m->TR32, dinv, m->ncells, m->state, limit, stall_now ? 1 : 0,
          m->tab32);
    else
      k_dir32_bulk<N, false><<<gb, Dir32Bulk<N, false>::THREADS, Dir32Bulk<N, false>::SMEM, s>>>(
          m->r32, m->p32, m->TR32, dinv, m->ncells, m->state, limit, stall_now ? 1 : 0,
          m->tab32);
    const size_t sm2 = sizeof(float) * 4 * C * N3;
    k_cell32<N><<<blocks, Cfg<N>::THREADS, sm2, s>>>(m->p32, m->TR32, m->kt32, m->gh32, m->q32,
                                                     m->ncells, m->N, m->partials_cells,
                                                     m->state, m->tab32);
    return cudaGetLastError();
  }
};

// Kernel attributes and the persistent grid of the bulk-copy direction kernel
// (host calls that must not run inside stream capture).
template <int N>
struct PrepareMixed32F {
  template <typename T>
  static cudaError_t run(dg_mesh* m) {
    const long long ngroups = (m->ncells + Dir32Bulk<N, false>::G - 1) / Dir32Bulk<N, false>::G;
    for (int pc = 0; pc < 2; ++pc) {
      const void* fn = pc ? (const void*)k_dir32_bulk<N, true> : (const void*)k_dir32_bulk<N, false>;
      const size_t smem = pc ? Dir32Bulk<N, true>::SMEM : Dir32Bulk<N, false>::SMEM;
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, Dir32Bulk<N, false>::THREADS,
                                                        smem);
      if (e != cudaSuccess) return e;
      if (occ < 1) return cudaErrorInvalidConfiguration;
      const long long full = (long long)occ * m->sm_count;
      m->dir_bulk_grid[pc] = (int)(ngroups < full ? ngroups : full);
    }
    return cudaSuccess;
  }
};

}  // namespace dgk

int dg_prepare_mixed32(dg_mesh* m) {
  cudaError_t e = dgk::dispatch_n<float, dgk::PrepareMixed32F>(m->n, m);
  if (e != cudaSuccess) return dg_cuda_fail(e, "mixed-precision FP32 kernel attributes");
  return DG_OK;
}

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
