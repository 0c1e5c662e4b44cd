// FP32 kernels of the mixed-precision CG iteration (DG_CG_MIXED_IR).
//
// FP32 arithmetic is ~75x cheaper than FP64 on GB300, so the FP32 operator is
// bound by memory traffic, instruction issue and latency, not arithmetic.
// These kernels trade arithmetic for bytes and fold the CG vector work into the
// operator passes:
//   k_dir32_bulk: p = z + beta p (z = M^-1 r; beta from the device CG state,
//             0 on a restart, formed once by k_update_xr / k_refine_r), then
//             pass 1 of p writing only the face traces (no U, X).  Its inputs
//             are staged in shared memory by bulk copies (TMA engine),
//             double-buffered over groups of cells in a persistent grid.
//   k_cell32x2: reloads p, recomputes its nodal and x-modal values in shared
//             memory (each line-thread forms its own face traces from its
//             line's values), reads the neighbours' traces, forms the face
//             weights from h*gamma, computes q = A p, and folds <p, q>
//             (FP64-accurate: exact products summed in compensated float-float)
//             into its epilogue; the last block to finish commits rho = rho_new
//             (formed with beta by the kernel that updated r) and sets
//             alpha = rho / <p, q>.  It works on pairs of cells in packed FP32
//             arithmetic (FFMA2 / FADD2 / FMUL2, dg_pair32.cuh): every
//             instruction serves two cells.
// Per DOF this moves ~38 B for the operator (instead of ~66 B in the generic
// two-pass FP32 path) and removes the separate direction and dot kernels.
// Measured at 48^3 Q4 (13.8 M DOFs): the cell kernel on single cells ran at
// 6.7 warp instructions per DOF, issue-bound (123 us); on cell pairs it runs
// 3.4 per DOF and is bound by load latency (about 100 us), the whole FP32
// iteration 0.219 ms instead of 0.242 ms.
#include <cstdlib>

#include "dg_apply_impl.cuh"
#include "dg_pair32.cuh"

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

// Pass 1 in the scaled Gauss-point basis (DG_CG_NODAL solves) on a group of
// cells staged in shared memory (s, n^3 values per cell): the z-line threads
// produce their lines with the loader (the direction update), keep them in
// shared memory for the y- and x-lines and form the z-face traces at once;
// after one barrier the same threads form the y- and x-face traces.  Traces
// (value, full reference derivative) by the scaled Lagrange end values, layout
// TR[c][2f + {0, 1}][n^2] as in the Legendre basis.
template <int N, typename T, typename ZL>
__device__ __forceinline__ void trace_core_nd(T* __restrict__ TR, long long c0, int nblk,
                                              const DGTabN<T>& tn, T* s, const ZL& zload) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  T* sc = s + lc * N3;
  T* tr = TR + (c0 + lc) * (12 * N2) + t2;
  auto ends = [&](const T (&u)[N], T* trf) {
    using ::fma;  // the scalar one (dgk::fma is the packed pair's)
    T vm = tn.l0[0] * u[0], vp = tn.l1[0] * u[0];
    T gm = tn.dl0[0] * u[0], gp = tn.dl1[0] * u[0];
#pragma unroll
    for (int e = 1; e < N; ++e) {
      vm = fma(tn.l0[e], u[e], vm);
      vp = fma(tn.l1[e], u[e], vp);
      gm = fma(tn.dl0[e], u[e], gm);
      gp = fma(tn.dl1[e], u[e], gp);
    }
    trf[0] = vm;
    trf[N2] = gm;
    trf[2 * N2] = vp;
    trf[3 * N2] = gp;
  };
  if (active) {  // z-line (a = p, b = q)
    T v[N];
    zload.template operator()<N, T>(sc, lc, p, q, v);
#pragma unroll
    for (int e = 0; e < N; ++e) sc[e * N2 + q * N + p] = v[e];
    ends(v, tr + 8 * N2);
  }
  __syncthreads();
  if (active) {
    T u[N];
#pragma unroll
    for (int b = 0; b < N; ++b) u[b] = sc[q * N2 + b * N + p];  // y-line (a = p, e = q)
    ends(u, tr + 4 * N2);
#pragma unroll
    for (int a = 0; a < N; ++a) u[a] = sc[q * N2 + p * N + a];  // x-line (b = p, e = q)
    ends(u, tr);
  }
}

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

// ND: the scaled Gauss-point basis (point values in, trace_core_nd).
template <int N, bool PC, bool ND = false>
__global__ void __launch_bounds__(Dir32Bulk<N, PC>::THREADS)
k_dir32_bulk(const float* __restrict__ r, float* __restrict__ p, float* __restrict__ TR,
             const float* __restrict__ dinv, long long ncells, DGCGState* st,
             long long limit, int stall_test, const __grid_constant__ DGTab<float> tab,
             const __grid_constant__ DGTabN<float> tn) {
  using B = Dir32Bulk<N, PC>;
  constexpr int N3 = B::N3, G = B::G, NT = B::THREADS;
  // nothing to do once done, at the cap, or with an FP64 refinement pending
  if (st->done || st->iters >= st->maxit || st->ru_skip == 0) return;
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
      if constexpr (ND)
        trace_core_nd<N, float>(TR, cg0, nblk, tn, bp(b), zl);
      else
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

// ---------------------------------------------------------------------------
// k_cell32x2: the FP32 operator pass of the mixed iteration on pairs of
// consecutive cells (a = c0 + 2j, b = a + 1), each value a packed FP32 pair
// (dg_pair32.cuh): one FFMA2 / FADD2 / FMUL2, one 64-bit shared-memory access
// and one address computation serve both cells.  Every lane computes what a
// single-cell kernel computes for its cell, with the same FP32 operations in
// the same order.  Per-lane differences (a face on the boundary for one cell
// of the pair only, a last pair with one cell) are handled with per-lane data
// instead of branches: a boundary lane's neighbour trace is zero, and its
// derivative term and derivative weight take the factor e = 2 (e = 1 inside),
// which turns the interior flux into the one-sided one; a lane without a cell
// loads nothing.  The block: pass 1 of p in shared memory, the cell phase with
// own traces formed in the line threads and the neighbours' traces from the
// direction kernel, and <p, q> folded into the epilogue, where each z-line
// thread still holds its z-line of p and of q in registers.  Registers are
// capped at 64 for n <= 5 (eight blocks per SM).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS, N <= 5 ? 8 : 1)
k_cell32x2(const float* __restrict__ pg, const float* __restrict__ TR,
           const float* __restrict__ kt, const float* __restrict__ gh, float* __restrict__ qg,
           long long ncells, int Nc, double* __restrict__ partials, DGCGState* st,
           const __grid_constant__ DGTab<float> tab) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N, NT = Cfg<N>::THREADS;
  constexpr float S2 = 4.0f * N * N;  // 2 sigma, sigma = 2 (k+1)^2
  // nothing to do once done, at the cap, or with an FP64 refinement pending
  if (st->done || st->iters >= st->maxit || st->ru_skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F2* su = reinterpret_cast<F2*>(smem_raw);
  F2* sx = su + C * N3;
  F2* sr = sx + C * N3;
  F2* sk = sr + C * N3;
  __shared__ float rh[NT], rl[NT];
  __shared__ bool is_last;
  __shared__ int sbase[3];
  const long long c0 = (long long)blockIdx.x * (2 * C);
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const long long ca = c0 + 2 * lc, cb = ca + 1;
  const bool va = ca < ncells, vb = cb < ncells;
  const int o = lc * N3;
  if (threadIdx.x == 0) {
    const unsigned cu = (unsigned)c0, n = (unsigned)Nc;
    sbase[0] = (int)(cu % n);
    sbase[1] = (int)((cu / n) % n);
    sbase[2] = (int)(cu / n / n);
  }
  // h w K of the block's cell pairs into registers (stored to shared memory
  // after pass 1), in flight together with the z-line loads of p
  F2 kreg[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;  // < C N3 = N NT
    const int pr = t / N3, pos = t - pr * N3;
    const long long c = c0 + 2 * pr;
    kreg[k] = F2(c < ncells ? kt[c * N3 + pos] : 0.0f, c + 1 < ncells ? kt[(c + 1) * N3 + pos] : 0.0f);
  }
  // pass 1 in shared memory.  z-lines: thread owns (i = p, j = q); it loads its
  // z-line of p (both cells) and keeps it for <p, q>
  F2 preg[N];
  {
    F2 u[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const int idx = l * N2 + q * N + p;
      preg[l] = F2(va ? pg[ca * N3 + idx] : 0.0f, vb ? pg[cb * N3 + idx] : 0.0f);
    }
    b_fwd<N>(tab, preg, u);
#pragma unroll
    for (int e = 0; e < N; ++e) su[o + e * N2 + q * N + p] = u[e];
  }
  __syncthreads();
  {  // y-lines: (i = p, e = q)
    F2 v[N], u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = su[o + q * N2 + j * N + p];
    b_fwd<N>(tab, v, u);
#pragma unroll
    for (int b = 0; b < N; ++b) su[o + q * N2 + b * N + p] = u[b];
  }
  __syncthreads();
  {  // x-lines: (b = p, e = q); X (x-modal) kept in sx, nodal values in su
    F2 X[N], u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) X[i] = su[o + q * N2 + p * N + i];
#pragma unroll
    for (int i = 0; i < N; ++i) sx[o + q * N2 + p * N + i] = X[i];
    b_fwd<N>(tab, X, u);
#pragma unroll
    for (int a = 0; a < N; ++a) su[o + q * N2 + p * N + a] = u[a];
  }
#pragma unroll
  for (int k = 0; k < N; ++k) sk[threadIdx.x + k * NT] = kreg[k];
  // cell coordinates of both lanes; interior flags as bits (face f: bit f for
  // lane a, bit 8 + f for lane b)
  int cxa = sbase[0] + 2 * lc, cya = sbase[1], cza = sbase[2];
  while (cxa >= Nc) {
    cxa -= Nc;
    if (++cya == Nc) {
      cya = 0;
      ++cza;
    }
  }
  int cxb = cxa + 1, cyb = cya, czb = cza;
  if (cxb == Nc) {
    cxb = 0;
    if (++cyb == Nc) {
      cyb = 0;
      ++czb;
    }
  }
  const bool pairrow = vb && cxb != 0;  // both cells of the pair in one x-row
  const long long sy = Nc, sz = (long long)Nc * Nc;
  const int pt = p + N * q;
  const float hw2 = 0.5f * tab.w[pt % N] * tab.w[pt / N];
  // face f's neighbour trace (value, derivative) and weight W/2 for both lanes;
  // zero trace on a boundary lane
  auto face = [&](int f, bool ina, bool inb, long long cna, long long cnb, F2& un, F2& gn,
                  F2& wh, F2& e, bool lda = true, bool ldb = true) {
    float ua = 0.f, ga = 0.f, ub = 0.f, gb = 0.f;
    if (ina && lda) load_trace<N>(TR, cna, f ^ 1, pt, ua, ga);
    if (inb && ldb) load_trace<N>(TR, cnb, f ^ 1, pt, ub, gb);
    un = F2(ua, ub);
    gn = F2(ga, gb);
    wh = F2(va ? hw2 * gh[ca * 6 + f] : 0.0f, vb ? hw2 * gh[cb * 6 + f] : 0.0f);
    e = F2(ina ? 1.0f : 2.0f, inb ? 1.0f : 2.0f);
  };
  F2 un[4], gn[4], wh[4], ee[4];  // faces z-, z+, y-, y+ (then x-, x+ in slots 0, 1)
  // a lane without a cell (the second cell of an odd last pair, or a pair
  // past the end) loads no face data: its values stay zero and finite
  face(4, va && cza > 0, vb && czb > 0, ca - sz, cb - sz, un[0], gn[0], wh[0], ee[0]);
  face(5, va && cza < Nc - 1, vb && czb < Nc - 1, ca + sz, cb + sz, un[1], gn[1], wh[1], ee[1]);
  face(2, va && cya > 0, vb && cyb > 0, ca - sy, cb - sy, un[2], gn[2], wh[2], ee[2]);
  face(3, va && cya < Nc - 1, vb && cyb < Nc - 1, ca + sy, cb + sy, un[3], gn[3], wh[3], ee[3]);
  __syncthreads();
  // flux of one face point from the own trace (uo, go) and the face data:
  // cv multiplies the test value, -cd the test derivative
  auto flux = [&](bool upper, F2 uo, F2 go, F2 unf, F2 gnf, F2 whf, F2 ef, F2& cv, F2& cd) {
    const F2 J = upper ? uo - unf : unf - uo;
    const F2 G = fma(ef, go, gnf);
    const F2 tt = upper ? fma(S2, J, -G) : fma(-S2, J, G);
    cv = whf * tt;
    cd = (whf * ef) * J;
  };
  // z-lines then y-lines: collocation derivative, h w K, transpose, own and
  // neighbour face terms
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const int base = (dir == 0) ? (q * N + p) : (q * N2 + p);
    const int step = (dir == 0) ? N2 : N;
    F2 u[N], r[N], kg[N];
#pragma unroll
    for (int e = 0; e < N; ++e) u[e] = su[o + base + e * step];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      F2 g = tab.D[e][0] * u[0];
#pragma unroll
      for (int f = 1; f < N; ++f) g = fma(tab.D[e][f], u[f], g);
      kg[e] = sk[o + base + e * step] * g;
    }
#pragma unroll
    for (int e = 0; e < N; ++e) {
      F2 acc = (dir == 0) ? tab.D[0][e] * kg[0] : fma(tab.D[0][e], kg[0], sr[o + base + e * step]);
#pragma unroll
      for (int f = 1; f < N; ++f) acc = fma(tab.D[f][e], kg[f], acc);
      r[e] = acc;
    }
    F2 vm = tab.l0[0] * u[0], vp = tab.l1[0] * u[0];
    F2 gm = tab.dl0[0] * u[0], gp = tab.dl1[0] * u[0];
#pragma unroll
    for (int e = 1; e < N; ++e) {
      vm = fma(tab.l0[e], u[e], vm);
      vp = fma(tab.l1[e], u[e], vp);
      gm = fma(tab.dl0[e], u[e], gm);
      gp = fma(tab.dl1[e], u[e], gp);
    }
    const int su_ = 2 * dir + 1, sl_ = 2 * dir;  // slots of the upper and lower face
    F2 cv1, cd1, cv0, cd0;
    flux(true, vp, gp, un[su_], gn[su_], wh[su_], ee[su_], cv1, cd1);
    flux(false, vm, gm, un[sl_], gn[sl_], wh[sl_], ee[sl_], cv0, cd0);
#pragma unroll
    for (int e = 0; e < N; ++e) {
      F2 acc = fma(tab.l1[e], cv1, r[e]);
      acc = fma(-tab.dl1[e], cd1, acc);
      acc = fma(tab.l0[e], cv0, acc);
      r[e] = fma(-tab.dl0[e], cd0, acc);
    }
#pragma unroll
    for (int e = 0; e < N; ++e) sr[o + base + e * step] = r[e];
    if (dir == 1) {  // the x-faces' data, in flight during the barrier
      // b's x- neighbour and a's x+ neighbour are the pair's other cell when
      // both sit in one x-row: their traces are formed in this thread below
      face(0, va && cxa > 0, vb && cxb > 0, ca - 1, cb - 1, un[0], gn[0], wh[0], ee[0], true,
           !pairrow);
      face(1, va && cxa < Nc - 1, vb && cxb < Nc - 1, ca + 1, cb + 1, un[1], gn[1], wh[1],
           ee[1], !pairrow, true);
    }
    __syncthreads();
  }
  {  // x-lines: (b = p, e = q); result x-modal, yz-nodal
    const int base = q * N2 + p * N;
    F2 X[N], rr[N], R[N], g[N], kg[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      X[i] = sx[o + base + i];
      rr[i] = sr[o + base + i];
    }
    bd_fwd<N>(tab, X, g);
#pragma unroll
    for (int a = 0; a < N; ++a) kg[a] = sk[o + base + a] * g[a];
    bt_bdt<N>(tab, rr, kg, R);
    F2 Se = X[0], So = tab.a1[1] * X[1], Do = tab.d1[1] * X[1], De = F2(0.0f);
#pragma unroll
    for (int i = 2; i < N; i += 2) Se = fma(tab.a1[i], X[i], Se);
#pragma unroll
    for (int i = 3; i < N; i += 2) So = fma(tab.a1[i], X[i], So);
#pragma unroll
    for (int i = 3; i < N; i += 2) Do = fma(tab.d1[i], X[i], Do);
    if (N > 2) {
      De = tab.d1[2] * X[2];
#pragma unroll
      for (int i = 4; i < N; i += 2) De = fma(tab.d1[i], X[i], De);
    }
    F2 cv1, cd1, cv0, cd0;
    if (pairrow) {  // the face between the pair's cells: each lane's neighbour is the other lane
      const F2 xm = Se - So, xp = Se + So, dxm = Do - De, dxp = Do + De;
      un[1].v.x = xm.v.y;
      gn[1].v.x = dxm.v.y;
      un[0].v.y = xp.v.x;
      gn[0].v.y = dxp.v.x;
    }
    flux(true, Se + So, Do + De, un[1], gn[1], wh[1], ee[1], cv1, cd1);
    flux(false, Se - So, Do - De, un[0], gn[0], wh[0], ee[0], cv0, cd0);
    const F2 spl = cv1 + cv0, smn = cv1 - cv0;
    const F2 dpl = cd1 + cd0, dmn = cd1 - cd0;
    R[0] = R[0] + spl;
#pragma unroll
    for (int i = 1; i < N; ++i) {
      if (i % 2 == 0)
        R[i] = fma(tab.a1[i], spl, fma(-tab.d1[i], dmn, R[i]));
      else
        R[i] = fma(tab.a1[i], smn, fma(-tab.d1[i], dpl, R[i]));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) sx[o + base + i] = R[i];
  }
  __syncthreads();
  {  // back along y: (i = p, e = q)
    F2 v[N], R[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = sx[o + q * N2 + b * N + p];
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int j = 0; j < N; ++j) sx[o + q * N2 + j * N + p] = R[j];
  }
  __syncthreads();
  // back along z: (i = p, j = q), the thread's z-line of q: store it and fold
  // <p, q> over it (exact products, compensated float-float sums per lane)
  F2 hi = F2(0.0f), lo = F2(0.0f);
  {
    F2 v[N], R[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sx[o + e * N2 + q * N + p];
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const int idx = l * N2 + q * N + p;
      if (va) qg[ca * N3 + idx] = R[l].v.x;
      if (vb) qg[cb * N3 + idx] = R[l].v.y;
      const F2 pr = preg[l] * R[l];
      const F2 er = fma(preg[l], R[l], -pr);  // preg R = pr + er exactly
      const F2 s1 = hi + pr;
      const F2 bb = s1 - hi;
      const F2 t1 = (hi - (s1 - bb)) + (pr - bb);
      hi = s1;
      lo = lo + (t1 + er);
    }
  }
  {  // combine the lanes
    float s1, t1;
    two_sum_f(hi.v.x, hi.v.y, s1, t1);
    rh[threadIdx.x] = s1;
    rl[threadIdx.x] = (lo.v.x + lo.v.y) + t1;
  }
  __syncthreads();
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
  __shared__ double rd[NT];
  const double tot = last_block_total<NT>(partials, (int)gridDim.x, rd);
  if (threadIdx.x == 0) {
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
}

// ---------------------------------------------------------------------------
// k_cell32x2_nd: the FP32 operator pass of the mixed iteration in the scaled
// Gauss-point basis (DG_CG_NODAL), on pairs of consecutive cells in packed
// FP32 like k_cell32x2.  Per line of each direction (z, then y, then x):
// r += Dh^T (h K . Dh u) with Dh = sqrt(w) D / sqrt(w) (the collocation
// derivative of the scaled point values), plus the own and neighbour face
// terms with the scaled Lagrange end values and the face weight h gamma / 2.
// No basis transforms: the z-line threads load p from global memory, the
// partial sums of q stay in shared memory, the x-line threads finish q, store
// it and fold <p, q> (exact products, compensated float-float sums) as the
// Legendre-basis kernel does.  Three block barriers instead of eight.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS, N <= 5 ? 8 : 1)
k_cell32x2_nd(const float* __restrict__ pg, const float* __restrict__ TR,
              const float* __restrict__ hk, const float* __restrict__ gh, float* __restrict__ qg,
              long long ncells, int Nc, double* __restrict__ partials, DGCGState* st,
              const __grid_constant__ DGTabN<float> tn) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N, NT = Cfg<N>::THREADS;
  constexpr float S2 = 4.0f * N * N;  // 2 sigma, sigma = 2 (k+1)^2
  if (st->done || st->iters >= st->maxit || st->ru_skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F2* su = reinterpret_cast<F2*>(smem_raw);
  F2* sr = su + C * N3;
  F2* sk = sr + C * N3;
  __shared__ float rh[NT], rl[NT];
  __shared__ bool is_last;
  __shared__ int sbase[3];
  const long long c0 = (long long)blockIdx.x * (2 * C);
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const long long ca = c0 + 2 * lc, cb = ca + 1;
  const bool va = ca < ncells, vb = cb < ncells;
  const int o = lc * N3;
  if (threadIdx.x == 0) {
    const unsigned cu = (unsigned)c0, n = (unsigned)Nc;
    sbase[0] = (int)(cu % n);
    sbase[1] = (int)((cu / n) % n);
    sbase[2] = (int)(cu / n / n);
  }
  // h K of the block's cell pairs and the thread's z-line of p (a = p, b = q)
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int t = threadIdx.x + k * NT;  // < C N3 = N NT
    const int pr = t / N3, pos = t - pr * N3;
    const long long c = c0 + 2 * pr;
    sk[t] = F2(c < ncells ? hk[c * N3 + pos] : 0.0f, c + 1 < ncells ? hk[(c + 1) * N3 + pos] : 0.0f);
  }
  F2 u[N];
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const int idx = e * N2 + q * N + p;
    u[e] = F2(va ? pg[ca * N3 + idx] : 0.0f, vb ? pg[cb * N3 + idx] : 0.0f);
    su[o + idx] = u[e];
  }
  __syncthreads();
  int cxa = sbase[0] + 2 * lc, cya = sbase[1], cza = sbase[2];
  while (cxa >= Nc) {
    cxa -= Nc;
    if (++cya == Nc) {
      cya = 0;
      ++cza;
    }
  }
  int cxb = cxa + 1, cyb = cya, czb = cza;
  if (cxb == Nc) {
    cxb = 0;
    if (++cyb == Nc) {
      cyb = 0;
      ++czb;
    }
  }
  const bool pairrow = vb && cxb != 0;  // both cells of the pair in one x-row
  const long long sy = Nc, sz = (long long)Nc * Nc;
  const int pt = t2;
  // face f's neighbour trace, weight h gamma / 2 and boundary factor e for
  // both lanes (zero trace on a boundary lane; a lane without a cell loads
  // nothing and keeps finite zeros)
  auto face = [&](int f, bool ina, bool inb, long long cna, long long cnb, F2& un, F2& gn,
                  F2& wh, F2& e, bool lda = true, bool ldb = true) {
    float ua = 0.f, ga = 0.f, ub = 0.f, gb = 0.f;
    if (ina && lda) load_trace<N>(TR, cna, f ^ 1, pt, ua, ga);
    if (inb && ldb) load_trace<N>(TR, cnb, f ^ 1, pt, ub, gb);
    un = F2(ua, ub);
    gn = F2(ga, gb);
    wh = F2(va ? 0.5f * gh[ca * 6 + f] : 0.0f, vb ? 0.5f * gh[cb * 6 + f] : 0.0f);
    e = F2(ina ? 1.0f : 2.0f, inb ? 1.0f : 2.0f);
  };
  auto flux = [&](bool upper, F2 uo, F2 go, F2 unf, F2 gnf, F2 whf, F2 ef, F2& cv, F2& cd) {
    const F2 J = upper ? uo - unf : unf - uo;
    const F2 G = fma(ef, go, gnf);
    const F2 tt = upper ? fma(S2, J, -G) : fma(-S2, J, G);
    cv = whf * tt;
    cd = (whf * ef) * J;
  };
  // one line: r = r + Dh^T (hK . Dh u) + the line's two faces (slots sl, su_)
  // swap: the two faces are the x-faces and the pair shares one of them (the
  // lanes' own traces there are each other's neighbour traces)
  auto line = [&](int base, int step, F2 (&un)[2], F2 (&gn)[2], const F2 (&wh)[2],
                  const F2 (&ee)[2], F2 (&r)[N], bool swap = false) {
    F2 kg[N];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      F2 g = tn.Dh[e][0] * u[0];
#pragma unroll
      for (int f = 1; f < N; ++f) g = fma(tn.Dh[e][f], u[f], g);
      kg[e] = sk[o + base + e * step] * g;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int e = 0; e < N; ++e) r[i] = fma(tn.Dh[e][i], kg[e], r[i]);
    }
    F2 vm = tn.l0[0] * u[0], vp = tn.l1[0] * u[0];
    F2 gm = tn.dl0[0] * u[0], gp = tn.dl1[0] * u[0];
#pragma unroll
    for (int e = 1; e < N; ++e) {
      vm = fma(tn.l0[e], u[e], vm);
      vp = fma(tn.l1[e], u[e], vp);
      gm = fma(tn.dl0[e], u[e], gm);
      gp = fma(tn.dl1[e], u[e], gp);
    }
    if (swap) {
      un[1].v.x = vm.v.y;
      gn[1].v.x = gm.v.y;
      un[0].v.y = vp.v.x;
      gn[0].v.y = gp.v.x;
    }
    F2 cv1, cd1, cv0, cd0;
    flux(true, vp, gp, un[1], gn[1], wh[1], ee[1], cv1, cd1);
    flux(false, vm, gm, un[0], gn[0], wh[0], ee[0], cv0, cd0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      F2 acc = fma(tn.l1[i], cv1, r[i]);
      acc = fma(-tn.dl1[i], cd1, acc);
      acc = fma(tn.l0[i], cv0, acc);
      r[i] = fma(-tn.dl0[i], cd0, acc);
    }
  };
  F2 un[2], gn[2], wh[2], ee[2];
  {  // z-lines (a = p, b = q): the first partial sums of q
    face(4, va && cza > 0, vb && czb > 0, ca - sz, cb - sz, un[0], gn[0], wh[0], ee[0]);
    face(5, va && cza < Nc - 1, vb && czb < Nc - 1, ca + sz, cb + sz, un[1], gn[1], wh[1], ee[1]);
    const int base = q * N + p;
    F2 r[N];
#pragma unroll
    for (int e = 0; e < N; ++e) r[e] = F2(0.0f);
    line(base, N2, un, gn, wh, ee, r);
#pragma unroll
    for (int e = 0; e < N; ++e) sr[o + base + e * N2] = r[e];
  }
  __syncthreads();
  {  // y-lines (a = p, e = q)
    face(2, va && cya > 0, vb && cyb > 0, ca - sy, cb - sy, un[0], gn[0], wh[0], ee[0]);
    face(3, va && cya < Nc - 1, vb && cyb < Nc - 1, ca + sy, cb + sy, un[1], gn[1], wh[1], ee[1]);
    const int base = q * N2 + p;
    F2 r[N];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      u[b] = su[o + base + b * N];
      r[b] = sr[o + base + b * N];
    }
    line(base, N, un, gn, wh, ee, r);
#pragma unroll
    for (int b = 0; b < N; ++b) sr[o + base + b * N] = r[b];
  }
  __syncthreads();
  // x-lines (b = p, e = q): finish q, store it and fold <p, q> over the line
  F2 hi = F2(0.0f), lo = F2(0.0f);
  {
    // b's x- and a's x+ neighbour: the pair's other cell when both sit in one
    // x-row; their traces are formed in this thread (line(..., pairrow))
    face(0, va && cxa > 0, vb && cxb > 0, ca - 1, cb - 1, un[0], gn[0], wh[0], ee[0], true,
         !pairrow);
    face(1, va && cxa < Nc - 1, vb && cxb < Nc - 1, ca + 1, cb + 1, un[1], gn[1], wh[1], ee[1],
         !pairrow, true);
    const int base = q * N2 + p * N;
    F2 r[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      u[a] = su[o + base + a];
      r[a] = sr[o + base + a];
    }
    line(base, 1, un, gn, wh, ee, r, pairrow);
#pragma unroll
    for (int a = 0; a < N; ++a) {
      if (va) qg[ca * N3 + base + a] = r[a].v.x;
      if (vb) qg[cb * N3 + base + a] = r[a].v.y;
      const F2 pr = u[a] * r[a];
      const F2 er = fma(u[a], r[a], -pr);  // u r = pr + er exactly
      const F2 s1 = hi + pr;
      const F2 bb = s1 - hi;
      const F2 t1 = (hi - (s1 - bb)) + (pr - bb);
      hi = s1;
      lo = lo + (t1 + er);
    }
  }
  {  // combine the lanes
    float s1, t1;
    two_sum_f(hi.v.x, hi.v.y, s1, t1);
    rh[threadIdx.x] = s1;
    rl[threadIdx.x] = (lo.v.x + lo.v.y) + t1;
  }
  __syncthreads();
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
  __shared__ double rd[NT];
  const double tot = last_block_total<NT>(partials, (int)gridDim.x, rd);
  if (threadIdx.x == 0) {
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
}

template <int N>
struct Mixed32F {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const float* rin, const float* dinv,
                         cudaStream_t s) {
    constexpr int C = Cfg<N>::CPB, N3 = N * N * N;
    // test hook (read when the iteration is captured): the direction kernel
    // skips its first bulk copy and gives up its wait after a few polls
    const char* env = getenv("DG_TEST_BULK_STALL");
    const bool stall_now = env != nullptr && env[0] == '1';
    const long long limit = stall_now ? (1LL << 12) : (1LL << 22);
    const int pc = dinv != nullptr;
    const unsigned gb = (unsigned)m->dir_bulk_grid[pc];
    const unsigned blocks2 = (unsigned)((m->ncells + 2 * C - 1) / (2 * C));
    if (m->nodal_op) {  // the scaled Gauss-point basis (DG_CG_NODAL)
      if (pc)
        k_dir32_bulk<N, true, true><<<gb, Dir32Bulk<N, true>::THREADS, Dir32Bulk<N, true>::SMEM,
                                      s>>>(rin, m->p32, m->TR32, dinv, m->ncells, m->state, limit,
                                           stall_now ? 1 : 0, m->tab32, m->tabN32);
      else
        k_dir32_bulk<N, false, true><<<gb, Dir32Bulk<N, false>::THREADS,
                                       Dir32Bulk<N, false>::SMEM, s>>>(
            rin, m->p32, m->TR32, dinv, m->ncells, m->state, limit, stall_now ? 1 : 0, m->tab32,
            m->tabN32);
      k_cell32x2_nd<N><<<blocks2, Cfg<N>::THREADS, sizeof(F2) * 3 * C * N3, s>>>(
          m->p32, m->TR32, m->hk32, m->gh32, m->q32, m->ncells, m->N, m->partials_cells,
          m->state, m->tabN32);
      return cudaGetLastError();
    }
    if (pc)
      k_dir32_bulk<N, true><<<gb, Dir32Bulk<N, true>::THREADS, Dir32Bulk<N, true>::SMEM, s>>>(
          rin, m->p32, m->TR32, dinv, m->ncells, m->state, limit, stall_now ? 1 : 0,
          m->tab32, m->tabN32);
    else
      k_dir32_bulk<N, false><<<gb, Dir32Bulk<N, false>::THREADS, Dir32Bulk<N, false>::SMEM, s>>>(
          rin, m->p32, m->TR32, dinv, m->ncells, m->state, limit, stall_now ? 1 : 0,
          m->tab32, m->tabN32);
    k_cell32x2<N><<<blocks2, Cfg<N>::THREADS, sizeof(F2) * 4 * C * N3, s>>>(
        m->p32, m->TR32, m->kt32, m->gh32, m->q32, m->ncells, m->N, m->partials_cells,
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
    {
      cudaError_t e = cudaFuncSetAttribute(k_cell32x2<N>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(F2) * 4 * Cfg<N>::CPB * N * N * N));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cell32x2_nd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(F2) * 3 * Cfg<N>::CPB * N * N * N));
      if (e != cudaSuccess) return e;
    }
    for (int pc = 0; pc < 2; ++pc) {
      const void* fn = pc ? (const void*)k_dir32_bulk<N, true> : (const void*)k_dir32_bulk<N, false>;
      const void* fnd = pc ? (const void*)k_dir32_bulk<N, true, true>
                           : (const void*)k_dir32_bulk<N, false, true>;
      const size_t smem = pc ? Dir32Bulk<N, true>::SMEM : Dir32Bulk<N, false>::SMEM;
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fnd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

int dg_launch_mixed32_dir_cell(const dg_mesh* m, const float* rin, const float* dinv,
                               cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<float, dgk::Mixed32F>(m->n, m, rin, dinv, s);
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
