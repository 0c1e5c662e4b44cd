// Conjugate gradients on the device (Section 2.4, the PCG algorithm; M = I, or
// M = diag(A) with DG_CG_PRECOND_JACOBI):
//   q = A p,  alpha = rho / <p, q>,  x += alpha p,  r -= alpha q,  z = M^-1 r,
//   rho' = <z, r> and the convergence norm <r, r> in the same pass (merged
//   into the update as in Section 2.4's merged reduction),  p = z + (rho'/rho) p.
// Scalars live on the device (DGCGState); every kernel checks `done` first, so
// a CUDA graph of a fixed number of iterations can be replayed until the host
// sees convergence without overshooting.  Reductions are deterministic: a fixed
// grid writes per-block partial sums and the last block to finish adds them in
// a fixed order.
//
// Inner products of FP32 vectors are accumulated to FP64 accuracy without the
// FP64 pipe: each product a*b is split exactly into p + e (p = fl(a*b),
// e = fma(a, b, -p)), the pairs are summed in compensated float-float
// arithmetic (Knuth's TwoSum), and only each block's partial sum is converted
// to FP64.
//
// Mixed precision (DG_CG_MIXED_IR): the CG recurrence runs on the FP32 operator
// with FP32 vectors (fused kernels in dg_mixed32.cu); x and the true residual
// are kept in FP64.  When the FP32 residual has dropped below delta (0.2)
// times its value at the last refinement (or below the tolerance), the FP32
// correction d is added to x in FP64, r = b - A x is recomputed with the FP64
// operator, and r replaces the FP32 residual; the search direction p is kept,
// so the Krylov recurrence is not restarted.  When a refinement finds that the
// true residual fell by less than 2x since the last one (the FP32 operator's
// error, about u_32 times the condition number, then pollutes the kept
// directions), the direction is restarted with p = r.  The captured graph
// holds FP32 iterations only: an iteration that requests a refinement sets a
// sticky flag, the remaining iterations of the replayed chunk continue the FP32
// recurrence, and the host runs the FP64 refinement after the replay.
//
// DG_CG_MIXED_IR_RESTART: classical refinement, each correction solved from
// zero by FP32 CG to a fixed residual reduction, then x += ||r|| d in FP64.
#include <chrono>
#include <cmath>

#include "dg_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// s + t = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// Accumulators: FP64 for FP64 data, compensated float-float for FP32 data.
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ double block_total();  // valid in thread 0
};
struct AccF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);  // a*b = p + e exactly
    float s, t;
    two_sum(hi, p, s, t);
    hi = s;
    lo += t + e;
  }
  __device__ double block_total();
};
__device__ __forceinline__ void merge(AccD& a, const AccD& b) { a.s += b.s; }
__device__ __forceinline__ void merge(AccF& a, const AccF& b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  a.hi = s;
  a.lo += b.lo + t;
}

// Visit i = tid, tid + S, ... < n (S = grid size) four strides at a time; f(i, j)
// receives the lane j in 0..3 so that reductions keep four independent
// accumulators (more loads in flight, shorter dependency chains).
template <typename F>
__device__ __forceinline__ void grid_stride4(long long n, F&& f) {
  const long long S = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    f(i, 0);
    f(i + S, 1);
    f(i + 2 * S, 2);
    f(i + 3 * S, 3);
  }
  for (; i < n; i += S) f(i, 0);
}

template <typename A>
__device__ __forceinline__ A merge4(A (&a)[4]) {
  merge(a[0], a[1]);
  merge(a[2], a[3]);
  merge(a[0], a[2]);
  return a[0];
}

template <typename T> struct AccOf;
template <> struct AccOf<double> { using type = AccD; };
template <> struct AccOf<float> { using type = AccF; };

__device__ double AccD::block_total() {
  __shared__ double sw[DG_RED_THREADS / 32];
  double v = warp_sum(s);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sw[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) r = warp_sum((l < DG_RED_THREADS / 32) ? sw[l] : 0.0);
  return r;
}

__device__ double AccF::block_total() {
  __shared__ float sh[DG_RED_THREADS / 32], sl[DG_RED_THREADS / 32];
  float h = hi, lw = lo;
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, off);
    const float ol = __shfl_xor_sync(0xffffffffu, lw, off);
    float s, t;
    two_sum(h, oh, s, t);
    h = s;
    lw = lw + ol + t;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sh[w] = h;
    sl[w] = lw;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    double v = (l < DG_RED_THREADS / 32) ? (double)sh[l] + (double)sl[l] : 0.0;
    r = warp_sum(v);
  }
  return r;
}

// Publish this block's partial sums; returns true in the last block to finish,
// whose thread 0 then holds the totals in tot[0..K-1] (fixed-order sums).
template <int K, typename A>
__device__ bool last_block_sums(A (&part)[K], double* partials, unsigned int* ticket,
                                double (&tot)[K]) {
  static_assert(K <= DG_RED_SUMS, "partials holds DG_RED_SUMS x DG_RED_BLOCKS doubles");
  __shared__ bool is_last;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = part[k].block_total();
    if (threadIdx.x == 0) partials[k * DG_RED_BLOCKS + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    AccD a;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      a.s += ((volatile double*)partials)[k * DG_RED_BLOCKS + b];
    tot[k] = a.block_total();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

#define GRID_STRIDE(i, n)                                                         \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)

// r = b - q, p = z = M^-1 r (PC: M = diag(A), dinv = 1/diag; else M = I);
// rho = <z, r>, rr = <r, r>, bnorm2 = <b, b>; tol2 = rtol^2 bnorm2.
// The preconditioner is a template parameter so that the M = I kernels carry
// no per-element branch (a runtime test kept the compiler from batching the
// loads of the unrolled grid-stride loop and cost ~40 % of the bandwidth).
template <typename T, bool PC>
__global__ void __launch_bounds__(DG_RED_THREADS)
k_init(const T* __restrict__ b, const T* __restrict__ q, T* __restrict__ r, T* __restrict__ p,
       const T* __restrict__ dinv, long long n, double rtol, double* partials, DGCGState* st) {
  using A = typename AccOf<T>::type;
  A ar[4], ab[4], az[4];
  grid_stride4(n, [&](long long i, int j) {
    const T ri = b[i] - q[i];
    r[i] = ri;
    T zi = ri;
    if constexpr (PC) zi = dinv[i] * ri;
    p[i] = zi;
    ar[j].add_prod(ri, ri);
    ab[j].add_prod(b[i], b[i]);
    az[j].add_prod(zi, ri);
  });
  A acc[3] = {merge4(ar), merge4(ab), merge4(az)};
  double tot[3];
  if (last_block_sums<3>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->rho = tot[2];
    st->bnorm2 = tot[1];
    st->tol2 = rtol * rtol * tot[1];
    st->breakdown = !(finite(tot[0]) && finite(tot[1]) && finite(tot[2]));
    st->done = st->breakdown || tot[0] <= st->tol2 || st->iters >= st->maxit;
    st->ru_skip = 1;
  }
}

// 16-byte vectors for the vector kernels below (all operands 16-byte aligned).
template <typename T> struct V16;
template <> struct V16<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static void split(const float4& v, float (&a)[4]) {
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
  }
  __device__ static float4 join(const float (&a)[4]) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <> struct V16<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static void split(const double2& v, double (&a)[2]) { a[0] = v.x; a[1] = v.y; }
  __device__ static double2 join(const double (&a)[2]) { return make_double2(a[0], a[1]); }
};

// pq = <p, q>, alpha = rho / pq.
template <typename T, bool VEC>
__global__ void __launch_bounds__(DG_RED_THREADS)
k_dot_pq(const T* __restrict__ p, const T* __restrict__ q, long long n, double* partials,
         DGCGState* st) {
  if (st->done) return;
  using A = typename AccOf<T>::type;
  A a4[4];
  const long long S = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tail = 0;
  if constexpr (VEC) {
    using VT = V16<T>;
    using V = typename VT::type;
    constexpr int W = VT::W;
    const long long nv = n / W;
    const V* pv = reinterpret_cast<const V*>(p);
    const V* qv = reinterpret_cast<const V*>(q);
    for (long long iv = tid; iv < nv; iv += 2 * S) {
      const bool two = iv + S < nv;
      T ps[2][W], qs[2][W];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && !two) break;
        VT::split(pv[iv + u * S], ps[u]);
        VT::split(qv[iv + u * S], qs[u]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && !two) break;
#pragma unroll
        for (int c = 0; c < W; ++c) a4[(u * W + c) & 3].add_prod(ps[u][c], qs[u][c]);
      }
    }
    tail = nv * W;
  }
  for (long long i = tail + tid; i < n; i += S) a4[0].add_prod(p[i], q[i]);
  A acc[1] = {merge4(a4)};
  double tot[1];
  if (last_block_sums<1>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
    st->pq = tot[0];
    if (!(tot[0] > 0.0) || !finite(tot[0])) {
      st->breakdown = 1;
      st->done = 1;
      st->ru_skip = 1;
    } else {
      st->alpha = st->rho / tot[0];
    }
  }
}

// x += alpha p, r -= alpha q; rr' = <r, r> (convergence norm), rho' = <z, r>
// with z = M^-1 r (= rr' without M).
// MIXED = false: convergence test on rr', beta = rho'/rho, rho = rho'.
// MIXED = true: rho' goes to rho_new and beta is formed for the direction
// update; an FP64 refinement is requested (ru_skip = 0, until it runs) when
// rr' has dropped below delta2 * rmax2 or below tol2, or at the iteration
// cap; the FP32 iteration kernels then skip until the refinement has run.
// BLK = true (cell blocks, Kronecker blocks): only x, r, <r, r> and the
// convergence test (MIXED: the refinement request); rho and beta (MIXED:
// rho_new and beta) are formed from z = M^-1 r by the kernel that follows.
template <typename T, bool MIXED, bool PC, bool VEC, bool BLK = false>
__global__ void __launch_bounds__(DG_RED_THREADS)
k_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
            const T* __restrict__ q, const T* __restrict__ dinv, long long n, double* partials,
            DGCGState* st) {
  // MIXED: the FP32 iterations stop once an FP64 refinement is pending
  // (ru_skip = 0) until it has run: iterating on in FP32 after the FP32
  // residual has converged corrupts the search direction that the refinement
  // keeps (seen on systems of 64 DOFs, which converge within one graph chunk)
  if (st->done || (MIXED && (st->iters >= st->maxit || st->ru_skip == 0))) return;
  const T a = (T)st->alpha;
  using A = typename AccOf<T>::type;
  A a4[4], z4[4];
  const long long S = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tail = 0;  // first element left to the scalar loop
  if constexpr (VEC) {
    // U 16-byte vectors of every operand per step, all loaded before any
    // store (U = 2 without M; 1 with M, which has five operands and two
    // compensated sums and would otherwise need over 100 registers).
    using VT = V16<T>;
    using V = typename VT::type;
    constexpr int W = VT::W, U = PC ? 1 : 2;
    const long long nv = n / W;
    V* xv = reinterpret_cast<V*>(x);
    V* rv = reinterpret_cast<V*>(r);
    const V* pv = reinterpret_cast<const V*>(p);
    const V* qv = reinterpret_cast<const V*>(q);
    const V* dv = reinterpret_cast<const V*>(dinv);
    for (long long iv = tid; iv < nv; iv += U * S) {
      const bool two = iv + S < nv;
      T xs[U][W], rs[U][W], ps[U][W], qs[U][W], ds[U][W];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u == 1 && !two) break;
        const long long k = iv + u * S;
        VT::split(xv[k], xs[u]);
        VT::split(rv[k], rs[u]);
        VT::split(pv[k], ps[u]);
        VT::split(qv[k], qs[u]);
        if constexpr (PC) VT::split(dv[k], ds[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u == 1 && !two) break;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const int j = (u * W + c) & 3;
          xs[u][c] = fma(a, ps[u][c], xs[u][c]);
          rs[u][c] = fma(-a, qs[u][c], rs[u][c]);
          a4[j].add_prod(rs[u][c], rs[u][c]);
          if constexpr (PC) z4[j].add_prod(ds[u][c] * rs[u][c], rs[u][c]);
        }
        xv[iv + u * S] = VT::join(xs[u]);
        rv[iv + u * S] = VT::join(rs[u]);
      }
    }
    tail = nv * W;
  }
  for (long long i = tail + tid; i < n; i += S) {
    x[i] = fma(a, p[i], x[i]);
    const T ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    a4[0].add_prod(ri, ri);
    if constexpr (PC) z4[0].add_prod(dinv[i] * ri, ri);
  }
  constexpr int K = PC ? 2 : 1;
  A acc[K];
  acc[0] = merge4(a4);
  if constexpr (PC) acc[K - 1] = merge4(z4);
  double tot[K];
  if (last_block_sums<K>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    const double zr = tot[K - 1];  // = rr without M
    st->iters += 1;
    if (!finite(rr) || !finite(zr)) {
      st->breakdown = 1;
      st->done = 1;
      st->ru_skip = 1;
    } else if (BLK && !MIXED) {
      st->rr = rr;
      if (rr <= st->tol2 || st->iters >= st->maxit) st->done = 1;
    } else if (!MIXED) {
      st->beta = zr / st->rho;
      st->rho = zr;
      st->rr = rr;
      if (rr <= st->tol2 || st->iters >= st->maxit) st->done = 1;
    } else {
      st->rr = rr;
      if (!BLK) {
        st->rho_new = zr;
        st->beta = zr / st->rho;  // next direction update (k_dir32_bulk)
      }
      if (rr <= st->delta2 * st->rmax2 || rr <= st->tol2 || st->iters >= st->maxit)
        st->ru_skip = 0;
    }
  }
}

// p = z + beta p, z = M^-1 r
template <typename T, bool PC, bool VEC>
__global__ void __launch_bounds__(DG_RED_THREADS)
k_update_p(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ dinv, long long n,
           const DGCGState* st) {
  if (st->done) return;
  const T be = (T)st->beta;
  const long long S = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tail = 0;
  if constexpr (VEC) {
    using VT = V16<T>;
    using V = typename VT::type;
    constexpr int W = VT::W;
    const long long nv = n / W;
    V* pv = reinterpret_cast<V*>(p);
    const V* rv = reinterpret_cast<const V*>(r);
    const V* dv = reinterpret_cast<const V*>(dinv);
    for (long long iv = tid; iv < nv; iv += 2 * S) {
      const bool two = iv + S < nv;
      T ps[2][W], rs[2][W], ds[2][W];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && !two) break;
        VT::split(pv[iv + u * S], ps[u]);
        VT::split(rv[iv + u * S], rs[u]);
        if constexpr (PC) VT::split(dv[iv + u * S], ds[u]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && !two) break;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          T z = rs[u][c];
          if constexpr (PC) z = ds[u][c] * z;
          ps[u][c] = fma(be, ps[u][c], z);
        }
        pv[iv + u * S] = VT::join(ps[u]);
      }
    }
    tail = nv * W;
  }
  for (long long i = tail + tid; i < n; i += S) {
    T zi = r[i];
    if constexpr (PC) zi = dinv[i] * zi;
    p[i] = fma(be, p[i], zi);
  }
}

// refinement step 1 (mixed): x64 += d32, d32 = 0.
__global__ void __launch_bounds__(DG_RED_THREADS)
k_refine_x(double* __restrict__ x, float* __restrict__ d, long long n, const DGCGState* st) {
  if (st->ru_skip) return;
  GRID_STRIDE(i, n) {
    x[i] += (double)d[i];
    d[i] = 0.0f;
  }
}

// The FP32 operator's error bounds the accuracy the mixed solver can reach
// (about u_32 times the condition number, relative).  After this many
// consecutive refinements without a 2x residual reduction it gives up.
constexpr int kMaxStall = 30;

// refinement step 2 (mixed), after q = A64 x: r64 = b - q, r32 = (float) r64,
// rho_new = rmax2 = ||r64||^2; converged when <= tol2; cap on iterations and
// on stagnating refinements.
template <bool PC>
__global__ void __launch_bounds__(DG_RED_THREADS)
k_refine_r(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
           float* __restrict__ r32, const double* __restrict__ dinv, long long n,
           double* partials, DGCGState* st) {
  if (st->ru_skip) return;
  AccD a4[4], z4[4];
  grid_stride4(n, [&](long long i, int j) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    r32[i] = (float)ri;
    a4[j].add_prod(ri, ri);
    if constexpr (PC) z4[j].add_prod(dinv[i] * ri, ri);
  });
  constexpr int K = PC ? 2 : 1;
  AccD acc[K];
  acc[0] = merge4(a4);
  if constexpr (PC) acc[K - 1] = merge4(z4);
  double tot[K];
  if (last_block_sums<K>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    const double zr = tot[K - 1];  // = rr without M
    st->n_refine += 1;
    st->restart = rr > 0.25 * st->rmax2;  // true residual fell by less than 2x
    st->stall = st->restart ? st->stall + 1 : 0;
    st->rho_new = zr;
    st->rr = rr;
    st->beta = st->restart ? 0.0 : zr / st->rho;  // direction update after replacement
    st->rmax2 = rr;
    st->ru_skip = 1;
    if (!finite(rr) || !finite(zr)) {
      st->breakdown = 1;
      st->done = 1;
    } else if (rr <= st->tol2 || st->iters >= st->maxit || st->stall >= kMaxStall) {
      st->done = 1;
    }
  }
}

// r = b - q; res2 = <r, r>, b2 = <b, b> (no other state change).
__global__ void __launch_bounds__(DG_RED_THREADS)
k_residual(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
           long long n, double* partials, DGCGState* st) {
  AccD ar[4], ab[4];
  grid_stride4(n, [&](long long i, int j) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    ar[j].add_prod(ri, ri);
    ab[j].add_prod(b[i], b[i]);
  });
  AccD acc[2] = {merge4(ar), merge4(ab)};
  double tot[2];
  if (last_block_sums<2>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
    st->res2 = tot[0];
    st->b2 = tot[1];
  }
}

// r32 = (float)(r64 * inv), d32 = 0
__global__ void k_scale_to_f32(const double* __restrict__ r, float* __restrict__ r32,
                               float* __restrict__ d32, long long n, double inv) {
  GRID_STRIDE(i, n) {
    r32[i] = (float)(r[i] * inv);
    d32[i] = 0.0f;
  }
}

// x += scale * d32  (FP64 update)
__global__ void k_axpy_f32_into_f64(double* __restrict__ x, const float* __restrict__ d,
                                    long long n, double scale) {
  GRID_STRIDE(i, n) x[i] = fma(scale, (double)d[i], x[i]);
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

#define RED_LAUNCH DG_RED_BLOCKS, DG_RED_THREADS, 0, s

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// One iteration of plain CG on FP64 or FP32 vectors.  With f0 <= f1 the
// operator is restricted to the DOFs [f0, f1): q = A p is set to zero outside
// them (p, r and x then stay zero there too).
template <typename T>
int launch_iteration(dg_mesh* m, T* x, T* r, T* p, T* q, const T* dinv, cudaStream_t s,
                     long long f0 = -1, long long f1 = -1) {
  int rc = (sizeof(T) == 8)
               ? dg_launch_apply_f64(m, (const double*)p, (double*)q, &m->state->done, s)
               : dg_launch_apply_f32(m, (const float*)p, (float*)q, &m->state->done, s);
  if (rc) return rc;
  const long long n = m->ndofs;
  if (f0 > 0) DG_CUDA(cudaMemsetAsync(q, 0, sizeof(T) * (size_t)f0, s));
  if (f0 >= 0 && f1 < n) DG_CUDA(cudaMemsetAsync(q + f1, 0, sizeof(T) * (size_t)(n - f1), s));
  // 16-byte vector kernels when every operand allows it (x is the caller's)
  const bool vec = aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q) &&
                   aligned16(dinv);
  if (vec)
    k_dot_pq<T, true><<<RED_LAUNCH>>>(p, q, n, m->partials, m->state);
  else
    k_dot_pq<T, false><<<RED_LAUNCH>>>(p, q, n, m->partials, m->state);
  if (dinv && vec) {
    k_update_xr<T, false, true, true><<<RED_LAUNCH>>>(x, r, p, q, dinv, n, m->partials,
                                                      m->state);
    k_update_p<T, true, true><<<RED_LAUNCH>>>(p, r, dinv, n, m->state);
  } else if (dinv) {
    k_update_xr<T, false, true, false><<<RED_LAUNCH>>>(x, r, p, q, dinv, n, m->partials,
                                                       m->state);
    k_update_p<T, true, false><<<RED_LAUNCH>>>(p, r, dinv, n, m->state);
  } else if (vec) {
    k_update_xr<T, false, false, true><<<RED_LAUNCH>>>(x, r, p, q, dinv, n, m->partials,
                                                       m->state);
    k_update_p<T, false, true><<<RED_LAUNCH>>>(p, r, dinv, n, m->state);
  } else {
    k_update_xr<T, false, false, false><<<RED_LAUNCH>>>(x, r, p, q, dinv, n, m->partials,
                                                        m->state);
    k_update_p<T, false, false><<<RED_LAUNCH>>>(p, r, dinv, n, m->state);
  }
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// One iteration of FP64 PCG with the cell-block Jacobi preconditioner:
// q = A p, alpha, x and r updates with <r, r>, z = M^-1 r with <z, r> (rho,
// beta), p = z + beta p.
int launch_iteration_block(dg_mesh* m, double* x, cudaStream_t s) {
  int rc = dg_launch_apply_f64(m, m->p64, m->q64, &m->state->done, s);
  if (rc) return rc;
  const long long n = m->ndofs;
  const bool vec = aligned16(x);
  if (vec) {
    k_dot_pq<double, true><<<RED_LAUNCH>>>(m->p64, m->q64, n, m->partials, m->state);
    k_update_xr<double, false, false, true, true><<<RED_LAUNCH>>>(x, m->r64, m->p64, m->q64,
                                                                  nullptr, n, m->partials,
                                                                  m->state);
  } else {
    k_dot_pq<double, false><<<RED_LAUNCH>>>(m->p64, m->q64, n, m->partials, m->state);
    k_update_xr<double, false, false, false, true><<<RED_LAUNCH>>>(x, m->r64, m->p64, m->q64,
                                                                   nullptr, n, m->partials,
                                                                   m->state);
  }
  DG_CUDA(cudaGetLastError());
  rc = dg_launch_block_apply(m, m->r64, m->t64, nullptr, false, s);
  if (rc) return rc;
  k_update_p<double, false, true><<<RED_LAUNCH>>>(m->p64, m->t64, nullptr, n, m->state);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// One FP32 iteration of the mixed CG: direction update, operator and <p, q>
// (fused kernels of dg_mixed32.cu), then d += alpha p, r -= alpha q.  The FP64
// refinement is not in the captured iteration: it runs between graph replays
// when an iteration has requested it (refine_mixed).
int launch_iteration_mixed(dg_mesh* m, const float* dinv, cudaStream_t s, bool kron = false) {
  const long long n = m->ndofs;
  // with Kronecker blocks the direction update reads z = M^-1 r from q32
  // (formed after the previous update; q32 is free until the cell kernel)
  int rc = dg_launch_mixed32_dir_cell(m, kron ? m->q32 : m->r32, dinv, s);
  if (rc) return rc;
  if (kron) {
    k_update_xr<float, true, false, true, true><<<RED_LAUNCH>>>(m->d32, m->r32, m->p32, m->q32,
                                                                nullptr, n, m->partials,
                                                                m->state);
    DG_CUDA(cudaGetLastError());
    return dg_launch_kron_apply(m, m->r32, m->q32, nullptr, DG_KRON_FP32, s);
  }
  // all operands are the mesh's own allocations (256-byte aligned)
  if (dinv)
    k_update_xr<float, true, true, true><<<RED_LAUNCH>>>(m->d32, m->r32, m->p32, m->q32, dinv,
                                                         n, m->partials, m->state);
  else
    k_update_xr<float, true, false, true><<<RED_LAUNCH>>>(m->d32, m->r32, m->p32, m->q32, dinv,
                                                          n, m->partials, m->state);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// One FP64 PCG iteration with the Kronecker cell blocks: q = A p, alpha, x and
// r updates with <r, r>, z = M^-1 r with <z, r> (rho, beta), p = z + beta p.
int launch_iteration_kron(dg_mesh* m, double* x, cudaStream_t s) {
  int rc = dg_launch_apply_f64(m, m->p64, m->q64, &m->state->done, s);
  if (rc) return rc;
  const long long n = m->ndofs;
  if (aligned16(x)) {
    k_dot_pq<double, true><<<RED_LAUNCH>>>(m->p64, m->q64, n, m->partials, m->state);
    k_update_xr<double, false, false, true, true><<<RED_LAUNCH>>>(x, m->r64, m->p64, m->q64,
                                                                  nullptr, n, m->partials,
                                                                  m->state);
  } else {
    k_dot_pq<double, false><<<RED_LAUNCH>>>(m->p64, m->q64, n, m->partials, m->state);
    k_update_xr<double, false, false, false, true><<<RED_LAUNCH>>>(x, m->r64, m->p64, m->q64,
                                                                   nullptr, n, m->partials,
                                                                   m->state);
  }
  DG_CUDA(cudaGetLastError());
  rc = dg_launch_kron_apply(m, m->r64, m->t64, nullptr, DG_KRON_FP64, s);
  if (rc) return rc;
  k_update_p<double, false, true><<<RED_LAUNCH>>>(m->p64, m->t64, nullptr, n, m->state);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// FP64 refinement: x += d, r = b - A x (FP64), r32 = (float) r.
int refine_mixed(dg_mesh* m, const double* b, double* x, const double* dinv, cudaStream_t s,
                 bool kron = false) {
  const long long n = m->ndofs;
  k_refine_x<<<RED_LAUNCH>>>(x, m->d32, n, m->state);
  int rc = dg_launch_apply_f64(m, x, m->q64, nullptr, s);
  if (rc) return rc;
  if (dinv)
    k_refine_r<true><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->r32, dinv, n, m->partials, m->state);
  else
    k_refine_r<false><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->r32, dinv, n, m->partials, m->state);
  DG_CUDA(cudaGetLastError());
  if (kron) return dg_launch_kron_apply(m, m->r32, m->q32, nullptr, DG_KRON_FP32, s);
  return DG_OK;
}

// Capture `chunk` iterations into a graph and replay it until `done`.
template <typename F>
int run_graph(dg_mesh* m, cudaStream_t s, int chunk, F&& one_iteration) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = DG_OK;
  for (int i = 0; i < chunk && rc == DG_OK; ++i) rc = one_iteration();
  cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  DG_CUDA(ec);
  ec = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  DG_CUDA(ec);
  for (;;) {
    ec = cudaGraphLaunch(exec, s);
    if (ec == cudaSuccess)
      ec = cudaMemcpyAsync(m->state_host, m->state, sizeof(DGCGState), cudaMemcpyDeviceToHost, s);
    if (ec == cudaSuccess) ec = cudaStreamSynchronize(s);
    if (ec != cudaSuccess) {
      cudaGraphExecDestroy(exec);
      return dg_cuda_fail(ec, "CG iteration graph");
    }
    if (m->state_host->done) break;
  }
  cudaGraphExecDestroy(exec);
  return DG_OK;
}

int set_state(dg_mesh* m, int maxit, int iters, cudaStream_t s) {
  DGCGState h = {};
  h.maxit = maxit;
  h.iters = iters;
  h.ru_skip = 1;
  *m->state_host = h;
  DG_CUDA(cudaMemcpyAsync(m->state, m->state_host, sizeof(DGCGState), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

// ||b - A x||^2 and ||b||^2 in FP64 (r64 gets the residual).
int true_residual(dg_mesh* m, const double* b, const double* x, cudaStream_t s, double* res2,
                  double* b2) {
  int rc = dg_launch_apply_f64(m, x, m->q64, nullptr, s);
  if (rc) return rc;
  k_residual<<<RED_LAUNCH>>>(b, m->q64, m->r64, m->ndofs, m->partials, m->state);
  DG_CUDA(cudaGetLastError());
  DG_CUDA(cudaMemcpyAsync(m->state_host, m->state, sizeof(DGCGState), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  *res2 = m->state_host->res2;
  *b2 = m->state_host->b2;
  return DG_OK;
}

int chunk_for(const dg_mesh* m) { return m->ndofs < (1LL << 22) ? 32 : 8; }

int zero_solution(dg_mesh* m, double* x, dg_cg_stats* st, cudaStream_t s) {
  DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)m->ndofs, s));
  if (st) st->rel_residual = st->rel_residual_rec = 0.0;
  return DG_OK;
}

int cg_fp64(dg_mesh* m, const double* b, double* x, double rtol, int maxit, dg_cg_stats* st,
            bool jacobi, cudaStream_t s, bool block = false, bool kron = false) {
  const double* dinv = jacobi ? (m->nodal_op ? m->dinvN64 : m->dinv64) : nullptr;
  const int max_restarts = 5;
  int iters = 0, restarts = 0;
  double res2 = 0, b2 = 0;
  int rc = true_residual(m, b, x, s, &res2, &b2);
  if (rc) return rc;
  if (b2 == 0.0) return zero_solution(m, x, st, s);  // A x = 0 has the solution x = 0
  for (;;) {
    rc = set_state(m, maxit, iters, s);
    if (rc) return rc;
    rc = dg_launch_apply_f64(m, x, m->q64, nullptr, s);
    if (rc) return rc;
    if (dinv)
      k_init<double, true><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->p64, dinv, m->ndofs, rtol,
                                           m->partials, m->state);
    else
      k_init<double, false><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->p64, dinv, m->ndofs, rtol,
                                            m->partials, m->state);
    DG_CUDA(cudaGetLastError());
    if (block) {  // z = M^-1 r, p = z, rho = <z, r>
      rc = dg_launch_block_apply(m, m->r64, m->t64, m->p64, true, s);
      if (rc) return rc;
    }
    if (kron) {
      rc = dg_launch_kron_apply(m, m->r64, m->t64, m->p64, DG_KRON_FP64_INIT, s);
      if (rc) return rc;
    }
    rc = run_graph(m, s, chunk_for(m), [&] {
      return block ? launch_iteration_block(m, x, s)
             : kron ? launch_iteration_kron(m, x, s)
                    : launch_iteration<double>(m, x, m->r64, m->p64, m->q64, dinv, s);
    });
    if (rc) return rc;
    const DGCGState hs = *m->state_host;
    iters = hs.iters;
    if (st) st->rel_residual_rec = hs.bnorm2 > 0 ? std::sqrt(hs.rr / hs.bnorm2) : 0.0;
    rc = true_residual(m, b, x, s, &res2, &b2);
    if (rc) return rc;
    const double rel = std::sqrt(res2 / b2);
    if (st) {
      st->iterations = iters;
      st->outer_iterations = restarts;
      st->rel_residual = rel;
    }
    if (hs.breakdown)
      return dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve: breakdown (<p,Ap> <= 0 or non-finite) at "
                                       "iteration %d", iters);
    if (rel <= rtol) return DG_OK;
    if (iters >= maxit || restarts >= max_restarts)
      return dg_fail(DG_ERR_NOT_CONVERGED,
                     "dg_cg_solve: relative residual %.3e > rtol %.3e after %d iterations", rel,
                     rtol, iters);
    ++restarts;  // recursive residual drifted from the true one: restart from x
  }
}

// FP32 CG recurrence with FP64 residual refinement (search direction kept).
int cg_mixed(dg_mesh* m, const double* b, double* x, double rtol, int maxit, dg_cg_stats* st,
             bool jacobi, cudaStream_t s, bool kron = false) {
  const double* dinv = jacobi ? (m->nodal_op ? m->dinvN64 : m->dinv64) : nullptr;
  const float* dinv32 = jacobi ? (m->nodal_op ? m->dinvN32 : m->dinv32) : nullptr;
  // refine when the FP32 residual has dropped 5x: measured at 48^3 Q4 to 1e-10,
  // delta 0.2 needs 34,400 iterations (0.1: 41,320; 0.3: 34,664); 0.01 drifts
  // and stagnates
  const double delta = 0.2;
  const long long n = m->ndofs;
  double res2 = 0, b2 = 0;
  int rc = true_residual(m, b, x, s, &res2, &b2);
  if (rc) return rc;
  if (b2 == 0.0) return zero_solution(m, x, st, s);
  rc = set_state(m, maxit, 0, s);
  if (rc) return rc;
  // q32 = (float) r64 is the right-hand side of k_init and d32 = 0 the initial
  // correction, so r32 = p32 = (float) r64.
  const unsigned vblocks = (unsigned)(m->sm_count * 8);
  k_scale_to_f32<<<vblocks, 256, 0, s>>>(m->r64, m->q32, m->d32, n, 1.0);
  if (dinv32)
    k_init<float, true><<<RED_LAUNCH>>>(m->q32, m->d32, m->r32, m->p32, dinv32, n, rtol,
                                        m->partials, m->state);
  else
    k_init<float, false><<<RED_LAUNCH>>>(m->q32, m->d32, m->r32, m->p32, dinv32, n, rtol,
                                         m->partials, m->state);
  DG_CUDA(cudaGetLastError());
  // FP64 tolerance and reference norm from the FP64 residual
  DG_CUDA(cudaMemcpyAsync(m->state_host, m->state, sizeof(DGCGState), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  {
    DGCGState h = *m->state_host;
    h.bnorm2 = b2;
    h.tol2 = rtol * rtol * b2;
    h.rmax2 = res2;
    h.delta2 = delta * delta;
    h.done = h.breakdown || res2 <= h.tol2;
    h.ru_skip = 1;
    h.rho_new = h.rho;  // first direction update: p = r (restart)
    h.restart = 1;
    h.beta = 0.0;
    *m->state_host = h;
    DG_CUDA(cudaMemcpyAsync(m->state, m->state_host, sizeof(DGCGState), cudaMemcpyHostToDevice,
                            s));
  }
  if (kron) {  // z = M^-1 r into q32, rho_new = <z, r>, beta = 0 (restart)
    rc = dg_launch_kron_apply(m, m->r32, m->q32, nullptr, DG_KRON_FP32, s);
    if (rc) return rc;
  }
  // replay a graph of FP32 iterations; refine in FP64 whenever one asked for it
  {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk_for(m) && rc == DG_OK; ++i)
      rc = launch_iteration_mixed(m, dinv32, s, kron);
    cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    DG_CUDA(ec);
    ec = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    DG_CUDA(ec);
    for (;;) {
      ec = cudaMemcpyAsync(m->state_host, m->state, sizeof(DGCGState), cudaMemcpyDeviceToHost, s);
      if (ec == cudaSuccess) ec = cudaStreamSynchronize(s);
      if (ec != cudaSuccess) break;
      if (m->state_host->done) break;
      if (m->state_host->ru_skip == 0) {
        rc = refine_mixed(m, b, x, dinv, s, kron);
        if (rc) break;
        continue;
      }
      ec = cudaGraphLaunch(exec, s);
      if (ec != cudaSuccess) break;
    }
    cudaGraphExecDestroy(exec);
    if (rc) return rc;
    DG_CUDA(ec);
  }
  const DGCGState hs = *m->state_host;
  if (hs.timeout)
    return dg_fail(DG_ERR_TIMEOUT,
                   "dg_cg_solve(mixed): a bounded wait for a bulk copy in the FP32 direction "
                   "kernel ran out at iteration %d", hs.iters);
  rc = true_residual(m, b, x, s, &res2, &b2);
  if (rc) return rc;
  const double rel = std::sqrt(res2 / b2);
  if (st) {
    st->iterations = hs.iters;
    st->outer_iterations = hs.n_refine;
    st->rel_residual = rel;
    st->rel_residual_rec = std::sqrt(hs.rr / b2);
  }
  if (hs.breakdown)
    return dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve(mixed): breakdown at iteration %d", hs.iters);
  if (rel <= rtol) return DG_OK;
  return dg_fail(DG_ERR_NOT_CONVERGED,
                 "dg_cg_solve(mixed): relative residual %.3e > rtol %.3e after %d iterations "
                 "(%d refinements%s)", rel, rtol, hs.iters, hs.n_refine,
                 hs.stall >= kMaxStall ? "; stagnated: the FP32 operator limits the accuracy, "
                                         "use DG_CG_FP64 for this tolerance" : "");
}

// Classical refinement: restart an FP32 CG from zero for every correction.
int cg_mixed_restart(dg_mesh* m, const double* b, double* x, double rtol, int maxit,
                     dg_cg_stats* st, bool jacobi, cudaStream_t s) {
  const float* dinv32 = jacobi ? m->dinv32 : nullptr;
  const int max_outer = 60;
  const double inner_tol = 0.1;  // relative reduction per refinement step
  const long long n = m->ndofs;
  const unsigned vblocks = (unsigned)(m->sm_count * 8);
  int inner_total = 0;
  double res2 = 0, b2 = 0;
  for (int outer = 0;; ++outer) {
    int rc = true_residual(m, b, x, s, &res2, &b2);
    if (rc) return rc;
    if (b2 == 0.0) return zero_solution(m, x, st, s);
    const double rn = std::sqrt(res2);
    const double rel = rn / std::sqrt(b2);
    if (st) {
      st->iterations = inner_total;
      st->outer_iterations = outer;
      st->rel_residual = rel;
      st->rel_residual_rec = rel;
    }
    if (!std::isfinite(rel))
      return dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve(mixed restart): non-finite residual");
    if (rel <= rtol) return DG_OK;
    if (outer >= max_outer || inner_total >= maxit)
      return dg_fail(DG_ERR_NOT_CONVERGED,
                     "dg_cg_solve(mixed restart): relative residual %.3e > rtol %.3e after %d "
                     "outer / %d inner iterations", rel, rtol, outer, inner_total);
    k_scale_to_f32<<<vblocks, 256, 0, s>>>(m->r64, m->q32, m->d32, n, 1.0 / rn);
    DG_CUDA(cudaGetLastError());
    rc = set_state(m, maxit - inner_total, 0, s);
    if (rc) return rc;
    if (dinv32)
      k_init<float, true><<<RED_LAUNCH>>>(m->q32, m->d32, m->r32, m->p32, dinv32, n, inner_tol,
                                          m->partials, m->state);
    else
      k_init<float, false><<<RED_LAUNCH>>>(m->q32, m->d32, m->r32, m->p32, dinv32, n,
                                           inner_tol, m->partials, m->state);
    DG_CUDA(cudaGetLastError());
    rc = run_graph(m, s, chunk_for(m), [&] {
      return launch_iteration<float>(m, m->d32, m->r32, m->p32, m->q32, dinv32, s);
    });
    if (rc) return rc;
    const DGCGState hs = *m->state_host;
    inner_total += hs.iters;
    if (hs.breakdown && hs.iters == 0)
      return dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve(mixed restart): inner CG breakdown");
    k_axpy_f32_into_f64<<<vblocks, 256, 0, s>>>(x, m->d32, n, rn);
    DG_CUDA(cudaGetLastError());
  }
}

// ---------------------------------------------------------------------------
// Resilient FP64 CG: the in-memory backup and recovery of Section 2.3 on one
// GPU.  Every `backup_interval` iterations the solver copies a backup into
// pinned host memory (the stand-in for the remote rank's memory): the full
// state (x, r, p and the CG scalars: lossless), x in FP64, or x rounded to
// FP32 (a lossy compression to half the bytes).  A data loss is injected on
// the host (x, r and p of a range of cells set to zero, as if the rank that
// held them had failed) at the first check at or after `fault_iteration`.
// Recovery: global rollback (every DOF back to the backup: with the full state
// the iteration resumes exactly and the result is bit-identical to the
// fault-free solve; with an x backup CG restarts from it), or local recovery
// (only the lost cells take the backup's x, or zero without a backup, and CG
// restarts), optionally followed by the local auxiliary problem on the lost
// cells (aux_solve).  FP64 operator, M = I or M = diag(A).
// ---------------------------------------------------------------------------

__global__ void k_zero_range(double* __restrict__ a, double* __restrict__ b,
                             double* __restrict__ c, long long i0, long long i1) {
  for (long long i = i0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < i1;
       i += (long long)gridDim.x * blockDim.x) {
    a[i] = 0.0;
    b[i] = 0.0;
    c[i] = 0.0;
  }
}

// x[i] = src[i] (FP32 -> FP64) for i in [i0, i1)
__global__ void k_restore_x32(double* __restrict__ x, const float* __restrict__ src, long long i0,
                              long long i1) {
  for (long long i = i0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < i1;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (double)src[i];
}

__global__ void k_round_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  GRID_STRIDE(i, n) y[i] = (float)x[i];
}

__global__ void k_add_range(double* __restrict__ x, const double* __restrict__ e, long long i0,
                            long long i1) {
  for (long long i = i0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < i1;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += e[i];
}

// The local auxiliary problem of the third recovery method: with F the DOFs
// [i0, i1) of the lost cells and every other DOF held at its current value
// (the Dirichlet layer), solve A(F,F) e = (b - A x)(F) by (P)CG to aux_rtol
// relative to the initial local residual, then x(F) += e.  The backup (or
// zero) already in x(F) is the initial guess.  Vectors: s64 the local
// right-hand side, t64 the correction e.
int aux_solve(dg_mesh* m, const double* b, double* x, const double* dinv, long long i0,
              long long i1, double aux_rtol, int aux_maxit, int* its, cudaStream_t s) {
  const long long n = m->ndofs;
  *its = 0;
  if (i1 <= i0) return DG_OK;
  double res2 = 0, b2 = 0;
  int rc = true_residual(m, b, x, s, &res2, &b2);  // r64 = b - A x
  if (rc) return rc;
  DG_CUDA(cudaMemsetAsync(m->s64, 0, sizeof(double) * (size_t)n, s));
  DG_CUDA(cudaMemcpyAsync(m->s64 + i0, m->r64 + i0, sizeof(double) * (size_t)(i1 - i0),
                          cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaMemsetAsync(m->t64, 0, sizeof(double) * (size_t)n, s));
  DG_CUDA(cudaMemsetAsync(m->q64, 0, sizeof(double) * (size_t)n, s));
  rc = set_state(m, aux_maxit, 0, s);
  if (rc) return rc;
  if (dinv)
    k_init<double, true><<<RED_LAUNCH>>>(m->s64, m->q64, m->r64, m->p64, dinv, n, aux_rtol,
                                         m->partials, m->state);
  else
    k_init<double, false><<<RED_LAUNCH>>>(m->s64, m->q64, m->r64, m->p64, dinv, n, aux_rtol,
                                          m->partials, m->state);
  DG_CUDA(cudaGetLastError());
  rc = run_graph(m, s, chunk_for(m), [&] {
    return launch_iteration<double>(m, m->t64, m->r64, m->p64, m->q64, dinv, s, i0, i1);
  });
  if (rc) return rc;
  const DGCGState hs = *m->state_host;
  *its = hs.iters;
  if (hs.breakdown)
    return dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve_resilient: auxiliary problem broke down");
  k_add_range<<<(unsigned)(m->sm_count * 8), 256, 0, s>>>(x, m->t64, i0, i1);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

int cg_fp64_resilient(dg_mesh* m, const double* b, double* x, double rtol, int maxit,
                      bool jacobi, dg_resilience* o, dg_cg_stats* st, cudaStream_t s) {
  const double* dinv = jacobi ? m->dinv64 : nullptr;
  const long long n = m->ndofs, n3 = (long long)m->n * m->n * m->n;
  const int kind = o->backup;
  const size_t bytes64 = sizeof(double) * (size_t)n;
  o->fault_injected_at = -1;
  o->backup_iteration = -1;
  o->backups_taken = 0;
  o->aux_iterations = 0;
  o->backup_bytes = kind == DG_BACKUP_FULL ? (long long)(3 * bytes64 + sizeof(DGCGState))
                  : kind == DG_BACKUP_X64  ? (long long)bytes64
                  : kind == DG_BACKUP_X32  ? (long long)(bytes64 / 2) : 0;
  // pinned host backups
  void *hx = nullptr, *hr = nullptr, *hp = nullptr;
  DGCGState hstate = {};
  auto release = [&]() {
    if (hx) cudaFreeHost(hx);
    if (hr) cudaFreeHost(hr);
    if (hp) cudaFreeHost(hp);
  };
  if (kind != DG_BACKUP_NONE) {
    DG_CUDA(cudaMallocHost(&hx, kind == DG_BACKUP_X32 ? bytes64 / 2 : bytes64));
    if (kind == DG_BACKUP_FULL) {
      cudaError_t e = cudaMallocHost(&hr, bytes64);
      if (e == cudaSuccess) e = cudaMallocHost(&hp, bytes64);
      if (e != cudaSuccess) {
        release();
        return dg_cuda_fail(e, "dg_cg_solve_resilient: host backup");
      }
    }
  }
  double res2 = 0, b2 = 0;
  int rc = true_residual(m, b, x, s, &res2, &b2);
  if (rc || b2 == 0.0) {
    release();
    return rc ? rc : zero_solution(m, x, st, s);
  }
  // (re)start the recurrence from x with `iters` iterations already counted
  auto start = [&](int iters) -> int {
    int r = set_state(m, maxit, iters, s);
    if (r) return r;
    r = dg_launch_apply_f64(m, x, m->q64, nullptr, s);
    if (r) return r;
    if (dinv)
      k_init<double, true><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->p64, dinv, n, rtol, m->partials,
                                           m->state);
    else
      k_init<double, false><<<RED_LAUNCH>>>(b, m->q64, m->r64, m->p64, dinv, n, rtol,
                                            m->partials, m->state);
    DG_CUDA(cudaGetLastError());
    return DG_OK;
  };
  rc = start(0);
  if (rc) {
    release();
    return rc;
  }
  const int chunk = o->backup_interval;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < chunk && rc == DG_OK; ++i)
    rc = launch_iteration<double>(m, x, m->r64, m->p64, m->q64, dinv, s);
  cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (rc == DG_OK && ec == cudaSuccess) ec = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc || ec != cudaSuccess) {
    release();
    return rc ? rc : dg_cuda_fail(ec, "dg_cg_solve_resilient: graph");
  }
  long long executed = 0;  // iterations actually run, rolled-back ones included
  int restarts = 0, last_it = 0;
  const unsigned vblocks = (unsigned)(m->sm_count * 8);
  // the loop returns through DG_CUDA on a CUDA error; the graph and the host
  // backups are released after it on every path
  rc = [&]() -> int {
    int rc = DG_OK;
    for (;;) {
      ec = cudaGraphLaunch(exec, s);
      if (ec == cudaSuccess)
        ec = cudaMemcpyAsync(m->state_host, m->state, sizeof(DGCGState), cudaMemcpyDeviceToHost, s);
      if (ec == cudaSuccess) ec = cudaStreamSynchronize(s);
      if (ec != cudaSuccess) {
        rc = dg_cuda_fail(ec, "dg_cg_solve_resilient: iteration");
        break;
      }
      const DGCGState hs = *m->state_host;
      executed += hs.iters - last_it;
      last_it = hs.iters;
      if (hs.breakdown) {
        rc = dg_fail(DG_ERR_BREAKDOWN, "dg_cg_solve_resilient: breakdown at iteration %d",
                     hs.iters);
        break;
      }
      if (hs.done) {
        rc = true_residual(m, b, x, s, &res2, &b2);
        if (rc) break;
        const double rel = std::sqrt(res2 / b2);
        if (st) {
          st->iterations = (int)executed;
          st->outer_iterations = restarts;
          st->rel_residual = rel;
          st->rel_residual_rec = hs.bnorm2 > 0 ? std::sqrt(hs.rr / hs.bnorm2) : 0.0;
        }
        if (rel <= rtol) break;
        if (hs.iters >= maxit || restarts >= 5) {
          rc = dg_fail(DG_ERR_NOT_CONVERGED,
                       "dg_cg_solve_resilient: relative residual %.3e > rtol %.3e", rel, rtol);
          break;
        }
        ++restarts;
        rc = start(hs.iters);
        if (rc) break;
        continue;
      }
      if (o->fault_iteration >= 0 && o->fault_injected_at < 0 && hs.iters >= o->fault_iteration) {
        // the data loss: x, r and p of the lost cells are gone
        long long c0 = o->fault_cell_begin, c1 = o->fault_cell_end;
        c0 = c0 < 0 ? 0 : c0;
        c1 = c1 > m->ncells ? m->ncells : c1;
      c1 = c1 < c0 ? c0 : c1;  // an empty or reversed range loses nothing
        k_zero_range<<<vblocks, 256, 0, s>>>(x, m->r64, m->p64, c0 * n3, c1 * n3);
        o->fault_injected_at = hs.iters;
        const bool have = o->backups_taken > 0;
        if (have) o->backup_iteration = hstate.iters;
        if (kind == DG_BACKUP_FULL && o->recovery == DG_RECOVER_GLOBAL && have) {
          DG_CUDA(cudaMemcpyAsync(x, hx, bytes64, cudaMemcpyHostToDevice, s));
          DG_CUDA(cudaMemcpyAsync(m->r64, hr, bytes64, cudaMemcpyHostToDevice, s));
          DG_CUDA(cudaMemcpyAsync(m->p64, hp, bytes64, cudaMemcpyHostToDevice, s));
          *m->state_host = hstate;
          DG_CUDA(cudaMemcpyAsync(m->state, m->state_host, sizeof(DGCGState),
                                  cudaMemcpyHostToDevice, s));
          DG_CUDA(cudaStreamSynchronize(s));
          last_it = hstate.iters;
          continue;  // resumes exactly at the backup's iteration
        }
        if (have) {  // the backup's x: everywhere (global) or on the lost cells (local)
          const long long i0 = o->recovery == DG_RECOVER_GLOBAL ? 0 : c0 * n3;
          const long long i1 = o->recovery == DG_RECOVER_GLOBAL ? n : c1 * n3;
          if (kind == DG_BACKUP_X32) {
            DG_CUDA(cudaMemcpyAsync(m->d32 + i0, (float*)hx + i0, sizeof(float) * (size_t)(i1 - i0),
                                    cudaMemcpyHostToDevice, s));
            k_restore_x32<<<vblocks, 256, 0, s>>>(x, m->d32, i0, i1);
          } else {
            DG_CUDA(cudaMemcpyAsync(x + i0, (double*)hx + i0, sizeof(double) * (size_t)(i1 - i0),
                                    cudaMemcpyHostToDevice, s));
          }
        }
        if (o->recovery == DG_RECOVER_LOCAL_AUX) {
          rc = aux_solve(m, b, x, dinv, c0 * n3, c1 * n3, o->aux_rtol, o->aux_maxit,
                         &o->aux_iterations, s);
          if (rc) break;
        }
        rc = start(hs.iters);  // CG restarts from the recovered x
        if (rc) break;
        ++restarts;
        continue;
      }
      if (kind != DG_BACKUP_NONE) {  // backup of the state after this chunk
        if (kind == DG_BACKUP_X32) {
          k_round_f32<<<vblocks, 256, 0, s>>>(x, m->d32, n);
          DG_CUDA(cudaMemcpyAsync(hx, m->d32, bytes64 / 2, cudaMemcpyDeviceToHost, s));
        } else {
          DG_CUDA(cudaMemcpyAsync(hx, x, bytes64, cudaMemcpyDeviceToHost, s));
        }
        if (kind == DG_BACKUP_FULL) {
          DG_CUDA(cudaMemcpyAsync(hr, m->r64, bytes64, cudaMemcpyDeviceToHost, s));
          DG_CUDA(cudaMemcpyAsync(hp, m->p64, bytes64, cudaMemcpyDeviceToHost, s));
        }
        DG_CUDA(cudaStreamSynchronize(s));
        hstate = hs;
        o->backups_taken += 1;
      }
    }
    return rc;
  }();
  cudaGraphExecDestroy(exec);
  release();
  if (st) st->status = rc;
  return rc;
}

// Marks a solve in the scaled Gauss-point basis: while it lives, the internal
// FP64 apply launcher applies Q A Q^T and the Jacobi diagonal is diag(Q A Q^T).
struct NodalScope {
  dg_mesh* m;
  explicit NodalScope(dg_mesh* mm) : m(mm) { m->nodal_op = true; }
  ~NodalScope() { m->nodal_op = false; }
};

// CG in the scaled Gauss-point basis (DG_CG_NODAL): b_hat = Q b, x_hat = Q x,
// the FP64 CG of cg_fp64 (or the mixed CG of cg_mixed) on Q A Q^T,
// x = Q^T x_hat, then the residual in the Legendre basis.  The solve's own
// stopping test is on ||b_hat - Q A Q^T x_hat|| = ||b - A x|| (Q orthogonal);
// the mapping back rounds x, so if the Legendre-basis residual is still above
// rtol, the same solver (precision and preconditioner) continues from x in the
// Legendre basis.
int cg_nodal(dg_mesh* m, const double* b, double* x, double rtol, int maxit, dg_cg_stats* st,
             bool jacobi, bool kron, bool mixed, cudaStream_t s) {
  int rc = jacobi ? dg_ensure_nodal_diag(m, s) : dg_ensure_nodal(m, s);
  if (rc == DG_OK && mixed) rc = dg_ensure_nodal32(m, s);
  if (rc == DG_OK && kron) rc = dg_ensure_kron_nodal(m, s);
  if (rc) return rc;
  rc = dg_launch_collocation(m, b, m->bN64, true, s);
  if (rc == DG_OK) rc = dg_launch_collocation(m, x, m->xN64, true, s);
  if (rc) return rc;
  dg_cg_stats sn{};
  {
    NodalScope scope(m);
    rc = mixed ? cg_mixed(m, m->bN64, m->xN64, rtol, maxit, &sn, jacobi, s, kron)
               : cg_fp64(m, m->bN64, m->xN64, rtol, maxit, &sn, jacobi, s, false, kron);
  }
  // x holds the last iterate also when the solve stopped early
  int rc2 = dg_launch_collocation(m, m->xN64, x, false, s);
  if (rc2) return rc2;
  if (rc != DG_OK && rc != DG_ERR_NOT_CONVERGED) return rc;
  double res2 = 0.0, b2 = 0.0;
  rc2 = true_residual(m, b, x, s, &res2, &b2);
  if (rc2) return rc2;
  const double rel = b2 > 0.0 ? std::sqrt(res2 / b2) : 0.0;
  if (st) {
    *st = sn;
    st->rel_residual = rel;
  }
  // NOT_CONVERGED: the solver's message stands (its residual equals this one
  // up to the mapping's rounding) and x holds the last iterate
  if (rc != DG_OK) return rc;
  if (rel <= rtol) return DG_OK;
  // finish in the Legendre basis with the same precision and preconditioner
  // (a few iterations: only the mapping's rounding is left)
  dg_cg_stats sp{};
  const int left = maxit - sn.iterations;
  if (left < 1)
    return dg_fail(DG_ERR_NOT_CONVERGED,
                   "dg_cg_solve(nodal): relative residual %.3e > rtol %.3e after %d iterations",
                   rel, rtol, sn.iterations);
  if (jacobi && (rc = dg_ensure_diagonal(m, s))) return rc;
  rc = mixed ? cg_mixed(m, b, x, rtol, left, &sp, jacobi, s, kron)
             : cg_fp64(m, b, x, rtol, left, &sp, jacobi, s, false, kron);
  if (st) {
    st->iterations = sn.iterations + sp.iterations;
    st->outer_iterations = sn.outer_iterations + 1 + sp.outer_iterations;
    st->rel_residual = sp.rel_residual;
    st->rel_residual_rec = sp.rel_residual_rec;
  }
  return rc;
}

}  // namespace

extern "C" int dg_cg_solve(const dg_mesh* mc, const double* b, double* x, double rtol, int maxit,
                           int mode, dg_cg_stats* st, void* stream) {
  if (mc == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: mesh is NULL");
  if (!mc->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: coefficient not set");
  if (b == nullptr || x == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: NULL vector");
  if (b == x) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: b and x alias");
  if (!(rtol > 0.0) || !(rtol < 1.0))
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: rtol=%g outside (0, 1)", rtol);
  if (maxit < 1) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: maxit=%d < 1", maxit);
  const bool jacobi = (mode & DG_CG_PRECOND_JACOBI) != 0;
  const bool block = (mode & DG_CG_PRECOND_BLOCK) != 0;
  const bool kron = (mode & DG_CG_PRECOND_KRON) != 0;
  const bool nodal = (mode & DG_CG_NODAL) != 0;
  const int base = mode & ~(DG_CG_PRECOND_JACOBI | DG_CG_PRECOND_BLOCK | DG_CG_PRECOND_KRON |
                            DG_CG_NODAL);
  if (base != DG_CG_FP64 && base != DG_CG_MIXED_IR && base != DG_CG_MIXED_IR_RESTART)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve: unknown mode %d", mode);
  if (nodal && (block || base == DG_CG_MIXED_IR_RESTART))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve: DG_CG_NODAL goes with DG_CG_FP64 or DG_CG_MIXED_IR, with M = I, "
                   "DG_CG_PRECOND_JACOBI or DG_CG_PRECOND_KRON");
  if (block && (jacobi || kron || base != DG_CG_FP64))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve: DG_CG_PRECOND_BLOCK goes with DG_CG_FP64 only");
  if (kron && (jacobi || base == DG_CG_MIXED_IR_RESTART))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve: DG_CG_PRECOND_KRON goes with DG_CG_FP64 or DG_CG_MIXED_IR "
                   "only");
  if ((mc->affine || mc->multilinear) && mode != DG_CG_FP64)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve: on an affine or multilinear geometry only DG_CG_FP64 without "
                   "preconditioner");
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  int rc = dg_ensure_solver_ws(m);
  if (rc) return rc;
  const double t0 = now_s();
  // order the solve after the caller's prior work on its stream
  DG_CUDA(cudaEventRecord(m->ev, (cudaStream_t)stream));
  DG_CUDA(cudaStreamWaitEvent(m->solve_stream, m->ev, 0));
  if (st) *st = dg_cg_stats{};
  cudaStream_t s = m->solve_stream;
  if (jacobi && !nodal) rc = dg_ensure_diagonal(m, s);
  if (block) rc = dg_ensure_block(m, s);
  if (kron) rc = dg_ensure_kron(m, s);
  if (rc == DG_OK) {
    if (nodal)
      rc = cg_nodal(m, b, x, rtol, maxit, st, jacobi, kron, base == DG_CG_MIXED_IR, s);
    else if (base == DG_CG_FP64)
      rc = cg_fp64(m, b, x, rtol, maxit, st, jacobi, s, block, kron);
    else if (base == DG_CG_MIXED_IR)
      rc = cg_mixed(m, b, x, rtol, maxit, st, jacobi, s, kron);
    else
      rc = cg_mixed_restart(m, b, x, rtol, maxit, st, jacobi, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == DG_OK && e != cudaSuccess) rc = dg_cuda_fail(e, "dg_cg_solve: synchronize");
  if (st) {
    st->seconds = now_s() - t0;
    st->status = rc;
  }
  return rc;
}

extern "C" int dg_cg_solve_resilient(const dg_mesh* mc, const double* b, double* x, double rtol,
                                     int maxit, int mode, dg_resilience* res, dg_cg_stats* st,
                                     void* stream) {
  if (mc == nullptr || res == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_resilient: NULL mesh or options");
  if (!mc->has_coef)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_resilient: coefficient not set");
  if (b == nullptr || x == nullptr || b == x)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_resilient: NULL or aliased b, x");
  if (mode != DG_CG_FP64 && mode != (DG_CG_FP64 | DG_CG_PRECOND_JACOBI))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve_resilient: mode %d; DG_CG_FP64 with or without Jacobi", mode);
  if (!(rtol > 0.0) || !(rtol < 1.0) || maxit < 1)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_resilient: rtol or maxit out of range");
  if (res->backup_interval < 1 || res->backup < DG_BACKUP_NONE || res->backup > DG_BACKUP_X32 ||
      res->recovery < DG_RECOVER_GLOBAL || res->recovery > DG_RECOVER_LOCAL_AUX ||
      (res->recovery == DG_RECOVER_LOCAL_AUX && (!(res->aux_rtol > 0.0) || res->aux_maxit < 1)))
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_resilient: bad backup options");
  if (int rc0 = dg_require_cube(mc, "dg_cg_solve_resilient")) return rc0;
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  int rc = dg_ensure_solver_ws(m);
  if (rc) return rc;
  const double t0 = now_s();
  DG_CUDA(cudaEventRecord(m->ev, (cudaStream_t)stream));
  DG_CUDA(cudaStreamWaitEvent(m->solve_stream, m->ev, 0));
  if (st) *st = dg_cg_stats{};
  cudaStream_t s = m->solve_stream;
  const bool jacobi = (mode & DG_CG_PRECOND_JACOBI) != 0;
  if (jacobi) rc = dg_ensure_diagonal(m, s);
  if (rc == DG_OK) rc = cg_fp64_resilient(m, b, x, rtol, maxit, jacobi, res, st, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == DG_OK && e != cudaSuccess) rc = dg_cuda_fail(e, "dg_cg_solve_resilient: synchronize");
  if (st) {
    st->seconds = now_s() - t0;
    st->status = rc;
  }
  return rc;
}
