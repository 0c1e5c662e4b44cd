// Sum-factorised SIPG operator application y = A(K) x (Section 3.3 applied to
// the Section 4.1 form), in two passes over the cells.
//
// Pass 1 (trace kernel), per cell: modal -> nodal values by three 1D
// contractions with B[a][i] = L_i(xi_a) (along z, then y, then x).  It keeps
// the x-modal / yz-nodal intermediate X, the nodal values U, and the value and
// reference normal derivative of u on all six faces at the n^2 face Gauss points
// (x-faces from X with L_i(0|1), L_i'(0|1); y/z-faces from U with the Lagrange
// end values l_a(0|1), l_a'(0|1)).
//
// Pass 2 (cell kernel), per cell: reads U, X, the weighted coefficient
// Kt_q = h w_q K_q, precomputed face-point weights, its own face traces and its
// six neighbours' face traces, and forms
//   r = sum_d D_d^T (Kt . D_d u)   (collocation derivative along y and z;
//                                   L_i' contraction from X along x),
// adds the face terms -{d_n u}[phi] - {d_n phi}[u] + sigma [u][phi], and maps
// back to modal coefficients with B^T along x, y, z.
//
// FP64 operations are the scarce resource on GB300 (FP64 runs ~75x slower than
// FP32), so the kernels minimise them:
//   * the Gauss points are symmetric about 1/2 and L_i(1 - t) = (-1)^i L_i(t),
//     so every B, B^T, L', L'^T line contraction splits into even and odd
//     modes (about n^2/2 + n operations instead of n^2); L_0 = 1 and L_0' = 0
//     remove further terms;
//   * x-face traces and x-face test functions use the same parity split;
//   * face-point weights W/2 = h gamma_F w_s w_t / 2 and the derivative weight
//     (W/2 inside, W on the boundary) are precomputed when K is set, and
//     2 sigma = 4 n^2 is a compile-time constant, so a face point costs five
//     operations.
// The only duplicated arithmetic is the pointwise flux of an interior face,
// which both of its cells evaluate.
//
// Thread layout: n^2 threads per cell; a block holds CPB cells.  Each thread
// owns one 1D line of its cell at every stage; lines are exchanged through
// shared memory between stages.
#pragma once

#include "dg_internal.cuh"

namespace dgk {

// Sum of partials[0 .. count) in the last block of a grid reduction, by all
// NT threads of the block in a fixed order: each thread keeps four
// independent chains of L2 loads (ld.global.cg: the other blocks' partials,
// published before their ticket increment), then warp 0 adds the threads'
// sums with a fixed tree.  Valid in warp 0; every thread of the block calls it.
template <int NT>
__device__ __forceinline__ double last_block_total(const double* __restrict__ partials,
                                                   int count, double* scratch) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int b = threadIdx.x;
  for (; b + 3 * NT < count; b += 4 * NT) {
    a0 += __ldcg(partials + b);
    a1 += __ldcg(partials + b + NT);
    a2 += __ldcg(partials + b + 2 * NT);
    a3 += __ldcg(partials + b + 3 * NT);
  }
  for (; b < count; b += NT) a0 += __ldcg(partials + b);
  scratch[threadIdx.x] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < NT; i += 32) t += scratch[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  }
  return t;
}

template <int N>
struct Cfg {
  // cells per block, chosen so a block has ~128-256 threads
  static constexpr int CPB = (N == 2) ? 32 : (N == 3) ? 14 : (N == 4) ? 8 : (N == 5) ? 5
                           : (N == 6) ? 4 : (N == 7) ? 3 : 2;
  static constexpr int THREADS = CPB * N * N;
};

// ---------------------------------------------------------------------------
// 1D line contractions with the parity split (H = N/2 mirror pairs a, N-1-a;
// for odd N the middle point m = N/2 sits at xi = 1/2).
// ---------------------------------------------------------------------------

// The contractions take the table type TT separately from the value type T
// (the packed FP32 pair values of dg_pair32.cuh use the scalar FP32 tables).

// u[a] = sum_i B[a][i] X[i]   (modal -> nodal values)
template <int N, typename T, typename TT>
__device__ __forceinline__ void b_fwd(const DGTab<TT>& t, const T (&X)[N], T (&u)[N]) {
  constexpr int H = N / 2;
#pragma unroll
  for (int a = 0; a < H; ++a) {
    T E = X[0];  // L_0 = 1
#pragma unroll
    for (int i = 2; i < N; i += 2) E = fma(t.B[a][i], X[i], E);
    T O = t.B[a][1] * X[1];
#pragma unroll
    for (int i = 3; i < N; i += 2) O = fma(t.B[a][i], X[i], O);
    u[a] = E + O;
    u[N - 1 - a] = E - O;
  }
  if (N % 2 == 1) {  // L_odd(1/2) = 0
    T E = X[0];
#pragma unroll
    for (int i = 2; i < N; i += 2) E = fma(t.B[H][i], X[i], E);
    u[H] = E;
  }
}

// g[a] = sum_i L_i'(xi_a) X[i]   (modal -> nodal derivative; L_1' is constant)
template <int N, typename T, typename TT>
__device__ __forceinline__ void bd_fwd(const DGTab<TT>& t, const T (&X)[N], T (&g)[N]) {
  constexpr int H = N / 2;
  const T c1 = t.Bd[0][1] * X[1];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    T O = c1;
#pragma unroll
    for (int i = 3; i < N; i += 2) O = fma(t.Bd[a][i], X[i], O);
    if (N > 2) {
      T E = t.Bd[a][2] * X[2];
#pragma unroll
      for (int i = 4; i < N; i += 2) E = fma(t.Bd[a][i], X[i], E);
      g[a] = O + E;
      g[N - 1 - a] = O - E;
    } else {
      g[a] = O;
      g[N - 1 - a] = O;
    }
  }
  if (N % 2 == 1) {  // L_even'(1/2) = 0
    T O = c1;
#pragma unroll
    for (int i = 3; i < N; i += 2) O = fma(t.Bd[H][i], X[i], O);
    g[H] = O;
  }
}

// R[i] = sum_a B[a][i] r[a] + sum_a L_i'(xi_a) k[a]   (nodal -> modal, both parts)
template <int N, typename T, typename TT>
__device__ __forceinline__ void bt_bdt(const DGTab<TT>& t, const T (&r)[N], const T (&k)[N],
                                       T (&R)[N]) {
  constexpr int H = N / 2;
  T re[H > 0 ? H : 1], ro[H > 0 ? H : 1], ke[H > 0 ? H : 1], ko[H > 0 ? H : 1];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    re[a] = r[a] + r[N - 1 - a];
    ro[a] = r[a] - r[N - 1 - a];
    ke[a] = k[a] + k[N - 1 - a];
    ko[a] = k[a] - k[N - 1 - a];
  }
  // i = 0: L_0 = 1, L_0' = 0
  {
    T acc = re[0];
#pragma unroll
    for (int a = 1; a < H; ++a) acc = acc + re[a];
    if (N % 2 == 1) acc = acc + r[H];
    R[0] = acc;
  }
#pragma unroll
  for (int i = 1; i < N; ++i) {
    T acc;
    if (i % 2 == 0) {  // even mode: value part symmetric, derivative part antisymmetric
      acc = t.B[0][i] * re[0];
#pragma unroll
      for (int a = 1; a < H; ++a) acc = fma(t.B[a][i], re[a], acc);
      if (N % 2 == 1) acc = fma(t.B[H][i], r[H], acc);
#pragma unroll
      for (int a = 0; a < H; ++a) acc = fma(t.Bd[a][i], ko[a], acc);
    } else {           // odd mode: value part antisymmetric, derivative part symmetric
      acc = t.B[0][i] * ro[0];
#pragma unroll
      for (int a = 1; a < H; ++a) acc = fma(t.B[a][i], ro[a], acc);
#pragma unroll
      for (int a = 0; a < H; ++a) acc = fma(t.Bd[a][i], ke[a], acc);
      if (N % 2 == 1) acc = fma(t.Bd[H][i], k[H], acc);
    }
    R[i] = acc;
  }
}

// R[i] = sum_a B[a][i] r[a]   (nodal -> modal values)
template <int N, typename T, typename TT>
__device__ __forceinline__ void b_bwd(const DGTab<TT>& t, const T (&r)[N], T (&R)[N]) {
  constexpr int H = N / 2;
  T re[H > 0 ? H : 1], ro[H > 0 ? H : 1];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    re[a] = r[a] + r[N - 1 - a];
    ro[a] = r[a] - r[N - 1 - a];
  }
  {
    T acc = re[0];
#pragma unroll
    for (int a = 1; a < H; ++a) acc = acc + re[a];
    if (N % 2 == 1) acc = acc + r[H];
    R[0] = acc;
  }
#pragma unroll
  for (int i = 1; i < N; ++i) {
    T acc;
    if (i % 2 == 0) {
      acc = t.B[0][i] * re[0];
#pragma unroll
      for (int a = 1; a < H; ++a) acc = fma(t.B[a][i], re[a], acc);
      if (N % 2 == 1) acc = fma(t.B[H][i], r[H], acc);
    } else {
      acc = t.B[0][i] * ro[0];
#pragma unroll
      for (int a = 1; a < H; ++a) acc = fma(t.B[a][i], ro[a], acc);
    }
    R[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// Face flux at one face point.  Reference units: g = d/dxi along +axis.
// UPPER: this cell is the lower-index (-) side of the face (its xi = 1 face).
//   J = u- - u+, G = g- + g+ ; the (-) cell's test value gets
//   W (sigma J - G/2) = Wh (2 sigma J - G), the (+) cell's the negative; both
//   test derivatives get -Wd J (Wd = W/2 inside, W on the boundary).
// On a boundary face the missing side is (u, g) = (0, own g), which turns the
// interior formula into the one-sided form -(d_n u) phi - (d_n phi) u + sigma u phi.
// Returns cv (multiplier of the test value) and cdm = Wd J (the test
// derivative's multiplier is -cdm).
// ---------------------------------------------------------------------------
template <int N, bool UPPER, typename T>
__device__ __forceinline__ void flux(T uo, T go, T un, T gn, T Wh, T Wd, T& cv, T& cdm) {
  constexpr T S2 = T(4 * N * N);  // 2 sigma, sigma = 2 (k+1)^2
  const T J = UPPER ? uo - un : un - uo;
  const T G = go + gn;
  const T tt = UPPER ? fma(S2, J, -G) : fma(-S2, J, G);
  cv = Wh * tt;
  cdm = Wd * J;
}

// Load a face trace pair (value, derivative) of face f of cell c at point pt.
template <int N, typename T>
__device__ __forceinline__ void load_trace(const T* __restrict__ TR, long long c, int f, int pt,
                                           T& v, T& g) {
  constexpr int N2 = N * N;
  const T* tr = TR + c * (12 * N2) + (2 * f) * N2 + pt;
  v = tr[0];
  g = tr[N2];
}

// Own and neighbour traces plus weights of face f at point pt; on a boundary
// face the neighbour is (0, own derivative).
template <int N, bool UPPER, typename T>
__device__ __forceinline__ void face_point(const T* __restrict__ TR, const T* __restrict__ FW,
                                           long long c, int f, bool interior, long long cn, int fn,
                                           int pt, T& cv, T& cdm) {
  constexpr int N2 = N * N;
  T uo, go;
  load_trace<N>(TR, c, f, pt, uo, go);
  T un = T(0), gn = go;
  if (interior) load_trace<N>(TR, cn, fn, pt, un, gn);
  const T* fw = FW + c * (12 * N2) + (2 * f) * N2 + pt;
  flux<N, UPPER>(uo, go, un, gn, fw[0], fw[N2], cv, cdm);
}

// Where pass 2 gets its face data.  FaceGlobal: own and neighbour traces from
// the pass-1 buffer, face-point weights from the precomputed buffer.
template <typename T>
struct FaceGlobal {
  const T* TR;
  const T* FW;
  static constexpr bool OWN_IN_THREAD = false;  // own traces come from TR
  struct Pre {};  // nothing prefetched: the FP64 kernels hide load latency behind the FP64 pipe
  template <int N>
  __device__ __forceinline__ void prefetch(Pre&, long long, int, const bool (&)[6],
                                           const long long (&)[6]) const {}
  template <int N, bool UPPER>
  __device__ __forceinline__ void get(const Pre&, long long c, int lc, int f, bool in,
                                      long long cn, int fn, int pt, T, T, T& cv,
                                      T& cdm) const {
    (void)lc;
    face_point<N, UPPER>(TR, FW, c, f, in, cn, fn, pt, cv, cdm);
  }
};

// FaceNbr: only the neighbour part of an interior face's flux; the own-side
// part (and the whole boundary form) is inside the line operators.  With the
// neighbour trace (un, gn) and W/2 = Wh (equal to the derivative weight
// inside), the upper face gives cv = -Wh (2 sigma un + gn), cdm = -Wh un and
// the lower face cv = Wh (gn - 2 sigma un), cdm = Wh un: three operations
// and three loads per face point instead of five and six.
template <typename T>
struct FaceNbr {
  const T* TR;
  const T* FW;
  static constexpr bool OWN_IN_THREAD = false;  // own terms are in the line operators
  struct Pre {};
  template <int N>
  __device__ __forceinline__ void prefetch(Pre&, long long, int, const bool (&)[6],
                                           const long long (&)[6]) const {}
  template <int N, bool UPPER>
  __device__ __forceinline__ void get(const Pre&, long long c, int lc, int f, bool in,
                                      long long cn, int fn, int pt, T, T, T& cv,
                                      T& cdm) const {
    constexpr int N2 = N * N;
    constexpr T S2 = T(4 * N * N);
    (void)lc;
    cv = T(0);
    cdm = T(0);
    if (!in) return;
    T un, gn;
    load_trace<N>(TR, cn, fn, pt, un, gn);
    const T wh = FW[c * (12 * N2) + (2 * f) * N2 + pt];
    if (UPPER) {
      cv = -wh * fma(S2, un, gn);
      cdm = -wh * un;
    } else {
      cv = wh * fma(-S2, un, gn);
      cdm = wh * un;
    }
  }
};

// FaceLocal: own traces formed by the calling line-thread from its own line's
// values (passed in as uo, go), neighbour traces from the pass-1 buffer,
// weights from h*gamma per face (W/2 = h gamma w_s w_t / 2; the derivative
// weight doubles on the boundary).
// The global loads (neighbour traces, h*gamma) of all six faces are issued
// together by prefetch() when the cell phase starts, so their latency overlaps
// the volume work instead of stalling each direction's face step.
template <typename T>
struct FaceLocal {
  const T* TR;
  const T* gh;
  const DGTab<T>* tab;
  static constexpr bool OWN_IN_THREAD = true;
  struct Pre {
    T un[6], gn[6], wh[6];  // neighbour trace; W/2 = h gamma w_s w_t / 2 per face
  };
  // in[f], cn[f]: whether face f is interior and its neighbour cell; the
  // neighbour's face is f ^ 1 (x- <-> x+, ...).
  template <int N>
  __device__ __forceinline__ void prefetch(Pre& pre, long long c, int pt, const bool (&in)[6],
                                           const long long (&cn)[6]) const {
    // the line's face point has the same Gauss weights on all six faces
    const T hw2 = T(0.5) * tab->w[pt % N] * tab->w[pt / N];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      pre.un[f] = T(0);
      pre.gn[f] = T(0);
      if (in[f]) load_trace<N>(TR, cn[f], f ^ 1, pt, pre.un[f], pre.gn[f]);
      pre.wh[f] = hw2 * gh[c * 6 + f];
    }
  }
  template <int N, bool UPPER>
  __device__ __forceinline__ void get(const Pre& pre, long long c, int lc, int f, bool in,
                                      long long cn, int fn, int pt, T uo, T go, T& cv,
                                      T& cdm) const {
    (void)c;
    (void)lc;
    (void)cn;
    (void)fn;
    (void)pt;
    const T un = pre.un[f], gn = in ? pre.gn[f] : go;
    const T wh = pre.wh[f];
    flux<N, UPPER>(uo, go, un, gn, wh, in ? wh : wh + wh, cv, cdm);
  }
};

// ---------------------------------------------------------------------------
// Pass 1: nodal values and face traces.
// TR layout: TR[((c*6 + f)*2 + comp)*n^2 + pt], f = x-, x+, y-, y+, z-, z+,
// comp 0 = value, 1 = d/dxi along +axis; pt = (b + n e) on x-faces,
// (a + n e) on y-faces, (a + n b) on z-faces.
// ---------------------------------------------------------------------------
// Pass 1 over the cells c0 .. c0+nblk-1 (nblk <= CPB) by the calling block;
// s: CPB n^3 values of shared memory.  Threads beyond CPB n^2 only take part
// in the loads and barriers.
// trace_core: s already holds the cells' modal coefficients.
//   MODE 0 (pass 1): writes U, X and the face traces to global memory;
//   MODE 2: writes only the face traces to global memory;
//   MODE 3: leaves U in s and copies X to sx, no traces (the cell phase forms
//           each line's own traces itself, FaceLocal).
// Default z-line input of trace_core: the line's modal values already in s.
struct ZFromShared {
  template <int N, typename T>
  __device__ __forceinline__ void operator()(const T* sc, int lc, int p, int q,
                                             T (&v)[N]) const {
    (void)lc;
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = sc[l * N * N + q * N + p];
  }
};

// z-line input straight from global memory (xg: the block's first cell).
template <typename TG>
struct ZFromGlobal {
  const TG* xg;
  template <int N, typename T>
  __device__ __forceinline__ void operator()(const T* sc, int lc, int p, int q,
                                             T (&v)[N]) const {
    (void)sc;
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = xg[lc * N * N * N + l * N * N + q * N + p];
  }
};

// ZL: fills v[l] (l = 0..n-1) with the modal values of the thread's z-line
// (x-mode p, y-mode q of cell lc); a kernel that produces those values itself
// (a direction update, a load from global memory) passes its own loader and
// needs no barrier between producing them and the first contraction.
template <int N, typename T, int MODE, typename ZL = ZFromShared>
__device__ __forceinline__ void trace_core(T* __restrict__ U, T* __restrict__ Xm,
                                           T* __restrict__ TR, long long c0, int nblk,
                                           const DGTab<T>& tab, T* s, T* sx,
                                           const ZL& zload = ZL()) {
  constexpr int N2 = N * N, N3 = N * N * N, H = N / 2;

  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  T* sc = s + lc * N3;
  const long long c = c0 + lc;

  // along z: thread owns (i = p, j = q)
  if (active) {
    T v[N], u[N];
    zload.template operator()<N, T>(sc, lc, p, q, v);
    b_fwd<N>(tab, v, u);
#pragma unroll
    for (int e = 0; e < N; ++e) sc[e * N2 + q * N + p] = u[e];
  }
  __syncthreads();
  // along y: thread owns (i = p, e = q)
  if (active) {
    T v[N], u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = sc[q * N2 + j * N + p];
    b_fwd<N>(tab, v, u);
#pragma unroll
    for (int b = 0; b < N; ++b) sc[q * N2 + b * N + p] = u[b];
  }
  __syncthreads();
  // along x: thread owns (b = p, e = q); X is modal in x, nodal in y and z
  T* tr = (MODE == 3) ? nullptr : TR + c * (12 * N2);
  if (active) {
    T X[N], u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) X[i] = sc[q * N2 + p * N + i];
    if (MODE != 2) {
      T* xm = (MODE == 0) ? Xm + c * N3 + q * N2 + p * N : sx + lc * N3 + q * N2 + p * N;
#pragma unroll
      for (int i = 0; i < N; ++i) xm[i] = X[i];
    }
    // x-face traces from the modes: L_i(1) = a_i, L_i(0) = (-1)^i a_i,
    // L_i'(1) = d_i, L_i'(0) = (-1)^(i+1) d_i, a_0 = 1, d_0 = 0
    if (MODE != 3) {
      T Se = X[0], So = tab.a1[1] * X[1];
#pragma unroll
      for (int i = 2; i < N; i += 2) Se = fma(tab.a1[i], X[i], Se);
#pragma unroll
      for (int i = 3; i < N; i += 2) So = fma(tab.a1[i], X[i], So);
      T Do = tab.d1[1] * X[1];
#pragma unroll
      for (int i = 3; i < N; i += 2) Do = fma(tab.d1[i], X[i], Do);
      T De = T(0);
      if (N > 2) {
        De = tab.d1[2] * X[2];
#pragma unroll
        for (int i = 4; i < N; i += 2) De = fma(tab.d1[i], X[i], De);
      }
      const int pt = p + N * q;
      tr[0 * N2 + pt] = Se - So;                 // x- value
      tr[1 * N2 + pt] = (N > 2) ? Do - De : Do;  // x- derivative
      tr[2 * N2 + pt] = Se + So;                 // x+ value
      tr[3 * N2 + pt] = (N > 2) ? Do + De : Do;  // x+ derivative
    }
    b_fwd<N>(tab, X, u);
#pragma unroll
    for (int a = 0; a < N; ++a) {
      sc[q * N2 + p * N + a] = u[a];
      if (MODE == 0) U[c * N3 + q * N2 + p * N + a] = u[a];
    }
  }
  if (MODE == 3) return;  // the caller synchronises before reading s
  __syncthreads();
  if (active) {
    // y-faces: thread owns points (a = p, e = q); z-faces: (a = p, b = q)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      T u[N];
      if (dir == 0) {
#pragma unroll
        for (int b = 0; b < N; ++b) u[b] = sc[q * N2 + b * N + p];
      } else {
#pragma unroll
        for (int e = 0; e < N; ++e) u[e] = sc[e * N2 + q * N + p];
      }
      T vm = tab.l0[0] * u[0], vp = tab.l1[0] * u[0];
      T gm = tab.dl0[0] * u[0], gp = tab.dl1[0] * u[0];
#pragma unroll
      for (int b = 1; b < N; ++b) {
        vm = fma(tab.l0[b], u[b], vm);
        vp = fma(tab.l1[b], u[b], vp);
        gm = fma(tab.dl0[b], u[b], gm);
        gp = fma(tab.dl1[b], u[b], gp);
      }
      const int pt = p + N * q;
      const int f0 = 4 + 4 * dir;
      tr[(f0 + 0) * N2 + pt] = vm;
      tr[(f0 + 1) * N2 + pt] = gm;
      tr[(f0 + 2) * N2 + pt] = vp;
      tr[(f0 + 3) * N2 + pt] = gp;
    }
  }
  (void)H;
  (void)N3;
}

// Pass 1 over the cells c0 .. c0+nblk-1 (nblk <= CPB) by the calling block;
// s: CPB n^3 values of shared memory.  Threads beyond CPB n^2 only take part
// in the loads and barriers.
template <int N, typename T>
__device__ __forceinline__ void trace_cells(const T* __restrict__ x, T* __restrict__ U,
                                            T* __restrict__ Xm, T* __restrict__ TR, long long c0,
                                            int nblk, const DGTab<T>& tab, T* s) {
  constexpr int N3 = N * N * N;
  // each z-line thread loads its own line of x: no staging barrier
  const ZFromGlobal<T> zl{x + c0 * N3};
  trace_core<N, T, 0>(U, Xm, TR, c0, nblk, tab, s, nullptr, zl);
}

template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_trace(const T* __restrict__ x, T* __restrict__ U, T* __restrict__ Xm, T* __restrict__ TR,
        long long cbeg, long long cend, const int* __restrict__ skip,
        const __grid_constant__ DGTab<T> tab) {
  constexpr int C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long c0 = cbeg + (long long)blockIdx.x * C;
  const int nblk = (int)((cend - c0) < C ? (cend - c0) : C);
  trace_cells<N, T>(x, U, Xm, TR, c0, nblk, tab, reinterpret_cast<T*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Pass 2: volume and face terms, back to modal coefficients.
// FW layout: FW[((c*6 + f)*2 + comp)*n^2 + pt], comp 0 = W/2, 1 = derivative
// weight (W/2 inside, W on the boundary), W = h gamma_F w_s w_t.
// ---------------------------------------------------------------------------
// Pass 2 over the cells c0 .. c0+nblk-1 (nblk <= CPB) by the calling block;
// smem: 4 CPB n^3 values of shared memory.
// cell_core: su (nodal U), sx (x-modal X) and sk (h w K) already hold the
// cells' data in shared memory; face data come from the policy fs; y gets the
// result.
// Packed upper triangle of a symmetric n x n line operator: entry (i, j), i <= j.
template <int N>
__host__ __device__ constexpr int packed(int i, int j) {
  return i <= j ? i * N - i * (i - 1) / 2 + (j - i) : j * N - j * (j - 1) / 2 + (i - j);
}

// LINEOP = true: the volume term of a line and the own-side terms of its two
// face points are one precomputed symmetric operator per line (lineop:
// [c][x,y,z][line][packed n(n+1)/2], see k_line_ops) instead of
// D^T diag(Kt) D (y, z) and L'^T diag(Kt) L' (x); the face policy then adds
// only the neighbour part of interior faces (FaceNbr).
template <int N, typename T, typename FS, bool LINEOP = false>
__device__ __forceinline__ void cell_core(const FS& fs, T* __restrict__ y, long long c0,
                                          int nblk, int Nc, const DGTab<T>& tab, T* su, T* sx,
                                          T* sr, T* sk, const T* __restrict__ lineop = nullptr) {
  constexpr int N2 = N * N, N3 = N * N * N, NP = N * (N + 1) / 2;

  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  const long long c = c0 + lc;
  // Cell coordinates: the block's first cell once (thread 0, one division),
  // then step forward to this thread's cell; 64-bit division per thread would
  // cost more instructions than the FP32 arithmetic of a line.
  __shared__ int sbase[3];
  if (threadIdx.x == 0) {
    const unsigned cu = (unsigned)c0, n = (unsigned)Nc;
    sbase[0] = (int)(cu % n);
    sbase[1] = (int)((cu / n) % n);
    sbase[2] = (int)(cu / n / n);
  }
  __syncthreads();
  int cx = sbase[0] + lc, cy = sbase[1], cz = sbase[2];
  while (cx >= Nc) {
    cx -= Nc;
    if (++cy == Nc) {
      cy = 0;
      ++cz;
    }
  }
  const long long sy = Nc, sz = (long long)Nc * Nc;
  const int o = lc * N3;
  const int pt = p + N * q;
  // face f = x-, x+, y-, y+, z-, z+: interior?  neighbour cell
  const bool in6[6] = {cx > 0, cx < Nc - 1, cy > 0, cy < Nc - 1, cz > 0, cz < Nc - 1};
  const long long cn6[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
  typename FS::Pre pre;
  if (active) fs.template prefetch<N>(pre, c, pt, in6, cn6);

  // z-lines then y-lines: collocation derivative, Kt, transpose, face terms
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    if (active) {
      // dir 0: z-line of (a = p, b = q); dir 1: y-line of (a = p, e = q)
      const int base = (dir == 0) ? (q * N + p) : (q * N2 + p);
      const int step = (dir == 0) ? N2 : N;
      T u[N], r[N];
#pragma unroll
      for (int e = 0; e < N; ++e) u[e] = su[o + base + e * step];
      if (LINEOP) {
        // dir 0 = z-lines (operator slot 2), dir 1 = y-lines (slot 1)
        const T* Mp = lineop + ((c * 3 + (2 - dir)) * N2 + pt) * NP;
        T Mv[NP];
#pragma unroll
        for (int t = 0; t < NP; ++t) Mv[t] = Mp[t];
#pragma unroll
        for (int e = 0; e < N; ++e) {
          T acc = (dir == 0) ? Mv[packed<N>(e, 0)] * u[0]
                             : fma(Mv[packed<N>(e, 0)], u[0], sr[o + base + e * step]);
#pragma unroll
          for (int f = 1; f < N; ++f) acc = fma(Mv[packed<N>(e, f)], u[f], acc);
          r[e] = acc;
        }
      } else {
        T kg[N];
#pragma unroll
        for (int e = 0; e < N; ++e) {
          T g = tab.D[e][0] * u[0];
#pragma unroll
          for (int f = 1; f < N; ++f) g = fma(tab.D[e][f], u[f], g);
          kg[e] = sk[o + base + e * step] * g;
        }
#pragma unroll
        for (int e = 0; e < N; ++e) {
          T acc = (dir == 0) ? tab.D[0][e] * kg[0]
                             : fma(tab.D[0][e], kg[0], sr[o + base + e * step]);
#pragma unroll
          for (int f = 1; f < N; ++f) acc = fma(tab.D[f][e], kg[f], acc);
          r[e] = acc;
        }
      }
      const int fu = (dir == 0) ? 5 : 3, fl = fu - 1;
      const bool inu = (dir == 0) ? (cz < Nc - 1) : (cy < Nc - 1);
      const bool inl = (dir == 0) ? (cz > 0) : (cy > 0);
      const long long st = (dir == 0) ? sz : sy;
      T cv1, cd1, cv0, cd0;
      // own traces of the line's end points (FaceLocal only): Lagrange end
      // values and derivatives of the line's nodal values
      T vm = T(0), vp = T(0), gm = T(0), gp = T(0);
      if constexpr (FS::OWN_IN_THREAD) {
        vm = tab.l0[0] * u[0];
        vp = tab.l1[0] * u[0];
        gm = tab.dl0[0] * u[0];
        gp = tab.dl1[0] * u[0];
#pragma unroll
        for (int e = 1; e < N; ++e) {
          vm = fma(tab.l0[e], u[e], vm);
          vp = fma(tab.l1[e], u[e], vp);
          gm = fma(tab.dl0[e], u[e], gm);
          gp = fma(tab.dl1[e], u[e], gp);
        }
      }
      fs.template get<N, true>(pre, c, lc, fu, inu, c + st, fl, pt, vp, gp, cv1, cd1);
      fs.template get<N, false>(pre, c, lc, fl, inl, c - st, fu, pt, vm, gm, cv0, cd0);
#pragma unroll
      for (int e = 0; e < N; ++e) {
        T acc = fma(tab.l1[e], cv1, r[e]);
        acc = fma(-tab.dl1[e], cd1, acc);
        acc = fma(tab.l0[e], cv0, acc);
        r[e] = fma(-tab.dl0[e], cd0, acc);
      }
#pragma unroll
      for (int e = 0; e < N; ++e) sr[o + base + e * step] = r[e];
    }
    __syncthreads();
  }
  // x-lines: thread owns (b = p, e = q); result is x-modal, yz-nodal
  if (active) {
    const int base = q * N2 + p * N;
    T X[N], rr[N], R[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      X[i] = sx[o + base + i];
      rr[i] = sr[o + base + i];
    }
    if (LINEOP) {
      b_bwd<N>(tab, rr, R);
      const T* Mp = lineop + ((c * 3 + 0) * N2 + pt) * NP;
      T Mv[NP];
#pragma unroll
      for (int t = 0; t < NP; ++t) Mv[t] = Mp[t];
#pragma unroll
      for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) R[i] = fma(Mv[packed<N>(i, j)], X[j], R[i]);
      }
    } else {
      T g[N], kg[N];
      bd_fwd<N>(tab, X, g);
#pragma unroll
      for (int a = 0; a < N; ++a) kg[a] = sk[o + base + a] * g[a];
      bt_bdt<N>(tab, rr, kg, R);
    }
    T cv1, cd1, cv0, cd0;
    // own x-face traces from the modes (FaceLocal only): L_i(1) = a_i,
    // L_i(0) = (-1)^i a_i, L_i'(1) = d_i, L_i'(0) = (-1)^(i+1) d_i
    T xm = T(0), xp = T(0), dxm = T(0), dxp = T(0);
    if constexpr (FS::OWN_IN_THREAD) {
      T Se = X[0], So = tab.a1[1] * X[1], Do = tab.d1[1] * X[1], De = T(0);
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
      xm = Se - So;
      xp = Se + So;
      dxm = Do - De;
      dxp = Do + De;
    }
    fs.template get<N, true>(pre, c, lc, 1, cx < Nc - 1, c + 1, 0, pt, xp, dxp, cv1, cd1);
    fs.template get<N, false>(pre, c, lc, 0, cx > 0, c - 1, 1, pt, xm, dxm, cv0, cd0);
    // modal test functions: value a_i at 1, (-1)^i a_i at 0; derivative -d_i cd
    // at 1, -(-1)^(i+1) d_i cd at 0 (a_0 = 1, d_0 = 0)
    const T sp = cv1 + cv0, sm = cv1 - cv0;
    const T dp = cd1 + cd0, dm = cd1 - cd0;
    R[0] = R[0] + sp;
#pragma unroll
    for (int i = 1; i < N; ++i) {
      if (i % 2 == 0)
        R[i] = fma(tab.a1[i], sp, fma(-tab.d1[i], dm, R[i]));
      else
        R[i] = fma(tab.a1[i], sm, fma(-tab.d1[i], dp, R[i]));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) sx[o + base + i] = R[i];
  }
  __syncthreads();
  // back along y: thread owns (i = p, e = q)
  if (active) {
    T v[N], R[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = sx[o + q * N2 + b * N + p];
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int j = 0; j < N; ++j) sx[o + q * N2 + j * N + p] = R[j];
  }
  __syncthreads();
  // back along z: thread owns (i = p, j = q)
  if (active) {
    T v[N], R[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sx[o + e * N2 + q * N + p];
    b_bwd<N>(tab, v, R);
#pragma unroll
    for (int l = 0; l < N; ++l) sx[o + l * N2 + q * N + p] = R[l];
  }
  __syncthreads();
  T* yb = y + c0 * N3;
  for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) yb[t] = sx[t];
}

// Pass 2 over the cells c0 .. c0+nblk-1 (nblk <= CPB) by the calling block;
// smem: 4 CPB n^3 values of shared memory.
// LINEOP: the volume term uses the precomputed line operators (kt unused).
template <int N, typename T, bool LINEOP = false>
__device__ __forceinline__ void cell_cells(const T* __restrict__ U, const T* __restrict__ Xm,
                                           const T* __restrict__ TR, const T* __restrict__ kt,
                                           const T* __restrict__ FW, T* __restrict__ y,
                                           long long c0, int nblk, int Nc, const DGTab<T>& tab,
                                           T* smem, const T* __restrict__ lineop = nullptr) {
  constexpr int N3 = N * N * N, C = Cfg<N>::CPB;
  T* su = smem;
  T* sx = su + C * N3;
  T* sr = sx + C * N3;
  T* sk = sr + C * N3;
  {
    const T* ub = U + c0 * N3;
    const T* xb = Xm + c0 * N3;
    const T* kb = kt + c0 * N3;
    for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) {
      su[t] = ub[t];
      sx[t] = xb[t];
      if (!LINEOP) sk[t] = kb[t];
    }
  }
  __syncthreads();
  if constexpr (LINEOP) {
    // the line operators hold the volume term and the own-side face terms
    const FaceNbr<T> fs{TR, FW};
    cell_core<N, T, FaceNbr<T>, true>(fs, y, c0, nblk, Nc, tab, su, sx, sr, sk, lineop);
  } else {
    const FaceGlobal<T> fs{TR, FW};
    cell_core<N, T, FaceGlobal<T>, false>(fs, y, c0, nblk, Nc, tab, su, sx, sr, sk, lineop);
  }
}

template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_cell(const T* __restrict__ U, const T* __restrict__ Xm, const T* __restrict__ TR,
       const T* __restrict__ kt, const T* __restrict__ FW, T* __restrict__ y, long long cbeg,
       long long cend, int Nc, const int* __restrict__ skip,
       const __grid_constant__ DGTab<T> tab) {
  constexpr int C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long c0 = cbeg + (long long)blockIdx.x * C;
  const int nblk = (int)((cend - c0) < C ? (cend - c0) : C);
  cell_cells<N, T>(U, Xm, TR, kt, FW, y, c0, nblk, Nc, tab, reinterpret_cast<T*>(smem_raw));
}

// Pass 2 with the precomputed line operators (FP64 path of dg_apply).
template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_cell_lo(const T* __restrict__ U, const T* __restrict__ Xm, const T* __restrict__ TR,
          const T* __restrict__ lineop, const T* __restrict__ FW, T* __restrict__ y,
          long long cbeg, long long cend, int Nc, const int* __restrict__ skip,
          const __grid_constant__ DGTab<T> tab) {
  constexpr int C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long c0 = cbeg + (long long)blockIdx.x * C;
  const int nblk = (int)((cend - c0) < C ? (cend - c0) : C);
  cell_cells<N, T, true>(U, Xm, TR, nullptr, FW, y, c0, nblk, Nc, tab,
                         reinterpret_cast<T*>(smem_raw), lineop);
}

// Line operators from Kt = h w K and h gamma (one thread per cell, direction
// and line):
//   x-line (b, e):  M[i][j] = sum_a L_i'(xi_a) Kt(a, b, e) L_j'(xi_a)   (acts on x-modes)
//   y-line (a, e):  M[i][j] = sum_f D[f][i] Kt(a, f, e) D[f][j]         (acts on nodal values)
//   z-line (a, b):  M[i][j] = sum_f D[f][i] Kt(a, b, f) D[f][j]
// plus the own-side part of the flux at the line's two face points, so that
// pass 2 only adds the neighbour part of interior faces (FaceNbr).
// Stored as lineop[((c*3 + dir)*n^2 + line)*n(n+1)/2 + packed(i, j)].
// NODAL: the line operators of Q A Q^T in the scaled Gauss-point basis
// (dg_nodal.cu): x-lines in the collocation form like y and z, every entry
// (i, j) of the line (s, t) multiplied by isw_i isw_j / (w_s w_t), which
// removes the tangential weights of Kt and of the face weight.
template <int N, bool NODAL = false>
__global__ void k_line_ops(const double* __restrict__ kt, const double* __restrict__ gh,
                           double* __restrict__ lineop, long long ncells, int Nc,
                           const __grid_constant__ DGTab<double> tab,
                           const __grid_constant__ DGTabN<double> tn) {
  constexpr int N2 = N * N, N3 = N * N * N, NP = N * (N + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells * 3 * N2) return;
  const long long c = t / (3 * N2);
  const int dir = (int)((t / N2) % 3);
  const int line = (int)(t % N2);
  const int p = line % N, q = line / N;
  double k[N];
#pragma unroll
  for (int f = 0; f < N; ++f) {
    // point index a + N(b + N e) along the line
    const int qi = dir == 0 ? f + N * (p + N * q)      // x-line (b = p, e = q)
                 : dir == 1 ? p + N * (f + N * q)      // y-line (a = p, e = q)
                            : p + N * (q + N * f);     // z-line (a = p, b = q)
    k[f] = kt[c * N3 + qi];
  }
  double* M = lineop + (t)*NP;
  // volume: M[i][j] = sum_f g_i(f) k_f g_j(f), with gk[i][f] = g_i(f) k_f formed once
  double gk[N][N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int f = 0; f < N; ++f)
      gk[i][f] = (dir == 0 && !NODAL ? tab.Bd[f][i] : tab.D[f][i]) * k[f];
  }
  // Own-side face terms of the line's two faces (both trial and test function
  // on this cell's side).  At the face point of this line, with v the test
  // values and d the test derivatives (d/dxi) at the face (modal a, L' on
  // x-lines; Lagrange l, l' on y- and z-lines), the flux adds
  //   Wh (2 sigma v v^T -+ c (v d^T + d v^T)),  Wh = h gamma_F w_s w_t / 2,
  // "-" on the upper face, "+" on the lower one, c = 1 inside and 2 on the
  // boundary (where the whole one-sided form is own-side).  Entry (i, j) of
  // each face term is v_i P_j + d_i Q_j with P = Wh (2 sigma v -+ c d) and
  // Q = -+ Wh c v.
  const long long crd = dir == 0 ? c % Nc : dir == 1 ? (c / Nc) % Nc : c / ((long long)Nc * Nc);
  const double w2 = tab.w[p] * tab.w[q];
  const double whl = 0.5 * gh[c * 6 + 2 * dir] * w2, whu = 0.5 * gh[c * 6 + 2 * dir + 1] * w2;
  const double cl = (crd > 0 ? 1.0 : 2.0) * whl, cu = (crd < Nc - 1 ? 1.0 : 2.0) * whu;
  constexpr double S2 = 4.0 * N * N;  // 2 sigma, sigma = 2 (k+1)^2
  double v0[N], d0[N], v1[N], d1[N], P0[N], Q0[N], P1[N], Q1[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const bool modal = dir == 0 && !NODAL;
    v0[j] = modal ? tab.a0[j] : tab.l0[j];
    d0[j] = modal ? tab.d0[j] : tab.dl0[j];
    v1[j] = modal ? tab.a1[j] : tab.l1[j];
    d1[j] = modal ? tab.d1[j] : tab.dl1[j];
    P0[j] = fma(whl * S2, v0[j], cl * d0[j]);
    Q0[j] = cl * v0[j];
    P1[j] = fma(whu * S2, v1[j], -cu * d1[j]);
    Q1[j] = -cu * v1[j];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = i; j < N; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int f = 0; f < N; ++f)
        acc = fma(gk[i][f], dir == 0 && !NODAL ? tab.Bd[f][j] : tab.D[f][j], acc);
      acc = fma(v0[i], P0[j], acc);
      acc = fma(d0[i], Q0[j], acc);
      acc = fma(v1[i], P1[j], acc);
      acc = fma(d1[i], Q1[j], acc);
      if (NODAL) acc *= (tn.isw[i] * tn.isw[j]) / w2;
      M[packed<N>(i, j)] = acc;
    }
  }
}

template <int N, typename T>
inline size_t trace_smem() { return sizeof(T) * Cfg<N>::CPB * N * N * N; }
template <int N, typename T>
inline size_t cell_smem() { return 4 * sizeof(T) * Cfg<N>::CPB * N * N * N; }

// Face-point weights from h*gamma per face side (one thread per cell).
template <typename T>
__global__ void k_face_weights(const double* __restrict__ gh, T* __restrict__ FW, int Nc, int n,
                               const __grid_constant__ DGTab<double> tab) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)Nc * Nc * Nc) return;
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  const int n2 = n * n;
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1;
    const bool upper = f & 1;
    const bool interior = upper ? (crd[d] < Nc - 1) : (crd[d] > 0);
    const double g = gh[c * 6 + f];
    for (int pt = 0; pt < n2; ++pt) {
      const double wh = 0.5 * g * tab.w[pt % n] * tab.w[pt / n];
      FW[(c * 12 + 2 * f) * n2 + pt] = (T)wh;
      FW[(c * 12 + 2 * f + 1) * n2 + pt] = (T)(interior ? wh : 2.0 * wh);
    }
  }
}


// Launch both passes for one precision.  U, X, TR: workspaces of the mesh.
template <int N, typename T>
cudaError_t launch_apply_n(const dg_mesh* m, const T* x, T* y, T* U, T* X, T* TR, const T* kt,
                           const T* fw, long long ncells, int Nc, const int* skip,
                           const DGTab<T>& tab, cudaStream_t s) {
  const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
  const size_t s1 = trace_smem<N, T>(), s2 = cell_smem<N, T>();
  dg_timing_mark(m, 0, s);
  k_trace<N, T><<<blocks, Cfg<N>::THREADS, s1, s>>>(x, U, X, TR, 0, ncells, skip, tab);
  dg_timing_mark(m, 1, s);
  if (sizeof(T) == 8 && m != nullptr && m->lineop64 != nullptr)
    k_cell_lo<N, T><<<blocks, Cfg<N>::THREADS, s2, s>>>(U, X, TR, (const T*)m->lineop64, fw, y,
                                                        0, ncells, Nc, skip, tab);
  else
    k_cell<N, T><<<blocks, Cfg<N>::THREADS, s2, s>>>(U, X, TR, kt, fw, y, 0, ncells, Nc, skip,
                                                     tab);
  dg_timing_mark(m, 2, s);
  return cudaGetLastError();
}

// One pass over the cells [cbeg, cend) (pipelined host-buffer apply).
// Pass 1 reads x and writes U, X, TR of those cells only; pass 2 reads the
// traces of their face neighbours, so it may run on a range only after pass 1
// has run on every neighbour of the range.
template <int N, typename T>
cudaError_t launch_pass_n(const dg_mesh* m, int pass, const T* x, T* y, T* U, T* X, T* TR,
                          const T* kt, const T* fw, long long cbeg, long long cend, int Nc,
                          const DGTab<T>& tab, cudaStream_t s) {
  if (cend <= cbeg) return cudaSuccess;
  const unsigned blocks = (unsigned)((cend - cbeg + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
  if (pass == 1)
    k_trace<N, T><<<blocks, Cfg<N>::THREADS, trace_smem<N, T>(), s>>>(x, U, X, TR, cbeg, cend,
                                                                       nullptr, tab);
  else if (sizeof(T) == 8 && m->lineop64 != nullptr)
    k_cell_lo<N, T><<<blocks, Cfg<N>::THREADS, cell_smem<N, T>(), s>>>(
        U, X, TR, (const T*)m->lineop64, fw, y, cbeg, cend, Nc, nullptr, tab);
  else
    k_cell<N, T><<<blocks, Cfg<N>::THREADS, cell_smem<N, T>(), s>>>(U, X, TR, kt, fw, y, cbeg,
                                                                     cend, Nc, nullptr, tab);
  return cudaGetLastError();
}

template <int N, typename T>
cudaError_t launch_trace_n(const T* x, T* U, T* X, T* TR, long long ncells, const DGTab<T>& tab,
                           cudaStream_t s) {
  const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
  k_trace<N, T><<<blocks, Cfg<N>::THREADS, trace_smem<N, T>(), s>>>(x, U, X, TR, 0, ncells,
                                                                     nullptr, tab);
  return cudaGetLastError();
}

template <typename T, template <int> class F, typename... Args>
cudaError_t dispatch_n(int n, Args... args) {
  switch (n) {
    case 2: return F<2>::template run<T>(args...);
    case 3: return F<3>::template run<T>(args...);
    case 4: return F<4>::template run<T>(args...);
    case 5: return F<5>::template run<T>(args...);
    case 6: return F<6>::template run<T>(args...);
    case 7: return F<7>::template run<T>(args...);
    case 8: return F<8>::template run<T>(args...);
    case 9: return F<9>::template run<T>(args...);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
struct ApplyF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const T* x, T* y, T* U, T* X, T* TR, const T* kt,
                         const T* fw, long long ncells, int Nc, const int* skip,
                         const DGTab<T>* tab, cudaStream_t s) {
    return launch_apply_n<N, T>(m, x, y, U, X, TR, kt, fw, ncells, Nc, skip, *tab, s);
  }
};

template <int N>
struct PassF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, int pass, const T* x, T* y, T* U, T* X, T* TR,
                         const T* kt, const T* fw, long long cbeg, long long cend, int Nc,
                         const DGTab<T>* tab, cudaStream_t s) {
    return launch_pass_n<N, T>(m, pass, x, y, U, X, TR, kt, fw, cbeg, cend, Nc, *tab, s);
  }
};

// Opt in to the dynamic shared memory the kernels use (above 48 KB for large n).
template <int N>
struct PrepareF {
  template <typename T>
  static cudaError_t run() {
    cudaError_t e = cudaFuncSetAttribute(k_cell<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cell_smem<N, T>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_cell_lo<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)cell_smem<N, T>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_trace<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)trace_smem<N, T>());
    return e;
  }
};

template <int N>
struct TraceF {
  template <typename T>
  static cudaError_t run(const T* x, T* U, T* X, T* TR, long long ncells, const DGTab<T>* tab,
                         cudaStream_t s) {
    return launch_trace_n<N, T>(x, U, X, TR, ncells, *tab, s);
  }
};

}  // namespace dgk

namespace dgk {
template <int N>
struct LineOpsF {
  template <typename T>
  static cudaError_t run(const double* kt, const double* gh, double* lineop, long long ncells,
                         int Nc, const DGTab<double>* tab, cudaStream_t s) {
    const long long threads = ncells * 3 * N * N;
    k_line_ops<N><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(kt, gh, lineop, ncells, Nc,
                                                                    *tab, DGTabN<double>{});
    return cudaGetLastError();
  }
};
}  // namespace dgk
