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
// h w_q K_q, its own face traces and its six neighbours' face traces, and forms
//   r = sum_d D_d^T (Kt . D_d u)  (collocation derivative along y and z,
//       L_i' contraction from X along x),
// adds the face terms -{d_n u}[phi] - {d_n phi}[u] + sigma [u][phi] with weight
// h gamma_F w_s w_t at each face point, and maps back to modal coefficients
// with B^T along x, y, z.  No FP64 work is repeated between the passes: the
// only duplicated arithmetic is the pointwise flux of an interior face, which
// both of its cells evaluate.
//
// Thread layout: n^2 threads per cell; a block holds CPB cells.  Each thread
// owns one 1D line of its cell at every stage; lines are exchanged through
// shared memory between stages.
#pragma once

#include "dg_internal.cuh"

namespace dgk {

template <int N>
struct Cfg {
  // cells per block, chosen so a block has ~128-256 threads
  static constexpr int CPB = (N == 2) ? 32 : (N == 3) ? 14 : (N == 4) ? 8 : (N == 5) ? 5
                           : (N == 6) ? 4 : (N == 7) ? 3 : 2;
  static constexpr int THREADS = CPB * N * N;
};

// Face flux at one face point (reference units: derivatives d/dxi along +axis,
// weight W = h gamma_F w_s w_t).  `upper`: this cell is the lower-index (-)
// side of the face (its xi = 1 face).  Interior:  J = u- - u+, G = g- + g+,
//   s_v = W (sigma J - G/2),  s_d = -W J / 2;
// the (-) cell adds  s_v phi + s_d dphi, the (+) cell  -s_v phi + s_d dphi.
// Boundary faces are the one-sided form with outward normal:
//   -(d_n u) phi - (d_n phi) u + sigma u phi,
// obtained from the same expressions with the missing side's value set to 0,
// its derivative set to the own one, and the factor 1/2 of s_d replaced by 1.
// Returns the multipliers (cv, cd) of the own test function's value and
// reference normal derivative.
template <bool UPPER, typename T>
__device__ __forceinline__ void face_flux(bool interior, T uo, T go, T un, T gn, T W, T sigma,
                                          T& cv, T& cd) {
  T um, gm, up, gp;
  if (UPPER) {
    um = uo; gm = go;
    up = interior ? un : T(0);
    gp = interior ? gn : go;
  } else {
    up = uo; gp = go;
    um = interior ? un : T(0);
    gm = interior ? gn : go;
  }
  const T J = um - up;
  const T G = gm + gp;
  const T sv = W * (sigma * J - T(0.5) * G);
  const T hw = interior ? T(-0.5) * W : -W;
  cv = UPPER ? sv : -sv;
  cd = hw * J;
}

// ---------------------------------------------------------------------------
// Pass 1: nodal values and face traces.
// TR layout: TR[((c*6 + f)*2 + comp)*n^2 + pt], f = x-, x+, y-, y+, z-, z+,
// comp 0 = value, 1 = d/dxi along +axis; pt = (b + n e) on x-faces,
// (a + n e) on y-faces, (a + n b) on z-faces.
// ---------------------------------------------------------------------------
template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_trace(const T* __restrict__ x, T* __restrict__ U, T* __restrict__ Xm, T* __restrict__ TR,
        long long ncells, const int* __restrict__ skip, const __grid_constant__ DGTab<T> tab) {
  constexpr int N2 = N * N, N3 = N * N * N, C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  const T* xb = x + c0 * N3;
  for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) s[t] = xb[t];
  __syncthreads();

  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  T* sc = s + lc * N3;
  const long long c = c0 + lc;

  // along z: thread owns (i = p, j = q)
  if (active) {
    T v[N];
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = sc[l * N2 + q * N + p];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      T acc = tab.B[e][0] * v[0];
#pragma unroll
      for (int l = 1; l < N; ++l) acc = fma(tab.B[e][l], v[l], acc);
      sc[e * N2 + q * N + p] = acc;
    }
  }
  __syncthreads();
  // along y: thread owns (i = p, e = q)
  if (active) {
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = sc[q * N2 + j * N + p];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T acc = tab.B[b][0] * v[0];
#pragma unroll
      for (int j = 1; j < N; ++j) acc = fma(tab.B[b][j], v[j], acc);
      sc[q * N2 + b * N + p] = acc;
    }
  }
  __syncthreads();
  // along x: thread owns (b = p, e = q); X is modal in x, nodal in y and z
  T* tr = TR + c * (12 * N2);
  if (active) {
    T X[N];
#pragma unroll
    for (int i = 0; i < N; ++i) X[i] = sc[q * N2 + p * N + i];
    T* xm = Xm + c * N3 + q * N2 + p * N;
#pragma unroll
    for (int i = 0; i < N; ++i) xm[i] = X[i];
    T vm = tab.a0[0] * X[0], vp = tab.a1[0] * X[0];
    T gm = tab.d0[0] * X[0], gp = tab.d1[0] * X[0];
#pragma unroll
    for (int i = 1; i < N; ++i) {
      vm = fma(tab.a0[i], X[i], vm);
      vp = fma(tab.a1[i], X[i], vp);
      gm = fma(tab.d0[i], X[i], gm);
      gp = fma(tab.d1[i], X[i], gp);
    }
    const int pt = p + N * q;
    tr[0 * N2 + pt] = vm;
    tr[1 * N2 + pt] = gm;
    tr[2 * N2 + pt] = vp;
    tr[3 * N2 + pt] = gp;
    T* ug = U + c * N3 + q * N2 + p * N;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T acc = tab.B[a][0] * X[0];
#pragma unroll
      for (int i = 1; i < N; ++i) acc = fma(tab.B[a][i], X[i], acc);
      sc[q * N2 + p * N + a] = acc;
      ug[a] = acc;
    }
  }
  __syncthreads();
  if (active) {
    // y-faces: thread owns points (a = p, e = q)
    {
      T u[N];
#pragma unroll
      for (int b = 0; b < N; ++b) u[b] = sc[q * N2 + b * N + p];
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
      tr[4 * N2 + pt] = vm;
      tr[5 * N2 + pt] = gm;
      tr[6 * N2 + pt] = vp;
      tr[7 * N2 + pt] = gp;
    }
    // z-faces: thread owns points (a = p, b = q)
    {
      T u[N];
#pragma unroll
      for (int e = 0; e < N; ++e) u[e] = sc[e * N2 + q * N + p];
      T vm = tab.l0[0] * u[0], vp = tab.l1[0] * u[0];
      T gm = tab.dl0[0] * u[0], gp = tab.dl1[0] * u[0];
#pragma unroll
      for (int e = 1; e < N; ++e) {
        vm = fma(tab.l0[e], u[e], vm);
        vp = fma(tab.l1[e], u[e], vp);
        gm = fma(tab.dl0[e], u[e], gm);
        gp = fma(tab.dl1[e], u[e], gp);
      }
      const int pt = p + N * q;
      tr[8 * N2 + pt] = vm;
      tr[9 * N2 + pt] = gm;
      tr[10 * N2 + pt] = vp;
      tr[11 * N2 + pt] = gp;
    }
  }
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

// ---------------------------------------------------------------------------
// Pass 2: volume and face terms, back to modal coefficients.
// ---------------------------------------------------------------------------
template <int N, typename T>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_cell(const T* __restrict__ U, const T* __restrict__ Xm, const T* __restrict__ TR,
       const T* __restrict__ kt, const T* __restrict__ gh, T* __restrict__ y, long long ncells,
       int Nc, const int* __restrict__ skip, const __grid_constant__ DGTab<T> tab) {
  constexpr int N2 = N * N, N3 = N * N * N, C = Cfg<N>::CPB;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sx = su + C * N3;
  T* sr = sx + C * N3;
  T* sk = sr + C * N3;
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  {
    const T* ub = U + c0 * N3;
    const T* xb = Xm + c0 * N3;
    const T* kb = kt + c0 * N3;
    for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) {
      su[t] = ub[t];
      sx[t] = xb[t];
      sk[t] = kb[t];
    }
  }
  __syncthreads();

  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  const long long c = c0 + lc;
  const int cx = (int)(c % Nc);
  const int cy = (int)((c / Nc) % Nc);
  const int cz = (int)(c / ((long long)Nc * Nc));
  const long long sy = Nc, sz = (long long)Nc * Nc;
  const int o = lc * N3;
  const T sigma = tab.sigma;
  const T* ghc = gh + c * 6;

  // z-lines: thread owns (a = p, b = q)
  if (active) {
    T u[N], kg[N], r[N];
#pragma unroll
    for (int e = 0; e < N; ++e) u[e] = su[o + e * N2 + q * N + p];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      T g = tab.D[e][0] * u[0];
#pragma unroll
      for (int f = 1; f < N; ++f) g = fma(tab.D[e][f], u[f], g);
      kg[e] = sk[o + e * N2 + q * N + p] * g;
    }
#pragma unroll
    for (int e = 0; e < N; ++e) {
      T acc = tab.D[0][e] * kg[0];
#pragma unroll
      for (int f = 1; f < N; ++f) acc = fma(tab.D[f][e], kg[f], acc);
      r[e] = acc;
    }
    const int pt = p + N * q;
    const T ww = tab.w[p] * tab.w[q];
    {  // z+ face: this cell is the (-) side
      const bool in = cz < Nc - 1;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 5, pt, uo, go);
      if (in) load_trace<N>(TR, c + sz, 4, pt, un, gn);
      T cv, cd;
      face_flux<true>(in, uo, go, un, gn, ghc[5] * ww, sigma, cv, cd);
#pragma unroll
      for (int e = 0; e < N; ++e) r[e] = fma(tab.l1[e], cv, fma(tab.dl1[e], cd, r[e]));
    }
    {  // z- face: this cell is the (+) side
      const bool in = cz > 0;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 4, pt, uo, go);
      if (in) load_trace<N>(TR, c - sz, 5, pt, un, gn);
      T cv, cd;
      face_flux<false>(in, uo, go, un, gn, ghc[4] * ww, sigma, cv, cd);
#pragma unroll
      for (int e = 0; e < N; ++e) r[e] = fma(tab.l0[e], cv, fma(tab.dl0[e], cd, r[e]));
    }
#pragma unroll
    for (int e = 0; e < N; ++e) sr[o + e * N2 + q * N + p] = r[e];
  }
  __syncthreads();
  // y-lines: thread owns (a = p, e = q)
  if (active) {
    T u[N], kg[N], r[N];
#pragma unroll
    for (int b = 0; b < N; ++b) u[b] = su[o + q * N2 + b * N + p];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T g = tab.D[b][0] * u[0];
#pragma unroll
      for (int f = 1; f < N; ++f) g = fma(tab.D[b][f], u[f], g);
      kg[b] = sk[o + q * N2 + b * N + p] * g;
    }
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T acc = sr[o + q * N2 + b * N + p];
#pragma unroll
      for (int f = 0; f < N; ++f) acc = fma(tab.D[f][b], kg[f], acc);
      r[b] = acc;
    }
    const int pt = p + N * q;
    const T ww = tab.w[p] * tab.w[q];
    {  // y+ face
      const bool in = cy < Nc - 1;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 3, pt, uo, go);
      if (in) load_trace<N>(TR, c + sy, 2, pt, un, gn);
      T cv, cd;
      face_flux<true>(in, uo, go, un, gn, ghc[3] * ww, sigma, cv, cd);
#pragma unroll
      for (int b = 0; b < N; ++b) r[b] = fma(tab.l1[b], cv, fma(tab.dl1[b], cd, r[b]));
    }
    {  // y- face
      const bool in = cy > 0;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 2, pt, uo, go);
      if (in) load_trace<N>(TR, c - sy, 3, pt, un, gn);
      T cv, cd;
      face_flux<false>(in, uo, go, un, gn, ghc[2] * ww, sigma, cv, cd);
#pragma unroll
      for (int b = 0; b < N; ++b) r[b] = fma(tab.l0[b], cv, fma(tab.dl0[b], cd, r[b]));
    }
#pragma unroll
    for (int b = 0; b < N; ++b) sr[o + q * N2 + b * N + p] = r[b];
  }
  __syncthreads();
  // x-lines: thread owns (b = p, e = q); result is x-modal, yz-nodal
  if (active) {
    T X[N], kg[N], R[N];
#pragma unroll
    for (int i = 0; i < N; ++i) X[i] = sx[o + q * N2 + p * N + i];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T g = tab.Bd[a][0] * X[0];
#pragma unroll
      for (int i = 1; i < N; ++i) g = fma(tab.Bd[a][i], X[i], g);
      kg[a] = sk[o + q * N2 + p * N + a] * g;
    }
    T rr[N];
#pragma unroll
    for (int a = 0; a < N; ++a) rr[a] = sr[o + q * N2 + p * N + a];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T acc = tab.Bd[0][i] * kg[0];
#pragma unroll
      for (int a = 1; a < N; ++a) acc = fma(tab.Bd[a][i], kg[a], acc);
#pragma unroll
      for (int a = 0; a < N; ++a) acc = fma(tab.B[a][i], rr[a], acc);
      R[i] = acc;
    }
    const int pt = p + N * q;
    const T ww = tab.w[p] * tab.w[q];
    {  // x+ face
      const bool in = cx < Nc - 1;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 1, pt, uo, go);
      if (in) load_trace<N>(TR, c + 1, 0, pt, un, gn);
      T cv, cd;
      face_flux<true>(in, uo, go, un, gn, ghc[1] * ww, sigma, cv, cd);
#pragma unroll
      for (int i = 0; i < N; ++i) R[i] = fma(tab.a1[i], cv, fma(tab.d1[i], cd, R[i]));
    }
    {  // x- face
      const bool in = cx > 0;
      T uo, go, un = T(0), gn = T(0);
      load_trace<N>(TR, c, 0, pt, uo, go);
      if (in) load_trace<N>(TR, c - 1, 1, pt, un, gn);
      T cv, cd;
      face_flux<false>(in, uo, go, un, gn, ghc[0] * ww, sigma, cv, cd);
#pragma unroll
      for (int i = 0; i < N; ++i) R[i] = fma(tab.a0[i], cv, fma(tab.d0[i], cd, R[i]));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) sx[o + q * N2 + p * N + i] = R[i];
  }
  __syncthreads();
  // back along y: thread owns (i = p, e = q)
  if (active) {
    T v[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = sx[o + q * N2 + b * N + p];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T acc = tab.B[0][j] * v[0];
#pragma unroll
      for (int b = 1; b < N; ++b) acc = fma(tab.B[b][j], v[b], acc);
      sx[o + q * N2 + j * N + p] = acc;
    }
  }
  __syncthreads();
  // back along z: thread owns (i = p, j = q)
  if (active) {
    T v[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sx[o + e * N2 + q * N + p];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      T acc = tab.B[0][l] * v[0];
#pragma unroll
      for (int e = 1; e < N; ++e) acc = fma(tab.B[e][l], v[e], acc);
      sx[o + l * N2 + q * N + p] = acc;
    }
  }
  __syncthreads();
  T* yb = y + c0 * N3;
  for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) yb[t] = sx[t];
}

template <int N, typename T>
inline size_t trace_smem() { return sizeof(T) * Cfg<N>::CPB * N * N * N; }
template <int N, typename T>
inline size_t cell_smem() { return 4 * sizeof(T) * Cfg<N>::CPB * N * N * N; }

// Launch both passes for one precision.  U, X, TR: workspaces of the mesh.
template <int N, typename T>
cudaError_t launch_apply_n(const dg_mesh* m, const T* x, T* y, T* U, T* X, T* TR, const T* kt,
                           const T* gh, long long ncells, int Nc, const int* skip,
                           const DGTab<T>& tab, cudaStream_t s) {
  const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
  const size_t s1 = trace_smem<N, T>(), s2 = cell_smem<N, T>();
  dg_timing_mark(m, 0, s);
  k_trace<N, T><<<blocks, Cfg<N>::THREADS, s1, s>>>(x, U, X, TR, ncells, skip, tab);
  dg_timing_mark(m, 1, s);
  k_cell<N, T><<<blocks, Cfg<N>::THREADS, s2, s>>>(U, X, TR, kt, gh, y, ncells, Nc, skip, tab);
  dg_timing_mark(m, 2, s);
  return cudaGetLastError();
}

template <int N, typename T>
cudaError_t launch_trace_n(const T* x, T* U, T* X, T* TR, long long ncells, const DGTab<T>& tab,
                           cudaStream_t s) {
  const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
  k_trace<N, T><<<blocks, Cfg<N>::THREADS, trace_smem<N, T>(), s>>>(x, U, X, TR, ncells, nullptr,
                                                                     tab);
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
                         const T* gh, long long ncells, int Nc, const int* skip,
                         const DGTab<T>* tab, cudaStream_t s) {
    return launch_apply_n<N, T>(m, x, y, U, X, TR, kt, gh, ncells, Nc, skip, *tab, s);
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
