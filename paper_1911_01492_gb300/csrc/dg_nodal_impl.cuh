// The two FP64 passes of the operator in the scaled Gauss-point basis, as
// block-level device functions over a group of up to CPB cells (used by the
// stand-alone kernels of dg_nodal.cu and by the batched persistent kernel).
// The basis, its scaling and the derivation of the data are described in
// dg_nodal.cu.  Every thread of the block calls these functions (they hold
// block barriers); threads beyond the group's n^2 lines per cell only take
// part in the loads and barriers.
#pragma once

#include "dg_apply_impl.cuh"

namespace dgk {

// Pass 1: the value and half the reference normal derivative of u_h on the six
// faces, TR[c][2f + {0, 1}][n^2] (the layout of the Legendre-basis pass), from
// each line's scaled point values with the scaled Lagrange end values.  The
// stored traces lack the tangential factor isw_s isw_t, which the face weight
// absorbs in pass 2; the factor 1/2 is the average's (pass 2 then multiplies
// by h gamma instead of h gamma / 2).  s: CPB n^3 values of shared memory.
template <int N, typename T>
__device__ __forceinline__ void trace_cells_nd(const T* __restrict__ x, T* __restrict__ TR,
                                               long long c0, int nblk, const DGTabN<T>& tn,
                                               T* s) {
  constexpr int N2 = N * N, N3 = N * N * N;
  {
    const T* xb = x + c0 * N3;
    for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) s[t] = xb[t];
  }
  __syncthreads();
  const int lc = threadIdx.x / N2;
  if (lc >= nblk) return;  // no barrier follows
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N, pt = t2;
  const T* sc = s + lc * N3;
  T* tr = TR + (c0 + lc) * (12 * N2);
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    // x-line (b = p, e = q), y-line (a = p, e = q), z-line (a = p, b = q)
    const int base = dir == 0 ? q * N2 + p * N : dir == 1 ? q * N2 + p : q * N + p;
    const int step = dir == 0 ? 1 : dir == 1 ? N : N2;
    T u[N];
#pragma unroll
    for (int e = 0; e < N; ++e) u[e] = sc[base + e * step];
    T vm = tn.l0[0] * u[0], vp = tn.l1[0] * u[0];
    T gm = tn.hdl0[0] * u[0], gp = tn.hdl1[0] * u[0];
#pragma unroll
    for (int e = 1; e < N; ++e) {
      vm = fma(tn.l0[e], u[e], vm);
      vp = fma(tn.l1[e], u[e], vp);
      gm = fma(tn.hdl0[e], u[e], gm);
      gp = fma(tn.hdl1[e], u[e], gp);
    }
    tr[(4 * dir + 0) * N2 + pt] = vm;  // lower face: value, derivative / 2
    tr[(4 * dir + 1) * N2 + pt] = gm;
    tr[(4 * dir + 2) * N2 + pt] = vp;  // upper face
    tr[(4 * dir + 3) * N2 + pt] = gp;
  }
}

// Pass 2: per line r = M u with the precomputed symmetric line operator of
// Q A Q^T (volume term and own-side face terms), plus the neighbour part of
// the line's two interior faces, summed over the z-, y- and x-lines through
// every point.  The z-line threads read their lines from global memory and
// publish them in shared memory for the other two directions; the partial
// sums stay in shared memory; the x-line threads write y.  smem: 2 CPB n^3
// doubles.
template <int N>
__device__ __forceinline__ void cell_cells_nd(const double* __restrict__ x,
                                              const double* __restrict__ TR,
                                              const double* __restrict__ lineop,
                                              const double* __restrict__ gh,
                                              double* __restrict__ y, long long c0, int nblk,
                                              int Nc, const DGTabN<double>& tn, double* smem) {
  constexpr int C = Cfg<N>::CPB, N2 = N * N, N3 = N * N * N, NP = N * (N + 1) / 2;
  constexpr double S2 = 4.0 * N * N;  // 2 sigma, sigma = 2 (k+1)^2
  double* su = smem;
  double* sr = su + C * N3;
  __shared__ int sbase[3];
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N, pt = t2;
  const bool active = lc < nblk;
  const long long c = c0 + lc;
  const int o = lc * N3;
  if (threadIdx.x == 0) {
    const unsigned cu = (unsigned)c0, n = (unsigned)Nc;
    sbase[0] = (int)(cu % n);
    sbase[1] = (int)((cu / n) % n);
    sbase[2] = (int)(cu / n / n);
  }
  // z-lines (a = p, b = q) from global memory
  double u[N];
  if (active) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
      u[e] = x[c * N3 + e * N2 + q * N + p];
      su[o + e * N2 + q * N + p] = u[e];
    }
  }
  __syncthreads();
  int crd[3] = {sbase[0] + lc, sbase[1], sbase[2]};
  while (crd[0] >= Nc) {
    crd[0] -= Nc;
    if (++crd[1] == Nc) {
      crd[1] = 0;
      ++crd[2];
    }
  }
  const long long stride[3] = {1, Nc, (long long)Nc * Nc};
  // r = r0 + M u + the neighbour terms of the line's faces 2 dir (lower) and
  // 2 dir + 1 (upper); r0: the partial sums of the directions already done
  // (none for the first).  The neighbour's trace (un, gn/2) comes with the
  // derivative halved (pass 1), and g = h gamma is the face weight h gamma / 2
  // times 2, so with l, dl the scaled end values:
  //   upper face (this cell the (-) side):
  //     r += -l1 g (sigma un + gn/2) + (dl1/2) g un,
  //   lower face (this cell the (+) side):
  //     r += l0 g (gn/2 - sigma un) - (dl0/2) g un.
  auto line = [&](int dir, const double* r0, double (&r)[N]) {
    const double* Mp = lineop + ((c * 3 + dir) * N2 + pt) * NP;
    double Mv[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) Mv[t] = Mp[t];
    double cv1 = 0.0, cd1 = 0.0, cv0 = 0.0, cd0 = 0.0;
    if (crd[dir] < Nc - 1) {  // upper face: this cell is the (-) side
      double un, gn;
      load_trace<N>(TR, c + stride[dir], 2 * dir, pt, un, gn);
      const double g = gh[c * 6 + 2 * dir + 1];
      cv1 = g * fma(0.5 * S2, un, gn);  // enters with -l1
      cd1 = g * un;                     // enters with +dl1 / 2
    }
    if (crd[dir] > 0) {  // lower face: this cell is the (+) side
      double un, gn;
      load_trace<N>(TR, c - stride[dir], 2 * dir + 1, pt, un, gn);
      const double g = gh[c * 6 + 2 * dir];
      cv0 = g * fma(-0.5 * S2, un, gn);  // enters with +l0
      cd0 = g * un;                      // enters with -dl0 / 2
    }
#pragma unroll
    for (int e = 0; e < N; ++e) {
      double acc = r0 != nullptr ? fma(-tn.l1[e], cv1, r0[e]) : -tn.l1[e] * cv1;
      acc = fma(tn.hdl1[e], cd1, acc);
      acc = fma(tn.l0[e], cv0, acc);
      acc = fma(-tn.hdl0[e], cd0, acc);
#pragma unroll
      for (int f = 0; f < N; ++f) acc = fma(Mv[packed<N>(e, f)], u[f], acc);
      r[e] = acc;
    }
  };
  if (active) {  // z-lines
    double r[N];
    line(2, nullptr, r);
#pragma unroll
    for (int e = 0; e < N; ++e) sr[o + e * N2 + q * N + p] = r[e];
  }
  __syncthreads();
  if (active) {  // y-lines (a = p, e = q), continuing the z-lines' sums
    double r0[N], r[N];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      u[b] = su[o + q * N2 + b * N + p];
      r0[b] = sr[o + q * N2 + b * N + p];
    }
    line(1, r0, r);
#pragma unroll
    for (int b = 0; b < N; ++b) sr[o + q * N2 + b * N + p] = r[b];
  }
  __syncthreads();
  if (active) {  // x-lines (b = p, e = q): the sum of all three directions
    double r0[N], r[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      u[a] = su[o + q * N2 + p * N + a];
      r0[a] = sr[o + q * N2 + p * N + a];
    }
    line(0, r0, r);
#pragma unroll
    for (int a = 0; a < N; ++a) y[c * N3 + q * N2 + p * N + a] = r[a];
  }
}

template <int N, typename T>
inline size_t trace_smem_nd() { return sizeof(T) * Cfg<N>::CPB * N * N * N; }
template <int N>
inline size_t cell_smem_nd() { return 2 * sizeof(double) * Cfg<N>::CPB * N * N * N; }

}  // namespace dgk
