// Packed FP32 pairs for the mixed CG's cell kernel.
//
// Blackwell executes two FP32 fused multiply-adds (or adds, or multiplies) in
// one instruction (FFMA2, FADD2, FMUL2), each lane rounded to nearest exactly
// as the scalar instruction would.  The FP32 cell kernel is bound by
// instruction issue, so it processes two cells per thread: every value is a
// pair (cell a, cell b) and every arithmetic instruction, shared-memory access
// (64-bit) and address computation serves both cells.
//
// F2 wraps float2 so that the generic line contractions of dg_apply_impl.cuh
// (templated on the value type; their unqualified fma() finds the overload
// below by argument-dependent lookup) run on pairs unchanged.  This header is
// included after dg_apply_impl.cuh.
#pragma once

#include "dg_apply_impl.cuh"

namespace dgk {

struct __align__(8) F2 {
  float2 v;
  F2() = default;
  __host__ __device__ constexpr F2(float a) : v{a, a} {}
  __host__ __device__ constexpr F2(float a, float b) : v{a, b} {}
  __host__ __device__ explicit constexpr F2(int a) : v{(float)a, (float)a} {}
};

__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
  F2 r;
  r.v = __ffma2_rn(a.v, b.v, c.v);
  return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  r.v = __fadd2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  r.v = __fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  r.v = __fmul2_rn(a.v, b.v);
  return r;
}

// Host: the FP32 tables with every entry duplicated into both lanes.
inline void pair_tables(const DGTab<float>& s, DGTab<F2>* d) {
  for (int a = 0; a < DG_MAXN; ++a) {
    for (int b = 0; b < DG_MAXN; ++b) {
      d->B[a][b] = F2(s.B[a][b]);
      d->Bd[a][b] = F2(s.Bd[a][b]);
      d->D[a][b] = F2(s.D[a][b]);
    }
    d->w[a] = F2(s.w[a]);
    d->a0[a] = F2(s.a0[a]);
    d->a1[a] = F2(s.a1[a]);
    d->d0[a] = F2(s.d0[a]);
    d->d1[a] = F2(s.d1[a]);
    d->l0[a] = F2(s.l0[a]);
    d->l1[a] = F2(s.l1[a]);
    d->dl0[a] = F2(s.dl0[a]);
    d->dl1[a] = F2(s.dl1[a]);
  }
  d->sigma = F2(s.sigma);
}

}  // namespace dgk
