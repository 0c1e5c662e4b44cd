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
// (templated on the value type; their unqualified fma() finds the overloads
// below by argument-dependent lookup) run on pairs unchanged, with the scalar
// FP32 tables: a table entry is a scalar broadcast into both lanes.  Measured
// on GB300: FFMA2 with a broadcast kernel-parameter constant issues one
// instruction per pair of FMAs, while a packed pair constant from the kernel
// parameters costs an extra move per FFMA2 and ran at half the scalar rate.
// This header is included after dg_apply_impl.cuh.
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

// A scalar table entry times a pair: the entry is broadcast into both lanes,
// which the packed instructions take as an operand directly (no extra move).
__device__ __forceinline__ F2 fma(float a, F2 b, F2 c) {
  F2 r;
  r.v = __ffma2_rn(make_float2(a, a), b.v, c.v);
  return r;
}
__device__ __forceinline__ F2 operator*(float a, F2 b) {
  F2 r;
  r.v = __fmul2_rn(make_float2(a, a), b.v);
  return r;
}

}  // namespace dgk
