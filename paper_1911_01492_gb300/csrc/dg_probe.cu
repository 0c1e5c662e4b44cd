// Arithmetic-throughput probes for measurement tools (the paper has no
// counterpart).  The benchmark divides the executed FP64 (or FP32) operation
// rate of the operator kernels by a peak measured on the same GPU in the same
// run, rather than by a nominal datasheet figure.
//
// Each probe kernel runs independent chains of fused multiply-adds in every
// thread of a grid that fills the GPU (8 blocks of 256 threads per SM), so the
// arithmetic pipe, not latency, bounds it.  The chains depend on a kernel
// argument and end in a conditional store, so the compiler can neither fold
// nor drop them.  The result is the best of several timed launches (CUDA
// events on the caller's stream), in TFLOP/s with an FMA counted as 2 flops.
#include "dg_internal.cuh"

namespace {

constexpr int kChains = 8;        // independent accumulators per thread
constexpr int kIters = 2048;      // loop trips per launch
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_f64(double a, double b, double* sink) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = b + c * 1e-3 + threadIdx.x * 1e-9;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == 12345.678) sink[0] = s;  // never true for the probe's arguments
}

__global__ void __launch_bounds__(kThreads) k_peak_f32(float a, float b, float* sink) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = b + c * 1e-3f + threadIdx.x * 1e-7f;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == 12345.678f) sink[0] = s;
}

// Packed FP32x2 fused multiply-add (two lanes per instruction).
__global__ void __launch_bounds__(kThreads) k_peak_f32x2(float a, float b, float* sink) {
  float2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    acc[c] = make_float2(b + c * 1e-3f + threadIdx.x * 1e-7f, b - c * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
  if (s == 12345.678f) sink[0] = s;
}

}  // namespace

extern "C" int dg_peak_probe(int kind, double* tflops, void* stream) {
  if (tflops == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_peak_probe: tflops is NULL");
  if (kind < 0 || kind > 2)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_peak_probe: kind=%d is not 0 (FP64), 1 (FP32) or "
                                       "2 (FP32x2)", kind);
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)(8 * sms);
  void* sink = nullptr;
  DG_CUDA(cudaMalloc(&sink, 64));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_ms = 1e300;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e != cudaSuccess) break;
    if (kind == 0)
      k_peak_f64<<<blocks, kThreads, 0, s>>>(0.999999, 1e-6, (double*)sink);
    else if (kind == 1)
      k_peak_f32<<<blocks, kThreads, 0, s>>>(0.9999f, 1e-4f, (float*)sink);
    else
      k_peak_f32x2<<<blocks, kThreads, 0, s>>>(0.9999f, 1e-4f, (float*)sink);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;  // rep 0 warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return dg_cuda_fail(e, "dg_peak_probe");
  const double lanes = kind == 2 ? 2.0 : 1.0;
  const double flops = 2.0 * lanes * kChains * (double)kIters * kThreads * blocks;
  *tflops = flops / (best_ms * 1e-3) / 1e12;
  return DG_OK;
}
