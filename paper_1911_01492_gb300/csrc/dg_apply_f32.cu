// FP32 instantiation of the two-pass operator application (FP32 tables,
// coefficients and accumulation).
#include "dg_apply_impl.cuh"

int dg_launch_apply_f32(const dg_mesh* m, const float* x, float* y, const int* skip,
                        cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<float, dgk::ApplyF>(m->n, m, x, y, m->U32, m->X32, m->TR32,
                                                      (const float*)m->kt32,
                                                      (const float*)m->fw32, m->ncells, m->N,
                                                      skip, &m->tab32, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply (fp32) launch");
  return DG_OK;
}

int dg_launch_pass_f32(const dg_mesh* m, int pass, const float* x, float* y, long long cbeg,
                       long long cend, cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<float, dgk::PassF>(m->n, m, pass, x, y, m->U32, m->X32,
                                                     m->TR32, (const float*)m->kt32,
                                                     (const float*)m->fw32, cbeg, cend, m->N,
                                                     &m->tab32, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply pass (fp32) launch");
  return DG_OK;
}

int dg_prepare_apply_f32(int n) {
  cudaError_t e = dgk::dispatch_n<float, dgk::PrepareF>(n);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply (fp32) kernel attributes");
  return DG_OK;
}
