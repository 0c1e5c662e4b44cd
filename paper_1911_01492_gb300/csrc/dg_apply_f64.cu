// FP64 instantiation of the two-pass operator application.
#include "dg_apply_impl.cuh"

int dg_launch_apply_f64(const dg_mesh* m, const double* x, double* y, const int* skip,
                        cudaStream_t s) {
  // inside a solve in the scaled Gauss-point basis (DG_CG_NODAL): Q A Q^T
  if (m != nullptr && m->nodal_op) return dg_launch_apply_nodal_f64(m, x, y, skip, s);
  if (m != nullptr && m->multilinear) return dg_launch_apply_multilinear(m, x, y, skip, s);
  if (m != nullptr && m->affine) return dg_launch_apply_affine(m, x, y, skip, s);
  cudaError_t e = dgk::dispatch_n<double, dgk::ApplyF>(m->n, m, x, y, m->U64, m->X64, m->TR64,
                                                       (const double*)m->kt64,
                                                       (const double*)m->fw64, m->ncells, m->N,
                                                       skip, &m->tab64, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply (fp64) launch");
  return DG_OK;
}

int dg_launch_trace_f64(const dg_mesh* m, const double* x, double* U, double* X, double* TR,
                        cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, dgk::TraceF>(m->n, x, U, X, TR, m->ncells, &m->tab64, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "trace (fp64) launch");
  return DG_OK;
}

int dg_launch_pass_f64(const dg_mesh* m, int pass, const double* x, double* y, long long cbeg,
                       long long cend, cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, dgk::PassF>(m->n, m, pass, x, y, m->U64, m->X64,
                                                      m->TR64, (const double*)m->kt64,
                                                      (const double*)m->fw64, cbeg, cend, m->N,
                                                      &m->tab64, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply pass (fp64) launch");
  return DG_OK;
}

int dg_prepare_apply_f64(int n) {
  cudaError_t e = dgk::dispatch_n<double, dgk::PrepareF>(n);
  if (e != cudaSuccess) return dg_cuda_fail(e, "apply (fp64) kernel attributes");
  return DG_OK;
}
