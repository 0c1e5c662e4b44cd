// Batched CG over independent samples (persistent lock-step kernel).
#include "dg_internal.cuh"

extern "C" int dg_cg_solve_batched(const dg_mesh* const* meshes, int count, const double* const* b,
                                   double* const* x, double rtol, int maxit, dg_cg_stats* st,
                                   void* stream) {
  (void)meshes; (void)count; (void)b; (void)x; (void)rtol; (void)maxit; (void)st; (void)stream;
  return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: not built yet");
}
