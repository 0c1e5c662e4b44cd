// dg_apply_static: the FP64 operator application for callers that cannot
// allocate device memory.  The paper has no counterpart; this is a deployment
// variant of dg_apply.
//
// Some callers may not call cudaMalloc: allocator-free embedded or real-time
// runtimes that reserve all device memory when they start, and host frameworks
// that own every device allocation and forbid libraries to make their own.
// dg_create_mesh allocates (coefficient data and workspaces), so those callers
// get this entry point instead.  It takes the raw coefficient K, the input x
// and the output y from the caller, and calls no cudaMalloc, cudaFree or
// allocating library routine.  Its temporaries live in one file-scope
// __device__ array of DG_STATIC_SCRATCH_BYTES:
//   the derived coefficients h w_q K, h gamma_F and the face-point weights,
//   the per-cell Kbar,
//   the validity flag,
//   the nodal values, the x-modal values and the face traces of x.
// Every GPU that loads the library holds this array until the process exits.
// The coefficient kernels are the ones dg_set_coefficient runs (FP64 outputs
// only); the two passes are the generic FP64 trace and cell kernels.
//
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in).  The first call on each device therefore looks up the array's
// device address with cudaGetSymbolAddress, with that device current, and
// caches it; that first call should come before any stream capture.  Every
// call shares the array and leaves its contents behind; the only value that
// must start at zero, the flag, is cleared on every call.  Calls that overlap
// on the GPU (on different streams or devices sharing a context) race on the
// array and must be serialised by the caller.  The call blocks: it copies the
// K validity flag back to the host and synchronises the stream.
#include <mutex>

#include "dg_apply_impl.cuh"

#define DG_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

static __device__ __align__(256) unsigned char g_dg_static_scratch[DG_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_static: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dg_static_scratch);
    if (e != cudaSuccess) return dg_cuda_fail(e, "dg_apply_static: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DG_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <int N>
struct StaticApplyF {
  template <typename T>
  static cudaError_t run(const double* x, double* y, double* U, double* X, double* TR,
                         const double* kt, const double* fw, long long ncells, int Nc,
                         const DGTab<double>* tab, cudaStream_t s) {
    using dgk::Cfg;
    const unsigned blocks = (unsigned)((ncells + Cfg<N>::CPB - 1) / Cfg<N>::CPB);
    dgk::k_trace<N, double><<<blocks, Cfg<N>::THREADS, dgk::trace_smem<N, double>(), s>>>(
        x, U, X, TR, 0, ncells, nullptr, *tab);
    dgk::k_cell<N, double><<<blocks, Cfg<N>::THREADS, dgk::cell_smem<N, double>(), s>>>(
        U, X, TR, kt, fw, y, 0, ncells, Nc, nullptr, *tab);
    return cudaGetLastError();
  }
};

}  // namespace

extern "C" int dg_apply_static(int n_cells, int degree, const double* K, const double* x,
                               double* y, void* stream) {
  if (n_cells < 1 || n_cells > 1024)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_static: n_cells=%d outside [1, 1024]", n_cells);
  if (degree < 1 || degree > DG_MAXN - 1)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_static: degree=%d outside [1, %d]", degree,
                   DG_MAXN - 1);
  if (K == nullptr || x == nullptr || y == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_static: NULL pointer");
  if ((const void*)x == (const void*)y || (const void*)K == (const void*)y)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_apply_static: y aliases x or K");
  const int n = degree + 1;
  const long long ncells = (long long)n_cells * n_cells * n_cells;
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  const size_t ndofs = (size_t)ncells * n3;
  // scratch layout (256-byte aligned parts)
  const size_t o_flag = 0;
  const size_t o_kbar = o_flag + 256;
  const size_t o_gh = o_kbar + align256(sizeof(double) * (size_t)ncells);
  const size_t o_kt = o_gh + align256(sizeof(double) * 6 * (size_t)ncells);
  const size_t o_U = o_kt + align256(sizeof(double) * ndofs);
  const size_t o_X = o_U + align256(sizeof(double) * ndofs);
  const size_t o_TR = o_X + align256(sizeof(double) * ndofs);
  const size_t o_FW = o_TR + align256(sizeof(double) * 12 * n2 * (size_t)ncells);
  const size_t total = o_FW + align256(sizeof(double) * 12 * n2 * (size_t)ncells);
  if (total > DG_STATIC_SCRATCH_BYTES)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_apply_static: %d^3 cells of degree %d need %zu bytes of scratch; the "
                   "static scratch holds %zu bytes (use dg_create_mesh + dg_apply)",
                   n_cells, degree, total, (size_t)DG_STATIC_SCRATCH_BYTES);
  unsigned char* base = nullptr;
  int rc = scratch_address((void**)&base);
  if (rc) return rc;
  rc = dg_prepare_apply_f64(n);  // kernel attributes only (no allocation)
  if (rc) return rc;
  int* flag = (int*)(base + o_flag);
  double* kbar = (double*)(base + o_kbar);
  double* gh = (double*)(base + o_gh);
  double* kt = (double*)(base + o_kt);
  double* U = (double*)(base + o_U);
  double* X = (double*)(base + o_X);
  double* TR = (double*)(base + o_TR);
  double* FW = (double*)(base + o_FW);

  DGTab<double> tab;
  DGTab<float> tab32;
  const double h = 1.0 / n_cells;
  dg_build_tables(n, 2.0 * n * n, &tab, &tab32);
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  // the coefficient kernels of dg_set_coefficient, FP64 outputs only
  k_coef_cells<<<(unsigned)((ncells * 32 + 255) / 256), 256, 0, s>>>(K, kt, nullptr, kbar, ncells,
                                                                     n, h, flag, tab);
  k_coef_faces<<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(kbar, gh, nullptr, nullptr,
                                                                n_cells, h, DG_BC_DIRICHLET);
  dgk::k_face_weights<double><<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(gh, FW, n_cells, n,
                                                                              tab);
  DG_CUDA(cudaGetLastError());
  cudaError_t e = dgk::dispatch_n<double, StaticApplyF>(n, x, y, U, X, TR, (const double*)kt,
                                                        (const double*)FW, ncells, n_cells,
                                                        (const DGTab<double>*)&tab, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "dg_apply_static: launch");
  int hflag = 0;
  DG_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (hflag)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_apply_static: K has a value <= 0 or non-finite; y is not valid");
  return DG_OK;
}
