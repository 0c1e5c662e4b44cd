// Mesh handle, coefficient setup, error reporting and the apply entry points.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "dg_apply_impl.cuh"

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

int dg_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int dg_cuda_fail(cudaError_t e, const char* what) {
  int code = (e == cudaErrorMemoryAllocation) ? DG_ERR_OOM : DG_ERR_CUDA;
  return dg_fail(code, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

extern "C" const char* dg_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// coefficient setup kernels
// ---------------------------------------------------------------------------

// One warp per cell: Kt = h w_q K (FP64, and FP32 unless kt32 is NULL),
// Kbar = exp(sum_q w_q log K).  Invalid K (<= 0, NaN, inf) raises bit 0 of *flag.
__global__ void k_coef_cells(const double* __restrict__ K, double* __restrict__ kt64,
                             float* __restrict__ kt32, double* __restrict__ kbar,
                             long long ncells, int n, double h, int* flag,
                             const __grid_constant__ DGTab<double> tab) {
  const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (c >= ncells) return;
  const int n3 = n * n * n;
  double acc = 0.0;
  bool bad = false;
  for (int q = lane; q < n3; q += 32) {
    const int a = q % n, b = (q / n) % n, e = q / (n * n);
    const double wq = tab.w[a] * tab.w[b] * tab.w[e];
    const double Kq = K[c * n3 + q];
    if (!(Kq > 0.0) || !(Kq < INFINITY)) bad = true;
    const double v = h * wq * Kq;
    kt64[c * n3 + q] = v;
    if (kt32 != nullptr) kt32[c * n3 + q] = (float)v;
    acc += wq * log(Kq);
  }
  if (bad) atomicOr(flag, 1);
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) kbar[c] = exp(acc);
}

// One thread per cell: h*gamma (FP64, and FP32 unless gh32 is NULL) and, unless
// dgam is NULL, d gamma / d log Kbar_c on its six faces.  A boundary face on a
// side whose bit is clear in dmask carries zero flux (homogeneous Neumann): no
// face term at all, i.e. gamma = 0 there.
__global__ void k_coef_faces(const double* __restrict__ kbar, double* __restrict__ gh64,
                             float* __restrict__ gh32, double* __restrict__ dgam, int Nc,
                             double h, int dmask) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)Nc * Nc * Nc;
  if (c >= nc) return;
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  const long long stride[3] = {1, Nc, (long long)Nc * Nc};
  const double k = kbar[c];
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1;
    const bool upper = f & 1;
    const bool interior = upper ? (crd[d] < Nc - 1) : (crd[d] > 0);
    double g, dg;
    if (interior) {
      const double kn = kbar[upper ? c + stride[d] : c - stride[d]];
      g = 2.0 * k * kn / (k + kn);
      dg = g * kn / (k + kn);
    } else if ((dmask >> f) & 1) {
      g = k;
      dg = k;
    } else {
      g = 0.0;
      dg = 0.0;
    }
    gh64[c * 6 + f] = h * g;
    if (gh32 != nullptr) gh32[c * 6 + f] = (float)(h * g);
    if (dgam != nullptr) dgam[c * 6 + f] = dg;
  }
}

// ---------------------------------------------------------------------------
// mesh lifetime
// ---------------------------------------------------------------------------
template <typename P>
static cudaError_t dmalloc(P** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(P));
}

static void free_all(dg_mesh* m) {
  void* ptrs[] = {m->kt64, m->kt32, m->gh64, m->gh32, m->dgam, m->kbar, m->dflag, m->fw64, m->fw32, m->lineop64, m->diag64, m->dinv64, m->dinv32, m->binv64, m->kron64, m->kron32, m->lineopN64, m->dinvN64, m->dinvN32, m->bN64, m->xN64, m->hk32, m->kronN64, m->kronN32, m->geo_vol, m->geo_det, m->geo_face, m->geo_pen,
                  m->U64,  m->X64,  m->TR64, m->U32,  m->X32,  m->TR32, m->U64b,
                  m->X64b, m->TR64b, m->hx_dev, m->hy_dev, m->r64, m->p64, m->q64,
                  m->t64,  m->s64, m->d32,  m->r32, m->p32, m->q32, m->partials, m->state,
                  m->partials_cells};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->state_host) cudaFreeHost(m->state_host);
  if (m->tev) {
    for (int i = 0; i < 3 * m->tev_cap; ++i) cudaEventDestroy(m->tev[i]);
    free(m->tev);
  }
  if (m->solve_stream) cudaStreamDestroy(m->solve_stream);
  if (m->ev) cudaEventDestroy(m->ev);
  for (cudaStream_t hs : m->hstream)
    if (hs) cudaStreamDestroy(hs);
  for (cudaEvent_t he : m->hev)
    if (he) cudaEventDestroy(he);
}

extern "C" int dg_create_mesh(int n_cells, int degree, dg_mesh** out) {
  if (out == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_create_mesh: out is NULL");
  *out = nullptr;
  if (n_cells < 1 || n_cells > 1024)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_create_mesh: n_cells=%d outside [1, 1024]", n_cells);
  if (degree < 1 || degree > DG_MAXN - 1)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_create_mesh: degree=%d outside [1, %d]", degree,
                   DG_MAXN - 1);
  dg_mesh* m = (dg_mesh*)calloc(1, sizeof(dg_mesh));
  if (!m) return dg_fail(DG_ERR_OOM, "dg_create_mesh: host allocation failed");
  m->N = n_cells;
  m->k = degree;
  m->n = degree + 1;
  m->ncells = (long long)n_cells * n_cells * n_cells;
  const long long n3 = (long long)m->n * m->n * m->n;
  const long long n2 = (long long)m->n * m->n;
  m->ndofs = m->ncells * n3;
  m->h = 1.0 / n_cells;
  m->sigma = 2.0 * (degree + 1) * (degree + 1);
  m->dirichlet_mask = DG_BC_DIRICHLET;
  m->affine = false;
  m->geomDet = 1.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) m->geomG[i][j] = i == j ? 1.0 : 0.0;
    m->geomKappa[i] = 1.0;
  }
  dg_build_tables(m->n, m->sigma, &m->tab64, &m->tab32);
  dg_build_nodal_tables(m->tab64, m->n, &m->tabN64, &m->tabN32);
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
  const size_t nd = (size_t)m->ndofs, nc = (size_t)m->ncells, ntr = (size_t)(12 * n2) * nc;
  if (e == cudaSuccess) e = dmalloc(&m->kt64, nd);
  if (e == cudaSuccess) e = dmalloc(&m->kt32, nd);
  if (e == cudaSuccess) e = dmalloc(&m->gh64, 6 * nc);
  if (e == cudaSuccess) e = dmalloc(&m->gh32, 6 * nc);
  if (e == cudaSuccess) e = dmalloc(&m->dgam, 6 * nc);
  if (e == cudaSuccess) e = dmalloc(&m->fw64, ntr);
  if (e == cudaSuccess) e = dmalloc(&m->fw32, ntr);
  if (e == cudaSuccess)
    e = dmalloc(&m->lineop64, (size_t)3 * n2 * (size_t)(m->n * (m->n + 1) / 2) * nc);
  if (e == cudaSuccess) e = dmalloc(&m->kbar, nc);
  if (e == cudaSuccess) e = dmalloc(&m->dflag, 1);
  if (e == cudaSuccess) e = dmalloc(&m->U64, nd);
  if (e == cudaSuccess) e = dmalloc(&m->X64, nd);
  if (e == cudaSuccess) e = dmalloc(&m->TR64, ntr);
  if (e == cudaSuccess) e = dmalloc(&m->U32, nd);
  if (e == cudaSuccess) e = dmalloc(&m->X32, nd);
  if (e == cudaSuccess) e = dmalloc(&m->TR32, ntr);
  if (e != cudaSuccess) {
    int rc = dg_cuda_fail(e, "dg_create_mesh: device allocation");
    free_all(m);
    free(m);
    return rc;
  }
  int rc = dg_prepare_apply_f64(m->n);
  if (rc == DG_OK) rc = dg_prepare_apply_f32(m->n);
  if (rc == DG_OK) rc = dg_prepare_affine(m->n);
  if (rc == DG_OK) rc = dg_prepare_grad(m->n);
  if (rc != DG_OK) {
    free_all(m);
    free(m);
    return rc;
  }
  *out = m;
  return DG_OK;
}

extern "C" int dg_destroy_mesh(dg_mesh* m) {
  if (m == nullptr) return DG_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_all(m);
  free(m);
  if (e != cudaSuccess) return dg_cuda_fail(e, "dg_destroy_mesh: device synchronize");
  return DG_OK;
}

extern "C" int dg_mesh_info(const dg_mesh* m, long long* n_dofs, long long* n_cells_total,
                            int* n_points_1d, double* sigma) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_mesh_info: mesh is NULL");
  if (n_dofs) *n_dofs = m->ndofs;
  if (n_cells_total) *n_cells_total = m->ncells;
  if (n_points_1d) *n_points_1d = m->n;
  if (sigma) *sigma = m->sigma;
  return DG_OK;
}

extern "C" int dg_set_boundary(dg_mesh* m, int dirichlet_mask) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_set_boundary: mesh is NULL");
  if (dirichlet_mask < 0 || dirichlet_mask > 0x3F)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_set_boundary: mask 0x%x outside 0..0x3f",
                   dirichlet_mask);
  if (dirichlet_mask == 0)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_set_boundary: at least one side must be Dirichlet (the operator would "
                   "be singular)");
  m->dirichlet_mask = dirichlet_mask;
  m->has_coef = false;  // the face weights depend on it: set the coefficient again
  m->has_diag = false;
  m->has_block = false;
  m->has_kron = false;
  m->has_nodal = false;
  m->has_nodal_diag = false;
  m->has_nodal32 = false;
  m->has_kron_nodal = false;
  return DG_OK;
}

int dg_require_cube(const dg_mesh* m, const char* who) {
  if (m != nullptr && (m->affine || m->multilinear))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "%s: not available on an affine or multilinear geometry (FP64 dg_apply, "
                   "dg_apply_adjoint, dg_load_vector and the FP64 CG without preconditioner "
                   "are)", who);
  return DG_OK;
}

int dg_ensure_grad_ws(dg_mesh* m) {
  if (m->U64b) return DG_OK;
  const size_t nd = (size_t)m->ndofs;
  const size_t ntr = (size_t)(12 * m->n * m->n) * (size_t)m->ncells;
  DG_CUDA(dmalloc(&m->U64b, nd));
  DG_CUDA(dmalloc(&m->X64b, nd));
  DG_CUDA(dmalloc(&m->TR64b, ntr));
  return DG_OK;
}

int dg_ensure_solver_ws(dg_mesh* m) {
  if (m->state) return DG_OK;
  const size_t nd = (size_t)m->ndofs;
  DG_CUDA(dmalloc(&m->r64, nd));
  DG_CUDA(dmalloc(&m->p64, nd));
  DG_CUDA(dmalloc(&m->q64, nd));
  DG_CUDA(dmalloc(&m->t64, nd));
  DG_CUDA(dmalloc(&m->s64, nd));
  DG_CUDA(dmalloc(&m->d32, nd));
  DG_CUDA(dmalloc(&m->r32, nd));
  DG_CUDA(dmalloc(&m->p32, nd));
  DG_CUDA(dmalloc(&m->q32, nd));
  DG_CUDA(dmalloc(&m->partials, DG_RED_SUMS * DG_RED_BLOCKS));
  DG_CUDA(dmalloc(&m->partials_cells, (size_t)dg_mixed32_blocks(m->n, m->ncells)));
  DG_CUDA(cudaMallocHost((void**)&m->state_host, sizeof(DGCGState)));
  DG_CUDA(cudaStreamCreateWithFlags(&m->solve_stream, cudaStreamNonBlocking));
  DG_CUDA(cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming));
  DG_CUDA(dmalloc(&m->state, 1));
  DG_CUDA(cudaMemset(m->state, 0, sizeof(DGCGState)));
  return dg_prepare_mixed32(m);
}

// ---------------------------------------------------------------------------
// coefficient
// ---------------------------------------------------------------------------
extern "C" int dg_set_coefficient(dg_mesh* m, const double* K, void* stream) {
  if (m == nullptr || K == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_set_coefficient: NULL mesh or K");
  cudaStream_t s = (cudaStream_t)stream;
  m->has_coef = false;
  m->has_diag = false;
  m->has_block = false;
  m->has_kron = false;
  m->has_nodal = false;
  m->has_nodal_diag = false;
  m->has_nodal32 = false;
  m->has_kron_nodal = false;
  DG_CUDA(cudaMemsetAsync(m->dflag, 0, sizeof(int), s));
  {
    const long long threads = m->ncells * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    k_coef_cells<<<blocks, 256, 0, s>>>(K, m->kt64, m->kt32, m->kbar, m->ncells, m->n, m->h,
                                        m->dflag, m->tab64);
    DG_CUDA(cudaGetLastError());
  }
  {
    const unsigned blocks = (unsigned)((m->ncells + 255) / 256);
    k_coef_faces<<<blocks, 256, 0, s>>>(m->kbar, m->gh64, m->gh32, m->dgam, m->N, m->h,
                                        m->dirichlet_mask);
    dgk::k_face_weights<double><<<blocks, 256, 0, s>>>(m->gh64, m->fw64, m->N, m->n, m->tab64);
    dgk::k_face_weights<float><<<blocks, 256, 0, s>>>(m->gh64, m->fw32, m->N, m->n, m->tab64);
    DG_CUDA(cudaGetLastError());
    cudaError_t e = dgk::dispatch_n<double, dgk::LineOpsF>(m->n, (const double*)m->kt64,
                                                           (const double*)m->gh64, m->lineop64,
                                                           m->ncells, m->N,
                                                           (const DGTab<double>*)&m->tab64, s);
    if (e != cudaSuccess) return dg_cuda_fail(e, "dg_set_coefficient: line operators");
  }
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, m->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (flag)
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_set_coefficient: K has a value <= 0 or non-finite; coefficient not set");
  m->has_coef = true;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// operator application
// ---------------------------------------------------------------------------
static int check_apply_args(const dg_mesh* m, const void* x, const void* y, int prec,
                            const char* who) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "%s: mesh is NULL", who);
  if (!m->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "%s: coefficient not set", who);
  if (x == nullptr || y == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "%s: NULL vector", who);
  if (x == y) return dg_fail(DG_ERR_INVALID_ARG, "%s: input and output alias", who);
  if (prec != DG_FP64 && prec != DG_FP32)
    return dg_fail(DG_ERR_INVALID_ARG, "%s: prec=%d is neither DG_FP64 nor DG_FP32", who, prec);
  return DG_OK;
}

extern "C" int dg_apply(const dg_mesh* m, const void* x, void* y, int prec, void* stream) {
  int rc = check_apply_args(m, x, y, prec, "dg_apply");
  if (rc) return rc;
  if (prec == DG_FP32 && (rc = dg_require_cube(m, "dg_apply(FP32)"))) return rc;
  if (prec == DG_FP64)
    return dg_launch_apply_f64(m, (const double*)x, (double*)y, nullptr, (cudaStream_t)stream);
  return dg_launch_apply_f32(m, (const float*)x, (float*)y, nullptr, (cudaStream_t)stream);
}

extern "C" int dg_apply_adjoint(const dg_mesh* m, const void* ybar, void* xbar, int prec,
                                void* stream) {
  int rc = check_apply_args(m, ybar, xbar, prec, "dg_apply_adjoint");
  if (rc) return rc;
  if (prec == DG_FP32 && (rc = dg_require_cube(m, "dg_apply_adjoint(FP32)"))) return rc;
  // a(u, v) = a(v, u): the transposed data flow performs the same contractions.
  if (prec == DG_FP64)
    return dg_launch_apply_f64(m, (const double*)ybar, (double*)xbar, nullptr,
                               (cudaStream_t)stream);
  return dg_launch_apply_f32(m, (const float*)ybar, (float*)xbar, nullptr, (cudaStream_t)stream);
}

// Host-buffer apply, pipelined over z-slabs of cells so that both copies
// overlap the kernels.  Four streams:
//   copy-in   H2D of x, slab by slab;
//   pass 1    pass 1 of slab s once its x has arrived (runs ahead of pass 2);
//   caller's  pass 2 of slab s once pass 1 has covered slab s+1 (the upper
//             neighbours of slab s are the first layer of slab s+1);
//   copy-out  D2H of y of slab s once pass 2 has written it.
// Pass 1 and pass 2 of different slabs may run at the same time, which fills
// the last partial wave of each launch.  Every event is recorded before any
// wait on it is enqueued.
static int ensure_host_pipeline(dg_mesh* m) {
  if (m->hx_dev == nullptr) {
    DG_CUDA(cudaMalloc(&m->hx_dev, (size_t)m->ndofs * sizeof(double)));
    DG_CUDA(cudaMalloc(&m->hy_dev, (size_t)m->ndofs * sizeof(double)));
  }
  for (cudaStream_t& hs : m->hstream)
    if (hs == nullptr) DG_CUDA(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
  for (cudaEvent_t& he : m->hev)
    if (he == nullptr) DG_CUDA(cudaEventCreateWithFlags(&he, cudaEventDisableTiming));
  return DG_OK;
}

extern "C" int dg_apply_host(const dg_mesh* mc, const void* x_host, void* y_host, int prec,
                             void* stream) {
  int rc = check_apply_args(mc, x_host, y_host, prec, "dg_apply_host");
  if (rc) return rc;
  if ((rc = dg_require_cube(mc, "dg_apply_host"))) return rc;
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaStream_t s = (cudaStream_t)stream;
  rc = ensure_host_pipeline(m);
  if (rc) return rc;
  const size_t esz = prec == DG_FP64 ? sizeof(double) : sizeof(float);
  const long long layer = (long long)m->N * m->N;  // cells per z-layer
  const int nslab_max = m->N < DG_HOST_SLABS ? m->N : DG_HOST_SLABS;
  const int lps = (m->N + nslab_max - 1) / nslab_max;  // layers per slab
  const int nslab = (m->N + lps - 1) / lps;
  const long long n3 = (long long)m->n * m->n * m->n;
  auto cells = [&](int sl) { return (long long)(sl * lps < m->N ? sl * lps : m->N) * layer; };
  cudaStream_t cin = m->hstream[0], cout = m->hstream[1], p1 = m->hstream[2];
  cudaEvent_t* ev_in = m->hev;                       // H2D of slab s done
  cudaEvent_t* ev_p1 = m->hev + DG_HOST_SLABS;       // pass 1 of slab s done
  cudaEvent_t* ev_out = m->hev + 2 * DG_HOST_SLABS;  // pass 2 of slab s done
  cudaEvent_t ev_start = m->hev[3 * DG_HOST_SLABS];
  // order after the caller's earlier work on its stream
  DG_CUDA(cudaEventRecord(ev_start, s));
  DG_CUDA(cudaStreamWaitEvent(cin, ev_start, 0));
  DG_CUDA(cudaStreamWaitEvent(p1, ev_start, 0));
  DG_CUDA(cudaStreamWaitEvent(cout, ev_start, 0));
  char* xd = (char*)m->hx_dev;
  char* yd = (char*)m->hy_dev;
  auto span = [&](int sl, size_t* off, size_t* bytes) {
    *off = (size_t)(cells(sl) * n3) * esz;
    *bytes = (size_t)((cells(sl + 1) - cells(sl)) * n3) * esz;
  };
  auto pass = [&](int p, int sl, cudaStream_t st) {
    return prec == DG_FP64
               ? dg_launch_pass_f64(m, p, (const double*)xd, (double*)yd, cells(sl),
                                    cells(sl + 1), st)
               : dg_launch_pass_f32(m, p, (const float*)xd, (float*)yd, cells(sl),
                                    cells(sl + 1), st);
  };
  for (int sl = 0; sl < nslab; ++sl) {
    size_t off, bytes;
    span(sl, &off, &bytes);
    DG_CUDA(cudaMemcpyAsync(xd + off, (const char*)x_host + off, bytes, cudaMemcpyHostToDevice,
                            cin));
    DG_CUDA(cudaEventRecord(ev_in[sl], cin));
  }
  for (int sl = 0; sl < nslab; ++sl) {
    DG_CUDA(cudaStreamWaitEvent(p1, ev_in[sl], 0));
    rc = pass(1, sl, p1);
    if (rc) return rc;
    DG_CUDA(cudaEventRecord(ev_p1[sl], p1));
  }
  for (int sl = 0; sl < nslab; ++sl) {
    // pass 1 of slabs sl - 1, sl, sl + 1 (in stream order on p1)
    DG_CUDA(cudaStreamWaitEvent(s, ev_p1[sl + 1 < nslab ? sl + 1 : sl], 0));
    rc = pass(2, sl, s);
    if (rc) return rc;
    DG_CUDA(cudaEventRecord(ev_out[sl], s));
  }
  for (int sl = 0; sl < nslab; ++sl) {
    size_t off, bytes;
    span(sl, &off, &bytes);
    DG_CUDA(cudaStreamWaitEvent(cout, ev_out[sl], 0));
    DG_CUDA(cudaMemcpyAsync((char*)y_host + off, yd + off, bytes, cudaMemcpyDeviceToHost, cout));
  }
  DG_CUDA(cudaStreamSynchronize(cout));
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

// ---------------------------------------------------------------------------
// coefficient gradient
// ---------------------------------------------------------------------------
extern "C" int dg_coeff_grad(const dg_mesh* mc, const double* u, const double* v, double* g,
                             void* stream) {
  if (mc == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_coeff_grad: mesh is NULL");
  if (!mc->has_coef) return dg_fail(DG_ERR_INVALID_ARG, "dg_coeff_grad: coefficient not set");
  if (u == nullptr || v == nullptr || g == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_coeff_grad: NULL vector");
  if (g == u || g == v) return dg_fail(DG_ERR_INVALID_ARG, "dg_coeff_grad: g aliases u or v");
  if (int rc0 = dg_require_cube(mc, "dg_coeff_grad")) return rc0;
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  int rc = dg_ensure_grad_ws(m);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = dg_launch_trace_f64(m, u, m->U64, m->X64, m->TR64, s);
  if (rc) return rc;
  rc = dg_launch_trace_f64(m, v, m->U64b, m->X64b, m->TR64b, s);
  if (rc) return rc;
  return dg_launch_coeff_grad(m, g, s);
}

// ---------------------------------------------------------------------------
// per-pass kernel timing
// ---------------------------------------------------------------------------
void dg_timing_mark(const dg_mesh* mc, int slot, cudaStream_t s) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  if (!m->timing || m->tev_used >= m->tev_cap) return;
  cudaEventRecord(m->tev[3 * m->tev_used + slot], s);
  if (slot == 2) m->tev_used += 1;
}

extern "C" int dg_timing_enable(dg_mesh* m, int max_applies) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_timing_enable: mesh is NULL");
  if (max_applies < 1 || max_applies > 65536)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_timing_enable: max_applies=%d outside [1, 65536]",
                   max_applies);
  if (m->tev_cap < max_applies) {
    if (m->tev) {
      for (int i = 0; i < 3 * m->tev_cap; ++i) cudaEventDestroy(m->tev[i]);
      free(m->tev);
      m->tev = nullptr;
      m->tev_cap = 0;
    }
    m->tev = (cudaEvent_t*)calloc((size_t)3 * max_applies, sizeof(cudaEvent_t));
    if (!m->tev) return dg_fail(DG_ERR_OOM, "dg_timing_enable: host allocation failed");
    for (int i = 0; i < 3 * max_applies; ++i) DG_CUDA(cudaEventCreate(&m->tev[i]));
    m->tev_cap = max_applies;
  }
  m->tev_used = 0;
  m->timing = true;
  return DG_OK;
}

extern "C" int dg_timing_read(dg_mesh* m, int* n_applies, double* ms1, double* ms2) {
  if (m == nullptr) return dg_fail(DG_ERR_INVALID_ARG, "dg_timing_read: mesh is NULL");
  m->timing = false;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < m->tev_used; ++i) {
    DG_CUDA(cudaEventSynchronize(m->tev[3 * i + 2]));
    float t1 = 0.f, t2 = 0.f;
    DG_CUDA(cudaEventElapsedTime(&t1, m->tev[3 * i], m->tev[3 * i + 1]));
    DG_CUDA(cudaEventElapsedTime(&t2, m->tev[3 * i + 1], m->tev[3 * i + 2]));
    a += t1;
    b += t2;
  }
  if (n_applies) *n_applies = m->tev_used;
  if (ms1) *ms1 = a;
  if (ms2) *ms2 = b;
  return DG_OK;
}
