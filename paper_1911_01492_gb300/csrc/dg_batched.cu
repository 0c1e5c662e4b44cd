// Batched CG: many independent systems A_s x_s = b_s (different coefficient
// samples, mesh sizes and degrees, as in the multilevel Monte-Carlo setting of
// Section 5) solved by lock-step CG in one persistent kernel.
//
// Each sample runs the PCG of Section 2.4 (M = I, or M = diag(A) with
// DG_CG_PRECOND_JACOBI) with its own scalars, like
// the k independent solvers running in lock-step of the horizontal
// vectorisation in Section 3.5.  The cells of all samples are cut into work
// units (one block's worth of cells of one sample); every iteration of every
// unfinished sample is executed by one persistent cooperative launch:
//   A  p = z + beta p (z = M^-1 r) on the unit's cells, then pass 1 (nodal
//      values, face traces) of p;
//   B  pass 2 (volume + face terms) -> q, and the unit's partial <p, q>;
//   C  per sample: alpha = rho / <p, q>  (partials summed in a fixed order);
//   D  x += alpha p, r -= alpha q, the unit's partials <r, r> and <z, r>;
//   E  per sample: rho' = <z, r>, convergence test on <r, r>, beta = rho'/rho;
// separated by grid-wide barriers.  Each barrier spins a bounded number of
// times; on expiry the kernel raises an error flag and returns, and the host
// reports DG_ERR_TIMEOUT.  Work units of finished samples are skipped, so
// uneven samples cost what they need (work proportional to size x iterations,
// as in the proportional allocation rule of Section 5).
//
// The launch is captured in a CUDA graph and replayed until every sample is
// done.  An autotuner picks the number of resident blocks per SM by timing the
// first graph replays (real CG iterations) for each candidate.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "dg_apply_impl.cuh"

namespace {

constexpr int BT = 128;        // threads per block (>= n^2 * cells per unit for n <= 5)
constexpr int MAXN_B = 5;      // batched solver supports n = 2..5 (degree 1..4)
constexpr int ITERS_PER_LAUNCH = 64;  // lock-step iterations per persistent launch
constexpr int ITERS_TUNE = 4;         // iterations per launch while autotuning

__constant__ DGTab<double> c_btab[MAXN_B - 1];  // tables for n = 2..5

struct SampleDev {
  const double* b;
  double* x;
  double *r, *p, *q;
  double *U, *X, *TR;
  const double* kt;
  const double* fw;
  const double* lineop;
  const double* dinv;  // 1 / diag(A) for M = diag(A); nullptr for M = I
  long long ncells;
  int Nc;       // cells per direction
  int n;        // points per direction
  int ubeg, uend;  // work units of this sample
};

struct BState {
  double rho, rho_new, alpha, beta, tol2, bnorm2, pq;
  double rr;  // <r, r>, the convergence norm (rho = <z, r>)
  int done, breakdown, iters, maxit;
};

struct BCtl {
  unsigned count;     // barrier arrivals
  unsigned gen;       // barrier generation
  int err;            // 1: a barrier wait expired
  int active;         // samples not done (written by block 0 after phase E)
  unsigned long long iterations_run;  // lock-step iterations executed
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block sum (blockDim.x == BT); result valid in every thread.
__device__ double block_sum(double v, double* sred) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sred[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < BT / 32; ++i) r += sred[i];
  return r;
}

// Grid barrier with a bounded wait.  Returns false (in every thread) once any
// block's wait has expired.
__device__ bool grid_sync(BCtl* ctl, unsigned nblocks, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &ctl->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&ctl->count, 1u) == nblocks - 1) {
      atomicExch(&ctl->count, 0u);
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (((volatile int*)&ctl->err)[0] || ++spins > limit) {
          atomicOr(&ctl->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ((volatile int*)&ctl->err)[0] == 0;
}

template <int N>
__device__ __forceinline__ void unit_pass1(const SampleDev& S, long long c0, int nblk,
                                           double* smem) {
  dgk::trace_cells<N, double>(S.p, S.U, S.X, S.TR, c0, nblk, c_btab[N - 2], smem);
}
template <int N>
__device__ __forceinline__ void unit_pass2(const SampleDev& S, long long c0, int nblk,
                                           double* smem) {
  dgk::cell_cells<N, double, true>(S.U, S.X, S.TR, S.kt, S.fw, S.q, c0, nblk, S.Nc,
                                   c_btab[N - 2], smem, S.lineop);
}

__device__ __forceinline__ int unit_cells(int n) {
  return n == 2 ? dgk::Cfg<2>::CPB : n == 3 ? dgk::Cfg<3>::CPB : n == 4 ? dgk::Cfg<4>::CPB
                                                                        : dgk::Cfg<5>::CPB;
}

__global__ void __launch_bounds__(BT)
kb_persistent(const SampleDev* __restrict__ S, int ns, const int2* __restrict__ units, int nu,
              BState* st, double* part, BCtl* ctl, int iters, long long limit, int stall_test) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* smem = reinterpret_cast<double*>(smem_raw);
  __shared__ double sred[BT / 32];
  const unsigned nb = gridDim.x;
  if (stall_test && blockIdx.x == 0) return;  // test hook: one block never arrives
  for (int it = 0; it < iters; ++it) {
    if (((volatile int*)&ctl->active)[0] == 0) break;
    // A: p = r + beta p on the unit, then pass 1 of p
    for (int u = blockIdx.x; u < nu; u += nb) {
      const int s = units[u].x;
      if (st[s].done) continue;
      const SampleDev& sd = S[s];
      const long long c0 = units[u].y;
      const int cpu = unit_cells(sd.n);
      const int nblk = (int)((sd.ncells - c0) < cpu ? (sd.ncells - c0) : cpu);
      const long long n3 = (long long)sd.n * sd.n * sd.n;
      const double be = st[s].beta;
      if (sd.dinv)
        for (long long i = c0 * n3 + threadIdx.x; i < (c0 + nblk) * n3; i += BT)
          sd.p[i] = fma(be, sd.p[i], sd.dinv[i] * sd.r[i]);
      else
        for (long long i = c0 * n3 + threadIdx.x; i < (c0 + nblk) * n3; i += BT)
          sd.p[i] = fma(be, sd.p[i], sd.r[i]);
      __syncthreads();
      switch (sd.n) {
        case 2: unit_pass1<2>(sd, c0, nblk, smem); break;
        case 3: unit_pass1<3>(sd, c0, nblk, smem); break;
        case 4: unit_pass1<4>(sd, c0, nblk, smem); break;
        default: unit_pass1<5>(sd, c0, nblk, smem); break;
      }
      __syncthreads();
    }
    if (!grid_sync(ctl, nb, limit)) return;
    // B: pass 2 -> q, partial <p, q>
    for (int u = blockIdx.x; u < nu; u += nb) {
      const int s = units[u].x;
      if (st[s].done) continue;
      const SampleDev& sd = S[s];
      const long long c0 = units[u].y;
      const int cpu = unit_cells(sd.n);
      const int nblk = (int)((sd.ncells - c0) < cpu ? (sd.ncells - c0) : cpu);
      switch (sd.n) {
        case 2: unit_pass2<2>(sd, c0, nblk, smem); break;
        case 3: unit_pass2<3>(sd, c0, nblk, smem); break;
        case 4: unit_pass2<4>(sd, c0, nblk, smem); break;
        default: unit_pass2<5>(sd, c0, nblk, smem); break;
      }
      __syncthreads();
      const long long n3 = (long long)sd.n * sd.n * sd.n;
      double a = 0.0;
      for (long long i = c0 * n3 + threadIdx.x; i < (c0 + nblk) * n3; i += BT)
        a = fma(sd.p[i], sd.q[i], a);
      a = block_sum(a, sred);
      if (threadIdx.x == 0) part[3 * u] = a;
    }
    if (!grid_sync(ctl, nb, limit)) return;
    // C: alpha per sample
    for (int s = blockIdx.x; s < ns; s += nb) {
      if (st[s].done) continue;
      double a = 0.0;
      for (int u = S[s].ubeg + threadIdx.x; u < S[s].uend; u += BT) a += part[3 * u];
      a = block_sum(a, sred);
      if (threadIdx.x == 0) {
        st[s].pq = a;
        if (!(a > 0.0) || !isfinite(a)) {
          st[s].breakdown = 1;
          st[s].done = 1;
        } else {
          st[s].alpha = st[s].rho / a;
        }
      }
    }
    if (!grid_sync(ctl, nb, limit)) return;
    // D: x += alpha p, r -= alpha q, partials <r, r> and <z, r>
    for (int u = blockIdx.x; u < nu; u += nb) {
      const int s = units[u].x;
      if (st[s].done) continue;
      const SampleDev& sd = S[s];
      const long long c0 = units[u].y;
      const int cpu = unit_cells(sd.n);
      const int nblk = (int)((sd.ncells - c0) < cpu ? (sd.ncells - c0) : cpu);
      const long long n3 = (long long)sd.n * sd.n * sd.n;
      const double al = st[s].alpha;
      double a = 0.0, z = 0.0;
      if (sd.dinv) {  // two loops: no per-element branch between the loads
        for (long long i = c0 * n3 + threadIdx.x; i < (c0 + nblk) * n3; i += BT) {
          sd.x[i] = fma(al, sd.p[i], sd.x[i]);
          const double ri = fma(-al, sd.q[i], sd.r[i]);
          sd.r[i] = ri;
          a = fma(ri, ri, a);
          z = fma(sd.dinv[i] * ri, ri, z);
        }
      } else {
        for (long long i = c0 * n3 + threadIdx.x; i < (c0 + nblk) * n3; i += BT) {
          sd.x[i] = fma(al, sd.p[i], sd.x[i]);
          const double ri = fma(-al, sd.q[i], sd.r[i]);
          sd.r[i] = ri;
          a = fma(ri, ri, a);
        }
      }
      a = block_sum(a, sred);
      if (sd.dinv) z = block_sum(z, sred);  // uniform: the block works on one unit
      if (threadIdx.x == 0) {
        part[3 * u + 1] = a;
        part[3 * u + 2] = z;
      }
    }
    if (!grid_sync(ctl, nb, limit)) return;
    // E: rho' = <z, r>, convergence on <r, r>, beta
    for (int s = blockIdx.x; s < ns; s += nb) {
      if (st[s].done) continue;
      const bool pc = S[s].dinv != nullptr;
      double a = 0.0, z = 0.0;
      for (int u = S[s].ubeg + threadIdx.x; u < S[s].uend; u += BT) {
        a += part[3 * u + 1];
        if (pc) z += part[3 * u + 2];
      }
      a = block_sum(a, sred);
      if (pc) z = block_sum(z, sred);
      if (threadIdx.x == 0) {
        BState& b = st[s];
        const double zr = pc ? z : a;
        b.iters += 1;
        if (!isfinite(a) || !isfinite(zr)) {
          b.breakdown = 1;
          b.done = 1;
        } else {
          b.beta = zr / b.rho;
          b.rho = zr;
          b.rr = a;
          if (a <= b.tol2 || b.iters >= b.maxit) b.done = 1;
        }
      }
    }
    if (!grid_sync(ctl, nb, limit)) return;
    if (blockIdx.x == 0) {
      int act = 0;
      for (int s = threadIdx.x; s < ns; s += BT) act += st[s].done ? 0 : 1;
      act = (int)block_sum((double)act, sred);
      if (threadIdx.x == 0) {
        ctl->active = act;
        ctl->iterations_run += 1;
      }
    }
    if (!grid_sync(ctl, nb, limit)) return;
  }
}

// Per-sample start: r = b - q (q = A x), p = z = M^-1 r (dinv, or M = I when
// dinv is null), rho = <z, r>, rr = <r, r>, bnorm2 = <b, b>, beta = 0.  One
// launch per sample; the last block publishes the sums.
__global__ void __launch_bounds__(256)
kb_init(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
        double* __restrict__ p, const double* __restrict__ dinv, long long n, double rtol,
        double* partials, unsigned* ticket, BState* st, int maxit, int keep_iters) {
  __shared__ double sw[8];
  __shared__ bool last;
  double rr = 0.0, bb = 0.0, zr = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - q[i];
    const double zi = dinv ? dinv[i] * ri : ri;
    r[i] = ri;
    p[i] = zi;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
    zr = fma(zi, ri, zr);
  }
  double tot[3] = {rr, bb, zr};
  for (int k = 0; k < 3; ++k) {
    double v = warp_sum(tot[k]);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += sw[i];
    if (threadIdx.x == 0) partials[3 * blockIdx.x + k] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0, z = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      a += ((volatile double*)partials)[3 * i];
      c += ((volatile double*)partials)[3 * i + 1];
      z += ((volatile double*)partials)[3 * i + 2];
    }
    BState s = {};
    s.rho = z;
    s.rr = a;
    s.bnorm2 = c;
    s.tol2 = rtol * rtol * c;
    s.beta = 0.0;
    s.maxit = maxit;
    s.iters = keep_iters;
    s.breakdown = !(isfinite(a) && isfinite(c) && isfinite(z));
    // b = 0: the solution is x = 0 (set by the host), nothing to iterate
    s.done = s.breakdown || c == 0.0 || a <= s.tol2 || keep_iters >= maxit;
    *st = s;
    *ticket = 0u;
  }
}

// ||b - q||^2 and ||b||^2 into out[0..1] (single block, fixed order).
__global__ void __launch_bounds__(256)
kb_residual(const double* __restrict__ b, const double* __restrict__ q, long long n,
            double* out) {
  __shared__ double sw[8];
  double rr = 0.0, bb = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double ri = b[i] - q[i];
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  double tot[2] = {rr, bb};
  for (int k = 0; k < 2; ++k) {
    double v = warp_sum(tot[k]);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < 8; ++i) t += sw[i];
      out[k] = t;
    }
  }
}

size_t persistent_smem() {
  size_t m = 0;
  m = std::max(m, dgk::cell_smem<2, double>());
  m = std::max(m, dgk::cell_smem<3, double>());
  m = std::max(m, dgk::cell_smem<4, double>());
  m = std::max(m, dgk::cell_smem<5, double>());
  return m;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Autotuner cache: batch signature -> blocks per SM.
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tune;

struct Batch {
  std::vector<dg_mesh*> meshes;
  SampleDev* d_samples = nullptr;
  int2* d_units = nullptr;
  BState* d_state = nullptr;
  double* d_part = nullptr;
  BCtl* d_ctl = nullptr;
  BCtl* h_ctl = nullptr;
  double* d_aux = nullptr;      // init partials, residual outputs
  unsigned* d_ticket = nullptr;
  int nunits = 0;
  ~Batch() {
    cudaFree(d_samples);
    cudaFree(d_units);
    cudaFree(d_state);
    cudaFree(d_part);
    cudaFree(d_ctl);
    cudaFree(d_aux);
    cudaFree(d_ticket);
    if (h_ctl) cudaFreeHost(h_ctl);
  }
};

int launch_persistent(Batch& B, int ns, int blocks, int iters, long long limit, int stall,
                      cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = persistent_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DG_CUDA(cudaLaunchKernelEx(&cfg, kb_persistent, (const SampleDev*)B.d_samples, ns,
                             (const int2*)B.d_units, B.nunits, B.d_state, B.d_part, B.d_ctl,
                             iters, limit, stall));
  return DG_OK;
}

}  // namespace

extern "C" int dg_cg_solve_batched_mode(const dg_mesh* const* meshes, int count,
                                        const double* const* b, double* const* x, double rtol,
                                        int maxit, int mode, dg_cg_stats* st, void* stream) {
  if (mode != DG_CG_FP64 && mode != (DG_CG_FP64 | DG_CG_PRECOND_JACOBI))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve_batched: mode %d; the batched solver runs DG_CG_FP64, with or "
                   "without DG_CG_PRECOND_JACOBI", mode);
  const bool jacobi = (mode & DG_CG_PRECOND_JACOBI) != 0;
  if (meshes == nullptr || b == nullptr || x == nullptr || count < 1)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: NULL array or count < 1");
  if (!(rtol > 0.0) || !(rtol < 1.0))
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: rtol=%g outside (0, 1)", rtol);
  if (maxit < 1) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: maxit=%d < 1", maxit);
  const double t0 = now_s();
  Batch B;
  B.meshes.resize(count);
  std::vector<SampleDev> hs(count);
  std::vector<int2> hu;
  std::vector<long long> sig;
  for (int s = 0; s < count; ++s) {
    dg_mesh* m = const_cast<dg_mesh*>(meshes[s]);
    if (m == nullptr || b[s] == nullptr || x[s] == nullptr)
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: NULL mesh or vector (sample %d)", s);
    if (!m->has_coef)
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: sample %d has no coefficient", s);
    if (m->n > MAXN_B)
      return dg_fail(DG_ERR_INVALID_ARG,
                     "dg_cg_solve_batched: sample %d has degree %d; the batched solver supports "
                     "degree 1..%d", s, m->k, MAXN_B - 1);
    if ((const void*)b[s] == (const void*)x[s])
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: b and x alias (sample %d)", s);
    for (int t = 0; t < s; ++t)
      if (meshes[t] == meshes[s])
        return dg_fail(DG_ERR_INVALID_ARG,
                       "dg_cg_solve_batched: samples %d and %d share a mesh (its workspaces)", t,
                       s);
    int rc = dg_ensure_solver_ws(m);
    if (rc) return rc;
    B.meshes[s] = m;
    SampleDev& d = hs[s];
    d.b = b[s];
    d.x = x[s];
    d.r = m->r64;
    d.p = m->p64;
    d.q = m->q64;
    d.U = m->U64;
    d.X = m->X64;
    d.TR = m->TR64;
    d.kt = m->kt64;
    d.fw = m->fw64;
    d.lineop = m->lineop64;
    d.dinv = nullptr;
    if (jacobi) {
      rc = dg_ensure_diagonal(m, m->solve_stream);
      if (rc) return rc;
      d.dinv = m->dinv64;
    }
    d.ncells = m->ncells;
    d.Nc = m->N;
    d.n = m->n;
    d.ubeg = (int)hu.size();
    const int cpu = m->n == 2 ? dgk::Cfg<2>::CPB : m->n == 3 ? dgk::Cfg<3>::CPB
                  : m->n == 4 ? dgk::Cfg<4>::CPB : dgk::Cfg<5>::CPB;
    for (long long c = 0; c < m->ncells; c += cpu) hu.push_back(make_int2(s, (int)c));
    d.uend = (int)hu.size();
    sig.push_back(m->N);
    sig.push_back(m->n);
  }
  sig.push_back(mode);
  B.nunits = (int)hu.size();
  cudaStream_t us = (cudaStream_t)stream;
  // a private non-blocking stream (capture needs one); ordered after the caller's work
  cudaStream_t s = B.meshes[0]->solve_stream;
  DG_CUDA(cudaEventRecord(B.meshes[0]->ev, us));
  DG_CUDA(cudaStreamWaitEvent(s, B.meshes[0]->ev, 0));

  DG_CUDA(cudaMalloc(&B.d_samples, sizeof(SampleDev) * count));
  DG_CUDA(cudaMalloc(&B.d_units, sizeof(int2) * B.nunits));
  DG_CUDA(cudaMalloc(&B.d_state, sizeof(BState) * count));
  DG_CUDA(cudaMalloc(&B.d_part, sizeof(double) * 3 * B.nunits));
  DG_CUDA(cudaMalloc(&B.d_ctl, sizeof(BCtl)));
  DG_CUDA(cudaMalloc(&B.d_aux, sizeof(double) * 2 * 1024));
  DG_CUDA(cudaMalloc(&B.d_ticket, sizeof(unsigned)));
  DG_CUDA(cudaMallocHost(&B.h_ctl, sizeof(BCtl)));
  *B.h_ctl = BCtl{};
  DG_CUDA(cudaMemcpyAsync(B.d_samples, hs.data(), sizeof(SampleDev) * count,
                          cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemcpyAsync(B.d_units, hu.data(), sizeof(int2) * B.nunits, cudaMemcpyHostToDevice,
                          s));
  DG_CUDA(cudaMemsetAsync(B.d_ticket, 0, sizeof(unsigned), s));
  {
    DGTab<double> t64[MAXN_B - 1];
    DGTab<float> t32;
    for (int n = 2; n <= MAXN_B; ++n) dg_build_tables(n, 2.0 * n * n, &t64[n - 2], &t32);
    DG_CUDA(cudaMemcpyToSymbolAsync(c_btab, t64, sizeof(t64), 0, cudaMemcpyHostToDevice, s));
  }
  const size_t smem = persistent_smem();
  DG_CUDA(cudaFuncSetAttribute(kb_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  int max_bpsm = 0;
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_bpsm, kb_persistent, BT, smem));
  if (max_bpsm < 1)
    return dg_fail(DG_ERR_CUDA, "dg_cg_solve_batched: persistent kernel cannot be resident");
  const int sms = B.meshes[0]->sm_count;

  // bounded barrier waits: ~1 s by default; the test hook shortens it and
  // holds one block back so that the waits expire
  long long limit = 1LL << 24;
  int stall = 0;
  if (const char* e = std::getenv("DG_TEST_BARRIER_STALL")) {
    if (e[0] == '1') {
      stall = 1;
      limit = 1LL << 12;
    }
  }

  std::vector<int> iters_total(count, 0);
  std::vector<int> status(count, DG_OK);
  std::vector<double> rel(count, 0.0);
  int first_bad = DG_OK;
  const int max_rounds = 5;
  for (int round = 0; round < max_rounds; ++round) {
    // (re)start the samples that are not finished: r = b - A x, p = r
    int nstart = 0;
    for (int i = 0; i < count; ++i) {
      if (round > 0 && status[i] != DG_ERR_NOT_CONVERGED) continue;
      dg_mesh* m = B.meshes[i];
      int rc = dg_launch_apply_f64(m, x[i], m->q64, nullptr, s);
      if (rc) return rc;
      kb_init<<<256, 256, 0, s>>>(b[i], m->q64, m->r64, m->p64, hs[i].dinv, m->ndofs, rtol,
                                  B.d_aux, B.d_ticket, B.d_state + i, maxit, iters_total[i]);
      DG_CUDA(cudaGetLastError());
      ++nstart;
    }
    if (round > 0 && nstart == 0) break;
    if (round > 0) {  // the others stay finished
      for (int i = 0; i < count; ++i)
        if (status[i] != DG_ERR_NOT_CONVERGED) {
          BState done = {};
          done.done = 1;
          DG_CUDA(cudaMemcpyAsync(B.d_state + i, &done, sizeof(BState), cudaMemcpyHostToDevice,
                                  s));
        }
    }
    DG_CUDA(cudaStreamSynchronize(s));
    BCtl c0 = {};
    c0.active = count;
    DG_CUDA(cudaMemcpyAsync(B.d_ctl, &c0, sizeof(BCtl), cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaStreamSynchronize(s));
    *B.h_ctl = c0;

    // autotuned blocks per SM; one captured graph per candidate
    int bpsm = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(sig);
      if (it != g_tune.end()) bpsm = it->second;
    }
    std::vector<int> cands;
    if (bpsm > 0) cands.push_back(bpsm);
    else
      for (int c = 1; c <= max_bpsm; ++c) cands.push_back(c);
    // graphs: [c] = production launch (64 iterations), [max_bpsm + 1 + c] = tuning launch
    std::vector<cudaGraphExec_t> execs(2 * (max_bpsm + 1), nullptr);
    auto get_exec = [&](int c, bool tune, cudaGraphExec_t* out) -> int {
      const int slot = tune ? max_bpsm + 1 + c : c;
      if (!execs[slot]) {
        cudaGraph_t g = nullptr;
        DG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = launch_persistent(B, count, c * sms, tune ? ITERS_TUNE : ITERS_PER_LAUNCH,
                                   limit, stall, s);
        cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        DG_CUDA(ec);
        ec = cudaGraphInstantiate(&execs[slot], g, 0);
        cudaGraphDestroy(g);
        DG_CUDA(ec);
      }
      *out = execs[slot];
      return DG_OK;
    };
    auto destroy_execs = [&]() {
      for (auto& e : execs)
        if (e) cudaGraphExecDestroy(e);
    };
    cudaEvent_t e0, e1;
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    double best_t = 1e300;
    int best_c = cands[0];
    size_t ci = 0;
    int rc = DG_OK;
    for (;;) {
      const bool tuning = ci < cands.size() && cands.size() > 1;
      if (!tuning && ci < cands.size()) ci = cands.size();  // one candidate: nothing to tune
      const int c = tuning ? cands[ci] : best_c;
      cudaGraphExec_t ex;
      rc = get_exec(c, tuning, &ex);
      if (rc) break;
      const unsigned long long before = B.h_ctl->iterations_run;
      cudaError_t ec = cudaEventRecord(e0, s);
      if (ec == cudaSuccess) ec = cudaGraphLaunch(ex, s);
      if (ec == cudaSuccess) ec = cudaEventRecord(e1, s);
      if (ec == cudaSuccess)
        ec = cudaMemcpyAsync(B.h_ctl, B.d_ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, s);
      if (ec == cudaSuccess) ec = cudaStreamSynchronize(s);
      if (ec != cudaSuccess) {
        rc = dg_cuda_fail(ec, "dg_cg_solve_batched: persistent launch");
        break;
      }
      if (B.h_ctl->err) {
        rc = dg_fail(DG_ERR_TIMEOUT,
                     "dg_cg_solve_batched: a grid barrier wait expired (%lld spins); the "
                     "persistent kernel stopped", limit);
        break;
      }
      if (tuning) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const unsigned long long ran = B.h_ctl->iterations_run - before;
        if (ran > 0) {
          const double per = ms / (double)ran;
          if (per < best_t) {
            best_t = per;
            best_c = c;
          }
        }
        ++ci;
        if (ci == cands.size() && best_t < 1e300) {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tune[sig] = best_c;
        }
      }
      if (B.h_ctl->active == 0) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    destroy_execs();
    if (rc) return rc;

    // per-sample outcome, with the residual recomputed in FP64
    std::vector<BState> hst(count);
    DG_CUDA(cudaMemcpyAsync(hst.data(), B.d_state, sizeof(BState) * count,
                            cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    bool any_restart = false;
    for (int i = 0; i < count; ++i) {
      if (round > 0 && status[i] != DG_ERR_NOT_CONVERGED) continue;
      dg_mesh* m = B.meshes[i];
      iters_total[i] = hst[i].iters;
      rc = dg_launch_apply_f64(m, x[i], m->q64, nullptr, s);
      if (rc) return rc;
      kb_residual<<<1, 256, 0, s>>>(b[i], m->q64, m->ndofs, B.d_aux);
      double out[2];
      DG_CUDA(cudaMemcpyAsync(out, B.d_aux, sizeof(out), cudaMemcpyDeviceToHost, s));
      DG_CUDA(cudaStreamSynchronize(s));
      rel[i] = out[1] > 0 ? std::sqrt(out[0] / out[1]) : 0.0;
      if (out[1] == 0.0 && !hst[i].breakdown)  // A x = 0 has the solution x = 0
        DG_CUDA(cudaMemsetAsync(x[i], 0, sizeof(double) * (size_t)m->ndofs, s));
      if (hst[i].breakdown) status[i] = DG_ERR_BREAKDOWN;
      else if (out[1] == 0.0 || rel[i] <= rtol) status[i] = DG_OK;
      else {
        status[i] = DG_ERR_NOT_CONVERGED;
        if (hst[i].iters < maxit) any_restart = true;
      }
    }
    if (!any_restart) break;
  }
  const double dt = now_s() - t0;
  for (int i = 0; i < count; ++i) {
    if (st) {
      st[i].iterations = iters_total[i];
      st[i].outer_iterations = 0;
      st[i].rel_residual = rel[i];
      st[i].rel_residual_rec = rel[i];
      st[i].seconds = dt;
      st[i].status = status[i];
    }
    if (status[i] != DG_OK && first_bad == DG_OK) {
      first_bad = status[i];
      dg_fail(first_bad, "dg_cg_solve_batched: sample %d: %s (relative residual %.3e)", i,
              status[i] == DG_ERR_BREAKDOWN ? "breakdown" : "not converged", rel[i]);
    }
  }
  return first_bad;
}

extern "C" int dg_cg_solve_batched(const dg_mesh* const* meshes, int count, const double* const* b,
                                   double* const* x, double rtol, int maxit, dg_cg_stats* st,
                                   void* stream) {
  return dg_cg_solve_batched_mode(meshes, count, b, x, rtol, maxit, DG_CG_FP64, st, stream);
}
