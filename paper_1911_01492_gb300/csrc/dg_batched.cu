// Batched CG: many independent systems A_s x_s = b_s (different coefficient
// samples, mesh sizes and degrees, as in the multilevel Monte-Carlo setting of
// Section 5) solved in lock-step by one persistent kernel.
//
// Each sample runs preconditioned CG (M = I, or M = diag(A) with
// DG_CG_PRECOND_JACOBI) with its own scalars, like the k independent solvers
// running in lock-step of the horizontal vectorisation in Section 3.5.  The
// recurrence is the single-reduction variant of Section 2.4 (Chronopoulos and
// Gear): s = A p is carried by its own recurrence, so every iteration applies
// the operator once, to u = M^-1 r, and needs the three inner products
// (r, u), (w, u) and (r, r) (w = A u) at one point:
//   phase 1, per work unit:  p = u + beta p,  s = w + beta s,  x += alpha p,
//                            r -= alpha s,  u = M^-1 r,  pass 1 of u
//                            (nodal values and face traces);
//   phase 2, per work unit:  pass 2 -> w = A u; the unit's partial sums of
//                            (r, u), (w, u), (r, r); the last unit of a sample
//                            to finish (a per-sample ticket) adds the sample's
//                            partials in a fixed order and forms
//                            gamma' = (r, u), beta = gamma' / gamma and
//                            alpha = gamma' / ((w, u) - beta gamma' / alpha),
//                            and tests (r, r) against the tolerance.
// Two grid-wide barriers per iteration: between the passes (pass 2 reads the
// neighbours' traces) and after the scalars.  Each barrier spins a bounded
// number of times; on expiry the kernel raises an error flag and returns, and
// the host reports DG_ERR_TIMEOUT.  Work units of finished samples are
// skipped, so uneven samples cost what they need (work proportional to size x
// iterations, the proportional allocation of Section 5).  A launch runs until
// every sample is done or for a number of iterations sized to about two
// seconds of work, and is captured in a CUDA graph that is replayed until the
// device-side count of active samples reaches zero.
//
// An autotuner picks the launch shape: resident blocks per SM and the tile of
// cells a block takes per work unit (1, 2 or 4 groups of the operator kernels'
// cells per block), by timing the first graph replays (real CG iterations)
// of each candidate.  Choices are cached per batch signature in the process
// and, if DG_TUNE_CACHE names a file, in that file.  DG_BATCHED_SHAPE="B,T"
// forces B blocks per SM (at most the resident maximum) and tile index T.
//
// Degrees 1..4 run in 128-thread blocks; a batch with any degree 5..8 runs in
// a 256-thread instantiation (the operator kernels' cell groups need up to
// 256 threads there).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dg_nodal_impl.cuh"

namespace {

constexpr int ITERS_TUNE = 4;         // iterations per launch while autotuning
constexpr int TILES[3] = {1, 2, 4};   // cell groups per work unit (tuned)
constexpr double LAUNCH_SECONDS = 2.0;   // work per production launch (estimate)
constexpr double EST_DOF_RATE = 7.0e9;   // DOF-iterations per second for that estimate

__constant__ DGTab<double> c_btab[DG_MAXN - 1];  // tables for n = 2..9
__constant__ DGTabN<double> c_btabN[DG_MAXN - 1];  // scaled Gauss-point basis, n = 2..9

struct SampleDev {
  const double* b;
  double* x;
  double *r, *u, *w, *p, *s;  // u == r when M = I
  double *U, *X, *TR;
  const double* kt;      // h w K (not read: the line operators hold the volume term)
  const double* fw;
  const double* lineop;  // line operators of A, or of Q A Q^T in the scaled Gauss-point basis
  const double* gh;      // h gamma per face side (the point basis's face weights)
  const double* dinv;  // 1 / diag(A) for M = diag(A); nullptr for M = I
  long long ncells;
  int Nc;          // cells per direction
  int n;           // points per direction
  int ubeg, uend;  // work units of this sample in the launch's unit list
};

struct BState {
  double gamma, delta, alpha, beta, rr, tol2, bnorm2;
  int done, breakdown, iters, maxit;
};

struct BCtl {
  unsigned count;     // barrier arrivals
  unsigned gen;       // barrier generation
  int err;            // 1: a barrier wait expired
  int active;         // samples not done (decremented by the sample's last unit)
  unsigned long long iterations_run;  // lock-step iterations executed
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block sum in a fixed order; result valid in every thread.
template <int BT>
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

__host__ __device__ constexpr int group_cells(int n) {
  return n == 2 ? dgk::Cfg<2>::CPB : n == 3 ? dgk::Cfg<3>::CPB : n == 4 ? dgk::Cfg<4>::CPB
       : n == 5 ? dgk::Cfg<5>::CPB : n == 6 ? dgk::Cfg<6>::CPB : n == 7 ? dgk::Cfg<7>::CPB
       : n == 8 ? dgk::Cfg<8>::CPB : dgk::Cfg<9>::CPB;
}

// ND: the samples' vectors are in the scaled Gauss-point basis (DG_CG_NODAL)
// and the passes are the transform-free ones of dg_nodal_impl.cuh.
template <int N, bool ND>
__device__ __forceinline__ void group_pass1(const SampleDev& S, long long c0, int nblk,
                                            double* smem) {
  if constexpr (ND)
    dgk::trace_cells_nd<N, double>(S.u, S.TR, c0, nblk, c_btabN[N - 2], smem);
  else
    dgk::trace_cells<N, double>(S.u, S.U, S.X, S.TR, c0, nblk, c_btab[N - 2], smem);
}
template <int N, bool ND>
__device__ __forceinline__ void group_pass2(const SampleDev& S, long long c0, int nblk,
                                            double* smem) {
  if constexpr (ND)
    dgk::cell_cells_nd<N>(S.u, S.TR, S.lineop, S.gh, S.w, c0, nblk, S.Nc, c_btabN[N - 2], smem);
  else
    dgk::cell_cells<N, double, true>(S.U, S.X, S.TR, S.kt, S.fw, S.w, c0, nblk, S.Nc,
                                     c_btab[N - 2], smem, S.lineop);
}

template <int MAXN, bool ND>
__device__ __forceinline__ void pass1_dispatch(const SampleDev& sd, long long c, int nblk,
                                               double* smem) {
  switch (sd.n) {
    case 2: group_pass1<2, ND>(sd, c, nblk, smem); break;
    case 3: group_pass1<3, ND>(sd, c, nblk, smem); break;
    case 4: group_pass1<4, ND>(sd, c, nblk, smem); break;
    case 5: group_pass1<5, ND>(sd, c, nblk, smem); break;
    default:
      if constexpr (MAXN > 5) {
        switch (sd.n) {
          case 6: group_pass1<6, ND>(sd, c, nblk, smem); break;
          case 7: group_pass1<7, ND>(sd, c, nblk, smem); break;
          case 8: group_pass1<8, ND>(sd, c, nblk, smem); break;
          default: group_pass1<9, ND>(sd, c, nblk, smem); break;
        }
      }
      break;
  }
}

template <int MAXN, bool ND>
__device__ __forceinline__ void pass2_dispatch(const SampleDev& sd, long long c, int nblk,
                                               double* smem) {
  switch (sd.n) {
    case 2: group_pass2<2, ND>(sd, c, nblk, smem); break;
    case 3: group_pass2<3, ND>(sd, c, nblk, smem); break;
    case 4: group_pass2<4, ND>(sd, c, nblk, smem); break;
    case 5: group_pass2<5, ND>(sd, c, nblk, smem); break;
    default:
      if constexpr (MAXN > 5) {
        switch (sd.n) {
          case 6: group_pass2<6, ND>(sd, c, nblk, smem); break;
          case 7: group_pass2<7, ND>(sd, c, nblk, smem); break;
          case 8: group_pass2<8, ND>(sd, c, nblk, smem); break;
          default: group_pass2<9, ND>(sd, c, nblk, smem); break;
        }
      }
      break;
  }
}

// One persistent launch of up to `iters` lock-step iterations over every
// unfinished sample.  `tile`: cell groups per work unit.
template <int BT, int MAXN, bool ND>
__global__ void __launch_bounds__(BT, BT == 128 ? 6 : 3)
kb_persistent(const SampleDev* __restrict__ S, const int2* __restrict__ units, int nu, int tile,
              BState* st, double* part, unsigned* tickets, BCtl* ctl, int iters, long long limit,
              int stall_test) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* smem = reinterpret_cast<double*>(smem_raw);
  __shared__ double sred[BT / 32];
  __shared__ bool is_last;
  const unsigned nb = gridDim.x;
  if (stall_test && blockIdx.x == 0) return;  // test hook: one block never arrives
  for (int it = 0; it < iters; ++it) {
    if (((volatile int*)&ctl->active)[0] == 0) break;
    // phase 1: vector recurrences on the unit's cells, then pass 1 of u
    for (int uu = blockIdx.x; uu < nu; uu += nb) {
      const int s = units[uu].x;
      if (st[s].done) continue;
      const SampleDev& sd = S[s];
      const int cpb = group_cells(sd.n);
      const long long c0 = units[uu].y;
      const long long c1 = (c0 + (long long)tile * cpb) < sd.ncells ? c0 + (long long)tile * cpb
                                                                    : sd.ncells;
      const long long n3 = (long long)sd.n * sd.n * sd.n;
      const double al = st[s].alpha, be = st[s].beta;
      if (sd.dinv) {  // two loops: no per-element branch between the loads
        for (long long i = c0 * n3 + threadIdx.x; i < c1 * n3; i += BT) {
          const double pi = fma(be, sd.p[i], sd.u[i]);
          const double si = fma(be, sd.s[i], sd.w[i]);
          sd.p[i] = pi;
          sd.s[i] = si;
          sd.x[i] = fma(al, pi, sd.x[i]);
          const double ri = fma(-al, si, sd.r[i]);
          sd.r[i] = ri;
          sd.u[i] = sd.dinv[i] * ri;
        }
      } else {
        for (long long i = c0 * n3 + threadIdx.x; i < c1 * n3; i += BT) {
          const double pi = fma(be, sd.p[i], sd.r[i]);
          const double si = fma(be, sd.s[i], sd.w[i]);
          sd.p[i] = pi;
          sd.s[i] = si;
          sd.x[i] = fma(al, pi, sd.x[i]);
          sd.r[i] = fma(-al, si, sd.r[i]);
        }
      }
      __syncthreads();
      for (long long c = c0; c < c1; c += cpb) {
        const int nblk = (int)((c1 - c) < cpb ? (c1 - c) : cpb);
        pass1_dispatch<MAXN, ND>(sd, c, nblk, smem);
        __syncthreads();
      }
    }
    if (!grid_sync(ctl, nb, limit)) return;
    // phase 2: w = A u, the unit's partial sums, the sample's scalars
    for (int uu = blockIdx.x; uu < nu; uu += nb) {
      const int s = units[uu].x;
      if (st[s].done) continue;
      const SampleDev& sd = S[s];
      const int cpb = group_cells(sd.n);
      const long long c0 = units[uu].y;
      const long long c1 = (c0 + (long long)tile * cpb) < sd.ncells ? c0 + (long long)tile * cpb
                                                                    : sd.ncells;
      for (long long c = c0; c < c1; c += cpb) {
        const int nblk = (int)((c1 - c) < cpb ? (c1 - c) : cpb);
        pass2_dispatch<MAXN, ND>(sd, c, nblk, smem);
        __syncthreads();
      }
      const long long n3 = (long long)sd.n * sd.n * sd.n;
      double ru = 0.0, wu = 0.0, rr = 0.0;
      for (long long i = c0 * n3 + threadIdx.x; i < c1 * n3; i += BT) {
        const double ri = sd.r[i], ui = sd.u[i];
        ru = fma(ri, ui, ru);
        wu = fma(sd.w[i], ui, wu);
        rr = fma(ri, ri, rr);
      }
      ru = block_sum<BT>(ru, sred);
      wu = block_sum<BT>(wu, sred);
      rr = block_sum<BT>(rr, sred);
      if (threadIdx.x == 0) {
        part[3 * uu] = ru;
        part[3 * uu + 1] = wu;
        part[3 * uu + 2] = rr;
        __threadfence();
        is_last = atomicAdd(&tickets[s], 1u) == (unsigned)(sd.uend - sd.ubeg) - 1;
      }
      __syncthreads();
      if (!is_last) continue;
      __threadfence();
      // the sample's last unit: fixed-order sums of all its units' partials
      double a = 0.0, b = 0.0, c = 0.0;
      const volatile double* vp = part;
      for (int v = sd.ubeg + threadIdx.x; v < sd.uend; v += BT) {
        a += vp[3 * v];
        b += vp[3 * v + 1];
        c += vp[3 * v + 2];
      }
      a = block_sum<BT>(a, sred);
      b = block_sum<BT>(b, sred);
      c = block_sum<BT>(c, sred);
      if (threadIdx.x == 0) {
        BState& q = st[s];
        q.iters += 1;
        if (!isfinite(a) || !isfinite(b) || !isfinite(c)) {
          q.breakdown = 1;
          q.done = 1;
        } else {
          q.rr = c;
          if (c <= q.tol2 || q.iters >= q.maxit) {
            q.done = 1;
          } else {
            const double beta = a / q.gamma;
            const double den = b - beta * a / q.alpha;  // (p, A p) of the next direction
            if (!(den > 0.0) || !(a > 0.0)) {
              q.breakdown = 1;
              q.done = 1;
            } else {
              q.beta = beta;
              q.alpha = a / den;
              q.gamma = a;
              q.delta = b;
            }
          }
        }
        if (q.done) atomicSub(&ctl->active, 1);
        tickets[s] = 0u;
      }
      __syncthreads();
    }
    if (!grid_sync(ctl, nb, limit)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->iterations_run += 1;
  }
}

// Deterministic sums of up to three products over a vector: a fixed grid of
// 256 blocks writes partials, the last block adds them in a fixed order.
// Start of a sample (after w = A x):
//   r = b - w, u = M^-1 r (dinv; u is r itself for M = I), p = s = 0,
//   bnorm2 = (b, b), rr = (r, r), tol2 = rtol^2 bnorm2.
__global__ void __launch_bounds__(256)
kb_init_r(const double* __restrict__ b, const double* __restrict__ w, double* __restrict__ r,
          double* __restrict__ u, double* __restrict__ p, double* __restrict__ sv,
          const double* __restrict__ dinv, long long n, double rtol, double* partials,
          unsigned* ticket, BState* st, int maxit, int keep_iters) {
  __shared__ double sred[8];
  __shared__ bool last;
  double rr = 0.0, bb = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - w[i];
    r[i] = ri;
    if (dinv) u[i] = dinv[i] * ri;
    p[i] = 0.0;
    sv[i] = 0.0;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  rr = block_sum<256>(rr, sred);
  bb = block_sum<256>(bb, sred);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rr;
    partials[2 * blockIdx.x + 1] = bb;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      a += ((volatile double*)partials)[2 * i];
      c += ((volatile double*)partials)[2 * i + 1];
    }
    BState s = {};
    s.rr = a;
    s.bnorm2 = c;
    s.tol2 = rtol * rtol * c;
    s.maxit = maxit;
    s.iters = keep_iters;
    s.breakdown = !(isfinite(a) && isfinite(c));
    // b = 0: the solution is x = 0 (set by the host), nothing to iterate
    s.done = s.breakdown || c == 0.0 || a <= s.tol2 || keep_iters >= maxit;
    *st = s;
    *ticket = 0u;
  }
}

// After w = A u: gamma = (r, u), delta = (w, u), alpha = gamma / delta, beta = 0.
__global__ void __launch_bounds__(256)
kb_init_scalars(const double* __restrict__ r, const double* __restrict__ u,
                const double* __restrict__ w, long long n, double* partials, unsigned* ticket,
                BState* st) {
  __shared__ double sred[8];
  __shared__ bool last;
  double g = 0.0, d = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    g = fma(r[i], u[i], g);
    d = fma(w[i], u[i], d);
  }
  g = block_sum<256>(g, sred);
  d = block_sum<256>(d, sred);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = g;
    partials[2 * blockIdx.x + 1] = d;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      a += ((volatile double*)partials)[2 * i];
      c += ((volatile double*)partials)[2 * i + 1];
    }
    BState s = *st;
    if (!s.done) {
      if (!isfinite(a) || !isfinite(c) || !(c > 0.0) || !(a > 0.0)) {
        s.breakdown = 1;
        s.done = 1;
      } else {
        s.gamma = a;
        s.delta = c;
        s.alpha = a / c;
        s.beta = 0.0;
      }
    }
    *st = s;
    *ticket = 0u;
  }
}

// ||b - q||^2 and ||b||^2 into out[0..1] (single block, fixed order).
__global__ void __launch_bounds__(256)
kb_residual(const double* __restrict__ b, const double* __restrict__ q, long long n,
            double* out) {
  __shared__ double sred[8];
  double rr = 0.0, bb = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double ri = b[i] - q[i];
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  rr = block_sum<256>(rr, sred);
  bb = block_sum<256>(bb, sred);
  if (threadIdx.x == 0) {
    out[0] = rr;
    out[1] = bb;
  }
}

template <int MAXN, bool ND>
size_t persistent_smem() {
  if constexpr (ND) {  // the point basis's passes need half the shared memory
    size_t m = 0;
    m = std::max(m, dgk::cell_smem_nd<2>());
    m = std::max(m, dgk::cell_smem_nd<3>());
    m = std::max(m, dgk::cell_smem_nd<4>());
    m = std::max(m, dgk::cell_smem_nd<5>());
    if (MAXN > 5) {
      m = std::max(m, dgk::cell_smem_nd<6>());
      m = std::max(m, dgk::cell_smem_nd<7>());
      m = std::max(m, dgk::cell_smem_nd<8>());
      m = std::max(m, dgk::cell_smem_nd<9>());
    }
    return m;
  }
  size_t m = 0;
  m = std::max(m, dgk::cell_smem<2, double>());
  m = std::max(m, dgk::cell_smem<3, double>());
  m = std::max(m, dgk::cell_smem<4, double>());
  m = std::max(m, dgk::cell_smem<5, double>());
  if (MAXN > 5) {
    m = std::max(m, dgk::cell_smem<6, double>());
    m = std::max(m, dgk::cell_smem<7, double>());
    m = std::max(m, dgk::cell_smem<8, double>());
    m = std::max(m, dgk::cell_smem<9, double>());
  }
  return m;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Autotuner cache: batch signature -> (blocks per SM, tile index), in the
// process and optionally in the file DG_TUNE_CACHE (one "signature bpsm tile"
// line per entry; the signature includes the GPU name).
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;
bool g_tune_file_read = false;

void tune_cache_load() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = std::getenv("DG_TUNE_CACHE");
  if (path == nullptr || path[0] == 0) return;
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return;
  char line[4096];
  while (std::fgets(line, sizeof(line), f)) {
    char sig[3800];
    int bpsm = 0, tile = 0;
    if (std::sscanf(line, "%3799s %d %d", sig, &bpsm, &tile) == 3 && bpsm > 0 && tile >= 0 &&
        tile < 3)
      g_tune[sig] = {bpsm, tile};
  }
  std::fclose(f);
}

void tune_cache_store(const std::string& sig, int bpsm, int tile) {
  g_tune[sig] = {bpsm, tile};
  const char* path = std::getenv("DG_TUNE_CACHE");
  if (path == nullptr || path[0] == 0 || sig.size() >= 3800) return;
  FILE* f = std::fopen(path, "a");
  if (f == nullptr) return;
  std::fprintf(f, "%s %d %d\n", sig.c_str(), bpsm, tile);
  std::fclose(f);
}

struct Batch {
  std::vector<dg_mesh*> meshes;
  SampleDev* d_samples = nullptr;  // 3 x count: one copy per tile choice
  int2* d_units = nullptr;         // unit lists of the three tile choices, concatenated
  int unit_off[3] = {0, 0, 0};
  int nunits[3] = {0, 0, 0};
  BState* d_state = nullptr;
  double* d_part = nullptr;
  unsigned* d_tickets = nullptr;
  BCtl* d_ctl = nullptr;
  BCtl* h_ctl = nullptr;
  double* d_aux = nullptr;      // init partials, residual outputs
  unsigned* d_ticket = nullptr;
  ~Batch() {
    cudaFree(d_samples);
    cudaFree(d_units);
    cudaFree(d_state);
    cudaFree(d_part);
    cudaFree(d_tickets);
    cudaFree(d_ctl);
    cudaFree(d_aux);
    cudaFree(d_ticket);
    if (h_ctl) cudaFreeHost(h_ctl);
  }
};

template <int BT, int MAXN, bool ND>
int launch_persistent(Batch& B, int count, int tsel, int blocks, int iters, long long limit,
                      int stall, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = persistent_smem<MAXN, ND>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DG_CUDA(cudaLaunchKernelEx(&cfg, kb_persistent<BT, MAXN, ND>,
                             (const SampleDev*)(B.d_samples + (size_t)tsel * count),
                             (const int2*)(B.d_units + B.unit_off[tsel]), B.nunits[tsel],
                             TILES[tsel], B.d_state, B.d_part, B.d_tickets, B.d_ctl, iters,
                             limit, stall));
  return DG_OK;
}

// Start (or restart) sample i: w = A x, r = b - w, u = M^-1 r, w = A u, scalars.
int start_sample(Batch& B, const SampleDev& d, dg_mesh* m, const double* b, const double* x,
                 double rtol, int maxit, int keep_iters, int i, cudaStream_t s) {
  int rc = dg_launch_apply_f64(m, x, d.w, nullptr, s);
  if (rc) return rc;
  kb_init_r<<<256, 256, 0, s>>>(b, d.w, d.r, d.u, d.p, d.s, d.dinv, m->ndofs, rtol, B.d_aux,
                                B.d_ticket, B.d_state + i, maxit, keep_iters);
  DG_CUDA(cudaGetLastError());
  rc = dg_launch_apply_f64(m, d.u, d.w, nullptr, s);
  if (rc) return rc;
  kb_init_scalars<<<256, 256, 0, s>>>(d.r, d.u, d.w, m->ndofs, B.d_aux, B.d_ticket,
                                      B.d_state + i);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int BT, int MAXN, bool ND>
int solve_batched(const dg_mesh* const* meshes, int count, const double* const* b,
                  double* const* x, double rtol, int maxit, bool jacobi, int mode,
                  dg_cg_stats* st, void* stream) {
  const double t0 = now_s();
  Batch B;
  B.meshes.resize(count);
  std::vector<SampleDev> hs(count);
  std::vector<int2> hu[3];
  std::vector<SampleDev> hst3;
  std::string sig = "bt" + std::to_string(BT) + "_mode" + std::to_string(mode);
  long long total_dofs = 0;
  for (int s = 0; s < count; ++s) {
    dg_mesh* m = const_cast<dg_mesh*>(meshes[s]);
    int rc = dg_ensure_solver_ws(m);
    if (rc) return rc;
    B.meshes[s] = m;
    SampleDev& d = hs[s];
    d.b = b[s];
    d.x = x[s];
    d.r = m->r64;
    d.p = m->p64;
    d.w = m->q64;
    d.s = m->s64;
    d.u = m->r64;  // M = I: u is r itself
    d.U = m->U64;
    d.X = m->X64;
    d.TR = m->TR64;
    d.kt = m->kt64;
    d.fw = m->fw64;
    d.lineop = ND ? m->lineopN64 : m->lineop64;
    d.gh = m->gh64;
    d.dinv = nullptr;
    if (jacobi) {
      rc = dg_ensure_diagonal(m, m->solve_stream);
      if (rc) return rc;
      d.dinv = m->dinv64;
      d.u = m->t64;
    }
    d.ncells = m->ncells;
    d.Nc = m->N;
    d.n = m->n;
    total_dofs += m->ndofs;
    sig += "_" + std::to_string(m->N) + "x" + std::to_string(m->n);
  }
  for (int t = 0; t < 3; ++t) {
    for (int s = 0; s < count; ++s) {
      SampleDev d = hs[s];
      const int step = TILES[t] * group_cells(d.n);
      d.ubeg = (int)hu[t].size();
      for (long long c = 0; c < d.ncells; c += step) hu[t].push_back(make_int2(s, (int)c));
      d.uend = (int)hu[t].size();
      hst3.push_back(d);
    }
    B.nunits[t] = (int)hu[t].size();
    B.unit_off[t] = t == 0 ? 0 : B.unit_off[t - 1] + B.nunits[t - 1];
  }
  cudaStream_t us = (cudaStream_t)stream;
  // a private non-blocking stream (capture needs one); ordered after the caller's work
  cudaStream_t s = B.meshes[0]->solve_stream;
  DG_CUDA(cudaEventRecord(B.meshes[0]->ev, us));
  DG_CUDA(cudaStreamWaitEvent(s, B.meshes[0]->ev, 0));
  const int nu_all = B.unit_off[2] + B.nunits[2];
  DG_CUDA(cudaMalloc(&B.d_samples, sizeof(SampleDev) * 3 * count));
  DG_CUDA(cudaMalloc(&B.d_units, sizeof(int2) * nu_all));
  DG_CUDA(cudaMalloc(&B.d_state, sizeof(BState) * count));
  DG_CUDA(cudaMalloc(&B.d_part, sizeof(double) * 3 * B.nunits[0]));
  DG_CUDA(cudaMalloc(&B.d_tickets, sizeof(unsigned) * count));
  DG_CUDA(cudaMalloc(&B.d_ctl, sizeof(BCtl)));
  DG_CUDA(cudaMalloc(&B.d_aux, sizeof(double) * 2 * 1024));
  DG_CUDA(cudaMalloc(&B.d_ticket, sizeof(unsigned)));
  DG_CUDA(cudaMallocHost(&B.h_ctl, sizeof(BCtl)));
  *B.h_ctl = BCtl{};
  DG_CUDA(cudaMemcpyAsync(B.d_samples, hst3.data(), sizeof(SampleDev) * 3 * count,
                          cudaMemcpyHostToDevice, s));
  for (int t = 0; t < 3; ++t)
    DG_CUDA(cudaMemcpyAsync(B.d_units + B.unit_off[t], hu[t].data(), sizeof(int2) * B.nunits[t],
                            cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(B.d_ticket, 0, sizeof(unsigned), s));
  DG_CUDA(cudaMemsetAsync(B.d_tickets, 0, sizeof(unsigned) * count, s));
  {
    DGTab<double> t64[DG_MAXN - 1];
    DGTab<float> t32;
    for (int n = 2; n <= DG_MAXN; ++n) dg_build_tables(n, 2.0 * n * n, &t64[n - 2], &t32);
    DG_CUDA(cudaMemcpyToSymbolAsync(c_btab, t64, sizeof(t64), 0, cudaMemcpyHostToDevice, s));
    if (ND) {
      DGTabN<double> tn64[DG_MAXN - 1];
      DGTabN<float> tn32;
      for (int n = 2; n <= DG_MAXN; ++n) dg_build_nodal_tables(t64[n - 2], n, &tn64[n - 2], &tn32);
      DG_CUDA(cudaMemcpyToSymbolAsync(c_btabN, tn64, sizeof(tn64), 0, cudaMemcpyHostToDevice, s));
    }
  }
  const size_t smem = persistent_smem<MAXN, ND>();
  DG_CUDA(cudaFuncSetAttribute(kb_persistent<BT, MAXN, ND>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int max_bpsm = 0;
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_bpsm, kb_persistent<BT, MAXN, ND>, BT,
                                                        smem));
  if (max_bpsm < 1)
    return dg_fail(DG_ERR_CUDA, "dg_cg_solve_batched: persistent kernel cannot be resident");
  const int sms = B.meshes[0]->sm_count;
  {
    cudaDeviceProp prop;
    DG_CUDA(cudaGetDeviceProperties(&prop, B.meshes[0]->device));
    std::string name(prop.name);
    for (char& ch : name)
      if (ch == ' ') ch = '_';
    sig = name + "_" + sig;
  }

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
  // iterations per production launch: about LAUNCH_SECONDS of work
  int iters_launch = (int)(LAUNCH_SECONDS * EST_DOF_RATE / (double)(total_dofs > 0 ? total_dofs : 1));
  iters_launch = iters_launch < 64 ? 64 : iters_launch > 4096 ? 4096 : iters_launch;

  std::vector<int> iters_total(count, 0);
  std::vector<int> status(count, DG_OK);
  std::vector<double> rel(count, 0.0);
  int first_bad = DG_OK;
  const int max_rounds = 5;
  for (int round = 0; round < max_rounds; ++round) {
    // (re)start the samples that are not finished
    int nstart = 0;
    for (int i = 0; i < count; ++i) {
      if (round > 0 && status[i] != DG_ERR_NOT_CONVERGED) continue;
      int rc = start_sample(B, hs[i], B.meshes[i], b[i], x[i], rtol, maxit, iters_total[i], i, s);
      if (rc) return rc;
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
    std::vector<BState> h0(count);
    DG_CUDA(cudaMemcpyAsync(h0.data(), B.d_state, sizeof(BState) * count, cudaMemcpyDeviceToHost,
                            s));
    DG_CUDA(cudaStreamSynchronize(s));
    BCtl c0 = {};
    for (int i = 0; i < count; ++i) c0.active += h0[i].done ? 0 : 1;
    DG_CUDA(cudaMemcpyAsync(B.d_ctl, &c0, sizeof(BCtl), cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaStreamSynchronize(s));
    *B.h_ctl = c0;

    // autotuned launch shape: (blocks per SM, tile); one captured graph per candidate
    std::pair<int, int> chosen = {0, 0};
    if (const char* e = std::getenv("DG_BATCHED_SHAPE")) {  // "blocks_per_sm,tile_index"
      int bp = 0, ti = -1;
      if (std::sscanf(e, "%d,%d", &bp, &ti) == 2 && bp >= 1 && ti >= 0 && ti < 3)
        chosen = {bp < max_bpsm ? bp : max_bpsm, ti};
    }
    if (chosen.first == 0) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_cache_load();
      auto it = g_tune.find(sig);
      if (it != g_tune.end() && it->second.first <= max_bpsm) chosen = it->second;
    }
    std::vector<std::pair<int, int>> cands;
    if (chosen.first > 0) cands.push_back(chosen);
    else
      for (int t = 0; t < 3; ++t)
        for (int c = 1; c <= max_bpsm; ++c) cands.push_back({c, t});
    std::map<std::pair<int, int>, cudaGraphExec_t> execs;  // key: (candidate index, tuning)
    auto get_exec = [&](int ci, bool tune, cudaGraphExec_t* out) -> int {
      const auto key = std::make_pair(ci, tune ? 1 : 0);
      auto f = execs.find(key);
      if (f == execs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        DG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = launch_persistent<BT, MAXN, ND>(B, count, cands[ci].second,
                                                 cands[ci].first * sms,
                                             tune ? ITERS_TUNE : iters_launch, limit, stall, s);
        cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        DG_CUDA(ec);
        ec = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        DG_CUDA(ec);
        f = execs.emplace(key, ex).first;
      }
      *out = f->second;
      return DG_OK;
    };
    cudaEvent_t e0, e1;
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    double best_t = 1e300;
    int best_ci = 0;
    size_t ci = 0;
    int rc = DG_OK;
    for (;;) {
      const bool tuning = ci < cands.size() && cands.size() > 1;
      if (!tuning && ci < cands.size()) ci = cands.size();  // one candidate: nothing to tune
      const int cidx = tuning ? (int)ci : best_ci;
      cudaGraphExec_t ex;
      rc = get_exec(cidx, tuning, &ex);
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
            best_ci = (int)ci;
          }
        }
        ++ci;
        if (ci == cands.size() && best_t < 1e300) {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          tune_cache_store(sig, cands[best_ci].first, cands[best_ci].second);
        }
      }
      if (B.h_ctl->active == 0) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto& kv : execs) cudaGraphExecDestroy(kv.second);
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

// The batch in the scaled Gauss-point basis (DG_CG_NODAL, M = I): every
// sample's b and x mapped into the basis, the lock-step solve on Q A Q^T with
// the transform-free passes, x mapped back, and the residual recomputed in the
// Legendre basis; a sample that the mapping's rounding left above rtol is
// finished by the one-sample FP64 CG from its x.
int solve_batched_nodal(const dg_mesh* const* meshes, int count, const double* const* b,
                        double* const* x, double rtol, int maxit, int maxn, int mode,
                        dg_cg_stats* st, void* stream) {
  cudaStream_t us = (cudaStream_t)stream;
  std::vector<const double*> bn(count);
  std::vector<double*> xn(count);
  for (int i = 0; i < count; ++i) {
    dg_mesh* m = const_cast<dg_mesh*>(meshes[i]);
    int rc = dg_ensure_solver_ws(m);
    if (rc == DG_OK) rc = dg_ensure_nodal(m, us);
    if (rc == DG_OK) rc = dg_launch_collocation(m, b[i], m->bN64, true, us);
    if (rc == DG_OK) rc = dg_launch_collocation(m, x[i], m->xN64, true, us);
    if (rc) return rc;
    bn[i] = m->bN64;
    xn[i] = m->xN64;
  }
  std::vector<dg_cg_stats> local(st ? 0 : count);
  dg_cg_stats* sts = st ? st : local.data();
  int rc;
  {
    struct Scope {  // the internal FP64 launcher applies Q A Q^T while it lives
      const dg_mesh* const* ms;
      int n;
      Scope(const dg_mesh* const* a, int c) : ms(a), n(c) {
        for (int i = 0; i < n; ++i) const_cast<dg_mesh*>(ms[i])->nodal_op = true;
      }
      ~Scope() {
        for (int i = 0; i < n; ++i) const_cast<dg_mesh*>(ms[i])->nodal_op = false;
      }
    } scope(meshes, count);
    rc = maxn <= 5 ? solve_batched<128, 5, true>(meshes, count, bn.data(), xn.data(), rtol, maxit,
                                                 false, mode, sts, stream)
                   : solve_batched<256, DG_MAXN, true>(meshes, count, bn.data(), xn.data(), rtol,
                                                       maxit, false, mode, sts, stream);
  }
  if (rc != DG_OK && rc != DG_ERR_NOT_CONVERGED && rc != DG_ERR_BREAKDOWN) return rc;
  for (int i = 0; i < count; ++i) {
    dg_mesh* m = const_cast<dg_mesh*>(meshes[i]);
    int r2 = dg_launch_collocation(m, xn[i], x[i], false, us);
    if (r2) return r2;
    r2 = dg_launch_apply_f64(m, x[i], m->q64, nullptr, us);
    if (r2) return r2;
    kb_residual<<<1, 256, 0, us>>>(b[i], m->q64, m->ndofs, m->partials);
    double out[2];
    DG_CUDA(cudaMemcpyAsync(out, m->partials, sizeof(out), cudaMemcpyDeviceToHost, us));
    DG_CUDA(cudaStreamSynchronize(us));
    const double rel = out[1] > 0 ? std::sqrt(out[0] / out[1]) : 0.0;
    sts[i].rel_residual = sts[i].rel_residual_rec = rel;
    if (sts[i].status == DG_OK && rel > rtol) {
      dg_cg_stats ps{};
      const int left = maxit - sts[i].iterations;
      const int prc = left >= 1 ? dg_cg_solve(m, b[i], x[i], rtol, left, DG_CG_FP64, &ps, stream)
                                : DG_ERR_NOT_CONVERGED;
      sts[i].iterations += ps.iterations;
      sts[i].outer_iterations += 1;
      if (left >= 1) sts[i].rel_residual = sts[i].rel_residual_rec = ps.rel_residual;
      sts[i].status = prc;
      if (prc != DG_OK && rc == DG_OK) {
        rc = prc;
        dg_fail(prc, "dg_cg_solve_batched: sample %d: not converged after the point-basis "
                     "solve (relative residual %.3e)", i, sts[i].rel_residual);
      }
    }
  }
  return rc;
}

}  // namespace

extern "C" int dg_cg_solve_batched_mode(const dg_mesh* const* meshes, int count,
                                        const double* const* b, double* const* x, double rtol,
                                        int maxit, int mode, dg_cg_stats* st, void* stream) {
  const bool nodal = (mode & DG_CG_NODAL) != 0;
  if (mode != DG_CG_FP64 && mode != (DG_CG_FP64 | DG_CG_PRECOND_JACOBI) &&
      mode != (DG_CG_FP64 | DG_CG_NODAL))
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_cg_solve_batched: mode %d; the batched solver runs DG_CG_FP64, with "
                   "DG_CG_PRECOND_JACOBI or with DG_CG_NODAL", mode);
  const bool jacobi = (mode & DG_CG_PRECOND_JACOBI) != 0;
  if (meshes == nullptr || b == nullptr || x == nullptr || count < 1)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: NULL array or count < 1");
  if (!(rtol > 0.0) || !(rtol < 1.0))
    return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: rtol=%g outside (0, 1)", rtol);
  if (maxit < 1) return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: maxit=%d < 1", maxit);
  int maxn = 0;
  for (int s = 0; s < count; ++s) {
    const dg_mesh* m = meshes[s];
    if (m == nullptr || b[s] == nullptr || x[s] == nullptr)
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: NULL mesh or vector (sample %d)", s);
    if (!m->has_coef)
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: sample %d has no coefficient", s);
    if ((const void*)b[s] == (const void*)x[s])
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: b and x alias (sample %d)", s);
    if (m->affine || m->multilinear)
      return dg_fail(DG_ERR_INVALID_ARG,
                     "dg_cg_solve_batched: sample %d has an affine or multilinear geometry (not "
                     "batched)", s);
    if (m->lineop64 == nullptr)
      return dg_fail(DG_ERR_INVALID_ARG, "dg_cg_solve_batched: sample %d has no line operators", s);
    for (int t = 0; t < s; ++t)
      if (meshes[t] == meshes[s])
        return dg_fail(DG_ERR_INVALID_ARG,
                       "dg_cg_solve_batched: samples %d and %d share a mesh (its workspaces)", t,
                       s);
    maxn = m->n > maxn ? m->n : maxn;
  }
  if (nodal) return solve_batched_nodal(meshes, count, b, x, rtol, maxit, maxn, mode, st, stream);
  if (maxn <= 5)
    return solve_batched<128, 5, false>(meshes, count, b, x, rtol, maxit, jacobi, mode, st,
                                        stream);
  return solve_batched<256, DG_MAXN, false>(meshes, count, b, x, rtol, maxit, jacobi, mode, st,
                                            stream);
}

extern "C" int dg_cg_solve_batched(const dg_mesh* const* meshes, int count, const double* const* b,
                                   double* const* x, double rtol, int maxit, dg_cg_stats* st,
                                   void* stream) {
  return dg_cg_solve_batched_mode(meshes, count, b, x, rtol, maxit, DG_CG_FP64, st, stream);
}
