// FP64 operator on an affine mesh (the paper's problem B, Section 3.3): the
// unit-cube mesh mapped by x = A xi with a constant matrix A (det A > 0).
// Every cell is the image of its reference cube with Jacobian J = h A, so in
// reference units (the gradients of the tensor basis on [0,1]^3):
//   volume:  sum_q Kt_q grad u . G grad v,    G = det A A^-1 A^-T,  Kt = h w K;
//   face of axis d (points p, weight W_p = h gamma_F w_p):
//     W_p ( -{(G e_d) . grad u}[v] - {(G e_d) . grad v}[u] + sigma kappa_d [u][v] ),
//     kappa_d = det A |A^-T e_d|^2,
// which are the physical SWIPDG terms (face area |det J| |J^-T e_d|, unit
// normal J^-T e_d / |J^-T e_d|, penalty length |T| / |F|).  For A = I, G = I
// and kappa = 1: the cube operator.
//
// Pass 1 is the cube kernel's trace kernel (nodal values U, x-modal values X,
// face traces of the value and of the reference derivative along the face
// axis).  Pass 2 (k_cell_aff) differs from the cube kernel in two places:
//   * the metric G couples the three derivatives, so the kernel first forms
//     all three reference gradients at every point (z- and y-lines by the
//     collocation derivative of the nodal values, x-lines by L' from the
//     x-modes), then the flux K G grad u per point, then the transposed
//     contractions;
//   * (G e_d) has tangential components, so a face flux needs the tangential
//     derivatives of the averaged trace along the face, and the test side's
//     tangential derivatives become, after the transposed collocation
//     derivative on the face grid, value multipliers.  Each needs one exchange
//     of the face's n^2 values through shared memory.
// Every face point: J = [u] = u- - u+ (u+ = 0 on a boundary), the average value
// and normal derivative (one-sided on a boundary),
//   F   = G_dd {d_d u} + sum_t G_td d_t {u},
//   cv  = W s (sigma kappa_d J - F)            (value multiplier; s = +1 on the
//                                               upper face, -1 on the lower),
//   cD  = -c W J,  c = 1/2 inside, 1 on the boundary,
//   the test function then gets cv + sum_t G_td (D_t^T cD) as value multiplier
//   and G_dd cD as multiplier of its derivative along d.
// A zero-flux side has gamma_F = 0 (W = 0).  FP64 only.
#include <cmath>

#include "dg_apply_impl.cuh"

namespace {

struct AffineGeom {
  double G[3][3];   // det A A^-1 A^-T
  double kappa[3];  // det A |A^-T e_d|^2
};

template <int N>
struct AffCfg {
  static constexpr int CPB = dgk::Cfg<N>::CPB;
  static constexpr int THREADS = CPB * N * N;
  static constexpr int N2 = N * N, N3 = N * N * N;
  // per cell: U, X, gx, gy, gz, r, kt (n^3 each), face buffers 2 x 2 x n^2
  static constexpr int PER_CELL = 7 * N3 + 4 * N2;
  static size_t smem() { return sizeof(double) * (size_t)CPB * PER_CELL; }
};

// One direction's face step for the two faces of the calling thread's line.
// pt: the thread's face point (s1 + N s2 on the face grid: s1 along t1, s2
// along t2, the tangential axes in increasing order); fA/fC: this cell's face
// buffers [2 faces][n^2]; returns the value multipliers cvl/cvu and the
// normal-derivative multipliers cdl/cdu of the lower / upper face point.
template <int N>
__device__ __forceinline__ void face_pair(const DGTab<double>& tab, const AffineGeom& g, int d,
                                          int t1, int t2, int s1, int s2,
                                          const double (&uo)[2], const double (&go)[2],
                                          const double (&un)[2], const double (&gn)[2],
                                          const bool (&in)[2], const double (&W)[2], double* fA,
                                          double* fC, bool active, double (&cv)[2],
                                          double (&cd)[2]) {
  constexpr int N2 = N * N;
  const int pt = s1 + N * s2;
  double J[2], Gn[2];
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {  // f = 0 lower face (cell is the + side), 1 upper
      const double av = in[f] ? 0.5 * (uo[f] + un[f]) : uo[f];
      Gn[f] = in[f] ? 0.5 * (go[f] + gn[f]) : go[f];
      J[f] = f == 1 ? uo[f] - (in[f] ? un[f] : 0.0) : (in[f] ? un[f] : 0.0) - uo[f];
      fA[f * N2 + pt] = av;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      double d1 = 0.0, d2 = 0.0;  // tangential derivatives of the averaged trace
#pragma unroll
      for (int k = 0; k < N; ++k) {
        d1 = fma(tab.D[s1][k], fA[f * N2 + k + N * s2], d1);
        d2 = fma(tab.D[s2][k], fA[f * N2 + s1 + N * k], d2);
      }
      const double F = fma(g.G[d][d], Gn[f], fma(g.G[t1][d], d1, g.G[t2][d] * d2));
      const double s = f == 1 ? 1.0 : -1.0;
      cv[f] = W[f] * s * fma(tab.sigma * g.kappa[d], J[f], -F);
      const double cD = -(in[f] ? 0.5 : 1.0) * W[f] * J[f];
      cd[f] = g.G[d][d] * cD;
      fC[f * N2 + pt] = cD;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      double e1 = 0.0, e2 = 0.0;  // transposed tangential derivatives of cD
#pragma unroll
      for (int k = 0; k < N; ++k) {
        e1 = fma(tab.D[k][s1], fC[f * N2 + k + N * s2], e1);
        e2 = fma(tab.D[k][s2], fC[f * N2 + s1 + N * k], e2);
      }
      cv[f] = fma(g.G[t1][d], e1, fma(g.G[t2][d], e2, cv[f]));
    }
  }
}

template <int N>
__global__ void __launch_bounds__(AffCfg<N>::THREADS)
k_cell_aff(const double* __restrict__ U, const double* __restrict__ Xm,
           const double* __restrict__ TR, const double* __restrict__ kt,
           const double* __restrict__ gh, double* __restrict__ y, long long ncells, int Nc,
           const int* __restrict__ skip, const __grid_constant__ AffineGeom geom,
           const __grid_constant__ DGTab<double> tab) {
  using Cf = AffCfg<N>;
  constexpr int C = Cf::CPB, N2 = N * N, N3 = N * N * N;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) double sm[];
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  double* base = sm + lc * Cf::PER_CELL;
  double* su = base;
  double* sx = su + N3;
  double* sg[3] = {sx + N3, sx + 2 * N3, sx + 3 * N3};  // gradients, then fluxes
  double* sr = sx + 4 * N3;
  double* sk = sx + 5 * N3;
  double* fA = sx + 6 * N3;
  double* fC = fA + 2 * N2;
  {
    const double* ub = U + c0 * N3;
    const double* xb = Xm + c0 * N3;
    const double* kb = kt + c0 * N3;
    for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) {
      const int cl = t / N3, o = t - cl * N3;
      sm[cl * Cf::PER_CELL + o] = ub[t];
      sm[cl * Cf::PER_CELL + N3 + o] = xb[t];
      sm[cl * Cf::PER_CELL + 6 * N3 + o] = kb[t];
    }
  }
  __syncthreads();
  const long long c = c0 + lc;
  int crd[3] = {0, 0, 0};
  if (active) {
    crd[0] = (int)(c % Nc);
    crd[1] = (int)((c / Nc) % Nc);
    crd[2] = (int)(c / ((long long)Nc * Nc));
  }
  const long long stride[3] = {1, Nc, (long long)Nc * Nc};
  // gradients at every point: z-line (a=p, b=q), y-line (a=p, e=q), x-line (b=p, e=q)
  if (active) {
    double u[N], g[N];
#pragma unroll
    for (int e = 0; e < N; ++e) u[e] = su[e * N2 + q * N + p];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      double a = 0.0;
#pragma unroll
      for (int f = 0; f < N; ++f) a = fma(tab.D[e][f], u[f], a);
      sg[2][e * N2 + q * N + p] = a;
    }
#pragma unroll
    for (int b = 0; b < N; ++b) u[b] = su[q * N2 + b * N + p];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      double a = 0.0;
#pragma unroll
      for (int f = 0; f < N; ++f) a = fma(tab.D[b][f], u[f], a);
      sg[1][q * N2 + b * N + p] = a;
    }
    double X[N];
#pragma unroll
    for (int i = 0; i < N; ++i) X[i] = sx[q * N2 + p * N + i];
    dgk::bd_fwd<N>(tab, X, g);
#pragma unroll
    for (int a = 0; a < N; ++a) sg[0][q * N2 + p * N + a] = g[a];
  }
  __syncthreads();
  // flux K G grad u at the points of the thread's z-line
  if (active) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
      const int idx = e * N2 + q * N + p;
      const double gx = sg[0][idx], gy = sg[1][idx], gz = sg[2][idx], k = sk[idx];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        sg[d][idx] = k * fma(geom.G[d][0], gx, fma(geom.G[d][1], gy, geom.G[d][2] * gz));
    }
  }
  __syncthreads();
  // z-lines then y-lines: transposed collocation derivative of the flux, then
  // the two faces of the line
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const int d = dir == 0 ? 2 : 1;
    const int lbase = (dir == 0) ? (q * N + p) : (q * N2 + p);
    const int step = (dir == 0) ? N2 : N;
    double r[N];
    bool in[2] = {false, false};
    double uo[2] = {0, 0}, go[2] = {0, 0}, un[2] = {0, 0}, gn[2] = {0, 0}, W[2] = {0, 0};
    const int pt = p + N * q;  // face grid: z-faces (a, b), y-faces (a, e)
    if (active) {
      double fl[N];
#pragma unroll
      for (int e = 0; e < N; ++e) fl[e] = sg[d][lbase + e * step];
#pragma unroll
      for (int e = 0; e < N; ++e) {
        double a = (dir == 0) ? 0.0 : sr[lbase + e * step];
#pragma unroll
        for (int f = 0; f < N; ++f) a = fma(tab.D[f][e], fl[f], a);
        r[e] = a;
      }
      const double wpt = tab.w[p] * tab.w[q];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const int face = 2 * d + f;
        in[f] = f == 1 ? crd[d] < Nc - 1 : crd[d] > 0;
        dgk::load_trace<N>(TR, c, face, pt, uo[f], go[f]);
        if (in[f]) dgk::load_trace<N>(TR, f == 1 ? c + stride[d] : c - stride[d], face ^ 1, pt, un[f], gn[f]);
        W[f] = gh[c * 6 + face] * wpt;
      }
    }
    double cv[2] = {0, 0}, cd[2] = {0, 0};
    face_pair<N>(tab, geom, d, 0, dir == 0 ? 1 : 2, p, q, uo, go, un, gn, in, W, fA, fC, active,
                 cv, cd);
    if (active) {
#pragma unroll
      for (int e = 0; e < N; ++e) {
        double a = fma(tab.l1[e], cv[1], r[e]);
        a = fma(tab.dl1[e], cd[1], a);
        a = fma(tab.l0[e], cv[0], a);
        r[e] = fma(tab.dl0[e], cd[0], a);
      }
#pragma unroll
      for (int e = 0; e < N; ++e) sr[lbase + e * step] = r[e];
    }
    __syncthreads();
  }
  // x-lines (b = p, e = q): B^T of the nodal residual plus L'^T of the x-flux
  // into x-modes, then the x-faces in modal form
  {
    double R[N];
    bool in[2] = {false, false};
    double uo[2] = {0, 0}, go[2] = {0, 0}, un[2] = {0, 0}, gn[2] = {0, 0}, W[2] = {0, 0};
    const int pt = p + N * q;  // face grid (b, e)
    if (active) {
      double rr[N], fx[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        rr[i] = sr[q * N2 + p * N + i];
        fx[i] = sg[0][q * N2 + p * N + i];
      }
      dgk::bt_bdt<N>(tab, rr, fx, R);
      const double wpt = tab.w[p] * tab.w[q];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        in[f] = f == 1 ? crd[0] < Nc - 1 : crd[0] > 0;
        dgk::load_trace<N>(TR, c, f, pt, uo[f], go[f]);
        if (in[f]) dgk::load_trace<N>(TR, f == 1 ? c + 1 : c - 1, f ^ 1, pt, un[f], gn[f]);
        W[f] = gh[c * 6 + f] * wpt;
      }
    }
    double cv[2] = {0, 0}, cd[2] = {0, 0};
    face_pair<N>(tab, geom, 0, 1, 2, p, q, uo, go, un, gn, in, W, fA, fC, active, cv, cd);
    if (active) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double a = fma(tab.a1[i], cv[1], R[i]);
        a = fma(tab.d1[i], cd[1], a);
        a = fma(tab.a0[i], cv[0], a);
        R[i] = fma(tab.d0[i], cd[0], a);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) sx[q * N2 + p * N + i] = R[i];
    }
  }
  __syncthreads();
  if (active) {  // back along y: (i = p, e = q)
    double v[N], R[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = sx[q * N2 + b * N + p];
    dgk::b_bwd<N>(tab, v, R);
#pragma unroll
    for (int j = 0; j < N; ++j) sx[q * N2 + j * N + p] = R[j];
  }
  __syncthreads();
  if (active) {  // back along z: (i = p, j = q), straight to y
    double v[N], R[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sx[e * N2 + q * N + p];
    dgk::b_bwd<N>(tab, v, R);
#pragma unroll
    for (int l = 0; l < N; ++l) y[c * N3 + l * N2 + q * N + p] = R[l];
  }
}

template <int N>
struct AffineF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const double* x, double* yv, const int* skip,
                         cudaStream_t s) {
    using Cf = AffCfg<N>;
    const unsigned blocks = (unsigned)((m->ncells + Cf::CPB - 1) / Cf::CPB);
    dg_timing_mark(m, 0, s);
    dgk::k_trace<N, double><<<blocks, dgk::Cfg<N>::THREADS, dgk::trace_smem<N, double>(), s>>>(
        x, m->U64, m->X64, m->TR64, 0, m->ncells, skip, m->tab64);
    dg_timing_mark(m, 1, s);
    AffineGeom g;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) g.G[i][j] = m->geomG[i][j];
      g.kappa[i] = m->geomKappa[i];
    }
    k_cell_aff<N><<<blocks, Cf::THREADS, Cf::smem(), s>>>(m->U64, m->X64, m->TR64, m->kt64,
                                                          m->gh64, yv, m->ncells, m->N, skip,
                                                          g, m->tab64);
    dg_timing_mark(m, 2, s);
    return cudaGetLastError();
  }
};

template <int N>
struct AffinePrepareF {
  template <typename T>
  static cudaError_t run() {
    return cudaFuncSetAttribute(k_cell_aff<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)AffCfg<N>::smem());
  }
};

}  // namespace

int dg_launch_apply_affine(const dg_mesh* m, const double* x, double* y, const int* skip,
                           cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, AffineF>(m->n, m, x, y, skip, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "affine apply: launch");
  return DG_OK;
}

extern "C" int dg_set_geometry(dg_mesh* m, const double* A) {
  if (m == nullptr || A == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_set_geometry: NULL mesh or matrix");
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(A[i])) return dg_fail(DG_ERR_INVALID_ARG, "dg_set_geometry: A not finite");
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(det > 0.0))
    return dg_fail(DG_ERR_INVALID_ARG, "dg_set_geometry: det A = %g, must be positive", det);
  // inverse by cofactors: Ainv[i][j]
  double Ai[3][3];
  Ai[0][0] = (A[4] * A[8] - A[5] * A[7]) / det;
  Ai[0][1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[0][2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[1][0] = (A[5] * A[6] - A[3] * A[8]) / det;
  Ai[1][1] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[1][2] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[2][0] = (A[3] * A[7] - A[4] * A[6]) / det;
  Ai[2][1] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[2][2] = (A[0] * A[4] - A[1] * A[3]) / det;
  bool identity = true;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) identity = identity && A[3 * i + j] == (i == j ? 1.0 : 0.0);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Ai[i][k] * Ai[j][k];
      m->geomG[i][j] = det * s;  // det A (A^-1 A^-T)_{ij}
    }
    double a2 = 0.0;  // |A^-T e_i|^2 = sum_k Ainv[i][k]^2
    for (int k = 0; k < 3; ++k) a2 += Ai[i][k] * Ai[i][k];
    m->geomKappa[i] = det * a2;
  }
  m->geomDet = det;
  m->affine = !identity;
  m->multilinear = false;
  m->has_coef = false;  // the coefficient is set again for the new geometry
  m->has_diag = false;
  m->has_block = false;
  m->has_kron = false;
  return dg_prepare_affine(m->n);
}

int dg_prepare_affine(int n) {
  cudaError_t e = dgk::dispatch_n<double, AffinePrepareF>(n);
  if (e != cudaSuccess) return dg_cuda_fail(e, "affine apply: kernel attributes");
  return DG_OK;
}
