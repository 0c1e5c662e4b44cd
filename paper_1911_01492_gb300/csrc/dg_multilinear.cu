// FP64 operator on a multilinear mesh (the paper's problem C, Section 3.3):
// the N^3 cells of the structured mesh with vertices at given positions, each
// cell the trilinear image of its reference cube, so the Jacobian J varies
// from point to point.  Written in reference gradients (the tensor basis on
// [0,1]^3), with physical quantities at every quadrature point:
//   volume:  sum_q h w_q K_q grad u . G_q grad v,   G_q = |det J_q| J_q^-1 J_q^-T / h;
//   face point p of a face with reference axis d (shared surface: the unit
//   normal n along +e_d and the area element A_p are the same from both
//   cells; each side's normal derivative is m_side . grad u_side with
//   m_side = J_side^-1 n):
//     W_p ( -{m . grad u}[v] - {m . grad v}[u] + (sigma / h_F)[u][v] ),
//     W_p = gamma_F A_p,  h_F = (|T-| + |T+|) / (2 |F|) inside, |T| / |F| on
//     the boundary (|T| cell volume, |F| face area).
// Affine vertices give the affine operator exactly.
//
// dg_set_vertices forms the per-point data once (k_geo_points, k_geo_penalty).
// The pass-2 kernel k_cell_ml is the affine kernel with those per-point
// values; since the two sides of a face have different Jacobians, each side's
// normal flux m . grad u needs the tangential derivatives of that side's own
// trace, so the face step exchanges both traces (and the test side's
// tangential multipliers) on the face grid.  FP64 only.
#include <cmath>
#include <vector>

#include "dg_apply_impl.cuh"

namespace {

// Trilinear map of one cell: Jacobian J[i][j] = d x_i / d xi_j at xi from the
// corner positions C[dz][dy][dx][3].
__device__ void tri_jacobian(const double (&C)[2][2][2][3], double x1, double x2, double x3,
                             double (&J)[3][3]) {
  const double s1[2] = {1.0 - x1, x1}, s2[2] = {1.0 - x2, x2}, s3[2] = {1.0 - x3, x3};
  const double ds[2] = {-1.0, 1.0};
  for (int i = 0; i < 3; ++i) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const double v = C[dz][dy][dx][i];
          a = fma(v, s3[dz] * s2[dy] * ds[dx], a);
          b = fma(v, s3[dz] * ds[dy] * s1[dx], b);
          c = fma(v, ds[dz] * s2[dy] * s1[dx], c);
        }
    J[i][0] = a;
    J[i][1] = b;
    J[i][2] = c;
  }
}

// inverse by cofactors; returns det J
__device__ double inv3(const double (&J)[3][3], double (&Ji)[3][3]) {
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  const double r = 1.0 / det;
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * r;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * r;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * r;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
  return det;
}

struct GaussPts {
  double xi[DG_MAXN];
};

// One thread per cell: volume metric and |det J| at the volume Gauss points,
// area element / h and J^-1 n at the face points, cell volume and face areas.
// A non-positive det J raises *flag.
__global__ void k_geo_points(const double* __restrict__ V, int Nc, int n, double h,
                             double* __restrict__ gvol, double* __restrict__ gdet,
                             double* __restrict__ gface, double* __restrict__ cellvol,
                             double* __restrict__ facearea, int* flag,
                             const __grid_constant__ GaussPts gp,
                             const __grid_constant__ DGTab<double> tab) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)Nc * Nc * Nc;
  if (c >= nc) return;
  const int cx = (int)(c % Nc), cy = (int)((c / Nc) % Nc), cz = (int)(c / ((long long)Nc * Nc));
  const long long V1 = Nc + 1;
  double C[2][2][2][3];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const long long v = ((cz + dz) * V1 + (cy + dy)) * V1 + (cx + dx);
        for (int i = 0; i < 3; ++i) C[dz][dy][dx][i] = V[3 * v + i];
      }
  const int n2 = n * n, n3 = n2 * n;
  double vol = 0.0;
  bool bad = false;
  for (int q = 0; q < n3; ++q) {
    const int a = q % n, b = (q / n) % n, e = q / n2;
    double J[3][3], Ji[3][3];
    tri_jacobian(C, gp.xi[a], gp.xi[b], gp.xi[e], J);
    const double det = inv3(J, Ji);
    if (!(det > 0.0)) bad = true;
    const double ad = fabs(det);
    // G = |det J| J^-1 J^-T / h, components xx, yy, zz, xy, xz, yz
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
    for (int t = 0; t < 6; ++t) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s = fma(Ji[ii[t]][k], Ji[jj[t]][k], s);
      gvol[(c * 6 + t) * n3 + q] = ad * s / h;
    }
    gdet[c * n3 + q] = ad;
    vol = fma(tab.w[a] * tab.w[b] * tab.w[e], ad, vol);
  }
  cellvol[c] = vol;
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, sd = f & 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    double area = 0.0;
    for (int p = 0; p < n2; ++p) {
      const int s1 = p % n, s2 = p / n;
      double xi3[3];
      xi3[d] = (double)sd;
      xi3[t1] = gp.xi[s1];
      xi3[t2] = gp.xi[s2];
      double J[3][3], Ji[3][3];
      tri_jacobian(C, xi3[0], xi3[1], xi3[2], J);
      const double det = inv3(J, Ji);
      if (!(det > 0.0)) bad = true;
      // J^-T e_d = row d of J^-1; unit normal n; m = J^-1 n
      const double v0 = Ji[d][0], v1 = Ji[d][1], v2 = Ji[d][2];
      const double len = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      const double nn[3] = {v0 / len, v1 / len, v2 / len};
      const double A = fabs(det) * len * tab.w[s1] * tab.w[s2];
      area += A;
      double* gf = gface + (c * 6 + f) * 4 * n2;
      gf[p] = A / h;
      for (int i = 0; i < 3; ++i)
        gf[(1 + i) * n2 + p] = Ji[i][0] * nn[0] + Ji[i][1] * nn[1] + Ji[i][2] * nn[2];
    }
    facearea[c * 6 + f] = area;
  }
  if (bad) atomicOr(flag, 1);
}

// sigma / h_F per cell face: h_F = (|T-| + |T+|) / (2 |F|) inside, |T| / |F| on
// the boundary.
__global__ void k_geo_penalty(const double* __restrict__ cellvol,
                              const double* __restrict__ facearea, double* __restrict__ pen,
                              int Nc, double sigma) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)Nc * Nc * Nc;
  if (c >= nc) return;
  const int crd[3] = {(int)(c % Nc), (int)((c / Nc) % Nc), (int)(c / ((long long)Nc * Nc))};
  const long long stride[3] = {1, Nc, (long long)Nc * Nc};
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1;
    const bool upper = f & 1;
    const bool inside = upper ? crd[d] < Nc - 1 : crd[d] > 0;
    const double F = facearea[c * 6 + f];
    const double T = inside ? 0.5 * (cellvol[c] + cellvol[upper ? c + stride[d] : c - stride[d]])
                            : cellvol[c];
    pen[c * 6 + f] = sigma * F / T;
  }
}

template <int N>
struct MlCfg {
  static constexpr int CPB = dgk::Cfg<N>::CPB;
  static constexpr int THREADS = CPB * N * N;
  static constexpr int N2 = N * N, N3 = N * N * N;
  // per cell: U, X, gx, gy, gz, r, kt (n^3 each), face buffers 2 faces x 4 x n^2
  static constexpr int PER_CELL = 7 * N3 + 8 * N2;
  static size_t smem() { return sizeof(double) * (size_t)CPB * PER_CELL; }
};

// One direction's face step (both faces of the thread's line) on a
// multilinear mesh: per side the normal flux m . grad u with that side's own
// tangential trace derivatives.  mo/mn: J^-1 n of the own and the neighbour
// side; Ah: area element / h; pen: sigma / h_F; gh: h gamma.
template <int N>
__device__ __forceinline__ void face_pair_ml(const DGTab<double>& tab, int d, int t1, int t2,
                                             int s1, int s2, const double (&uo)[2],
                                             const double (&go)[2], const double (&un)[2],
                                             const double (&gn)[2], const bool (&in)[2],
                                             const double (&mo)[2][3], const double (&mn)[2][3],
                                             const double (&W)[2], const double (&pen)[2],
                                             double* fb, bool active, double (&cv)[2],
                                             double (&cd)[2]) {
  constexpr int N2 = N * N;
  const int pt = s1 + N * s2;
  double J[2];
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      J[f] = f == 1 ? uo[f] - (in[f] ? un[f] : 0.0) : (in[f] ? un[f] : 0.0) - uo[f];
      fb[(4 * f + 0) * N2 + pt] = uo[f];
      fb[(4 * f + 1) * N2 + pt] = in[f] ? un[f] : 0.0;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      double o1 = 0.0, o2 = 0.0, n1 = 0.0, n2v = 0.0;  // tangential derivatives of each trace
#pragma unroll
      for (int k = 0; k < N; ++k) {
        o1 = fma(tab.D[s1][k], fb[(4 * f) * N2 + k + N * s2], o1);
        o2 = fma(tab.D[s2][k], fb[(4 * f) * N2 + s1 + N * k], o2);
        n1 = fma(tab.D[s1][k], fb[(4 * f + 1) * N2 + k + N * s2], n1);
        n2v = fma(tab.D[s2][k], fb[(4 * f + 1) * N2 + s1 + N * k], n2v);
      }
      const double Fo = fma(mo[f][d], go[f], fma(mo[f][t1], o1, mo[f][t2] * o2));
      double F = Fo;
      if (in[f]) F = 0.5 * (Fo + fma(mn[f][d], gn[f], fma(mn[f][t1], n1, mn[f][t2] * n2v)));
      const double s = f == 1 ? 1.0 : -1.0;
      cv[f] = W[f] * s * fma(pen[f], J[f], -F);
      const double cD = -(in[f] ? 0.5 : 1.0) * W[f] * J[f];
      cd[f] = mo[f][d] * cD;
      fb[(4 * f + 2) * N2 + pt] = mo[f][t1] * cD;
      fb[(4 * f + 3) * N2 + pt] = mo[f][t2] * cD;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      double e = cv[f];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        e = fma(tab.D[k][s1], fb[(4 * f + 2) * N2 + k + N * s2], e);
        e = fma(tab.D[k][s2], fb[(4 * f + 3) * N2 + s1 + N * k], e);
      }
      cv[f] = e;
    }
  }
}

template <int N>
__global__ void __launch_bounds__(MlCfg<N>::THREADS)
k_cell_ml(const double* __restrict__ U, const double* __restrict__ Xm,
          const double* __restrict__ TR, const double* __restrict__ kt,
          const double* __restrict__ gh, const double* __restrict__ gvol,
          const double* __restrict__ gface, const double* __restrict__ gpen,
          double* __restrict__ y, long long ncells, int Nc, const int* __restrict__ skip,
          const __grid_constant__ DGTab<double> tab) {
  using Cf = MlCfg<N>;
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
  double* sg[3] = {sx + N3, sx + 2 * N3, sx + 3 * N3};
  double* sr = sx + 4 * N3;
  double* sk = sx + 5 * N3;
  double* fb = sx + 6 * N3;
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
  if (active) {  // gradients at every point (as the affine kernel)
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
  if (active) {  // flux h w K G_q grad u at the points of the thread's z-line
    const double* Gc = gvol + c * 6 * N3;
#pragma unroll
    for (int e = 0; e < N; ++e) {
      const int idx = e * N2 + q * N + p;
      const double gx = sg[0][idx], gy = sg[1][idx], gz = sg[2][idx], k = sk[idx];
      const double xx = Gc[idx], yy = Gc[N3 + idx], zz = Gc[2 * N3 + idx];
      const double xy = Gc[3 * N3 + idx], xz = Gc[4 * N3 + idx], yz = Gc[5 * N3 + idx];
      sg[0][idx] = k * fma(xx, gx, fma(xy, gy, xz * gz));
      sg[1][idx] = k * fma(xy, gx, fma(yy, gy, yz * gz));
      sg[2][idx] = k * fma(xz, gx, fma(yz, gy, zz * gz));
    }
  }
  __syncthreads();
  // face data of face f at the thread's face point pt
  auto load_face = [&](int face, int pt, int f, double (&uo)[2], double (&go)[2],
                       double (&un)[2], double (&gn)[2], bool (&in)[2], double (&mo)[2][3],
                       double (&mn)[2][3], double (&W)[2], double (&pen)[2]) {
    const int d = face >> 1;
    in[f] = f == 1 ? crd[d] < Nc - 1 : crd[d] > 0;
    dgk::load_trace<N>(TR, c, face, pt, uo[f], go[f]);
    const double* gf = gface + (c * 6 + face) * 4 * N2;
    W[f] = gh[c * 6 + face] * gf[pt];
    for (int i = 0; i < 3; ++i) mo[f][i] = gf[(1 + i) * N2 + pt];
    pen[f] = gpen[c * 6 + face];
    un[f] = gn[f] = 0.0;
    for (int i = 0; i < 3; ++i) mn[f][i] = 0.0;
    if (in[f]) {
      const long long cn = f == 1 ? c + stride[d] : c - stride[d];
      dgk::load_trace<N>(TR, cn, face ^ 1, pt, un[f], gn[f]);
      const double* gn_ = gface + (cn * 6 + (face ^ 1)) * 4 * N2;
      for (int i = 0; i < 3; ++i) mn[f][i] = gn_[(1 + i) * N2 + pt];
    }
  };
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const int d = dir == 0 ? 2 : 1;
    const int lbase = (dir == 0) ? (q * N + p) : (q * N2 + p);
    const int step = (dir == 0) ? N2 : N;
    double r[N];
    bool in[2] = {false, false};
    double uo[2] = {0, 0}, go[2] = {0, 0}, un[2] = {0, 0}, gn[2] = {0, 0}, W[2] = {0, 0},
           pen[2] = {0, 0}, mo[2][3] = {}, mn[2][3] = {};
    const int pt = p + N * q;
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
      load_face(2 * d, pt, 0, uo, go, un, gn, in, mo, mn, W, pen);
      load_face(2 * d + 1, pt, 1, uo, go, un, gn, in, mo, mn, W, pen);
    }
    double cv[2] = {0, 0}, cd[2] = {0, 0};
    face_pair_ml<N>(tab, d, 0, dir == 0 ? 1 : 2, p, q, uo, go, un, gn, in, mo, mn, W, pen, fb,
                    active, cv, cd);
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
  {  // x-lines (b = p, e = q)
    double R[N];
    bool in[2] = {false, false};
    double uo[2] = {0, 0}, go[2] = {0, 0}, un[2] = {0, 0}, gn[2] = {0, 0}, W[2] = {0, 0},
           pen[2] = {0, 0}, mo[2][3] = {}, mn[2][3] = {};
    const int pt = p + N * q;
    if (active) {
      double rr[N], fx[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        rr[i] = sr[q * N2 + p * N + i];
        fx[i] = sg[0][q * N2 + p * N + i];
      }
      dgk::bt_bdt<N>(tab, rr, fx, R);
      load_face(0, pt, 0, uo, go, un, gn, in, mo, mn, W, pen);
      load_face(1, pt, 1, uo, go, un, gn, in, mo, mn, W, pen);
    }
    double cv[2] = {0, 0}, cd[2] = {0, 0};
    face_pair_ml<N>(tab, 0, 1, 2, p, q, uo, go, un, gn, in, mo, mn, W, pen, fb, active, cv, cd);
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
  if (active) {
    double v[N], R[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = sx[q * N2 + b * N + p];
    dgk::b_bwd<N>(tab, v, R);
#pragma unroll
    for (int j = 0; j < N; ++j) sx[q * N2 + j * N + p] = R[j];
  }
  __syncthreads();
  if (active) {
    double v[N], R[N];
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = sx[e * N2 + q * N + p];
    dgk::b_bwd<N>(tab, v, R);
#pragma unroll
    for (int l = 0; l < N; ++l) y[c * N3 + l * N2 + q * N + p] = R[l];
  }
}

template <int N>
struct MlApplyF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, const double* x, double* yv, const int* skip,
                         cudaStream_t s) {
    using Cf = MlCfg<N>;
    const unsigned blocks = (unsigned)((m->ncells + Cf::CPB - 1) / Cf::CPB);
    dg_timing_mark(m, 0, s);
    dgk::k_trace<N, double><<<blocks, dgk::Cfg<N>::THREADS, dgk::trace_smem<N, double>(), s>>>(
        x, m->U64, m->X64, m->TR64, 0, m->ncells, skip, m->tab64);
    dg_timing_mark(m, 1, s);
    k_cell_ml<N><<<blocks, Cf::THREADS, Cf::smem(), s>>>(m->U64, m->X64, m->TR64, m->kt64,
                                                         m->gh64, m->geo_vol, m->geo_face,
                                                         m->geo_pen, yv, m->ncells, m->N, skip,
                                                         m->tab64);
    dg_timing_mark(m, 2, s);
    return cudaGetLastError();
  }
};

template <int N>
struct MlPrepareF {
  template <typename T>
  static cudaError_t run() {
    return cudaFuncSetAttribute(k_cell_ml<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)MlCfg<N>::smem());
  }
};

}  // namespace

int dg_launch_apply_multilinear(const dg_mesh* m, const double* x, double* y, const int* skip,
                                cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, MlApplyF>(m->n, m, x, y, skip, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "multilinear apply: launch");
  return DG_OK;
}

extern "C" int dg_set_vertices(dg_mesh* m, const double* X) {
  if (m == nullptr || X == nullptr)
    return dg_fail(DG_ERR_INVALID_ARG, "dg_set_vertices: NULL mesh or vertices");
  const long long nv = (long long)(m->N + 1) * (m->N + 1) * (m->N + 1);
  for (long long i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(X[i]))
      return dg_fail(DG_ERR_INVALID_ARG, "dg_set_vertices: vertex coordinate %lld not finite", i);
  const size_t n3 = (size_t)m->n * m->n * m->n, n2 = (size_t)m->n * m->n;
  const size_t nc = (size_t)m->ncells;
  if (m->geo_vol == nullptr) {
    DG_CUDA(cudaMalloc((void**)&m->geo_vol, sizeof(double) * 6 * n3 * nc));
    DG_CUDA(cudaMalloc((void**)&m->geo_det, sizeof(double) * n3 * nc));
    DG_CUDA(cudaMalloc((void**)&m->geo_face, sizeof(double) * 24 * n2 * nc));
    DG_CUDA(cudaMalloc((void**)&m->geo_pen, sizeof(double) * 6 * nc));
  }
  double *dV = nullptr, *dvol = nullptr, *darea = nullptr;
  cudaError_t e = cudaMalloc((void**)&dV, sizeof(double) * 3 * nv);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dvol, sizeof(double) * nc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&darea, sizeof(double) * 6 * nc);
  if (e == cudaSuccess) e = cudaMemcpy(dV, X, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->dflag, 0, sizeof(int));
  GaussPts gp = {};
  double w[DG_MAXN];
  dg_gauss_points(m->n, gp.xi, w);
  const unsigned blocks = (unsigned)((nc + 127) / 128);
  if (e == cudaSuccess) {
    k_geo_points<<<blocks, 128>>>(dV, m->N, m->n, m->h, m->geo_vol, m->geo_det, m->geo_face,
                                  dvol, darea, m->dflag, gp, m->tab64);
    k_geo_penalty<<<blocks, 128>>>(dvol, darea, m->geo_pen, m->N, m->sigma);
    e = cudaGetLastError();
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, m->dflag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dV);
  cudaFree(dvol);
  cudaFree(darea);
  if (e != cudaSuccess) return dg_cuda_fail(e, "dg_set_vertices");
  if (flag) {
    m->multilinear = false;
    return dg_fail(DG_ERR_INVALID_ARG,
                   "dg_set_vertices: a cell's Jacobian determinant is not positive (inverted "
                   "or degenerate cell)");
  }
  cudaError_t ea = dgk::dispatch_n<double, MlPrepareF>(m->n);
  if (ea != cudaSuccess) return dg_cuda_fail(ea, "multilinear apply: kernel attributes");
  m->multilinear = true;
  m->affine = false;
  m->geomDet = 1.0;
  m->has_coef = false;
  m->has_diag = false;
  m->has_block = false;
  m->has_kron = false;
  return DG_OK;
}
