// Gradient of v^T A(K) u with respect to log K at the volume Gauss points.
//
// With Kt_q = h w_q K_q the volume part of v^T A u is sum_q Kt_q grad u . grad v
// (reference gradients), so its derivative by log K_q is that product.  The
// face part is sum_F gamma_F b_F(u, v) with b_F the face form for gamma = 1
// (-{d_n u}[v] - {d_n v}[u] + sigma [u][v] weighted by h w_s w_t); gamma_F
// depends on K only through the cells' Kbar = exp(sum_q w_q log K_q), hence
//   g_q = Kt_q grad u . grad v + w_q sum_{F of the cell} (d gamma_F / d log Kbar_c) b_F(u, v).
// Inputs: pass-1 data (nodal U, x-modal X, face traces) of u and of v.
#include <type_traits>

#include "dg_apply_impl.cuh"

namespace dgk {

// b_F contribution at one face point for gamma = 1 (W = h w_s w_t).
template <bool UPPER>
__device__ __forceinline__ double face_form_point(bool interior, double uo, double go, double un,
                                                  double gn, double vo, double gvo, double vn,
                                                  double gvn, double W, double sigma) {
  double Ju, Au, Jv, Av;
  if (interior) {
    if (UPPER) {  // own cell is (-)
      Ju = uo - un; Jv = vo - vn;
    } else {      // own cell is (+)
      Ju = un - uo; Jv = vn - vo;
    }
    Au = 0.5 * (go + gn);
    Av = 0.5 * (gvo + gvn);
  } else {        // outward normal +e_d (upper) or -e_d (lower)
    Ju = uo; Jv = vo;
    Au = UPPER ? go : -go;
    Av = UPPER ? gvo : -gvo;
  }
  return W * (-Au * Jv - Av * Ju + sigma * Ju * Jv);
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_coeff_grad(const double* __restrict__ Uu, const double* __restrict__ Xu,
             const double* __restrict__ TRu, const double* __restrict__ Uv,
             const double* __restrict__ Xv, const double* __restrict__ TRv,
             const double* __restrict__ kt, const double* __restrict__ dgam, double h,
             double* __restrict__ g, long long ncells, int Nc,
             const __grid_constant__ DGTab<double> tab) {
  constexpr int N2 = N * N, N3 = N * N * N, C = Cfg<N>::CPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* su = reinterpret_cast<double*>(smem_raw);
  double* sv = su + C * N3;
  double* sxu = sv + C * N3;
  double* sxv = sxu + C * N3;
  double* sg = sxv + C * N3;         // grad u . grad v accumulated per point
  double* sf = sg + C * N3;          // per-face-point face form values [C][6][N2]
  const long long c0 = (long long)blockIdx.x * C;
  const int nblk = (int)((ncells - c0) < C ? (ncells - c0) : C);
  for (int t = threadIdx.x; t < nblk * N3; t += blockDim.x) {
    su[t] = Uu[c0 * N3 + t];
    sv[t] = Uv[c0 * N3 + t];
    sxu[t] = Xu[c0 * N3 + t];
    sxv[t] = Xv[c0 * N3 + t];
  }
  __syncthreads();
  const int lc = threadIdx.x / N2;
  const int t2 = threadIdx.x - lc * N2;
  const int p = t2 % N, q = t2 / N;
  const bool active = lc < nblk;
  const long long c = c0 + lc;
  const int cx = (int)(c % Nc);
  const int cy = (int)((c / Nc) % Nc);
  const int cz = (int)(c / ((long long)Nc * Nc));
  const long long sy = Nc, sz = (long long)Nc * Nc;
  const int o = lc * N3;
  double* sfc = sf + lc * 6 * N2;
  const double sigma = tab.sigma;
  const int pt = p + N * q;
  const double W = h * tab.w[p] * tab.w[q];

  auto face = [&](auto upper_tag, int f, int fn, bool in, long long cn) {
    constexpr bool UP = decltype(upper_tag)::value;
    double uo, go, un = 0.0, gn = 0.0, vo, gvo, vn = 0.0, gvn = 0.0;
    load_trace<N>(TRu, c, f, pt, uo, go);
    load_trace<N>(TRv, c, f, pt, vo, gvo);
    if (in) {
      load_trace<N>(TRu, cn, fn, pt, un, gn);
      load_trace<N>(TRv, cn, fn, pt, vn, gvn);
    }
    sfc[f * N2 + pt] = face_form_point<UP>(in, uo, go, un, gn, vo, gvo, vn, gvn, W, sigma);
  };
  using UpT = std::integral_constant<bool, true>;
  using LoT = std::integral_constant<bool, false>;

  // z-lines (a = p, b = q)
  if (active) {
    double u[N], v[N];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      u[e] = su[o + e * N2 + q * N + p];
      v[e] = sv[o + e * N2 + q * N + p];
    }
#pragma unroll
    for (int e = 0; e < N; ++e) {
      double gu = 0.0, gv = 0.0;
#pragma unroll
      for (int f = 0; f < N; ++f) {
        gu = fma(tab.D[e][f], u[f], gu);
        gv = fma(tab.D[e][f], v[f], gv);
      }
      sg[o + e * N2 + q * N + p] = gu * gv;
    }
    face(UpT{}, 5, 4, cz < Nc - 1, c + sz);
    face(LoT{}, 4, 5, cz > 0, c - sz);
  }
  __syncthreads();
  // y-lines (a = p, e = q)
  if (active) {
    double u[N], v[N];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      u[b] = su[o + q * N2 + b * N + p];
      v[b] = sv[o + q * N2 + b * N + p];
    }
#pragma unroll
    for (int b = 0; b < N; ++b) {
      double gu = 0.0, gv = 0.0;
#pragma unroll
      for (int f = 0; f < N; ++f) {
        gu = fma(tab.D[b][f], u[f], gu);
        gv = fma(tab.D[b][f], v[f], gv);
      }
      sg[o + q * N2 + b * N + p] = fma(gu, gv, sg[o + q * N2 + b * N + p]);
    }
    face(UpT{}, 3, 2, cy < Nc - 1, c + sy);
    face(LoT{}, 2, 3, cy > 0, c - sy);
  }
  __syncthreads();
  // x-lines (b = p, e = q): x-derivative from the x-modal data
  if (active) {
    double Xa[N], Xb[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Xa[i] = sxu[o + q * N2 + p * N + i];
      Xb[i] = sxv[o + q * N2 + p * N + i];
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
      double gu = 0.0, gv = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        gu = fma(tab.Bd[a][i], Xa[i], gu);
        gv = fma(tab.Bd[a][i], Xb[i], gv);
      }
      sg[o + q * N2 + p * N + a] = fma(gu, gv, sg[o + q * N2 + p * N + a]);
    }
    face(UpT{}, 1, 0, cx < Nc - 1, c + 1);
    face(LoT{}, 0, 1, cx > 0, c - 1);
  }
  __syncthreads();
  // per cell: s = sum_f dgam_f * sum_pt sf[f][pt]  (fixed summation order)
  if (active) {
    double s = 0.0;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      double b = 0.0;
      for (int k = 0; k < N2; ++k) b += sfc[f * N2 + k];
      s = fma(dgam[c * 6 + f], b, s);
    }
    // each thread writes the n points of its z-line (a = p, b = q)
#pragma unroll
    for (int e = 0; e < N; ++e) {
      const int qi = e * N2 + q * N + p;
      const double wq = tab.w[p] * tab.w[q] * tab.w[e];
      g[c * N3 + qi] = fma(kt[c * N3 + qi], sg[o + qi], wq * s);
    }
  }
}

template <int N>
struct GradF {
  template <typename T>
  static cudaError_t run(const dg_mesh* m, double* g, cudaStream_t s) {
    constexpr int C = Cfg<N>::CPB, N3 = N * N * N;
    const size_t smem = sizeof(double) * (5 * C * N3 + C * 6 * N * N);
    const unsigned blocks = (unsigned)((m->ncells + C - 1) / C);
    k_coeff_grad<N><<<blocks, Cfg<N>::THREADS, smem, s>>>(
        m->U64, m->X64, m->TR64, m->U64b, m->X64b, m->TR64b, m->kt64, m->dgam, m->h, g,
        m->ncells, m->N, m->tab64);
    return cudaGetLastError();
  }
};

template <int N>
struct GradPrepF {
  template <typename T>
  static cudaError_t run() {
    constexpr int C = Cfg<N>::CPB, N3 = N * N * N;
    const size_t smem = sizeof(double) * (5 * C * N3 + C * 6 * N * N);
    return cudaFuncSetAttribute(k_coeff_grad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
};

}  // namespace dgk

int dg_prepare_grad(int n) {
  cudaError_t e = dgk::dispatch_n<double, dgk::GradPrepF>(n);
  if (e != cudaSuccess) return dg_cuda_fail(e, "coefficient gradient kernel attributes");
  return DG_OK;
}

int dg_launch_coeff_grad(const dg_mesh* m, double* g, cudaStream_t s) {
  cudaError_t e = dgk::dispatch_n<double, dgk::GradF>(m->n, m, g, s);
  if (e != cudaSuccess) return dg_cuda_fail(e, "coefficient gradient launch");
  return DG_OK;
}
