// Host construction of the 1D tables on [0,1] for n Gauss points.
//
// Gauss-Legendre points: roots of P_n on [-1,1] by Newton's method from the
// Chebyshev-like initial guesses cos(pi (i + 3/4) / (n + 1/2)); weights
// 2 / ((1 - t^2) P_n'(t)^2); both mapped to [0,1] (points (t+1)/2, weights w/2).
// Legendre values by the three-term recurrence
//   (j+1) P_{j+1}(t) = (2j+1) t P_j(t) - j P_{j-1}(t),
// derivatives by P_{j+1}' = P_{j-1}' + (2j+1) P_j.
// Lagrange basis on the Gauss points in barycentric form: l_a(t) =
// lambda_a / (t - xi_a) * prod_b (t - xi_b) with lambda_a = 1 / prod_{b!=a}
// (xi_a - xi_b); collocation derivative D[a][b] = (lambda_b / lambda_a) /
// (xi_a - xi_b) for a != b and D[a][a] = -sum_{b!=a} D[a][b].
#include <cmath>
#include <cstring>

#include "dg_internal.cuh"

namespace {

// P_j(t) and P_j'(t) for j = 0..n-1 at t in [-1,1]
void legendre_all(int n, double t, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n > 1) {
    P[1] = t;
    dP[1] = 1.0;
  }
  for (int j = 1; j + 1 < n; ++j) {
    P[j + 1] = ((2.0 * j + 1.0) * t * P[j] - j * P[j - 1]) / (j + 1.0);
    dP[j + 1] = dP[j - 1] + (2.0 * j + 1.0) * P[j];
  }
}

// P_n(t) and P_n'(t)
void legendre_n(int n, double t, double* Pn, double* dPn) {
  double p0 = 1.0, p1 = t;
  if (n == 0) {
    *Pn = 1.0;
    *dPn = 0.0;
    return;
  }
  for (int j = 1; j < n; ++j) {
    double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *Pn = p1;
  *dPn = n * (t * p1 - p0) / (t * t - 1.0);  // (1 - t^2) P_n' = n (P_{n-1} - t P_n)
}

void gauss_01(int n, double* xi, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double t = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double Pn, dPn;
      legendre_n(n, t, &Pn, &dPn);
      double dt = Pn / dPn;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double Pn, dPn;
    legendre_n(n, t, &Pn, &dPn);
    // roots come out in decreasing t; store increasing on [0,1]
    xi[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dPn * dPn);
  }
  // exact symmetry of the rule about 1/2
  for (int i = 0; i < n / 2; ++i) {
    double s = 0.5 * ((1.0 - xi[n - 1 - i]) + xi[i]);
    xi[i] = s;
    xi[n - 1 - i] = 1.0 - s;
    double ww = 0.5 * (w[i] + w[n - 1 - i]);
    w[i] = w[n - 1 - i] = ww;
  }
  if (n % 2 == 1) xi[n / 2] = 0.5;
}

// orthonormal L_i(s) = sqrt(2i+1) P_i(2s-1) and L_i'(s) = 2 sqrt(2i+1) P_i'(2s-1)
void onb_all(int n, double s, double* L, double* dL) {
  double P[DG_MAXN], dP[DG_MAXN];
  legendre_all(n, 2.0 * s - 1.0, P, dP);
  for (int i = 0; i < n; ++i) {
    double a = std::sqrt(2.0 * i + 1.0);
    L[i] = a * P[i];
    dL[i] = 2.0 * a * dP[i];
  }
}

template <typename D, typename S>
void copy_round(const DGTab<S>& s, DGTab<D>* d) {
  for (int a = 0; a < DG_MAXN; ++a) {
    for (int b = 0; b < DG_MAXN; ++b) {
      d->B[a][b] = (D)s.B[a][b];
      d->Bd[a][b] = (D)s.Bd[a][b];
      d->D[a][b] = (D)s.D[a][b];
    }
    d->w[a] = (D)s.w[a];
    d->a0[a] = (D)s.a0[a];
    d->a1[a] = (D)s.a1[a];
    d->d0[a] = (D)s.d0[a];
    d->d1[a] = (D)s.d1[a];
    d->l0[a] = (D)s.l0[a];
    d->l1[a] = (D)s.l1[a];
    d->dl0[a] = (D)s.dl0[a];
    d->dl1[a] = (D)s.dl1[a];
  }
  d->sigma = (D)s.sigma;
}

}  // namespace

void dg_build_tables(int n, double sigma, DGTab<double>* t, DGTab<float>* t32) {
  std::memset(t, 0, sizeof(*t));
  double xi[DG_MAXN], w[DG_MAXN];
  gauss_01(n, xi, w);
  for (int a = 0; a < n; ++a) {
    double L[DG_MAXN], dL[DG_MAXN];
    onb_all(n, xi[a], L, dL);
    for (int i = 0; i < n; ++i) {
      t->B[a][i] = L[i];
      t->Bd[a][i] = dL[i];
    }
    t->w[a] = w[a];
  }
  {
    double L0[DG_MAXN], dL0[DG_MAXN], L1[DG_MAXN], dL1[DG_MAXN];
    onb_all(n, 0.0, L0, dL0);
    onb_all(n, 1.0, L1, dL1);
    for (int i = 0; i < n; ++i) {
      t->a0[i] = L0[i];
      t->a1[i] = L1[i];
      t->d0[i] = dL0[i];
      t->d1[i] = dL1[i];
    }
  }
  // barycentric weights of the Gauss points
  double lam[DG_MAXN];
  for (int a = 0; a < n; ++a) {
    double p = 1.0;
    for (int b = 0; b < n; ++b)
      if (b != a) p *= (xi[a] - xi[b]);
    lam[a] = 1.0 / p;
  }
  for (int a = 0; a < n; ++a) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) {
      if (b == a) continue;
      double v = (lam[b] / lam[a]) / (xi[a] - xi[b]);
      t->D[a][b] = v;
      s += v;
    }
    t->D[a][a] = -s;
  }
  // Lagrange values and derivatives at the ends s = 0, 1 (not nodes)
  for (int e = 0; e < 2; ++e) {
    double s = (double)e;
    for (int a = 0; a < n; ++a) {
      double l = 1.0, dsum = 0.0;
      for (int b = 0; b < n; ++b) {
        if (b == a) continue;
        l *= (s - xi[b]) / (xi[a] - xi[b]);
        dsum += 1.0 / (s - xi[b]);
      }
      if (e == 0) {
        t->l0[a] = l;
        t->dl0[a] = l * dsum;
      } else {
        t->l1[a] = l;
        t->dl1[a] = l * dsum;
      }
    }
  }
  t->sigma = sigma;
  copy_round<float, double>(*t, t32);
}

// Gauss-Legendre points and weights on [0,1] (the rule the tables use).
void dg_gauss_points(int n, double* xi, double* w) { gauss_01(n, xi, w); }
