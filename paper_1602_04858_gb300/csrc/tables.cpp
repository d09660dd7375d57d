// tables.cpp -- 1-D reference quantities on [0,1] for the nodal tensor basis.
//
// Basis (a reading: the paper does not fix one): along its own direction a
// velocity component is Lagrange of degree K+1 through the K+2 Gauss-Lobatto
// points; across it, and for the pressure, Lagrange of degree K through the
// K+1 Gauss points.  Integrals use a 12-point Gauss rule (exact here).
// The face matrices are the 1-D restriction of the interior-penalty form of
// eq. (ipbrinkman) with reference penalty (K+1)(K+2) (sigma_j h_j, Sec. 4.1)
// entering as 2 sigma, the average {.} = mean of both traces, the jump
// [.] = lower - upper trace, the normal pointing from the lower to the upper
// cell, and on boundary faces [v] = v, {v'} n = outward derivative.
#include "tables.h"

#include <cmath>
#include <vector>

namespace mgd {
namespace {

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n.
void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * t * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? t : p1, pm = (n == 1) ? 1.0 : p0;
      double dp = n * (t * pn - pm) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int m = 2; m <= n; ++m) {
      double p2 = ((2.0 * m - 1.0) * t * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? t : p1, pm = (n == 1) ? 1.0 : p0;
    double dp = n * (t * pn - pm) / (t * t - 1.0);
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) on [-1,1], halved
  }
}

std::vector<double> lobatto_nodes(int npts) {
  // K+2 <= 3 points are used: {0,1} and {0,1/2,1}
  if (npts == 2) return {0.0, 1.0};
  if (npts == 3) return {0.0, 0.5, 1.0};
  return {0.0, 0.5 - 0.5 / std::sqrt(5.0), 0.5 + 0.5 / std::sqrt(5.0), 1.0};
}

double lag(const std::vector<double>& z, int a, double x) {
  double v = 1.0;
  for (size_t m = 0; m < z.size(); ++m)
    if ((int)m != a) v *= (x - z[m]) / (z[a] - z[m]);
  return v;
}

double dlag(const std::vector<double>& z, int a, double x) {
  double s = 0.0;
  for (size_t l = 0; l < z.size(); ++l) {
    if ((int)l == a) continue;
    double t = 1.0 / (z[a] - z[l]);
    for (size_t m = 0; m < z.size(); ++m)
      if ((int)m != a && m != l) t *= (x - z[m]) / (z[a] - z[m]);
    s += t;
  }
  return s;
}

}  // namespace

template <int K>
void make_tables(Tab<K, double>& T, Tab<K, float>& F) {
  constexpr int K1 = K + 1, NG = K + 2;
  std::vector<double> gx, gw, qx, qw;
  gauss_rule(K1, gx, gw);
  gauss_rule(12, qx, qw);
  std::vector<double> lx = lobatto_nodes(NG);
  const double sig = (K + 1.0) * (K + 2.0);
  for (int b = 0; b < K1; ++b) T.wg[b] = gw[b];
  for (int a = 0; a < NG; ++a)
    for (int c = 0; c < NG; ++c) {
      double m = 0, k = 0;
      for (int q = 0; q < 12; ++q) {
        m += qw[q] * lag(lx, a, qx[q]) * lag(lx, c, qx[q]);
        k += qw[q] * dlag(lx, a, qx[q]) * dlag(lx, c, qx[q]);
      }
      T.Mcg[a][c] = m;
      T.Kcg[a][c] = k;
    }
  double V0[K1], V1[K1], D0[K1], D1[K1];
  for (int b = 0; b < K1; ++b) {
    V0[b] = lag(gx, b, 0.0);
    V1[b] = lag(gx, b, 1.0);
    D0[b] = dlag(gx, b, 0.0);
    D1[b] = dlag(gx, b, 1.0);
  }
  for (int b = 0; b < K1; ++b)
    for (int c = 0; c < K1; ++c) {
      double k = 0;
      for (int q = 0; q < 12; ++q) k += qw[q] * dlag(gx, b, qx[q]) * dlag(gx, c, qx[q]);
      T.Kdg[b][c] = k;
      T.F11[b][c] = 2 * sig * V1[b] * V1[c] - 0.5 * V1[b] * D1[c] - 0.5 * D1[b] * V1[c];
      T.F22[b][c] = 2 * sig * V0[b] * V0[c] + 0.5 * V0[b] * D0[c] + 0.5 * D0[b] * V0[c];
      T.F12[b][c] = -2 * sig * V1[b] * V0[c] - 0.5 * V1[b] * D0[c] + 0.5 * D1[b] * V0[c];
      T.F21[b][c] = -2 * sig * V0[b] * V1[c] + 0.5 * V0[b] * D1[c] - 0.5 * D0[b] * V1[c];
      T.Blo[b][c] = 2 * sig * V0[b] * V0[c] + V0[b] * D0[c] + D0[b] * V0[c];
      T.Bhi[b][c] = 2 * sig * V1[b] * V1[c] - V1[b] * D1[c] - D1[b] * V1[c];
    }
  for (int b = 0; b < K1; ++b)
    for (int a = 0; a < NG; ++a) {
      double g = 0;
      for (int q = 0; q < 12; ++q) g += qw[q] * lag(gx, b, qx[q]) * dlag(lx, a, qx[q]);
      T.G[b][a] = g;
    }
  for (int ch = 0; ch < 2; ++ch) {
    for (int af = 0; af < NG; ++af)
      for (int ac = 0; ac < NG; ++ac) T.Wgl[ch][af][ac] = lag(lx, ac, 0.5 * (ch + lx[af]));
    for (int bf = 0; bf < K1; ++bf)
      for (int bc = 0; bc < K1; ++bc) T.Wg[ch][bf][bc] = lag(gx, bc, 0.5 * (ch + gx[bf]));
  }
  // float copy
  const double* s = reinterpret_cast<const double*>(&T);
  float* d = reinterpret_cast<float*>(&F);
  static_assert(sizeof(Tab<K, double>) == 2 * sizeof(Tab<K, float>), "table layout");
  for (size_t i = 0; i < sizeof(Tab<K, double>) / sizeof(double); ++i) d[i] = (float)s[i];
}

template void make_tables<0>(Tab<0, double>&, Tab<0, float>&);
template void make_tables<1>(Tab<1, double>&, Tab<1, float>&);
template void make_tables<2>(Tab<2, double>&, Tab<2, float>&);

}  // namespace mgd
