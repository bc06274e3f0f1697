// Host-side 1D tables and small dense helpers of the CUDA library (FP64).
//
// Sec. 2 (Fig. 1): Q_k / Q_{k-1} shape functions are tensor products of 1D Lagrange
// polynomials on (0,1); nodes are the Gauss-Lobatto points of each degree, integrals use
// the (k+1)-point Gauss-Legendre rule.  Both point sets are computed here by Newton's
// method on the Legendre polynomials (three-term recurrence), independent of any library.
#include <cmath>
#include <vector>

#include "host_tables.h"

namespace smf {

// P_n(x) and P_n'(x) by the three-term recurrence (n >= 1).
static void legendre(int n, double x, double &p, double &dp) {
  double p0 = 1.0, p1 = x;
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  p = (n == 0) ? 1.0 : p1;
  // derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n)
  dp = (n == 0) ? 0.0 : n * (p0 - x * p1) / (1.0 - x * x);
}

void gauss_legendre01(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, p, dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, p, dp);
    // ascending order on [0,1]
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // = 2/((1-z^2)P'^2) / 2
  }
}

void gauss_lobatto01(int deg, double *x) {
  if (deg == 1) {
    x[0] = 0.0;
    x[1] = 1.0;
    return;
  }
  x[0] = 0.0;
  x[deg] = 1.0;
  // interior nodes: roots of P_deg'; Newton with P_deg'' from the Legendre equation
  for (int i = 1; i < deg; ++i) {
    double z = -std::cos(M_PI * i / deg);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(deg, z, p, dp);
      double d2p = (2.0 * z * dp - deg * (deg + 1.0) * p) / (1.0 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 + z);
  }
}

double lagrange(const double *nodes, int n, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
  return v;
}

double lagrange_deriv(const double *nodes, int n, int i, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double t = 1.0 / (nodes[i] - nodes[m]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != m) t *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    s += t;
  }
  return s;
}

void build_tables(int k, Tab1D<double> &t) {
  const int nq = k + 1, nv = k + 1, np = k;
  double xg[kMaxN1], wg[kMaxN1], xv[kMaxN1], xp[kMaxN1];
  gauss_legendre01(nq, xg, wg);
  gauss_lobatto01(k, xv);
  gauss_lobatto01(k - 1, xp);
  for (int i = 0; i < kMaxN1 * kMaxN1; ++i) t.S[i] = t.Sd[i] = t.D[i] = 0.0;
  for (int i = 0; i < kMaxN1 * kMaxDeg; ++i) t.Pv[i] = t.Pd[i] = 0.0;
  for (int m = 0; m < kMaxN1; ++m) t.nodes[m] = m < nv ? xv[m] : 0.0;
  for (int q = 0; q < nq; ++q) {
    t.x[q] = xg[q];
    t.w[q] = wg[q];
    for (int m = 0; m < nv; ++m) {
      t.S[q * nv + m] = lagrange(xv, nv, m, xg[q]);
      t.Sd[q * nv + m] = lagrange_deriv(xv, nv, m, xg[q]);
    }
    for (int m = 0; m < nq; ++m) t.D[q * nq + m] = lagrange_deriv(xg, nq, m, xg[q]);
    for (int m = 0; m < np; ++m) {
      t.Pv[q * np + m] = lagrange(xp, np, m, xg[q]);
      t.Pd[q * np + m] = lagrange_deriv(xp, np, m, xg[q]);
    }
  }
}

void build_transfer(int k, TransferTab<double> &tt) {
  for (auto &v : tt.vel) v = 0.0;
  for (auto &v : tt.pre) v = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    const int deg = pass == 0 ? k : k - 1;
    double t[kMaxN1];
    gauss_lobatto01(deg, t);
    for (int h = 0; h < 2; ++h)
      for (int a = 0; a <= deg; ++a) {
        const double xi = 0.5 * (h + t[a]);
        for (int m = 0; m <= deg; ++m) {
          double v = lagrange(t, deg + 1, m, xi);
          if (std::fabs(v) < 1e-15) v = 0.0;
          if (std::fabs(v - 1.0) < 1e-15) v = 1.0;
          if (pass == 0)
            tt.vel[(h * (deg + 1) + a) * (deg + 1) + m] = v;
          else
            tt.pre[(h * (deg + 1) + a) * (deg + 1) + m] = v;
        }
      }
  }
}

// Largest eigenvalue of the symmetric tridiagonal matrix (diag a[0..n), off-diag b[0..n-1))
// by bisection on the Sturm sequence count.
double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b) {
  const int n = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // number of eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) >= n)
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

}  // namespace smf
