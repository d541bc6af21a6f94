// Host construction of the 1D Gauss / Gauss-Lobatto tables (Sec. 5: Q_k
// Lagrange basis on Gauss-Lobatto nodes, k+1 Gauss-Legendre quadrature points).
#include "tables.h"

#include <cmath>
#include <utility>
#include <vector>

namespace sipg {
namespace {

// P_m(x) and P_m'(x) by the three-term recurrence.
void legendre(int m, double x, double* p, double* dp, double* d2p) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
  if (m == 0) { *p = 1.0; *dp = 0.0; *d2p = 0.0; return; }
  for (int j = 1; j < m; ++j) {
    const double p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
    const double d2 = ((2 * j + 1) * (p1 + x * d1) - j * d0) / (j + 1);
    const double e2 = ((2 * j + 1) * (2 * d1 + x * e1) - j * e0) / (j + 1);
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
  }
  *p = p1; *dp = d1; *d2p = e1;
}

std::vector<double> lagrange_values(const std::vector<double>& nodes, double x) {
  const int n = (int)nodes.size();
  std::vector<double> v(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) v[j] *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

std::vector<double> lagrange_derivs(const std::vector<double>& nodes, double x) {
  const int n = (int)nodes.size();
  std::vector<double> d(n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      double t = 1.0 / (nodes[j] - nodes[m]);
      for (int l = 0; l < n; ++l)
        if (l != j && l != m) t *= (x - nodes[l]) / (nodes[j] - nodes[l]);
      d[j] += t;
    }
  return d;
}

}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp, d2p;
      legendre(n, t, &p, &dp, &d2p);
      const double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double p, dp, d2p;
    legendre(n, t, &p, &dp, &d2p);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // half of 2/((1-t^2) P'^2)
  }
}

void gauss_lobatto(int n, double* x, double* w) {
  const int m = n - 1;
  std::vector<double> t(n);
  t[0] = -1.0;
  t[n - 1] = 1.0;
  for (int j = 1; j < n - 1; ++j) {
    double s = -std::cos(M_PI * j / m);
    for (int it = 0; it < 100; ++it) {
      double p, dp, d2p;
      legendre(m, s, &p, &dp, &d2p);
      const double step = dp / d2p;
      s -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    t[j] = s;
  }
  for (int j = 0; j < n; ++j) {
    double p, dp, d2p;
    legendre(m, t[j], &p, &dp, &d2p);
    x[j] = 0.5 * (t[j] + 1.0);
    w[j] = 1.0 / (n * m * p * p);
  }
}

Tab make_tab(int n) {
  Tab T{};
  T.n = n;
  std::vector<double> gll(n), gllw(n), gp(n), gw(n);
  gauss_lobatto(n, gll.data(), gllw.data());
  gauss_legendre(n, gp.data(), gw.data());
  for (int q = 0; q < n; ++q) {
    const auto s = lagrange_values(gll, gp[q]);
    const auto ds = lagrange_derivs(gll, gp[q]);
    const auto dg = lagrange_derivs(gp, gp[q]);
    for (int j = 0; j < n; ++j) {
      T.S[q * n + j] = s[j];
      T.DS[q * n + j] = ds[j];
      T.Dg[q * n + j] = dg[j];
    }
  }
  const auto d0 = lagrange_derivs(gll, 0.0), d1 = lagrange_derivs(gll, 1.0);
  for (int j = 0; j < n; ++j) {
    T.dS0[j] = d0[j];
    T.dS1[j] = d1[j];
    T.gw[j] = gw[j];
    T.gp[j] = gp[j];
    T.gll[j] = gll[j];
  }
  // 1D mass matrix with the n-point Gauss rule, and its inverse by Gauss-Jordan
  // elimination with partial pivoting (symmetric positive definite, n <= 6)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += gw[q] * T.S[q * n + i] * T.S[q * n + j];
      T.M1[i * n + j] = s;
    }
  std::vector<double> a(T.M1, T.M1 + n * n), inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[p * n + c])) p = r;
    for (int j = 0; j < n; ++j) {
      std::swap(a[c * n + j], a[p * n + j]);
      std::swap(inv[c * n + j], inv[p * n + j]);
    }
    const double d = a[c * n + c];
    for (int j = 0; j < n; ++j) {
      a[c * n + j] /= d;
      inv[c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      for (int j = 0; j < n; ++j) {
        a[r * n + j] -= f * a[c * n + j];
        inv[r * n + j] -= f * inv[c * n + j];
      }
    }
  }
  for (int i = 0; i < n * n; ++i) T.M1inv[i] = inv[i];
  return T;
}

SplitTab make_split_tab(int n) {
  SplitTab T{};
  T.n = n;
  std::vector<double> gll(n), gllw(n), gp(n), gw(n), pl(n - 1), plw(n - 1);
  gauss_lobatto(n, gll.data(), gllw.data());
  gauss_legendre(n, gp.data(), gw.data());
  if (n - 1 >= 2) gauss_lobatto(n - 1, pl.data(), plw.data());
  for (int q = 0; q < n; ++q) {
    const auto s = lagrange_values(gll, gp[q]);
    const auto ds = lagrange_derivs(gll, gp[q]);
    const auto dg = lagrange_derivs(gp, gp[q]);
    for (int j = 0; j < n; ++j) {
      T.S[q * n + j] = s[j];
      T.DS[q * n + j] = ds[j];
      T.Dg[q * n + j] = dg[j];
    }
    if (n - 1 >= 2) {
      const auto sp = lagrange_values(pl, gp[q]);
      const auto dsp = lagrange_derivs(pl, gp[q]);
      for (int j = 0; j < n - 1; ++j) {
        T.Sp[q * (n - 1) + j] = sp[j];
        T.DSp[q * (n - 1) + j] = dsp[j];
      }
    }
  }
  const auto d0 = lagrange_derivs(gll, 0.0), d1 = lagrange_derivs(gll, 1.0);
  const auto l0 = lagrange_values(gp, 0.0), l1 = lagrange_values(gp, 1.0);
  const auto e0 = lagrange_derivs(gp, 0.0), e1 = lagrange_derivs(gp, 1.0);
  for (int j = 0; j < n; ++j) {
    T.dS0[j] = d0[j];
    T.dS1[j] = d1[j];
    T.lg0[j] = l0[j];
    T.lg1[j] = l1[j];
    T.dlg0[j] = e0[j];
    T.dlg1[j] = e1[j];
    T.gw[j] = gw[j];
    T.gp[j] = gp[j];
  }
  for (int j = 0; j < n; ++j) {
    const auto lj = lagrange_values(gp, gll[j]);
    for (int q = 0; q < n; ++q) T.Sinv[j * n + q] = lj[q];
  }
  return T;
}

TransferTab make_p_transfer(int nf, int nc) {
  TransferTab T{};
  T.nf = nf;
  T.nc = nc;
  std::vector<double> xf(nf), wf(nf), xc(nc), wc(nc);
  gauss_lobatto(nf, xf.data(), wf.data());
  gauss_lobatto(nc, xc.data(), wc.data());
  for (int i = 0; i < nf; ++i) {
    const auto v = lagrange_values(xc, xf[i]);
    for (int j = 0; j < nc; ++j) T.E[i * nc + j] = v[j];
  }
  return T;
}

TransferTab make_h_transfer(int n) {
  TransferTab T{};
  T.nf = n;
  T.nc = n;
  std::vector<double> x(n), w(n);
  gauss_lobatto(n, x.data(), w.data());
  for (int i = 0; i < n; ++i) {
    const auto v0 = lagrange_values(x, 0.5 * x[i]);
    const auto v1 = lagrange_values(x, 0.5 * (x[i] + 1.0));
    for (int j = 0; j < n; ++j) {
      T.E[i * n + j] = v0[j];
      T.E1[i * n + j] = v1[j];
    }
  }
  return T;
}

// Downward interpolation (linearization velocity onto a coarse level):
// p: I[j*nf + i] = l^fine_i(xi^coarse_j); h: child of each coarse node and the
// fine-basis values at the node's position inside that child.
TransferTab make_p_interp_down(int nf, int nc) {
  TransferTab T{};
  T.nf = nf;
  T.nc = nc;
  std::vector<double> xf(nf), wf(nf), xc(nc), wc(nc);
  gauss_lobatto(nf, xf.data(), wf.data());
  gauss_lobatto(nc, xc.data(), wc.data());
  for (int j = 0; j < nc; ++j) {
    const auto v = lagrange_values(xf, xc[j]);
    for (int i = 0; i < nf; ++i) T.E[j * nf + i] = v[i];
  }
  return T;
}

TransferTab make_h_interp_down(int n, int* child) {
  TransferTab T{};
  T.nf = n;
  T.nc = n;
  std::vector<double> x(n), w(n);
  gauss_lobatto(n, x.data(), w.data());
  for (int j = 0; j < n; ++j) {
    child[j] = x[j] > 0.5 ? 1 : 0;  // a node on the child interface goes to child 0
    const double local = 2.0 * x[j] - child[j];
    const auto v = lagrange_values(x, local);
    for (int i = 0; i < n; ++i) T.E[j * n + i] = v[i];
  }
  return T;
}

LoadTab make_load_tab(int n) {
  LoadTab T{};
  T.n = n;
  T.nq = n + 3;
  std::vector<double> gll(n), gllw(n);
  gauss_lobatto(n, gll.data(), gllw.data());
  gauss_legendre(T.nq, T.gp, T.gw);
  for (int q = 0; q < T.nq; ++q) {
    const auto v = lagrange_values(gll, T.gp[q]);
    for (int j = 0; j < n; ++j) T.S[q * n + j] = v[j];
  }
  return T;
}

}  // namespace sipg
