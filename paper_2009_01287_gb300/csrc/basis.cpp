// Host 1D polynomial machinery: Gauss-Lobatto nodes (Section 2.2), Gauss
// rules and Lagrange values for the setup of the device tables.
#include <cmath>
#include <mutex>

#include "dg_internal.h"

namespace dg {

namespace {

// P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre(int n, double x, double& pn, double& pn1) {
  double a = 1.0, b = x;
  if (n == 0) { pn = 1.0; pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  pn = b;
  pn1 = a;
}

}  // namespace

std::vector<double> gll_nodes(int p) {
  // interior nodes: roots of P_p' on (-1,1), Newton with P_p'' from the
  // Legendre equation; start from the Chebyshev-Lobatto points.
  std::vector<double> x(p + 1);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double t = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(p, t, pn, pn1);
      double dp = p * (t * pn - pn1) / (t * t - 1.0);
      double ddp = (2.0 * t * dp - p * (p + 1.0) * pn) / (1.0 - t * t);
      double dt = dp / ddp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = t;
  }
  std::vector<double> out(p + 1);
  for (int j = 0; j <= p; ++j) out[j] = 0.5 * (x[j] + 1.0);
  // enforce the exact mirror symmetry of the rule
  for (int j = 0; j <= p / 2; ++j) {
    double a = 0.5 * (out[j] + (1.0 - out[p - j]));
    out[j] = a;
    out[p - j] = 1.0 - a;
  }
  out[0] = 0.0;
  out[p] = 1.0;
  if (p % 2 == 0) out[p / 2] = 0.5;
  return out;
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int j = 0; j < q; ++j) {
    double t = -std::cos(M_PI * (j + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(q, t, pn, pn1);
      dp = q * (t * pn - pn1) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double pn, pn1;
    legendre(q, t, pn, pn1);
    dp = q * (t * pn - pn1) / (t * t - 1.0);
    x[j] = 0.5 * (t + 1.0);
    w[j] = 1.0 / ((1.0 - t * t) * dp * dp);  // (2/((1-t^2)P'^2)) / 2
  }
}

void lagrange_eval(const std::vector<double>& nodes, double t, double* out) {
  const int n = (int)nodes.size();
  for (int j = 0; j < n; ++j) {
    if (t == nodes[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  }
  double denom = 0.0;
  for (int j = 0; j < n; ++j) {
    double lam = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) lam /= (nodes[j] - nodes[k]);
    out[j] = lam / (t - nodes[j]);
    denom += out[j];
  }
  for (int j = 0; j < n; ++j) out[j] /= denom;
}

void lagrange_deriv_eval(const std::vector<double>& nodes, double t, double* out) {
  const int n = (int)nodes.size();
  int hit = -1;
  for (int j = 0; j < n; ++j)
    if (t == nodes[j]) hit = j;
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (nodes[j] - nodes[k]);
  if (hit >= 0) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == hit) continue;
      out[j] = (lam[j] / lam[hit]) / (t - nodes[j]);
      s += 1.0 / (t - nodes[j]);
    }
    out[hit] = s;
    return;
  }
  std::vector<double> l(n);
  lagrange_eval(nodes, t, l.data());
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = 0; k < n; ++k)
      if (k != j) s += 1.0 / (t - nodes[k]);
    out[j] = l[j] * s;
  }
}

namespace {

void invert_spd(int n, const double* A, double* Ainv) {
  // Gauss-Jordan with partial pivoting (n <= 9)
  std::vector<double> a(A, A + n * n), b(n * n, 0.0);
  for (int i = 0; i < n; ++i) b[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    for (int j = 0; j < n; ++j) {
      std::swap(a[c * n + j], a[piv * n + j]);
      std::swap(b[c * n + j], b[piv * n + j]);
    }
    double d = a[c * n + c];
    for (int j = 0; j < n; ++j) { a[c * n + j] /= d; b[c * n + j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { a[r * n + j] -= f * a[c * n + j]; b[r * n + j] -= f * b[c * n + j]; }
    }
  }
  for (int i = 0; i < n * n; ++i) Ainv[i] = b[i];
}

Basis1D make_basis(int p) {
  Basis1D b;
  b.p = p;
  b.nodes = gll_nodes(p);
  const int n = p + 1;
  std::vector<double> gx, gw;
  gauss_rule(p + 1, gx, gw);
  b.M.assign(n * n, 0.0);
  b.K.assign(n * n, 0.0);
  std::vector<double> l(n), d(n);
  for (int g = 0; g < (int)gx.size(); ++g) {
    lagrange_eval(b.nodes, gx[g], l.data());
    lagrange_deriv_eval(b.nodes, gx[g], d.data());
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        b.M[i * n + j] += gw[g] * l[i] * l[j];
        b.K[i * n + j] += gw[g] * d[i] * d[j];
      }
  }
  b.Minv.assign(n * n, 0.0);
  invert_spd(n, b.M.data(), b.Minv.data());
  b.d0.assign(n, 0.0);
  b.d1.assign(n, 0.0);
  lagrange_deriv_eval(b.nodes, 0.0, b.d0.data());
  lagrange_deriv_eval(b.nodes, 1.0, b.d1.data());
  return b;
}

}  // namespace

const Basis1D& basis1d(int p) {
  static std::once_flag once;
  static std::vector<Basis1D> table;
  std::call_once(once, [] {
    table.resize(kMaxP + 1);
    for (int q = 1; q <= kMaxP; ++q) table[q] = make_basis(q);
  });
  if (p < 1 || p > kMaxP) throw Error(DG_EINVAL, "degree out of range");
  return table[p];
}

}  // namespace dg
