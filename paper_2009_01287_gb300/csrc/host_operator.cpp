// Host evaluation of one element's rows of the DG operator (same sub-face
// formulation as the device kernel).  Used at setup to read the diagonal of A
// on V_J and the dense blocks A_e = R_e A R_e^T of the V_e (Section 4.1, items
// 2: "assembly of the diagonal ... and of the diagonal blocks").
#include <algorithm>
#include <cmath>
#include <vector>

#include "dg_internal.h"
#include "host_state.h"

namespace dg {

void host_element_residual(const dg_mesh& M, int64_t k, const double* x, double* y, int64_t source) {
  if (M.host.mapped) {
    host_element_residual_map(M, k, x, y);
    return;
  }
  const HostMesh& m = M.host;
  const int P = m.p[k], NP = P + 1, NN = NP * NP;
  const Basis1D& B = basis1d(P);
  const double hk = M.h_h[k], ak = m.coef[k];
  // x vanishes outside element `source` (when >= 0): on another element the
  // volume term and every sub-face not shared with `source` add exact zeros
  const bool own_zero = source >= 0 && source != k;
  const double* xk = x + m.off[k];
  auto sn = [](int s, int i, int q, int np) { return (s < 2) ? (i * np + q) : (q * np + i); };
  // volume: (K (x) M + M (x) K) x  with local index iy*NP + ix, two passes
  if (own_zero) std::fill(y, y + NN, 0.0);
  else {
    double t1[kMaxN * kMaxN], t2[kMaxN * kMaxN];
    for (int qy = 0; qy < NP; ++qy)
      for (int ix = 0; ix < NP; ++ix) {
        double a = 0.0, b = 0.0;
        for (int qx = 0; qx < NP; ++qx) {
          a += B.K[ix * NP + qx] * xk[qy * NP + qx];
          b += B.M[ix * NP + qx] * xk[qy * NP + qx];
        }
        t1[qy * NP + ix] = a;
        t2[qy * NP + ix] = b;
      }
    for (int iy = 0; iy < NP; ++iy)
      for (int ix = 0; ix < NP; ++ix) {
        double v = 0.0;
        for (int qy = 0; qy < NP; ++qy) v += B.M[iy * NP + qy] * t1[qy * NP + ix] + B.K[iy * NP + qy] * t2[qy * NP + ix];
        y[iy * NP + ix] = ak * v;
      }
  }
  double dn[4 * kMaxN], r[4 * kMaxN] = {0.0}, c2[4 * kMaxN] = {0.0};
  for (int s = 0; s < 4; ++s)
    for (int i = 0; i < NP; ++i) {
      const double* dv = (s & 1) ? B.d1.data() : B.d0.data();
      double acc = 0.0;
      for (int q = 0; q < NP; ++q) acc += dv[q] * xk[sn(s, i, q, NP)];
      dn[s * NP + i] = ((s & 1) ? 1.0 : -1.0) * (ak / hk) * acc;   // a grad u . n
    }
  const double* T = M.h_tables.data();
  for (int s = 0; s < 4; ++s) {
    const int kedge = (s & 1) ? P : 0;
    for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
      const SubFaceRec& f = M.h_sf[j];
      if (own_zero && f.nb != source) continue;
      double un[kMaxN] = {0.0}, dnn[kMaxN] = {0.0};
      int np = 0;
      if (f.nb >= 0) {
        np = f.pn + 1;
        const Basis1D& Bn = basis1d(f.pn);
        const double* xn = x + m.off[f.nb];
        const int ke = (f.nb_side & 1) ? f.pn : 0;
        const double* dv = (f.nb_side & 1) ? Bn.d1.data() : Bn.d0.data();
        const double sg = ((f.nb_side & 1) ? -1.0 : 1.0) * (m.coef[f.nb] / M.h_h[f.nb]);
        for (int q = 0; q < np; ++q) {
          un[q] = xn[sn(f.nb_side, q, ke, np)];
          double acc = 0.0;
          for (int t = 0; t < np; ++t) acc += dv[t] * xn[sn(f.nb_side, q, t, np)];
          dnn[q] = sg * acc;
        }
      }
      double jo[kMaxN], cd[kMaxN], jn[kMaxN] = {0.0};
      for (int i = 0; i < NP; ++i) {
        double a = 0.0, c = 0.0, b = 0.0, d = 0.0;
        for (int q = 0; q < NP; ++q) {
          a += T[f.tab_oo + i * NP + q] * xk[sn(s, q, kedge, NP)];
          c += T[f.tab_oo + i * NP + q] * dn[s * NP + q];
        }
        for (int q = 0; q < np; ++q) {
          b += T[f.tab_on + i * np + q] * un[q];
          d += T[f.tab_on + i * np + q] * dnn[q];
        }
        a *= f.len; b *= f.len; c *= f.len; d *= f.len;
        if (f.nb < 0) {
          c2[s * NP + i] -= a;
          jo[i] = a;
          cd[i] = -c;
          if (M.opts.form == DG_FORM_SIPG) r[s * NP + i] += -c + f.sigma * a;
        } else {
          c2[s * NP + i] -= 0.5 * (a - b);
          jo[i] = a - b;
          cd[i] = -0.5 * (c + d);
          if (M.opts.form == DG_FORM_SIPG) r[s * NP + i] += -0.5 * (c + d) + f.sigma * (a - b);
        }
      }
      if (M.opts.form == DG_FORM_BR2) {
        for (int q = 0; q < np; ++q) {
          double v = 0.0;
          for (int i = 0; i < NP; ++i) v += T[f.tab_on + i * np + q] * xk[sn(s, i, kedge, NP)];
          for (int t = 0; t < np; ++t) v -= T[f.tab_nn + q * np + t] * un[t];
          jn[q] = v * f.len;
        }
        double go[kMaxN], gn[kMaxN] = {0.0};
        // both sides' liftings carry the larger a of the sub-face
        const double w = f.nb < 0 ? ak : std::max(ak, m.coef[f.nb]);
        for (int i = 0; i < NP; ++i) {
          double g = 0.0;
          for (int q = 0; q < NP; ++q) g += B.Minv[i * NP + q] * jo[q];
          go[i] = w * (g * B.Minv[0] / (hk * hk));
        }
        if (np) {
          const Basis1D& Bn = basis1d(f.pn);
          const double hn = M.h_h[f.nb];
          for (int q = 0; q < np; ++q) {
            double g = 0.0;
            for (int t = 0; t < np; ++t) g += Bn.Minv[q * np + t] * jn[t];
            gn[q] = w * (g * Bn.Minv[0] / (hn * hn));
          }
        }
        const double coef = (f.nb < 0) ? 1.0 : 0.25;
        for (int i = 0; i < NP; ++i) {
          double st = 0.0;
          for (int q = 0; q < NP; ++q) st += T[f.tab_oo + i * NP + q] * go[q];
          for (int q = 0; q < np; ++q) st += T[f.tab_on + i * np + q] * gn[q];
          r[s * NP + i] += cd[i] + M.eta * coef * f.len * st;
        }
      }
    }
  }
  for (int node = 0; node < NN; ++node) {
    const int ix = node % NP, iy = node / NP;
    double v = y[node];
    const double aih = ak / hk;
    v += -B.d0[ix] * aih * c2[0 * NP + iy];
    v += B.d1[ix] * aih * c2[1 * NP + iy];
    v += -B.d0[iy] * aih * c2[2 * NP + ix];
    v += B.d1[iy] * aih * c2[3 * NP + ix];
    if (ix == 0) v += r[0 * NP + iy];
    if (ix == P) v += r[1 * NP + iy];
    if (iy == 0) v += r[2 * NP + ix];
    if (iy == P) v += r[3 * NP + ix];
    y[node] = v;
  }
}

// Diagonal of element k's rows, in closed form: the volume diagonal plus, for
// every side holding the node, the sub-face terms of the node's own basis
// function (its trace is l_i on that side, its outward normal derivative is
// dv l_i, dv = l_edge'(edge) / h with the outward sign).
void host_element_diag(const dg_mesh& M, int64_t k, double* d) {
  if (M.host.mapped) {
    host_element_diag_map(M, k, d);
    return;
  }
  const HostMesh& m = M.host;
  const int P = m.p[k], NP = P + 1;
  const Basis1D& B = basis1d(P);
  const double hk = M.h_h[k], ak = m.coef[k];
  const double* T = M.h_tables.data();
  const bool br2 = M.opts.form == DG_FORM_BR2;
  for (int iy = 0; iy < NP; ++iy)
    for (int ix = 0; ix < NP; ++ix)
      d[iy * NP + ix] = ak * (B.K[ix * NP + ix] * B.M[iy * NP + iy] + B.M[ix * NP + ix] * B.K[iy * NP + iy]);
  double go[kMaxN], gn[kMaxN], jo[kMaxN], jn[kMaxN];
  for (int s = 0; s < 4; ++s) {
    const double dv = ((s & 1) ? B.d1[P] : -B.d0[0]) * (ak / hk);   // a times the normal derivative
    for (int i = 0; i < NP; ++i) {
      const int node = (s < 2) ? (i * NP + ((s & 1) ? P : 0)) : (((s & 1) ? P : 0) * NP + i);
      double add = 0.0;
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        const SubFaceRec& f = M.h_sf[j];
        const double moo = T[f.tab_oo + i * NP + i];
        const bool interior = f.nb >= 0;
        if (!br2) {
          add += f.len * moo * (f.sigma - (interior ? 1.0 : 2.0) * dv);
          continue;
        }
        add -= (interior ? 1.0 : 2.0) * f.len * moo * dv;
        const double w = interior ? std::max(ak, m.coef[f.nb]) : ak;   // larger a of the sub-face
        for (int q = 0; q < NP; ++q) jo[q] = f.len * T[f.tab_oo + q * NP + i];
        for (int a = 0; a < NP; ++a) {
          double g = 0.0;
          for (int q = 0; q < NP; ++q) g += B.Minv[a * NP + q] * jo[q];
          go[a] = w * (g * B.Minv[0] / (hk * hk));
        }
        double st = 0.0;
        for (int a = 0; a < NP; ++a) st += T[f.tab_oo + i * NP + a] * go[a];
        if (interior) {
          const int np = f.pn + 1;
          const Basis1D& Bn = basis1d(f.pn);
          const double hn = M.h_h[f.nb];
          for (int q = 0; q < np; ++q) jn[q] = f.len * T[f.tab_on + i * np + q];
          for (int a = 0; a < np; ++a) {
            double g = 0.0;
            for (int q = 0; q < np; ++q) g += Bn.Minv[a * np + q] * jn[q];
            gn[a] = w * (g * Bn.Minv[0] / (hn * hn));
          }
          for (int a = 0; a < np; ++a) st += T[f.tab_on + i * np + a] * gn[a];
        }
        add += M.eta * (interior ? 0.25 : 1.0) * f.len * st;
      }
      d[node] += add;
    }
  }
}

}  // namespace dg
