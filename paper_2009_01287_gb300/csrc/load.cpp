// Load vectors from caller-supplied data (host): b_i = int f phi_i over the
// elements plus, for u = g on the boundary imposed weakly by SIPG (Section 2
// with inhomogeneous Dirichlet data), the boundary terms
//   sum over boundary sub-faces of int g (sigma phi_i - a grad phi_i . n) ds
// that replacing [[u]] by u - g on the boundary moves to the right-hand side.
// Quadrature: p+3 Gauss points per direction on the volume and on every
// boundary sub-face.  Mapped meshes take the images and det J of the volume
// points and, on boundary sub-faces, the images, the weights with the arc
// length and m = J^-1 n stored when the mesh was made (grad phi . n =
// grad_X phi . m, grad_X the pre-image gradient).  The callbacks' outputs are
// NaN before each call, so values a callback leaves unwritten are reported.
#include <cmath>
#include <vector>

#include "dg_internal.h"
#include "host_state.h"

namespace dg {

void host_load(const dg_mesh& M, dg_field_fn f, dg_field_fn g, void* ctx, double* hb) {
  const HostMesh& m = M.host;
  if (m.dim != 2) throw Error(DG_EUNSUPPORTED, "load vectors from callbacks: square meshes only");
  if (g && M.opts.form != DG_FORM_SIPG) throw Error(DG_EUNSUPPORTED, "boundary data: SIPG only");
  std::fill(hb, hb + M.n_dofs, 0.0);
  std::vector<double> gx, gw, L, X, val;
  // a boundary sub-face of a mapped element: the stored images, weights and
  // m = J^-1 n at the p+3 Gauss points; grad phi . n = (d_t phi m_t + d_n phi
  // m_n) / h with d_t, d_n the reference derivatives along the side and along
  // the normal axis (increasing coordinate) and m_t, m_n the matching parts of m
  auto mapped_boundary = [&](int64_t k, int s, int j, int t0) {
    const int P = m.p[k], NP = P + 1, q = P + 3;
    const Basis1D& B = basis1d(P);
    const auto& sf = m.sf[j];
    const double h = m.size[k] * m.lh;
    const int edge = (s & 1) ? P : 0;
    const double* dv = (s & 1) ? B.d1.data() : B.d0.data();
    std::vector<double> rx, rw;
    gauss_rule(q, rx, rw);
    std::vector<double> Ls((size_t)q * NP), Ds((size_t)q * NP), pts(2 * (size_t)q), gv(q, std::nan(""));
    const double* geo = M.h_xbnd.data() + M.h_boff[j];
    for (int r = 0; r < q; ++r) {
      const double t = ((sf.t0 - t0) + (sf.t1 - sf.t0) * rx[r]) / (double)m.size[k];
      lagrange_eval(B.nodes, t, &Ls[(size_t)r * NP]);
      lagrange_deriv_eval(B.nodes, t, &Ds[(size_t)r * NP]);
      pts[2 * r] = geo[5 * r];
      pts[2 * r + 1] = geo[5 * r + 1];
    }
    g(q, pts.data(), gv.data(), ctx);
    const double sigma = M.h_sfm[j].sigma, a = m.coef[k];
    for (int r = 0; r < q; ++r) {
      DG_REQUIRE(std::isfinite(gv[r]), "g returned a non-finite value");
      const double* e = geo + 5 * r;
      const double mn = s < 2 ? e[3] : e[4], mt = s < 2 ? e[4] : e[3];
      const double w = e[2] * gv[r];
      for (int i = 0; i < NP; ++i) {
        const double li = Ls[(size_t)r * NP + i], di = Ds[(size_t)r * NP + i];
        for (int jn = 0; jn < NP; ++jn) {
          // node i along the side, jn along the normal
          const int node = s < 2 ? i * NP + jn : jn * NP + i;
          double dn = li * dv[jn] * mn;               // along the normal axis
          if (jn == edge) dn += di * mt;              // along the side
          double v = -a * dn / h;                     // - a grad phi . n
          if (jn == edge) v += sigma * li;            // sigma phi on the side
          hb[m.off[k] + node] += w * v;
        }
      }
    }
  };
  for (int64_t k = 0; k < m.n; ++k) {
    const int P = m.p[k], NP = P + 1, q = P + 3;
    const Basis1D& B = basis1d(P);
    gauss_rule(q, gx, gw);
    const double h = m.size[k] * m.lh;
    const double X0 = m.lo[2 * k] * m.lh, Y0 = m.lo[2 * k + 1] * m.lh;
    L.resize((size_t)q * NP);
    for (int r = 0; r < q; ++r) lagrange_eval(B.nodes, gx[r], &L[(size_t)r * NP]);
    if (f) {
      X.resize(2 * (size_t)q * q);
      val.assign((size_t)q * q, std::nan(""));
      std::vector<double> det((size_t)q * q, 1.0);
      for (int gy = 0; gy < q; ++gy)
        for (int gxi = 0; gxi < q; ++gxi) {
          const int pt = gy * q + gxi;
          if (m.mapped) {
            const double* s = M.h_xrhs.data() + M.h_roff[k] + 3 * pt;
            X[2 * pt] = s[0];
            X[2 * pt + 1] = s[1];
            det[pt] = s[2];
          } else {
            X[2 * pt] = X0 + h * gx[gxi];
            X[2 * pt + 1] = Y0 + h * gx[gy];
          }
        }
      f(q * q, X.data(), val.data(), ctx);
      for (int gy = 0; gy < q; ++gy)
        for (int gxi = 0; gxi < q; ++gxi) {
          const int pt = gy * q + gxi;
          DG_REQUIRE(std::isfinite(val[pt]), "f returned a non-finite value");
          const double w = gw[gxi] * gw[gy] * h * h * det[pt] * val[pt];
          for (int iy = 0; iy < NP; ++iy)
            for (int ix = 0; ix < NP; ++ix)
              hb[m.off[k] + iy * NP + ix] += w * L[(size_t)gy * NP + iy] * L[(size_t)gxi * NP + ix];
        }
    }
    if (!g) continue;
    for (int s = 0; s < 4; ++s) {
      int axis, c, t0, t1;
      m.side_segment((int)k, s, axis, c, t0, t1);
      const int edge = (s & 1) ? P : 0;
      const double* dv = (s & 1) ? B.d1.data() : B.d0.data();
      const double sgn = (s & 1) ? 1.0 : -1.0;   // outward along the normal axis
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        const auto& sf = m.sf[j];
        if (sf.nb >= 0) continue;
        if (m.mapped) {
          mapped_boundary(k, s, j, t0);
          continue;
        }
        const double len = (sf.t1 - sf.t0) * m.lh;
        X.resize(2 * (size_t)q);
        val.assign(q, std::nan(""));
        std::vector<double> Ls((size_t)q * NP);
        for (int r = 0; r < q; ++r) {
          const double t = (sf.t0 + (sf.t1 - sf.t0) * gx[r]) * m.lh;
          X[2 * r] = s < 2 ? c * m.lh : t;
          X[2 * r + 1] = s < 2 ? t : c * m.lh;
          lagrange_eval(B.nodes, ((sf.t0 - t0) + (sf.t1 - sf.t0) * gx[r]) / (double)m.size[k], &Ls[(size_t)r * NP]);
        }
        g(q, X.data(), val.data(), ctx);
        const double sigma = M.h_sf[j].sigma;
        const double aih = m.coef[k] / h;
        for (int r = 0; r < q; ++r) {
          DG_REQUIRE(std::isfinite(val[r]), "g returned a non-finite value");
          const double w = gw[r] * len * val[r];
          for (int i = 0; i < NP; ++i) {
            const double li = Ls[(size_t)r * NP + i];
            for (int jn = 0; jn < NP; ++jn) {
              // node i along the side, jn along the normal
              const int node = s < 2 ? i * NP + jn : jn * NP + i;
              double v = -aih * sgn * dv[jn] * li;    // - a grad phi . n
              if (jn == edge) v += sigma * li;        // sigma phi on the side
              hb[m.off[k] + node] += w * v;
            }
          }
        }
      }
    }
  }
}

}  // namespace dg
