// Mapped square meshes (Section 2: element maps T_kappa onto general
// quadrilaterals).  The leaf boxes of the lattice are pre-images; the bilinear
// map of the lattice domain onto the quadrilateral with the given corners, or
// the caller's smooth map (curved elements), carries them to the elements.
// This file builds what the mapped operator kernel reads - per degree the
// volume rule's basis tables, the geometric factors at every volume and
// sub-face Gauss point, per sub-face its rule size, both sides' 1D basis values
// and derivatives at the rule's points and its penalty, for BR2 the blocks of
// every element's mass inverse on its sides' nodes - and holds the host mirror
// of that kernel (element rows, their diagonal) and the LOR blocks on mapped
// cells (Section 3.4).  The map is evaluated here, inside dg_mesh_create, and
// nowhere else: what later calls need of it (the LOR cells' vertices, the load
// vector's points) is stored.
//
// The SIPG form is the one of boxes, evaluated at Gauss points:
//   volume  int a grad u . grad v = int a (grad_xi u)^T G (grad_xi v) dxi,
//           G = det(J) J^-1 J^-T of the domain map at the point (the box's own
//           scaling cancels in 2D), p+2 points per direction;
//   faces   on every sub-face, max(p-, p+)+2 points, arc length |J t| dt,
//           physical normal n = J^-T nu / |J^-T nu| (nu the pre-image normal),
//           grad u . n = grad_X u . (J^-1 n) with grad_X u from the side's trace
//           values (tangential) and its normal-derivative line (normal),
//           sigma = a_e eta p_e^2 / min(h-, h+) with h_kappa = sqrt(|kappa|);
//   BR2     the lifting of a sub-face's jump on each side with that element's
//           own mass matrix (the p+2 rule; not a Kronecker product on a mapped
//           element), of which only the block on the side's nodes is needed.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "dg_internal.h"
#include "host_state.h"

namespace dg {

namespace {

int append_rule(std::vector<double>& t, int q, std::map<int, int>& cache) {
  auto it = cache.find(q);
  if (it != cache.end()) return it->second;
  std::vector<double> x, w;
  gauss_rule(q, x, w);
  const int off = (int)t.size();
  t.insert(t.end(), x.begin(), x.end());
  t.insert(t.end(), w.begin(), w.end());
  cache.emplace(q, off);
  return off;
}

// degree-p values and derivatives at the points s_g = (num + len x_g) / den of
// the q-point Gauss rule: q rows of p+1 values, then q rows of derivatives
int append_side_table(std::vector<double>& t, int p, int q, int num, int len, int den,
                      std::map<std::tuple<int, int, int, int, int>, int>& cache) {
  const int g = std::gcd(std::gcd(num, len), den);
  const auto key = std::make_tuple(p, q, num / g, len / g, den / g);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::vector<double> x, w;
  gauss_rule(q, x, w);
  const int n = p + 1;
  const int off = (int)t.size();
  t.resize(off + 2 * (size_t)q * n);
  const auto& nodes = basis1d(p).nodes;
  for (int r = 0; r < q; ++r) {
    const double s = ((double)num + (double)len * x[r]) / (double)den;
    lagrange_eval(nodes, s, &t[off + (size_t)r * n]);
    lagrange_deriv_eval(nodes, s, &t[off + (size_t)(q + r) * n]);
  }
  cache.emplace(key, off);
  return off;
}

// The map at a batch of pre-image points: the caller's map, or the bilinear
// map of the corners in closed form.  x: 2 per point, J: 4 per point.
struct MapEval {
  const dg_mesh_desc* desc;
  const DomainMap* D;
  const double* c;
  double Lx, Ly;
  void operator()(int64_t n, const double* X, double* x, double* J) const {
    if (desc->map) {
      std::fill(x, x + 2 * n, std::nan(""));
      std::fill(J, J + 4 * n, std::nan(""));
      desc->map(n, X, x, J, desc->map_ctx);
      for (int64_t i = 0; i < 2 * n; ++i) DG_REQUIRE(std::isfinite(x[i]), "the map returned a non-finite point");
      for (int64_t i = 0; i < 4 * n; ++i) DG_REQUIRE(std::isfinite(J[i]), "the map returned a non-finite Jacobian");
    } else {
      for (int64_t i = 0; i < n; ++i) {
        const double s = X[2 * i] / Lx, t = X[2 * i + 1] / Ly;
        const double w[4] = {(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t};
        x[2 * i] = x[2 * i + 1] = 0.0;
        for (int a = 0; a < 4; ++a) {
          x[2 * i] += w[a] * c[2 * a];
          x[2 * i + 1] += w[a] * c[2 * a + 1];
        }
        const Jac2 j = domain_jacobian(*D, X[2 * i], X[2 * i + 1]);
        J[4 * i] = j.j0;
        J[4 * i + 1] = j.j1;
        J[4 * i + 2] = j.j2;
        J[4 * i + 3] = j.j3;
      }
    }
    for (int64_t i = 0; i < n; ++i)
      DG_REQUIRE(J[4 * i] * J[4 * i + 3] - J[4 * i + 1] * J[4 * i + 2] > 0.0,
                 "the map is not orientation preserving at a quadrature point");
  }
};

}  // namespace

void build_mesh_map(dg_mesh* M, const dg_mesh_desc* desc) {
  HostMesh& m = M->host;
  const double Lx = m.extent[0] * m.lh, Ly = m.extent[1] * m.lh;
  const double* c = m.corners;
  DomainMap& D = M->dmap;
  D = DomainMap{};
  if (!desc->map) {
    D.u1x = (c[2] - c[0]) / Lx;
    D.u1y = (c[3] - c[1]) / Lx;
    D.u2x = (c[4] - c[0]) / Ly;
    D.u2y = (c[5] - c[1]) / Ly;
    D.u3x = (c[6] - c[4] - c[2] + c[0]) / (Lx * Ly);
    D.u3y = (c[7] - c[5] - c[3] + c[1]) / (Lx * Ly);
    // det J is linear in (X, Y): positive everywhere iff at the four corners
    const double XY[4][2] = {{0.0, 0.0}, {Lx, 0.0}, {0.0, Ly}, {Lx, Ly}};
    for (const auto& p : XY) {
      const Jac2 J = domain_jacobian(D, p[0], p[1]);
      DG_REQUIRE(J.j0 * J.j3 - J.j1 * J.j2 > 0.0,
                 "corners do not bound a convex, counter-clockwise quadrilateral");
    }
  }
  const MapEval map{desc, &D, c, Lx, Ly};
  // tables, appended after the box tables
  std::vector<double>& T = M->h_tables;
  std::map<int, int> rules;
  std::map<std::tuple<int, int, int, int, int>, int> sides;
  for (int p = 1; p <= kMaxP; ++p) {
    const int q = p + 1 + kMapQExtra, n = p + 1;
    const int r = append_rule(T, q, rules);
    M->moff[p].gx = r;
    M->moff[p].gw = r + q;
    std::vector<double> x(T.begin() + r, T.begin() + r + q);
    const auto& nodes = basis1d(p).nodes;
    M->moff[p].B = (int)T.size();
    T.resize(T.size() + 2 * (size_t)q * n);
    M->moff[p].D = M->moff[p].B + q * n;
    for (int g = 0; g < q; ++g) {
      lagrange_eval(nodes, x[g], &T[M->moff[p].B + (size_t)g * n]);
      lagrange_deriv_eval(nodes, x[g], &T[M->moff[p].D + (size_t)g * n]);
    }
  }
  M->moff[0] = M->moff[1];
  // volume factors a w_g w_h G = a w_g w_h det(J) J^-1 J^-T at every Gauss
  // point (the box's own scaling cancels in 2D), three planes per element;
  // the element's area by the same rule gives its penalty size sqrt(|kappa|)
  M->h_goff.assign(m.n + 1, 0);
  for (int64_t k = 0; k < m.n; ++k) {
    const int64_t q = m.p[k] + 1 + kMapQExtra;
    M->h_goff[k + 1] = M->h_goff[k] + 3 * q * q;
  }
  M->h_gvol.assign(M->h_goff[m.n], 0.0);
  const bool br2 = M->opts.form == DG_FORM_BR2;
  M->h_gbr2.clear();
  M->h_g2off.assign(br2 ? m.n + 1 : 0, 0);
  std::vector<double> hpen(m.n), X, x, J, Mk;
  for (int64_t k = 0; k < m.n; ++k) {
    const int P = m.p[k], Q = P + 1 + kMapQExtra, QQ = Q * Q;
    const double* gx = T.data() + M->moff[P].gx;
    const double* gw = T.data() + M->moff[P].gw;
    const double X0 = m.lo[2 * k] * m.lh, Y0 = m.lo[2 * k + 1] * m.lh, h = m.size[k] * m.lh;
    X.resize(2 * QQ);
    x.resize(2 * QQ);
    J.resize(4 * QQ);
    for (int gy = 0; gy < Q; ++gy)
      for (int gxi = 0; gxi < Q; ++gxi) {
        X[2 * (gy * Q + gxi)] = X0 + h * gx[gxi];
        X[2 * (gy * Q + gxi) + 1] = Y0 + h * gx[gy];
      }
    map(QQ, X.data(), x.data(), J.data());
    double* G = M->h_gvol.data() + M->h_goff[k];
    double area = 0.0;
    for (int gy = 0; gy < Q; ++gy)
      for (int gxi = 0; gxi < Q; ++gxi) {
        const int pt = gy * Q + gxi;
        const double* j = &J[4 * pt];
        const double det = j[0] * j[3] - j[1] * j[2];
        const double w = m.coef[k] * gw[gxi] * gw[gy] / det;
        G[pt] = w * (j[1] * j[1] + j[3] * j[3]);
        G[QQ + pt] = -w * (j[0] * j[1] + j[2] * j[3]);
        G[2 * QQ + pt] = w * (j[0] * j[0] + j[2] * j[2]);
        area += gw[gxi] * gw[gy] * det * h * h;
      }
    hpen[k] = std::sqrt(area);
    if (br2) {
      // the element's mass matrix by the same rule, its inverse, and the
      // inverse's block on each side's nodes (the BR2 lifting, Section 4.4)
      const int NP = P + 1, NN = NP * NP;
      const double* Bq = T.data() + M->moff[P].B;
      Mk.assign((size_t)NN * NN, 0.0);
      for (int gy = 0; gy < Q; ++gy)
        for (int gxi = 0; gxi < Q; ++gxi) {
          const double* j = &J[4 * (gy * Q + gxi)];
          const double W = gw[gxi] * gw[gy] * (j[0] * j[3] - j[1] * j[2]) * h * h;
          for (int a = 0; a < NN; ++a) {
            const double va = W * Bq[gxi * NP + a % NP] * Bq[gy * NP + a / NP];
            for (int b = 0; b < NN; ++b) Mk[(size_t)a * NN + b] += va * Bq[gxi * NP + b % NP] * Bq[gy * NP + b / NP];
          }
        }
      dense_inverse_spd(NN, Mk);
      for (int sd = 0; sd < 4; ++sd) {
        auto node = [&](int i) {
          const int e = (sd & 1) ? P : 0;
          return sd < 2 ? i * NP + e : e * NP + i;
        };
        for (int i = 0; i < NP; ++i)
          for (int i2 = 0; i2 < NP; ++i2) M->h_gbr2.push_back(Mk[(size_t)node(i) * NN + node(i2)]);
      }
      M->h_g2off[k + 1] = (int64_t)M->h_gbr2.size();
    }
  }
  M->h_sfm.assign(m.sf.size(), SubFaceMap{});
  M->h_gface.clear();
  const dg_options& o = M->opts;
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 4; ++s) {
      int axis, cc, t0, t1;
      m.side_segment((int)k, s, axis, cc, t0, t1);
      const int P = m.p[k];
      const double so = (s & 1) ? 1.0 : -1.0;   // outward along the normal axis
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        const auto& f = m.sf[j];
        SubFaceMap& r = M->h_sfm[j];
        const int len = f.t1 - f.t0;
        int pe = P;
        double he = hpen[k], ae = m.coef[k];
        if (f.nb >= 0) {
          pe = std::max(P, m.p[f.nb]);
          he = std::min(he, hpen[f.nb]);
          ae = std::max(ae, m.coef[f.nb]);
        }
        const int qf = pe + 1 + kMapQExtra;
        r.qf = qf;
        r.tab_bo = append_side_table(T, P, qf, f.t0 - t0, len, m.size[k], sides);
        if (f.nb >= 0) {
          int na, nc, n0, n1;
          m.side_segment(f.nb, f.nb_side, na, nc, n0, n1);
          r.tab_bn = append_side_table(T, m.p[f.nb], qf, f.t0 - n0, len, m.size[f.nb], sides);
        } else {
          r.tab_bn = r.tab_bo;
        }
        const double pp = (o.penalty_form == DG_PENALTY_P1SQ) ? (pe + 1.0) : (double)pe;
        r.sigma = ae * (M->eta * pp * pp / he);
        r.cbr2 = br2 ? ae * M->eta * (f.nb >= 0 ? 0.25 : 1.0) : 0.0;
        // face factors at the rule's points: arc length |J t| dt, the physical
        // normal n = J^-T nu / |J^-T nu| (nu = so e_n), m = J^-1 n
        const int rg = append_rule(T, qf, rules);
        DG_REQUIRE(M->h_gface.size() + 3 * (size_t)qf < (1ULL << 31), "face geometry too large");
        r.geo = (int32_t)M->h_gface.size();
        M->h_gface.resize(M->h_gface.size() + 3 * (size_t)qf);
        double* G = M->h_gface.data() + r.geo;
        const double xc = cc * m.lh, xt0 = f.t0 * m.lh, xt1 = f.t1 * m.lh;
        X.resize(2 * qf);
        x.resize(2 * qf);
        J.resize(4 * qf);
        for (int g = 0; g < qf; ++g) {
          const double Xt = xt0 + (xt1 - xt0) * T[rg + g];
          X[2 * g] = s < 2 ? xc : Xt;
          X[2 * g + 1] = s < 2 ? Xt : xc;
        }
        map(qf, X.data(), x.data(), J.data());
        for (int g = 0; g < qf; ++g) {
          const double* jj = &J[4 * g];
          const double tx = s < 2 ? jj[1] : jj[0], ty = s < 2 ? jj[3] : jj[2];
          const double det = jj[0] * jj[3] - jj[1] * jj[2];
          double nx, ny;
          if (s < 2) { nx = so * jj[3]; ny = -so * jj[1]; }
          else { nx = -so * jj[2]; ny = so * jj[0]; }
          const double nl = std::sqrt(nx * nx + ny * ny);
          nx /= nl;
          ny /= nl;
          const double mX = (jj[3] * nx - jj[1] * ny) / det, mY = (jj[0] * ny - jj[2] * nx) / det;
          const double mn = s < 2 ? mX : mY, mt = s < 2 ? mY : mX;
          const double W = T[rg + qf + g] * (xt1 - xt0) * std::sqrt(tx * tx + ty * ty);
          G[g] = W;
          G[qf + g] = W * mt;
          G[2 * qf + g] = W * mn * so;
        }
      }
    }
  DG_REQUIRE(T.size() < (1ULL << 31), "face tables too large");
  // images of the Gauss-Lobatto nodes (LOR cells) and of the load-vector
  // rule's points with det J, kept so that no later call needs the map
  M->h_xnode.clear();
  M->h_xrhs.clear();
  M->h_roff.assign(m.n + 1, 0);
  for (int64_t k = 0; k < m.n; ++k) {
    const int P = m.p[k], NP = P + 1, q = P + 3;
    const auto& gn = basis1d(P).nodes;
    std::vector<double> rx, rw;
    gauss_rule(q, rx, rw);
    const double X0 = m.lo[2 * k] * m.lh, Y0 = m.lo[2 * k + 1] * m.lh, h = m.size[k] * m.lh;
    X.resize(2 * NP * NP);
    x.resize(2 * NP * NP);
    J.resize(4 * NP * NP);
    for (int j = 0; j < NP; ++j)
      for (int i = 0; i < NP; ++i) {
        X[2 * (j * NP + i)] = X0 + h * gn[i];
        X[2 * (j * NP + i) + 1] = Y0 + h * gn[j];
      }
    map(NP * NP, X.data(), x.data(), J.data());
    M->h_xnode.insert(M->h_xnode.end(), x.begin(), x.end());
    X.resize(2 * q * q);
    x.resize(2 * q * q);
    J.resize(4 * q * q);
    for (int gy = 0; gy < q; ++gy)
      for (int gxi = 0; gxi < q; ++gxi) {
        X[2 * (gy * q + gxi)] = X0 + h * rx[gxi];
        X[2 * (gy * q + gxi) + 1] = Y0 + h * rx[gy];
      }
    map(q * q, X.data(), x.data(), J.data());
    for (int pt = 0; pt < q * q; ++pt) {
      M->h_xrhs.push_back(x[2 * pt]);
      M->h_xrhs.push_back(x[2 * pt + 1]);
      M->h_xrhs.push_back(J[4 * pt] * J[4 * pt + 3] - J[4 * pt + 1] * J[4 * pt + 2]);
    }
    M->h_roff[k + 1] = (int64_t)M->h_xrhs.size();
  }
  // boundary sub-faces at the p+3 Gauss points of the element's degree: the
  // image, the weight with the arc length and m = J^-1 n, n the outward
  // physical normal (the boundary terms of weak Dirichlet data)
  M->h_xbnd.clear();
  M->h_boff.assign(m.sf.size(), -1);
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 4; ++s) {
      int axis, cc, t0, t1;
      m.side_segment((int)k, s, axis, cc, t0, t1);
      const double so = (s & 1) ? 1.0 : -1.0;
      const int q = m.p[k] + 3;
      std::vector<double> rx, rw;
      gauss_rule(q, rx, rw);
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        const auto& f = m.sf[j];
        if (f.nb >= 0) continue;
        const double xc = cc * m.lh, xt0 = f.t0 * m.lh, xt1 = f.t1 * m.lh;
        X.resize(2 * q);
        x.resize(2 * q);
        J.resize(4 * q);
        for (int g = 0; g < q; ++g) {
          const double Xt = xt0 + (xt1 - xt0) * rx[g];
          X[2 * g] = s < 2 ? xc : Xt;
          X[2 * g + 1] = s < 2 ? Xt : xc;
        }
        map(q, X.data(), x.data(), J.data());
        M->h_boff[j] = (int64_t)M->h_xbnd.size();
        for (int g = 0; g < q; ++g) {
          const double* jj = &J[4 * g];
          const double tx = s < 2 ? jj[1] : jj[0], ty = s < 2 ? jj[3] : jj[2];
          const double det = jj[0] * jj[3] - jj[1] * jj[2];
          double nx, ny;
          if (s < 2) { nx = so * jj[3]; ny = -so * jj[1]; }
          else { nx = -so * jj[2]; ny = so * jj[0]; }
          const double nl = std::sqrt(nx * nx + ny * ny);
          nx /= nl;
          ny /= nl;
          M->h_xbnd.push_back(x[2 * g]);
          M->h_xbnd.push_back(x[2 * g + 1]);
          M->h_xbnd.push_back(rw[g] * (xt1 - xt0) * std::sqrt(tx * tx + ty * ty));
          M->h_xbnd.push_back((jj[3] * nx - jj[1] * ny) / det);
          M->h_xbnd.push_back((jj[0] * ny - jj[2] * nx) / det);
        }
      }
    }
}

void map_stats(dg_mesh* M) {
  // operation and byte counts of one mapped operator apply, as the kernel does it
  const HostMesh& m = M->host;
  dg_mesh_stats& S = M->stats;
  double fl = 0.0;
  for (int64_t k = 0; k < m.n; ++k) {
    const double n1 = m.p[k] + 1.0, q = m.p[k] + 1.0 + kMapQExtra;
    // volume: two products per pass (x, then y), four passes, the point step
    // (two 2-term sums); the side traces' normal derivatives (trace kernel)
    // and the gather's normal-derivative terms
    fl += 2.0 * (2.0 * n1 * n1 * q + 2.0 * q * q * n1 + 2.0 * n1 * q * q + 2.0 * n1 * n1 * q) + 8.0 * q * q;
    fl += 2.0 * 4.0 * n1 * n1 + 2.0 * 4.0 * n1 * n1;
    for (int j = m.sf_ptr[4 * k]; j < m.sf_ptr[4 * k + 4]; ++j) {
      const auto& f = m.sf[j];
      const double qf = M->h_sfm[j].qf;
      const double nn = f.nb >= 0 ? m.p[f.nb] + 1.0 : 0.0;
      // per point: three own and three neighbour sums and the weights; per
      // side node and point: three sums
      fl += qf * (2.0 * 3.0 * (n1 + nn) + 16.0) + 2.0 * 3.0 * n1 * qf;
      // BR2: both sides' projections, side-block products and values at the points
      if (M->opts.form == DG_FORM_BR2) fl += 2.0 * (2.0 * qf * (n1 + nn) + n1 * n1 + nn * nn) + 4.0 * qf;
    }
  }
  S.apply_flops = fl;
  S.apply_bytes += 8.0 * (double)(M->h_gvol.size() + M->h_gface.size() + M->h_gbr2.size() + m.n) +
                   (double)m.sf.size() * sizeof(SubFaceMap);
}

// ---------------------------------------------------------------- host mirror
// The mapped kernel's formulation, written plainly, on the same stored
// geometric factors (so the CPU tests against the oracle check those too).
void host_element_residual_map(const dg_mesh& M, int64_t k, const double* x, double* y) {
  const HostMesh& m = M.host;
  const double* T = M.h_tables.data();
  const int P = m.p[k], NP = P + 1, Q = P + 1 + kMapQExtra, QQ = Q * Q;
  const MapOff& mo = M.moff[P];
  const double* Bq = T + mo.B;   // Bq[g * NP + j] = l_j(x_g)
  const double* Dq = T + mo.D;
  const double* G = M.h_gvol.data() + M.h_goff[k];
  const double hX = m.size[k] * m.lh;
  const double ak = m.coef[k], aih = ak / hX;
  const double* xk = x + m.off[k];
  // ---- volume
  std::vector<double> A1(NP * Q), A2(NP * Q), F1(QQ), F2(QQ);
  for (int jy = 0; jy < NP; ++jy)
    for (int g = 0; g < Q; ++g) {
      double a = 0.0, b = 0.0;
      for (int jx = 0; jx < NP; ++jx) {
        a += Dq[g * NP + jx] * xk[jy * NP + jx];
        b += Bq[g * NP + jx] * xk[jy * NP + jx];
      }
      A1[jy * Q + g] = a;
      A2[jy * Q + g] = b;
    }
  for (int gyi = 0; gyi < Q; ++gyi)
    for (int gxi = 0; gxi < Q; ++gxi) {
      double ux = 0.0, uy = 0.0;
      for (int jy = 0; jy < NP; ++jy) {
        ux += Bq[gyi * NP + jy] * A1[jy * Q + gxi];
        uy += Dq[gyi * NP + jy] * A2[jy * Q + gxi];
      }
      const int pt = gyi * Q + gxi;
      F1[pt] = G[pt] * ux + G[QQ + pt] * uy;
      F2[pt] = G[QQ + pt] * ux + G[2 * QQ + pt] * uy;
    }
  std::vector<double> C1(NP * Q), C2(NP * Q);
  for (int iy = 0; iy < NP; ++iy)
    for (int g = 0; g < Q; ++g) {
      double a = 0.0, b = 0.0;
      for (int gy = 0; gy < Q; ++gy) {
        a += Bq[gy * NP + iy] * F1[gy * Q + g];
        b += Dq[gy * NP + iy] * F2[gy * Q + g];
      }
      C1[iy * Q + g] = a;
      C2[iy * Q + g] = b;
    }
  for (int iy = 0; iy < NP; ++iy)
    for (int ix = 0; ix < NP; ++ix) {
      double v = 0.0;
      for (int g = 0; g < Q; ++g) v += Dq[g * NP + ix] * C1[iy * Q + g] + Bq[g * NP + ix] * C2[iy * Q + g];
      y[iy * NP + ix] = v;
    }
  // ---- faces: side traces (value, a times the outward pre-image normal
  // derivative) as the trace kernel writes them
  auto sn = [](int s, int i, int q, int np) { return (s < 2) ? (i * np + q) : (q * np + i); };
  auto trace = [&](int64_t e, int s, double* u, double* dn) {
    const int p = m.p[e], np = p + 1;
    const Basis1D& B = basis1d(p);
    const double* xe = x + m.off[e];
    const double* dv = (s & 1) ? B.d1.data() : B.d0.data();
    const double sg = ((s & 1) ? 1.0 : -1.0) * m.coef[e] / (m.size[e] * m.lh);
    for (int i = 0; i < np; ++i) {
      u[i] = xe[sn(s, i, (s & 1) ? p : 0, np)];
      double acc = 0.0;
      for (int q = 0; q < np; ++q) acc += dv[q] * xe[sn(s, i, q, np)];
      dn[i] = sg * acc;
    }
  };
  double r[4 * kMaxN] = {0.0}, c2[4 * kMaxN] = {0.0};
  for (int s = 0; s < 4; ++s) {
    double uo[kMaxN], fo[kMaxN];
    trace(k, s, uo, fo);
    for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
      const SubFaceRec& f = M.h_sf[j];
      const SubFaceMap& g = M.h_sfm[j];
      const int qf = g.qf;
      const double* W = M.h_gface.data() + g.geo;
      double un[kMaxN], fn[kMaxN];
      int npn = 0;
      double ihn = 0.0, an = 0.0;
      if (f.nb >= 0) {
        trace(f.nb, f.nb_side, un, fn);
        npn = f.pn + 1;
        ihn = 1.0 / (m.size[f.nb] * m.lh);
        an = m.coef[f.nb];
      }
      const bool br2 = M.opts.form == DG_FORM_BR2;
      double rho1v[kMapQMax], wj[kMapQMax];
      for (int q = 0; q < qf; ++q) {
        const double* Bo = T + g.tab_bo + (size_t)q * NP;
        const double* Do = T + g.tab_bo + (size_t)(qf + q) * NP;
        double u0 = 0.0, du0 = 0.0, f0 = 0.0;
        for (int i = 0; i < NP; ++i) {
          u0 += Bo[i] * uo[i];
          du0 += Do[i] * uo[i];
          f0 += Bo[i] * fo[i];
        }
        du0 /= hX;
        const double w = W[q], wmt = W[qf + q], wmn = W[2 * qf + q];
        const double Fo = f0 * wmn + ak * du0 * wmt;   // w (a grad u-) . n
        double jmp, flux, cc;
        if (f.nb >= 0) {
          const double* Bn = T + g.tab_bn + (size_t)q * npn;
          const double* Dn = T + g.tab_bn + (size_t)(qf + q) * npn;
          double u1 = 0.0, du1 = 0.0, f1 = 0.0;
          for (int i = 0; i < npn; ++i) {
            u1 += Bn[i] * un[i];
            du1 += Dn[i] * un[i];
            f1 += Bn[i] * fn[i];
          }
          du1 *= ihn;
          const double Fn = -f1 * wmn + an * du1 * wmt;   // w (a grad u+) . n
          jmp = u0 - u1;
          flux = 0.5 * (Fo + Fn);
          cc = 0.5;
        } else {
          jmp = u0;
          flux = Fo;
          cc = 1.0;
        }
        const double rho2 = -cc * jmp * wmt;
        const double rho3 = -cc * jmp * wmn;
        rho1v[q] = br2 ? -flux : g.sigma * jmp * w - flux;
        wj[q] = w * jmp;
        for (int i = 0; i < NP; ++i) {
          r[s * NP + i] += aih * Do[i] * rho2;
          c2[s * NP + i] += Bo[i] * rho3;
        }
      }
      if (br2) {
        // liftings on both sides: j = int phi_j [[u]] ds on each side's nodes,
        // z = (mass-inverse side block) j, and at every point the weight
        // eta coef a w (z-(x_g) + z+(x_g)) of the own test function's value
        double jo[kMaxN] = {0.0}, jn[kMaxN] = {0.0}, zo[kMaxN] = {0.0}, zn[kMaxN] = {0.0};
        for (int q = 0; q < qf; ++q)
          for (int i = 0; i < NP; ++i) jo[i] += T[g.tab_bo + (size_t)q * NP + i] * wj[q];
        const double* Go = M.h_gbr2.data() + M.h_g2off[k] + (size_t)s * NP * NP;
        for (int i = 0; i < NP; ++i)
          for (int i2 = 0; i2 < NP; ++i2) zo[i] += Go[i * NP + i2] * jo[i2];
        if (f.nb >= 0) {
          for (int q = 0; q < qf; ++q)
            for (int i = 0; i < npn; ++i) jn[i] += T[g.tab_bn + (size_t)q * npn + i] * wj[q];
          const double* Gn = M.h_gbr2.data() + M.h_g2off[f.nb] + (size_t)f.nb_side * npn * npn;
          for (int i = 0; i < npn; ++i)
            for (int i2 = 0; i2 < npn; ++i2) zn[i] += Gn[i * npn + i2] * jn[i2];
        }
        for (int q = 0; q < qf; ++q) {
          double v = 0.0;
          for (int i = 0; i < NP; ++i) v += T[g.tab_bo + (size_t)q * NP + i] * zo[i];
          for (int i = 0; i < npn; ++i) v += T[g.tab_bn + (size_t)q * npn + i] * zn[i];
          rho1v[q] += g.cbr2 * W[q] * v;
        }
      }
      for (int q = 0; q < qf; ++q)
        for (int i = 0; i < NP; ++i) r[s * NP + i] += T[g.tab_bo + (size_t)q * NP + i] * rho1v[q];
    }
  }
  const Basis1D& B = basis1d(P);
  for (int node = 0; node < NP * NP; ++node) {
    const int ix = node % NP, iy = node / NP;
    double v = y[node];
    double gg = -B.d0[ix] * c2[0 * NP + iy];
    gg += B.d1[ix] * c2[1 * NP + iy];
    gg += -B.d0[iy] * c2[2 * NP + ix];
    gg += B.d1[iy] * c2[3 * NP + ix];
    v += gg * aih;
    if (ix == 0) v += r[0 * NP + iy];
    if (ix == P) v += r[1 * NP + iy];
    if (iy == 0) v += r[2 * NP + ix];
    if (iy == P) v += r[3 * NP + ix];
    y[node] = v;
  }
}

void host_element_diag_map(const dg_mesh& M, int64_t k, double* d) {
  // column by column: the element's own rows of A e_i
  const HostMesh& m = M.host;
  thread_local std::vector<double> x;
  if ((int64_t)x.size() < M.n_dofs) x.assign(M.n_dofs, 0.0);
  const int NN = (m.p[k] + 1) * (m.p[k] + 1);
  std::vector<double> y(NN);
  for (int i = 0; i < NN; ++i) {
    x[m.off[k] + i] = 1.0;
    host_element_residual_map(M, k, x.data(), y.data());
    x[m.off[k] + i] = 0.0;
    d[i] = y[i];
  }
}

void host_lor_block_map(const dg_mesh& M, int64_t k, double* A) {
  // Q1 stiffness on the images of the Gauss-Lobatto cells, 2 x 2 Gauss
  const HostMesh& m = M.host;
  const int P = m.p[k], NP = P + 1, NN = NP * NP;
  // the element's node images: h_xnode holds 2 (p+1)^2 values per element,
  // element by element like the DOFs
  const double* xn = M.h_xnode.data() + 2 * m.off[k];
  std::vector<double> gx, gw;
  gauss_rule(2, gx, gw);
  std::fill(A, A + (size_t)NN * NN, 0.0);
  for (int cj = 0; cj < P; ++cj)
    for (int ci = 0; ci < P; ++ci) {
      double V[4][2];
      const int idx[4] = {cj * NP + ci, cj * NP + ci + 1, (cj + 1) * NP + ci, (cj + 1) * NP + ci + 1};
      for (int a = 0; a < 4; ++a) {
        V[a][0] = xn[2 * idx[a]];
        V[a][1] = xn[2 * idx[a] + 1];
      }
      double K[4][4] = {{0.0}};
      for (int qy = 0; qy < 2; ++qy)
        for (int qx = 0; qx < 2; ++qx) {
          const double s = gx[qx], t = gx[qy];
          const double ds[4] = {-(1 - t), 1 - t, -t, t};
          const double dt[4] = {-(1 - s), -s, 1 - s, s};
          double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
          for (int a = 0; a < 4; ++a) {
            j00 += ds[a] * V[a][0];
            j01 += dt[a] * V[a][0];
            j10 += ds[a] * V[a][1];
            j11 += dt[a] * V[a][1];
          }
          const double det = j00 * j11 - j01 * j10;
          double gxv[4], gyv[4];
          for (int a = 0; a < 4; ++a) {   // J^-T (ds, dt)
            gxv[a] = (j11 * ds[a] - j10 * dt[a]) / det;
            gyv[a] = (-j01 * ds[a] + j00 * dt[a]) / det;
          }
          const double w = gw[qx] * gw[qy] * det;
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) K[a][b] += w * (gxv[a] * gxv[b] + gyv[a] * gyv[b]);
        }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) A[(size_t)idx[a] * NN + idx[b]] += K[a][b];
    }
}

}  // namespace dg
