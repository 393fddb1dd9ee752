// Mesh topology on the host: sub-faces, hanging vertices, master edges
// (Section 2 mesh and skeleton; Section 3.2 hanging / regular / hp-vertices).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "dg_internal.h"
#include "host_state.h"

namespace dg {

void HostMesh::side_segment(int k, int s, int& axis, int& c, int& t0, int& t1) const {
  const int x0 = lo[2 * k], y0 = lo[2 * k + 1], h = size[k];
  switch (s) {
    case 0: axis = 0; c = x0; t0 = y0; t1 = y0 + h; break;
    case 1: axis = 0; c = x0 + h; t0 = y0; t1 = y0 + h; break;
    case 2: axis = 1; c = y0; t0 = x0; t1 = x0 + h; break;
    default: axis = 1; c = y0 + h; t0 = x0; t1 = x0 + h; break;
  }
}

bool HostMesh::corner_of(int k, int x, int y) const {
  const int x0 = lo[2 * k], y0 = lo[2 * k + 1], h = size[k];
  return (x == x0 || x == x0 + h) && (y == y0 || y == y0 + h);
}

int HostMesh::containing_side(int x, int y, int* side) const {
  for (int dy = -1; dy <= 0; ++dy)
    for (int dx = -1; dx <= 0; ++dx) {
      int cx = x + dx, cy = y + dy;
      if (cx < 0 || cy < 0 || cx >= extent[0] || cy >= extent[1]) continue;
      int e = elem_at(cx, cy);
      if (e < 0 || corner_of(e, x, y)) continue;   // a hole, or a corner of e
      const int x0 = lo[2 * e], y0 = lo[2 * e + 1], h = size[e];
      int s;
      if (x == x0) s = 0;
      else if (x == x0 + h) s = 1;
      else if (y == y0) s = 2;
      else if (y == y0 + h) s = 3;
      else continue;  // (x, y) inside e: not a vertex position
      if (side) *side = s;
      return e;
    }
  return -1;
}

bool HostMesh::is_hp_vertex(int x, int y) const {
  if (containing_side(x, y, nullptr) < 0) return false;
  int pv = -1;
  for (int dy = -1; dy <= 0; ++dy)
    for (int dx = -1; dx <= 0; ++dx) {
      int cx = x + dx, cy = y + dy;
      if (cx < 0 || cy < 0 || cx >= extent[0] || cy >= extent[1]) continue;
      int e = elem_at(cx, cy);
      if (e < 0) continue;   // a hole
      if (pv < 0) pv = p[e];
      else if (p[e] != pv) return true;
    }
  return false;
}

void build_topology(HostMesh& m) {
  const int64_t n = m.n;
  // ---- sub-faces seen from every element side
  m.sf_ptr.assign(4 * n + 1, 0);
  m.sf.clear();
  for (int64_t k = 0; k < n; ++k) {
    for (int s = 0; s < 4; ++s) {
      int axis, c, t0, t1;
      m.side_segment((int)k, s, axis, c, t0, t1);
      const bool outward_plus = (s == 1 || s == 3);
      const bool bdry = outward_plus ? (c == m.extent[axis]) : (c == 0);
      if (bdry) {
        m.sf.push_back({-1, -1, t0, t1});
      } else {
        // the cells across the side: elements (one sub-face each) or holes of
        // the domain (the side is then boundary; a side must not border a hole
        // in part only)
        int t = t0, holes = 0, elems = 0;
        while (t < t1) {
          int cx, cy;
          if (axis == 0) { cx = outward_plus ? c : c - 1; cy = t; }
          else { cx = t; cy = outward_plus ? c : c - 1; }
          int nb = m.elem_at(cx, cy);
          if (nb < 0) {
            ++holes;
            ++t;
            continue;
          }
          int u0 = m.lo[2 * nb + (1 - axis)];
          int u1 = u0 + m.size[nb];
          int e1 = std::min(t1, u1);
          m.sf.push_back({nb, s ^ 1, t, e1});
          ++elems;
          t = e1;
        }
        DG_REQUIRE(holes == 0 || elems == 0, "an element side borders a hole in part only");
        if (holes) m.sf.push_back({-1, -1, t0, t1});
      }
      m.sf_ptr[4 * k + s + 1] = (int32_t)m.sf.size();
    }
  }
  // ---- master edges
  m.side_master.assign(4 * n, -1);
  m.masters.clear();
  auto is_slave = [&](int64_t k, int s) {
    const auto& f = m.sf[m.sf_ptr[4 * k + s]];
    return f.nb >= 0 && m.size[f.nb] > m.size[k];
  };
  for (int64_t k = 0; k < n; ++k)
    for (int s = 0; s < 4; ++s) {
      if (is_slave(k, s) || m.side_master[4 * k + s] >= 0) continue;
      HostMesh::Master M;
      m.side_segment((int)k, s, M.axis, M.c, M.t0, M.t1);
      M.boundary = m.sf[m.sf_ptr[4 * k + s]].nb < 0;
      M.owners.push_back((int32_t)k);
      const int id = (int)m.masters.size();
      m.side_master[4 * k + s] = id;
      const int b = m.sf_ptr[4 * k + s], e = m.sf_ptr[4 * k + s + 1];
      if (!M.boundary && e - b == 1 && m.size[m.sf[b].nb] == m.size[k]) {
        M.owners.push_back(m.sf[b].nb);
        m.side_master[4 * m.sf[b].nb + (s ^ 1)] = id;
      } else if (!M.boundary) {
        for (int j = b; j < e; ++j) {
          M.slaves.push_back(m.sf[j].nb);
          if (j > b) {
            int t = m.sf[j].t0;
            M.hanging.push_back(M.axis == 0 ? std::make_pair(M.c, t) : std::make_pair(t, M.c));
          }
        }
      }
      m.masters.push_back(M);
    }
  for (int64_t k = 0; k < n; ++k)
    for (int s = 0; s < 4; ++s)
      if (m.side_master[4 * k + s] < 0) {
        const auto& f = m.sf[m.sf_ptr[4 * k + s]];
        m.side_master[4 * k + s] = m.side_master[4 * f.nb + (s ^ 1)];
      }
  for (auto& M : m.masters) {
    int pm = 1 << 30;
    for (int k : M.owners) pm = std::min(pm, m.p[k]);
    for (int k : M.slaves) pm = std::min(pm, m.p[k]);
    M.p = pm;
  }
}

int FaceTables::get(int p, int L, int off, int pn, int Ln, int offn) {
  auto key = std::make_tuple(p, L, off, pn, Ln, offn);
  auto it = index.find(key);
  if (it != index.end()) return it->second;
  const Basis1D& a = basis1d(p);
  const Basis1D& b = basis1d(pn);
  std::vector<double> gx, gw;
  gauss_rule(std::max(p, pn) + 1, gx, gw);
  const int o = (int)data.size();
  data.resize(o + (p + 1) * (pn + 1), 0.0);
  double la[kMaxN], lb[kMaxN];
  const double sa = std::ldexp(1.0, -L), sb = std::ldexp(1.0, -Ln);
  for (size_t g = 0; g < gx.size(); ++g) {
    lagrange_eval(a.nodes, (off + gx[g]) * sa, la);
    lagrange_eval(b.nodes, (offn + gx[g]) * sb, lb);
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= pn; ++j) data[o + i * (pn + 1) + j] += gw[g] * la[i] * lb[j];
  }
  index[key] = o;
  return o;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static void validate_and_copy(const dg_mesh_desc* d, HostMesh& m) {
  DG_REQUIRE(d != nullptr, "null mesh description");
  DG_REQUIRE(d->dim == 2, "dim must be 2 or 3");
  DG_REQUIRE(d->n_elems > 0 && d->n_elems < (1LL << 30), "n_elems out of range");
  DG_REQUIRE(d->lo && d->size && d->p && d->extent, "null array in mesh description");
  DG_REQUIRE(d->lattice_h > 0.0 && std::isfinite(d->lattice_h), "lattice_h must be positive");
  m.dim = 2;
  m.n = d->n_elems;
  m.extent[0] = d->extent[0];
  m.extent[1] = d->extent[1];
  DG_REQUIRE(m.extent[0] > 0 && m.extent[1] > 0, "extent must be positive");
  DG_REQUIRE((int64_t)m.extent[0] * m.extent[1] <= (1LL << 28), "lattice too large");
  m.lh = d->lattice_h;
  copy_coeff(d, m.coef);
  m.lo.assign(d->lo, d->lo + 2 * m.n);
  m.size.assign(d->size, d->size + m.n);
  m.p.assign(d->p, d->p + m.n);
  m.cellmap.assign((int64_t)m.extent[0] * m.extent[1], -1);
  m.off.assign(m.n + 1, 0);
  for (int64_t k = 0; k < m.n; ++k) {
    const int x0 = m.lo[2 * k], y0 = m.lo[2 * k + 1], h = m.size[k];
    DG_REQUIRE(m.p[k] >= 1 && m.p[k] <= kMaxP, "degree out of range 1..8");
    DG_REQUIRE(pow2(h), "element size must be a power of two");
    DG_REQUIRE(x0 >= 0 && y0 >= 0 && x0 % h == 0 && y0 % h == 0, "element corner not aligned to its size");
    DG_REQUIRE(x0 + h <= m.extent[0] && y0 + h <= m.extent[1], "element outside the domain");
    for (int y = y0; y < y0 + h; ++y)
      for (int x = x0; x < x0 + h; ++x) {
        int32_t& c = m.cellmap[(int64_t)y * m.extent[0] + x];
        DG_REQUIRE(c < 0, "elements overlap");
        c = (int32_t)k;
      }
    m.off[k + 1] = m.off[k] + (int64_t)(m.p[k] + 1) * (m.p[k] + 1);
  }
  // cells no element covers are holes of the domain (their edges are boundary)
  int64_t covered = 0;
  for (int32_t c : m.cellmap) covered += c >= 0;
  DG_REQUIRE(covered > 0, "no element");
}

static void append(std::vector<double>& t, const std::vector<double>& v, int& off) {
  off = (int)t.size();
  t.insert(t.end(), v.begin(), v.end());
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

void build_tiles(dg_mesh* M) {
  // tiles of the operator kernel: degree-descending element order, runs of
  // at most tile_epb[p] elements of one degree (apply_epb(p) unless tuned)
  const HostMesh& m = M->host;
  std::vector<int32_t> order(m.n);
  for (int64_t k = 0; k < m.n; ++k) order[k] = (int32_t)k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return m.p[a] > m.p[b]; });
  M->h_tiles.clear();
  for (int64_t i = 0; i < m.n;) {
    const int P = m.p[order[i]];
    int64_t j = i;
    while (j < m.n && m.p[order[j]] == P && j - i < M->tile_epb[P]) ++j;
    M->h_tiles.push_back({P, (int32_t)i, (int32_t)(j - i), 0});
    i = j;
  }
  M->n_tiles = (int)M->h_tiles.size();
  M->h_order = order;
  build_face_items(M);
}

void build_face_items(dg_mesh* M) {
  const HostMesh& m = M->host;
  M->h_items.clear();
  M->h_item_ptr.assign(1, 0);
  M->h_side_items.assign(8 * M->h_order.size(), 0);
  for (const ApplyTile& T : M->h_tiles) {
    for (int e = 0; e < T.count; ++e) {
      const int64_t pos = T.first + e;
      const int32_t k = M->h_order[pos];
      for (int s = 0; s < 4; ++s) {
        const int b = m.sf_ptr[4 * (int64_t)k + s], c = m.sf_ptr[4 * (int64_t)k + s + 1] - b;
        M->h_side_items[8 * pos + 2 * s] = (int32_t)(M->h_items.size() / 2);
        M->h_side_items[8 * pos + 2 * s + 1] = c;
        for (int j = 0; j < c; ++j) {
          M->h_items.push_back(b + j);
          M->h_items.push_back(4 * e + s);
        }
      }
    }
    // The tile's items in the order of the branches their threads take -
    // interior first, by neighbour degree (the loop bound), then the boundary
    // - so that a warp of the face pass spans fewer kinds of item.  The high
    // half of the side field keeps the item's position in sub-face order,
    // where the face pass writes its partials (the side sums read them there).
    const int64_t t0 = M->h_item_ptr.back(), t1 = (int64_t)M->h_items.size() / 2;
    DG_REQUIRE(t1 - t0 < 65536, "operator tile: too many sub-face items");
    std::vector<std::pair<int32_t, int32_t>> key;   // (branch key, position in the tile)
    for (int64_t g = t0; g < t1; ++g) {
      const SubFaceRec& f = M->h_sf[M->h_items[2 * g]];
      key.push_back({f.nb >= 0 ? 16 - f.pn : 32, (int32_t)(g - t0)});
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                       return a.first < b.first;
                     });
    const std::vector<int32_t> rec(M->h_items.begin() + 2 * t0, M->h_items.end());
    for (int64_t g = t0; g < t1; ++g) {
      const int32_t pos = key[g - t0].second;
      M->h_items[2 * g] = rec[2 * pos];
      M->h_items[2 * g + 1] = rec[2 * pos + 1] | (pos << 16);
    }
    M->h_item_ptr.push_back((int32_t)(M->h_items.size() / 2));
  }
}

void build_mesh_host(dg_mesh* M, const dg_mesh_desc* desc, const dg_options* opts) {
  HostMesh& m = M->host;
  dg_options o{};
  o.form = DG_FORM_SIPG;
  o.penalty_form = DG_PENALTY_PAPER;
  if (opts) o = *opts;
  DG_REQUIRE(o.form == DG_FORM_SIPG || o.form == DG_FORM_BR2, "unknown form");
  DG_REQUIRE(o.penalty_form == DG_PENALTY_PAPER || o.penalty_form == DG_PENALTY_P1SQ, "unknown penalty form");
  M->opts = o;
  DG_REQUIRE(desc != nullptr, "null mesh description");
  if (desc->dim == 3) {
    if (desc->corners || desc->map) throw Error(DG_EUNSUPPORTED, "mapped elements: square meshes only");
    build_mesh_host3(M, desc, o);
    return;
  }
  validate_and_copy(desc, m);
  if (desc->corners || desc->map) {
    DG_REQUIRE(!(desc->corners && desc->map), "give corners or a map, not both");
    if (desc->corners)
      for (int i = 0; i < 8; ++i) {
        DG_REQUIRE(std::isfinite(desc->corners[i]), "corners must be finite");
        m.corners[i] = desc->corners[i];
      }
    m.mapped = true;
  }
  build_topology(m);
  M->n_dofs = m.off[m.n];
  DG_REQUIRE(M->n_dofs < (1LL << 31), "too many unknowns for 32-bit indices");
  // element sizes
  M->h_h.resize(m.n);
  for (int64_t k = 0; k < m.n; ++k) M->h_h[k] = m.size[k] * m.lh;
  // penalty default
  if (o.eta > 0) {
    M->eta = o.eta;
  } else if (o.form == DG_FORM_BR2) {
    int mx = 0;
    for (int64_t k = 0; k < m.n; ++k) {
      int c = m.sf_ptr[4 * k + 4] - m.sf_ptr[4 * k];
      mx = std::max(mx, c);
    }
    M->eta = (double)mx;
  } else {
    M->eta = 100.0;
  }
  // tables: basis per degree, then face masses
  M->h_tables.clear();
  for (int p = 1; p <= kMaxP; ++p) {
    const Basis1D& b = basis1d(p);
    append(M->h_tables, b.M, M->boff[p].M);
    append(M->h_tables, b.K, M->boff[p].K);
    append(M->h_tables, b.Minv, M->boff[p].Minv);
    append(M->h_tables, b.d0, M->boff[p].d0);
    append(M->h_tables, b.d1, M->boff[p].d1);
  }
  M->boff[0] = M->boff[1];
  FaceTables ft;
  M->h_sf.resize(m.sf.size());
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 4; ++s) {
      int axis, c, t0, t1;
      m.side_segment((int)k, s, axis, c, t0, t1);
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        const auto& f = m.sf[j];
        SubFaceRec r{};
        const int len = f.t1 - f.t0;
        const int P = m.p[k];
        const int Lo = ilog2(m.size[k] / len), oo = (f.t0 - t0) / len;
        r.nb = f.nb;
        r.nb_side = f.nb_side;
        r.len = len * m.lh;
        r.tab_oo = ft.get(P, Lo, oo, P, Lo, oo);
        int pe = P;
        double he = M->h_h[k], ae = m.coef[k];
        if (f.nb >= 0) {
          const int pn = m.p[f.nb];
          int na, nc, n0, n1;
          m.side_segment(f.nb, f.nb_side, na, nc, n0, n1);
          const int Ln = ilog2(m.size[f.nb] / len), on = (f.t0 - n0) / len;
          r.pn = pn;
          r.tab_on = ft.get(P, Lo, oo, pn, Ln, on);
          r.tab_nn = ft.get(pn, Ln, on, pn, Ln, on);
          pe = std::max(P, pn);
          he = std::min(he, M->h_h[f.nb]);
          ae = std::max(ae, m.coef[f.nb]);
        } else {
          r.pn = P;
          r.tab_on = r.tab_oo;
          r.tab_nn = r.tab_oo;
        }
        const double pp = (o.penalty_form == DG_PENALTY_P1SQ) ? (pe + 1.0) : (double)pe;
        r.sigma = ae * (M->eta * pp * pp / he);   // the larger coefficient of the two sides
        M->h_sf[j] = r;
      }
    }
  // BR2: each sub-face's lifting multiplied out (SubFaceBr2), its product
  // tables appended after the face tables
  std::vector<double> prod;
  M->h_sfb.clear();
  if (o.form == DG_FORM_BR2) {
    std::map<std::tuple<int, int, int, int>, int> pindex;
    const int pbase = (int)ft.data.size();
    // kind 0: Z = M_oo Minv M_oo, 1: V = M_oo Minv M_on, 2: X = M_on Minv_n M_no,
    // 3: Y = M_on Minv_n M_nn (row-major, (p+1) rows)
    auto product = [&](int kind, int p, int pn, int oo, int on, int nn) {
      const auto key = std::make_tuple(kind, kind == 0 ? oo : on, kind == 3 ? nn : (kind == 1 ? oo : -1),
                                       p * 16 + pn);
      const auto it = pindex.find(key);
      if (it != pindex.end()) return it->second;
      const int a = p + 1, b = pn + 1;
      const double* Moo = ft.data.data() + oo;
      const double* Mon = ft.data.data() + on;
      const double* Mnn = ft.data.data() + nn;
      const std::vector<double>& Mi = basis1d(p).Minv;
      const std::vector<double>& Min = basis1d(pn).Minv;
      const int cols = (kind == 0 || kind == 2) ? a : b;
      const int off = (int)prod.size();
      prod.resize(off + (size_t)a * cols, 0.0);
      for (int i = 0; i < a; ++i)
        for (int j = 0; j < cols; ++j) {
          double v = 0.0;
          for (int u = 0; u < (kind < 2 ? a : b); ++u)
            for (int w = 0; w < (kind < 2 ? a : b); ++w) {
              if (kind == 0) v += Moo[i * a + u] * Mi[u * a + w] * Moo[w * a + j];
              else if (kind == 1) v += Moo[i * a + u] * Mi[u * a + w] * Mon[w * b + j];
              else if (kind == 2) v += Mon[i * b + u] * Min[u * b + w] * Mon[j * b + w];
              else v += Mon[i * b + u] * Min[u * b + w] * Mnn[w * b + j];
            }
          prod[off + (size_t)i * cols + j] = v;
        }
      pindex.emplace(key, pbase + off);
      return pbase + off;
    };
    M->h_sfb.assign(m.sf.size(), SubFaceBr2{});
    for (int64_t k = 0; k < m.n; ++k)
      for (int s = 0; s < 4; ++s)
        for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
          const SubFaceRec& r = M->h_sf[j];
          SubFaceBr2& g = M->h_sfb[j];
          const int P = m.p[k], len = m.sf[j].t1 - m.sf[j].t0;
          const bool in = r.nb >= 0;
          const double coef = in ? 0.25 : 1.0, hk = M->h_h[k];
          // both sides' lifting energies carry the larger coefficient of the sub-face
          const double w = in ? std::max(m.coef[k], m.coef[r.nb]) : m.coef[k];
          g.full = (m.size[k] == len ? 1 : 0) | (in && m.size[r.nb] == len ? 2 : 0);
          g.cz = w * (M->eta * coef * r.len * r.len * basis1d(P).Minv[0] / (hk * hk));
          g.tab_z = product(0, P, P, r.tab_oo, r.tab_oo, r.tab_oo);
          if (in) {
            const double hn = M->h_h[r.nb];
            g.cx = w * (M->eta * coef * r.len * r.len * basis1d(r.pn).Minv[0] / (hn * hn));
            g.tab_v = product(1, P, r.pn, r.tab_oo, r.tab_on, r.tab_nn);
            g.tab_x = product(2, P, r.pn, r.tab_oo, r.tab_on, r.tab_nn);
            g.tab_y = product(3, P, r.pn, r.tab_oo, r.tab_on, r.tab_nn);
          } else {
            g.tab_v = g.tab_x = g.tab_y = g.tab_z;
          }
        }
  }
  const int base = (int)M->h_tables.size();
  M->h_tables.insert(M->h_tables.end(), ft.data.begin(), ft.data.end());
  M->h_tables.insert(M->h_tables.end(), prod.begin(), prod.end());
  DG_REQUIRE(M->h_tables.size() < (1ULL << 31), "face tables too large");
  for (auto& r : M->h_sf) {
    r.tab_oo += base;
    r.tab_on += base;
    r.tab_nn += base;
  }
  for (auto& g : M->h_sfb) {
    g.tab_z += base;
    g.tab_v += base;
    g.tab_x += base;
    g.tab_y += base;
  }
  if (m.mapped) build_mesh_map(M, desc);   // the mapped records, tables and factors
  build_tiles(M);
  // operation and byte counts of one operator apply, as the kernel does it
  dg_mesh_stats& S = M->stats;
  S = dg_mesh_stats{};
  S.n_elems = m.n;
  S.n_dofs = M->n_dofs;
  S.n_subfaces = (int64_t)m.sf.size();
  double fl = 0.0;
  for (int64_t k = 0; k < m.n; ++k) {
    const double n1 = m.p[k] + 1.0;
    fl += 2.0 * (4.0 * n1 * n1 * n1 + 4.0 * n1 * n1 + 4.0 * n1 * n1);  // volume, own dn, gather
    for (int j = m.sf_ptr[4 * k]; j < m.sf_ptr[4 * k + 4]; ++j) {
      const auto& f = m.sf[j];
      // BR2 products (SubFaceBr2): Z and X on the own trace, V and Y on the
      // neighbour's; Z and V are not formed on the own element's whole side,
      // Y not on the neighbour's whole side
      const bool own_whole = m.size[k] == f.t1 - f.t0;
      if (f.nb < 0) {
        fl += 2.0 * (2.0 * n1 * n1);
        if (o.form == DG_FORM_BR2 && !own_whole) fl += 2.0 * (n1 * n1);
        continue;
      }
      const double nn = m.p[f.nb] + 1.0;
      fl += 2.0 * (2.0 * n1 * n1 + 2.0 * n1 * nn);
      if (o.form == DG_FORM_BR2) {
        const bool nb_whole = m.size[f.nb] == f.t1 - f.t0;
        fl += 2.0 * (n1 * n1 + (own_whole ? 0.0 : n1 * n1 + n1 * nn) + (nb_whole ? 0.0 : n1 * nn));
      }
      const int lg = std::abs(ilog2(m.size[k]) - ilog2(m.size[f.nb]));
      S.max_level_gap = std::max<int64_t>(S.max_level_gap, lg);
    }
  }
  S.apply_flops = fl;
  S.apply_bytes = 16.0 * (double)M->n_dofs + (double)m.n * (4 + 8 + 8 + 4 + 16) +
                  (double)m.sf.size() * sizeof(SubFaceRec);
  if (m.mapped) map_stats(M);
}

}  // namespace dg
