// Cube meshes (the method of Section 2 on hexahedra): topology, sub-face
// records, operator tiles and the host mirror of the 3D operator.
//
// A sub-face of two dyadic cubes is the smaller of the two touching squares;
// its face integrals are products of 1D integrals along the two tangential
// axes, so the 1D face-mass tables of the square meshes serve both
// directions.  Side s of a cube has normal axis s / 2 (upper face when s is
// odd); its (p+1)^2 side nodes are indexed (i, j) along the first and second
// tangential axis (increasing axis numbers).
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "dg_internal.h"
#include "host_state.h"

namespace dg {

namespace {

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// volume index of side node (i, j) at normal index q on side s
inline int side_node3(int s, int i, int j, int q, int np) {
  const int ax = s >> 1;
  if (ax == 0) return q + np * (i + np * j);
  if (ax == 1) return i + np * (q + np * j);
  return i + np * (j + np * q);
}

void validate_and_copy3(const dg_mesh_desc* d, HostMesh& m) {
  DG_REQUIRE(d->n_elems > 0 && d->n_elems < (1LL << 30), "n_elems out of range");
  DG_REQUIRE(d->lo && d->size && d->p && d->extent, "null array in mesh description");
  DG_REQUIRE(d->lattice_h > 0.0 && std::isfinite(d->lattice_h), "lattice_h must be positive");
  m.dim = 3;
  m.n = d->n_elems;
  for (int a = 0; a < 3; ++a) {
    m.extent[a] = d->extent[a];
    DG_REQUIRE(m.extent[a] > 0, "extent must be positive");
  }
  DG_REQUIRE((int64_t)m.extent[0] * m.extent[1] * m.extent[2] <= (1LL << 28), "lattice too large");
  m.lh = d->lattice_h;
  copy_coeff(d, m.coef);
  m.lo.assign(d->lo, d->lo + 3 * m.n);
  m.size.assign(d->size, d->size + m.n);
  m.p.assign(d->p, d->p + m.n);
  m.cellmap.assign((int64_t)m.extent[0] * m.extent[1] * m.extent[2], -1);
  m.off.assign(m.n + 1, 0);
  for (int64_t k = 0; k < m.n; ++k) {
    const int x0 = m.lo[3 * k], y0 = m.lo[3 * k + 1], z0 = m.lo[3 * k + 2], h = m.size[k];
    DG_REQUIRE(m.p[k] >= 1 && m.p[k] <= kMaxP, "degree out of range 1..8");
    DG_REQUIRE(pow2(h), "element size must be a power of two");
    DG_REQUIRE(x0 >= 0 && y0 >= 0 && z0 >= 0 && x0 % h == 0 && y0 % h == 0 && z0 % h == 0,
               "element corner not aligned to its size");
    DG_REQUIRE(x0 + h <= m.extent[0] && y0 + h <= m.extent[1] && z0 + h <= m.extent[2],
               "element outside the domain");
    for (int z = z0; z < z0 + h; ++z)
      for (int y = y0; y < y0 + h; ++y)
        for (int x = x0; x < x0 + h; ++x) {
          int32_t& c = m.cellmap[((int64_t)z * m.extent[1] + y) * m.extent[0] + x];
          DG_REQUIRE(c < 0, "elements overlap");
          c = (int32_t)k;
        }
    const int64_t np = m.p[k] + 1;
    m.off[k + 1] = m.off[k] + np * np * np;
  }
  for (int32_t c : m.cellmap) DG_REQUIRE(c >= 0, "elements do not cover the domain");
}

}  // namespace

void build_topology3(HostMesh& m) {
  const int64_t n = m.n;
  m.sf_ptr.assign(6 * n + 1, 0);
  m.sf3.clear();
  for (int64_t k = 0; k < n; ++k) {
    const int h = m.size[k];
    for (int s = 0; s < 6; ++s) {
      int ax, ta, tb;
      side_axes3(s, ax, ta, tb);
      const bool upper = s & 1;
      const int c = m.lo[3 * k + ax] + (upper ? h : 0);
      const int A0 = m.lo[3 * k + ta], B0 = m.lo[3 * k + tb];
      if (upper ? (c == m.extent[ax]) : (c == 0)) {
        m.sf3.push_back({-1, -1, A0, B0, h});
      } else {
        const int cn = upper ? c : c - 1;
        int cell[3];
        cell[ax] = cn;
        for (int v = B0; v < B0 + h; ++v) {
          int u = A0;
          while (u < A0 + h) {
            cell[ta] = u;
            cell[tb] = v;
            const int nb = m.elem_at3(cell[0], cell[1], cell[2]);
            const int nA = m.lo[3 * nb + ta], nB = m.lo[3 * nb + tb], nh = m.size[nb];
            const int a0 = std::max(A0, nA), b0 = std::max(B0, nB);
            if (u == a0 && v == b0) m.sf3.push_back({nb, s ^ 1, a0, b0, std::min(h, nh)});
            u = std::min(A0 + h, nA + nh);
          }
        }
      }
      m.sf_ptr[6 * k + s + 1] = (int32_t)m.sf3.size();
    }
  }
}

// degree-sorted element order and tiles of the 3D operator kernel.  Elements
// are sorted by (p, nq), descending, nq = max(p, neighbour degrees) + 1; a tile
// is a run of equal (p, nq) with as many elements as fill 256 threads while the
// volume and side arrays leave room for a chunk of at least kApply3MinChunk
// sub-face items.  The tile's sub-faces are a flat list of (record, side)
// items, processed in chunks that fit the shared-memory budget; per element
// side the first item and the count.
void build_tiles3(dg_mesh* M) {
  const HostMesh& m = M->host;
  const bool br2 = M->opts.form == DG_FORM_BR2;
  std::vector<int32_t> nq(m.n), nitem(m.n);
  for (int64_t k = 0; k < m.n; ++k) {
    int q = m.p[k] + 1;
    const int b = m.sf_ptr[6 * k], e = m.sf_ptr[6 * k + 6];
    for (int j = b; j < e; ++j)
      if (m.sf3[j].nb >= 0) q = std::max(q, m.p[m.sf3[j].nb] + 1);
    nq[k] = q;
    nitem[k] = e - b;
  }
  std::vector<int32_t> order(m.n);
  for (int64_t k = 0; k < m.n; ++k) order[k] = (int32_t)k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (m.p[a] != m.p[b]) return m.p[a] > m.p[b];
    return nq[a] > nq[b];
  });
  M->h_tiles.clear();
  M->h_items.clear();
  M->h_item_ptr.assign(1, 0);
  M->h_side_items.assign(12 * (size_t)m.n, 0);
  M->apply3_smem = 0;
  for (int64_t i = 0; i < m.n;) {
    const int P = m.p[order[i]], Q = nq[order[i]], NP = P + 1;
    const int fixed_per = apply3_elem_doubles(P);
    const int item_per = apply3_item_doubles(P, Q, br2);
    const int by_threads = std::max(1, kThreads / (NP * NP * NP));
    int64_t j = i, items = 0;
    while (j < m.n && m.p[order[j]] == P && nq[order[j]] == Q && j - i < by_threads) {
      const int64_t cnt = j - i + 1, it = items + nitem[order[j]];
      const int64_t need = 2 * NP * NP + cnt * fixed_per + std::min<int64_t>(it, kApply3MinChunk) * item_per;
      if (need > M->apply3_budget && j > i) break;
      items = it;
      ++j;
    }
    const int64_t fixed = 2 * NP * NP + (j - i) * fixed_per;
    const int64_t room = (M->apply3_budget - fixed) / item_per;
    DG_REQUIRE(room >= 1, "3D operator tile does not fit in shared memory");
    ApplyTile T{};
    T.p = P;
    T.first = (int32_t)i;
    T.count = (int32_t)(j - i);
    T.nq = Q;
    T.chunk = (int32_t)std::min<int64_t>(items, room);
    for (int64_t e = 0; e < T.count; ++e) {
      const int64_t pos = i + e;
      const int32_t k = order[pos];
      for (int s = 0; s < 6; ++s) {
        const int b = m.sf_ptr[6 * (int64_t)k + s], c = m.sf_ptr[6 * (int64_t)k + s + 1] - b;
        M->h_side_items[12 * pos + 2 * s] = (int32_t)(M->h_items.size() / 2);
        M->h_side_items[12 * pos + 2 * s + 1] = c;
        for (int q = 0; q < c; ++q) {
          M->h_items.push_back(b + q);
          M->h_items.push_back((int32_t)(6 * e + s));
        }
      }
    }
    // Within each chunk the items go in the order of the branches their
    // threads take - interior first, then the BR2 whole-face flags, then the
    // neighbour degree (the loop bound) - so that a warp of the two
    // contraction passes spans fewer kinds of item.  The high half of the
    // side field keeps the item's position in sub-face order: the second pass
    // writes the item's partials there, and the third adds them in that order.
    {
      const int64_t t0 = M->h_item_ptr.back(), t1 = (int64_t)M->h_items.size() / 2;
      DG_REQUIRE(T.chunk < 65536, "3D operator: sub-face chunk too long");
      std::vector<std::pair<int32_t, int32_t>> key;   // (branch key, position in the chunk)
      std::vector<int32_t> rec, side;
      for (int64_t c0 = t0; c0 < t1; c0 += T.chunk) {
        const int64_t c1 = std::min<int64_t>(c0 + T.chunk, t1);
        key.clear();
        rec.assign(M->h_items.begin() + 2 * c0, M->h_items.begin() + 2 * c1);
        for (int64_t g = c0; g < c1; ++g) {
          const SubFaceRec3& f = M->h_sf3[M->h_items[2 * g]];
          const bool in = f.nb >= 0;
          const int zv = (br2 && !(f.full & 1)) ? 1 : 0, yy = (br2 && in && !(f.full & 2)) ? 1 : 0;
          key.push_back({((in ? 0 : 1) << 12) | (zv << 11) | (yy << 10) | (in ? 16 - f.pn : 0),
                         (int32_t)(g - c0)});
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                           return a.first < b.first;
                         });
        for (int64_t g = c0; g < c1; ++g) {
          const int32_t pos = key[g - c0].second;
          M->h_items[2 * g] = rec[2 * pos];
          M->h_items[2 * g + 1] = rec[2 * pos + 1] | (pos << 16);
        }
      }
    }
    M->h_item_ptr.push_back((int32_t)(M->h_items.size() / 2));
    M->h_tiles.push_back(T);
    M->apply3_smem = std::max<int64_t>(M->apply3_smem, 8LL * (fixed + T.chunk * item_per));
    i = j;
  }
  M->n_tiles = (int)M->h_tiles.size();
  M->h_order = order;
}

void build_mesh_host3(dg_mesh* M, const dg_mesh_desc* desc, const dg_options& o) {
  HostMesh& m = M->host;
  validate_and_copy3(desc, m);
  build_topology3(m);
  M->n_dofs = m.off[m.n];
  DG_REQUIRE(M->n_dofs < (1LL << 31), "too many unknowns for 32-bit indices");
  M->h_h.resize(m.n);
  for (int64_t k = 0; k < m.n; ++k) M->h_h[k] = m.size[k] * m.lh;
  if (o.eta > 0) {
    M->eta = o.eta;
  } else if (o.form == DG_FORM_BR2) {
    int mx = 0;
    for (int64_t k = 0; k < m.n; ++k) mx = std::max(mx, m.sf_ptr[6 * k + 6] - m.sf_ptr[6 * k]);
    M->eta = (double)mx;
  } else {
    M->eta = 100.0;
  }
  M->h_tables.clear();
  for (int p = 1; p <= kMaxP; ++p) {
    const Basis1D& b = basis1d(p);
    auto app = [&](const std::vector<double>& v, int& off) {
      off = (int)M->h_tables.size();
      M->h_tables.insert(M->h_tables.end(), v.begin(), v.end());
    };
    app(b.M, M->boff[p].M);
    app(b.K, M->boff[p].K);
    app(b.Minv, M->boff[p].Minv);
    app(b.d0, M->boff[p].d0);
    app(b.d1, M->boff[p].d1);
  }
  M->boff[0] = M->boff[1];
  FaceTables ft;
  M->h_sf3.resize(m.sf3.size());
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 6; ++s) {
      int ax, ta, tb;
      side_axes3(s, ax, ta, tb);
      const int P = m.p[k];
      const int A0 = m.lo[3 * k + ta], B0 = m.lo[3 * k + tb], h = m.size[k];
      for (int j = m.sf_ptr[6 * k + s]; j < m.sf_ptr[6 * k + s + 1]; ++j) {
        const auto& f = m.sf3[j];
        SubFaceRec3 r{};
        const int Lo = ilog2(h / f.len);
        const int oa = (f.a0 - A0) / f.len, ob = (f.b0 - B0) / f.len;
        r.nb = f.nb;
        r.nb_side = f.nb_side;
        r.full = (Lo == 0) ? 1 : 0;
        r.area = (double)f.len * f.len * m.lh * m.lh;
        r.tab_oo[0] = ft.get(P, Lo, oa, P, Lo, oa);
        r.tab_oo[1] = ft.get(P, Lo, ob, P, Lo, ob);
        int pe = P;
        double he = M->h_h[k], ae = m.coef[k];
        if (f.nb >= 0) {
          const int pn = m.p[f.nb], nh = m.size[f.nb];
          const int nA = m.lo[3 * f.nb + ta], nB = m.lo[3 * f.nb + tb];
          const int Ln = ilog2(nh / f.len);
          const int na = (f.a0 - nA) / f.len, nbo = (f.b0 - nB) / f.len;
          r.pn = pn;
          if (Ln == 0) r.full |= 2;
          r.tab_on[0] = ft.get(P, Lo, oa, pn, Ln, na);
          r.tab_on[1] = ft.get(P, Lo, ob, pn, Ln, nbo);
          r.tab_nn[0] = ft.get(pn, Ln, na, pn, Ln, na);
          r.tab_nn[1] = ft.get(pn, Ln, nbo, pn, Ln, nbo);
          pe = std::max(P, pn);
          he = std::min(he, M->h_h[f.nb]);
          ae = std::max(ae, m.coef[f.nb]);
        } else {
          r.pn = P;
          for (int d = 0; d < 2; ++d) r.tab_on[d] = r.tab_nn[d] = r.tab_oo[d];
        }
        const double pp = (o.penalty_form == DG_PENALTY_P1SQ) ? (pe + 1.0) : (double)pe;
        r.sigma = ae * (M->eta * pp * pp / he);   // the larger coefficient of the two sides
        M->h_sf3[j] = r;
      }
    }
  // BR2 lifting products of the face tables (the lifting of a sub-face jump,
  // its element mass inverse and the face mass back onto the side nodes, per
  // tangential axis), appended after the face tables
  std::vector<double> prod;
  std::map<std::tuple<int, int, int, int>, int> pindex;
  const int pbase = (int)ft.data.size();
  auto product = [&](int kind, int p, int pn, int oo, int on, int nn) {
    const auto key = std::make_tuple(kind, kind == 0 ? oo : on, kind == 3 ? nn : (kind == 1 ? oo : -1), p * 16 + pn);
    auto it = pindex.find(key);
    if (it != pindex.end()) return it->second;
    const int a = p + 1, b = pn + 1;
    const double* Moo = ft.data.data() + oo;
    const double* Mon = ft.data.data() + on;
    const double* Mnn = ft.data.data() + nn;
    const std::vector<double>& Mi = basis1d(p).Minv;
    const std::vector<double>& Min = basis1d(pn).Minv;
    const int cols = (kind == 0 || kind == 2) ? a : b;
    const int o = (int)prod.size();
    prod.resize(o + (size_t)a * cols, 0.0);
    for (int i = 0; i < a; ++i)
      for (int j = 0; j < cols; ++j) {
        double v = 0.0;
        if (kind == 0) {          // Z = M_oo Minv M_oo
          for (int u = 0; u < a; ++u)
            for (int w = 0; w < a; ++w) v += Moo[i * a + u] * Mi[u * a + w] * Moo[w * a + j];
        } else if (kind == 1) {   // V = M_oo Minv M_on
          for (int u = 0; u < a; ++u)
            for (int w = 0; w < a; ++w) v += Moo[i * a + u] * Mi[u * a + w] * Mon[w * b + j];
        } else if (kind == 2) {   // X = M_on Minv_n M_no
          for (int u = 0; u < b; ++u)
            for (int w = 0; w < b; ++w) v += Mon[i * b + u] * Min[u * b + w] * Mon[j * b + w];
        } else {                  // Y = M_on Minv_n M_nn
          for (int u = 0; u < b; ++u)
            for (int w = 0; w < b; ++w) v += Mon[i * b + u] * Min[u * b + w] * Mnn[w * b + j];
        }
        prod[o + (size_t)i * cols + j] = v;
      }
    pindex.emplace(key, pbase + o);
    return pbase + o;
  };
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 6; ++s)
      for (int j = m.sf_ptr[6 * k + s]; j < m.sf_ptr[6 * k + s + 1]; ++j) {
        SubFaceRec3& r = M->h_sf3[j];
        const int P = m.p[k];
        const bool in = r.nb >= 0;
        const double coef = in ? 0.25 : 1.0;
        const double hk = M->h_h[k];
        // both sides' lifting energies carry the larger coefficient of the sub-face
        const double w = in ? std::max(m.coef[k], m.coef[r.nb]) : m.coef[k];
        r.cz = w * (M->eta * coef * r.area * r.area * basis1d(P).Minv[0] / (hk * hk * hk));
        for (int d = 0; d < 2; ++d) {
          r.tab_z[d] = product(0, P, P, r.tab_oo[d], r.tab_oo[d], r.tab_oo[d]);
          if (in) {
            r.tab_v[d] = product(1, P, r.pn, r.tab_oo[d], r.tab_on[d], r.tab_nn[d]);
            r.tab_x[d] = product(2, P, r.pn, r.tab_oo[d], r.tab_on[d], r.tab_nn[d]);
            r.tab_y[d] = product(3, P, r.pn, r.tab_oo[d], r.tab_on[d], r.tab_nn[d]);
          } else {
            r.tab_v[d] = r.tab_x[d] = r.tab_y[d] = r.tab_z[d];
          }
        }
        if (in) {
          const double hn = M->h_h[r.nb];
          r.cx = w * (M->eta * coef * r.area * r.area * basis1d(r.pn).Minv[0] / (hn * hn * hn));
        }
      }
  const int base = (int)M->h_tables.size();
  M->h_tables.insert(M->h_tables.end(), ft.data.begin(), ft.data.end());
  M->h_tables.insert(M->h_tables.end(), prod.begin(), prod.end());
  DG_REQUIRE(M->h_tables.size() < (1ULL << 31), "face tables too large");
  for (auto& r : M->h_sf3)
    for (int d = 0; d < 2; ++d) {
      r.tab_oo[d] += base;
      r.tab_on[d] += base;
      r.tab_nn[d] += base;
      r.tab_z[d] += base;
      r.tab_v[d] += base;
      r.tab_x[d] += base;
      r.tab_y[d] += base;
    }
  build_tiles3(M);
  // operation and byte counts of one operator apply, as the kernels do it
  dg_mesh_stats& S = M->stats;
  S = dg_mesh_stats{};
  S.n_elems = m.n;
  S.n_dofs = M->n_dofs;
  S.n_subfaces = (int64_t)m.sf3.size();
  const bool br2 = o.form == DG_FORM_BR2;
  double fma = 0.0;
  for (int64_t k = 0; k < m.n; ++k) {
    const double a = m.p[k] + 1.0, a2 = a * a, a3 = a2 * a;
    fma += 7.0 * a3 * a + 6.0 * a3 + 6.0 * a3;   // volume, traces' dn, gather
    for (int j = m.sf_ptr[6 * k]; j < m.sf_ptr[6 * k + 6]; ++j) {
      const auto& f = m.sf3[j];
      const bool own_full = f.len == m.size[k];
      if (f.nb < 0) {
        fma += 4.0 * a3 + ((br2 && !own_full) ? 2.0 * a3 : 0.0);   // M_oo on u, dn; BR2: Z on u
        continue;
      }
      const double b = m.p[f.nb] + 1.0, b2 = b * b;
      const bool nb_full = f.len == m.size[f.nb];
      fma += 4.0 * a3 + 2.0 * a * b2 + 2.0 * a2 * b;   // M_oo on u-, dn-; M_on on u+, dn+
      if (br2) {
        fma += 2.0 * a3;                                          // X on u-
        if (!own_full) fma += 2.0 * a3 + a * b2 + a2 * b;         // Z on u-, V on u+
        if (!nb_full) fma += a * b2 + a2 * b;                     // Y on u+
      }
      const int lg = std::abs(ilog2(m.size[k]) - ilog2(m.size[f.nb]));
      S.max_level_gap = std::max<int64_t>(S.max_level_gap, lg);
    }
  }
  S.apply_flops = 2.0 * fma;
  S.apply_bytes = 16.0 * (double)M->n_dofs + (double)m.n * (4 + 8 + 8 + 4 + 16) +
                  (double)m.sf3.size() * sizeof(SubFaceRec3);
}

// Rows of element k of y = A x on a cube mesh, with the records and tables the
// kernel uses and the same algebra, written as plain loops.
void host_element_residual3(const dg_mesh& M, int64_t k, const double* x, double* y, int64_t source) {
  const HostMesh& m = M.host;
  const int P = m.p[k], NP = P + 1, N2 = NP * NP, N3 = N2 * NP;
  const Basis1D& B = basis1d(P);
  const double hk = M.h_h[k];
  const double* xk = x + m.off[k];
  const double* T = M.h_tables.data();
  const bool br2 = M.opts.form == DG_FORM_BR2;
  // x vanishes outside element `source` (when >= 0): on another element k the
  // volume term and every sub-face not shared with `source` add exact zeros
  const bool own_zero = source >= 0 && source != k;
  if (own_zero) std::fill(y, y + N3, 0.0);
  // volume: h (K x M x M + M x K x M + M x M x K) x, index ix + NP (iy + NP iz),
  // sum factorised: along z A = M x, Bz = K x; along y C = M A, D = K A + M Bz;
  // along x y = h (K C + M D)
  if (!own_zero) {
    double A[kMaxN * kMaxN * kMaxN], Bz[kMaxN * kMaxN * kMaxN];
    double C[kMaxN * kMaxN * kMaxN], D[kMaxN * kMaxN * kMaxN];
    for (int iz = 0; iz < NP; ++iz)
      for (int r = 0; r < N2; ++r) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < NP; ++q) {
          a += B.M[iz * NP + q] * xk[q * N2 + r];
          b += B.K[iz * NP + q] * xk[q * N2 + r];
        }
        A[iz * N2 + r] = a;
        Bz[iz * N2 + r] = b;
      }
    for (int iz = 0; iz < NP; ++iz)
      for (int iy = 0; iy < NP; ++iy)
        for (int ix = 0; ix < NP; ++ix) {
          double c = 0.0, d = 0.0;
          for (int q = 0; q < NP; ++q) {
            const double av = A[iz * N2 + q * NP + ix];
            c += B.M[iy * NP + q] * av;
            d += B.K[iy * NP + q] * av + B.M[iy * NP + q] * Bz[iz * N2 + q * NP + ix];
          }
          C[iz * N2 + iy * NP + ix] = c;
          D[iz * N2 + iy * NP + ix] = d;
        }
    for (int r = 0; r < N3; r += NP)
      for (int ix = 0; ix < NP; ++ix) {
        double v = 0.0;
        for (int q = 0; q < NP; ++q) v += B.K[ix * NP + q] * C[r + q] + B.M[ix * NP + q] * D[r + q];
        y[r + ix] = (m.coef[k] * hk) * v;
      }
  }
  // traces (value, outward normal derivative) of an element side
  auto trace = [&](int64_t e, int s, std::vector<double>& u, std::vector<double>& dn) {
    const int pe = m.p[e], ne = pe + 1;
    const Basis1D& Be = basis1d(pe);
    const double* xe = x + m.off[e];
    const double* dv = (s & 1) ? Be.d1.data() : Be.d0.data();
    const double sg = ((s & 1) ? 1.0 : -1.0) * (m.coef[e] / M.h_h[e]);   // a grad u . n
    u.assign(ne * ne, 0.0);
    dn.assign(ne * ne, 0.0);
    for (int j = 0; j < ne; ++j)
      for (int i = 0; i < ne; ++i) {
        u[j * ne + i] = xe[side_node3(s, i, j, (s & 1) ? pe : 0, ne)];
        double acc = 0.0;
        for (int q = 0; q < ne; ++q) acc += dv[q] * xe[side_node3(s, i, j, q, ne)];
        dn[j * ne + i] = sg * acc;
      }
  };
  // 2D contraction out[i + ro*j] = sum_{m,n} Ta[i][m] Tb[j][n] in[m + ci*n]
  // (table rows of length ci; `tr` reads the tables transposed), in two passes
  auto contract = [&](int ta, int tb, int ro, int ci, bool tr, const std::vector<double>& in,
                      std::vector<double>& out) {
    double w[kMaxN * kMaxN];
    for (int nn = 0; nn < ci; ++nn)
      for (int i = 0; i < ro; ++i) {
        double v = 0.0;
        for (int mm = 0; mm < ci; ++mm) v += (tr ? T[ta + mm * ro + i] : T[ta + i * ci + mm]) * in[mm + ci * nn];
        w[i + ro * nn] = v;
      }
    out.assign(ro * ro, 0.0);
    for (int j = 0; j < ro; ++j)
      for (int i = 0; i < ro; ++i) {
        double v = 0.0;
        for (int nn = 0; nn < ci; ++nn) v += (tr ? T[tb + nn * ro + j] : T[tb + j * ci + nn]) * w[i + ro * nn];
        out[i + ro * j] = v;
      }
  };
  auto minv2 = [&](int pe, double he, const std::vector<double>& in, std::vector<double>& out) {
    const Basis1D& Be = basis1d(pe);
    const int ne = pe + 1;
    out.assign(ne * ne, 0.0);
    const double sc = Be.Minv[0] / (he * he * he);
    for (int j = 0; j < ne; ++j)
      for (int i = 0; i < ne; ++i) {
        double v = 0.0;
        for (int nn = 0; nn < ne; ++nn)
          for (int mm = 0; mm < ne; ++mm) v += Be.Minv[i * ne + mm] * Be.Minv[j * ne + nn] * in[mm + ne * nn];
        out[i + ne * j] = sc * v;
      }
  };
  std::vector<double> r(6 * N2, 0.0), c2(6 * N2, 0.0);
  std::vector<double> uo, dno, un, dnn, a, c, b, d, jo, jn, t1, t2, go, gn, st1, st2;
  for (int s = 0; s < 6; ++s) {
    trace(k, s, uo, dno);
    for (int j = m.sf_ptr[6 * k + s]; j < m.sf_ptr[6 * k + s + 1]; ++j) {
      const SubFaceRec3& f = M.h_sf3[j];
      if (own_zero && f.nb != source) continue;
      const double ar = f.area;
      contract(f.tab_oo[0], f.tab_oo[1], NP, NP, false, uo, a);
      contract(f.tab_oo[0], f.tab_oo[1], NP, NP, false, dno, c);
      const bool interior = f.nb >= 0;
      const int nn = f.pn + 1;
      if (interior) {
        trace(f.nb, f.nb_side, un, dnn);
        contract(f.tab_on[0], f.tab_on[1], NP, nn, false, un, b);
        contract(f.tab_on[0], f.tab_on[1], NP, nn, false, dnn, d);
      } else {
        b.assign(N2, 0.0);
        d.assign(N2, 0.0);
      }
      const double half = interior ? 0.5 : 1.0;
      jo.assign(N2, 0.0);
      for (int q = 0; q < N2; ++q) {
        const double jmp = a[q] - b[q];
        c2[s * N2 + q] -= half * ar * jmp;
        jo[q] = ar * jmp;
        const double cons = interior ? -0.5 * ar * (c[q] - d[q]) : -ar * c[q];
        r[s * N2 + q] += cons;
        if (!br2) r[s * N2 + q] += f.sigma * ar * jmp;
      }
      if (br2) {
        minv2(P, hk, jo, go);
        contract(f.tab_oo[0], f.tab_oo[1], NP, NP, false, go, st1);
        if (interior) {
          std::vector<double> p1, p2;
          contract(f.tab_on[0], f.tab_on[1], nn, NP, true, uo, p1);   // M_no u-
          contract(f.tab_nn[0], f.tab_nn[1], nn, nn, false, un, p2);  // M_nn u+
          jn.assign(nn * nn, 0.0);
          for (int q = 0; q < nn * nn; ++q) jn[q] = ar * (p1[q] - p2[q]);
          minv2(f.pn, M.h_h[f.nb], jn, gn);
          contract(f.tab_on[0], f.tab_on[1], NP, nn, false, gn, st2);
        } else {
          st2.assign(N2, 0.0);
        }
        const double coef = interior ? 0.25 : 1.0;
        // both sides' lifting energies carry the larger a of the sub-face
        const double w = interior ? std::max(m.coef[k], m.coef[f.nb]) : m.coef[k];
        for (int q = 0; q < N2; ++q)
          r[s * N2 + q] += M.eta * coef * ar * w * (st1[q] + st2[q]);
      }
    }
  }
  for (int node = 0; node < N3; ++node) {
    const int idx[3] = {node % NP, (node / NP) % NP, node / N2};
    double v = y[node];
    for (int s = 0; s < 6; ++s) {
      int ax, ta, tb;
      side_axes3(s, ax, ta, tb);
      const int q = idx[ax], i = idx[ta], j = idx[tb];
      const double dv = (s & 1) ? B.d1[q] : -B.d0[q];
      v += dv * (m.coef[k] / hk) * c2[s * N2 + j * NP + i];
      if (q == ((s & 1) ? P : 0)) v += r[s * N2 + j * NP + i];
    }
    y[node] = v;
  }
}

}  // namespace dg
