// Host setup of the preconditioner B = B_B + B_C on cube meshes (Sections
// 3.2-3.4 read for hexahedra).
//
// Master entities: every closed element splits into 27 entities (each axis at
// its lower end, its upper end, or spanning).  The master of an element entity
// Z is, among the entities of the elements touching the midpoint of Z whose
// relative interior holds that point, the one of largest dimension, then
// largest size: a hanging vertex belongs to a master edge or face, a hanging
// face to the larger face, a fine edge inside a coarse face to that face.
//
// V_C = V_h cap H^1_0: on every master entity M off the boundary a tensor
// polynomial of degree p_M at the Gauss-Lobatto points of M, p_M = the lowest
// degree of the elements touching relint(M), lowered to p_N for every master
// N whose boundary holds an edge or face of M (their traces must agree).
// Unknowns: the interior grid points of each master ((p_M-1)^dim, one for a
// vertex) and of each element.  Grid points on the boundary of M take the value
// of the master containing them, transitively; P evaluates the conforming basis
// at the DG nodes.  Numbering: first touch (elements in order, nodes
// lexicographic), a master is numbered by a node whose element entity has the
// master's dimension.
//
// V_J: nodes at regular vertices, and nodes of masters that are interior,
// unsubdivided and of one degree, or whose closure holds no hp-vertex (a
// hanging vertex whose elements differ in degree), or (remark_cases) whose
// coarse degree is <= every fine degree.  V_e: the E nodes of one master entity
// (the initial sets of the growth process; on hp cube meshes the growth to
// closure joins nearly all E nodes into a single block).
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>

#include "dg_internal.h"
#include "host_state.h"
#include "precond_setup.h"

namespace dg {

namespace {

using Row = std::vector<std::pair<int32_t, double>>;

struct BoxKey {
  std::array<int32_t, 6> v;   // lo[3], hi[3]
  bool operator==(const BoxKey& o) const { return v == o.v; }
};
struct BoxHash {
  size_t operator()(const BoxKey& b) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t c : b.v) {
      h ^= (uint32_t)c;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

int box_dim(const BoxKey& b) {
  int d = 0;
  for (int a = 0; a < 3; ++a) d += b.v[3 + a] > b.v[a];
  return d;
}
int box_size(const BoxKey& b) {
  int s = 0;
  for (int a = 0; a < 3; ++a) s = std::max(s, b.v[3 + a] - b.v[a]);
  return s;
}

struct Master {
  BoxKey box;
  int dim = 0;
  int p = 1 << 30;
  bool boundary = false, slaved = false;
  std::vector<int32_t> elems, owners;
  int64_t first = -1;   // first unknown; -1 not numbered, -2 none
};

struct Builder3 {
  const dg_mesh& M;
  const HostMesh& m;
  bool remark;
  std::vector<Master> ms;
  std::unordered_map<BoxKey, int32_t, BoxHash> master_id;   // master box -> id
  std::unordered_map<BoxKey, int32_t, BoxHash> memo;        // any box -> master id
  std::vector<int32_t> ent_master;                          // 27 per element
  int64_t nC = 0;
  std::vector<int32_t> conf_of_interior;

  Builder3(const dg_mesh& M_, bool remark_) : M(M_), m(M_.host), remark(remark_) {}

  BoxKey elem_entity(int64_t k, const int sel[3]) const {
    BoxKey b;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.lo[3 * k + a], hi = lo + m.size[k];
      b.v[a] = (sel[a] == 2) ? hi : lo;
      b.v[3 + a] = (sel[a] == 0) ? lo : hi;
    }
    return b;
  }
  bool on_boundary(const BoxKey& b) const {
    for (int a = 0; a < 3; ++a)
      if (b.v[a] == b.v[3 + a] && (b.v[a] == 0 || b.v[a] == m.extent[a])) return true;
    return false;
  }
  // elements whose closed box contains the point m2 / 2
  int touching(const int m2[3], int32_t* out) const {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      if (m2[a] % 2 == 0) {
        c0[a] = std::max(0, m2[a] / 2 - 1);
        c1[a] = std::min(m.extent[a] - 1, m2[a] / 2);
      } else {
        c0[a] = c1[a] = (m2[a] - 1) / 2;
      }
    }
    int n = 0;
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          const int32_t e = m.elem_at3(x, y, z);
          bool seen = false;
          for (int i = 0; i < n; ++i) seen = seen || out[i] == e;
          if (!seen) out[n++] = e;
        }
    return n;
  }
  int32_t master_of(const BoxKey& z) {
    auto it = memo.find(z);
    if (it != memo.end()) return it->second;
    int m2[3];
    for (int a = 0; a < 3; ++a) m2[a] = z.v[a] + z.v[3 + a];
    int32_t el[8];
    const int ne = touching(m2, el);
    BoxKey best{};
    int bd = -1, bs = -1;
    for (int i = 0; i < ne; ++i) {
      const int64_t k = el[i];
      int sel[3];
      for (int a = 0; a < 3; ++a) {
        const int lo = m.lo[3 * k + a], hi = lo + m.size[k];
        sel[a] = (m2[a] == 2 * lo) ? 0 : ((m2[a] == 2 * hi) ? 2 : 1);
      }
      const BoxKey c = elem_entity(k, sel);
      const int d = box_dim(c), s = box_size(c);
      if (d > bd || (d == bd && s > bs)) {
        best = c;
        bd = d;
        bs = s;
      }
    }
    auto mi = master_id.find(best);
    int32_t id;
    if (mi == master_id.end()) {
      id = (int32_t)ms.size();
      Master mm;
      mm.box = best;
      mm.dim = box_dim(best);
      mm.boundary = on_boundary(best);
      ms.push_back(mm);
      master_id.emplace(best, id);
    } else {
      id = mi->second;
    }
    memo.emplace(z, id);
    return id;
  }

  static void sel_of(int e, int sel[3]) {
    sel[0] = e % 3;
    sel[1] = (e / 3) % 3;
    sel[2] = e / 9;
  }

  void build_masters() {
    ent_master.assign(27 * m.n, -1);
    for (int64_t k = 0; k < m.n; ++k)
      for (int e = 0; e < 27; ++e) {
        int sel[3];
        sel_of(e, sel);
        const BoxKey z = elem_entity(k, sel);
        const int32_t id = master_of(z);
        ent_master[27 * k + e] = id;
        Master& mm = ms[id];
        mm.elems.push_back((int32_t)k);
        mm.p = std::min(mm.p, m.p[k]);
        if (z == mm.box) mm.owners.push_back((int32_t)k);
        else mm.slaved = true;
      }
    // trace-degree closure: masters holding an edge or face of M's boundary
    bool changed = true;
    while (changed) {
      changed = false;
      for (size_t i = 0; i < ms.size(); ++i) {
        if (ms[i].dim == 0) continue;
        const BoxKey b = ms[i].box;
        const int pm = ms[i].p;
        int span[3], ns = 0;
        for (int a = 0; a < 3; ++a)
          if (b.v[3 + a] > b.v[a]) span[ns++] = a;
        int total = 1;
        for (int t = 0; t < ns; ++t) total *= 3;
        for (int c = 0; c < total; ++c) {
          BoxKey z = b;
          int cc = c, sd = 0;
          bool whole = true;
          for (int t = 0; t < ns; ++t) {
            const int ch = cc % 3;
            cc /= 3;
            const int a = span[t];
            if (ch == 0) { z.v[3 + a] = z.v[a]; whole = false; }
            else if (ch == 2) { z.v[a] = z.v[3 + a]; whole = false; }
            else ++sd;
          }
          if (whole || sd == 0) continue;
          const int32_t j = master_of(z);
          if (ms[j].p > pm) {
            ms[j].p = pm;
            changed = true;
          }
        }
      }
    }
  }

  static int entity_index(int P, int ix, int iy, int iz) {
    auto s = [P](int i) { return i == 0 ? 0 : (i == P ? 2 : 1); };
    return s(ix) + 3 * s(iy) + 9 * s(iz);
  }
  static int entity_dim(int e) {
    int sel[3];
    sel_of(e, sel);
    return (sel[0] == 1) + (sel[1] == 1) + (sel[2] == 1);
  }

  void number() {
    conf_of_interior.assign(m.off[m.n], -1);
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      for (int iz = 0; iz <= P; ++iz)
        for (int iy = 0; iy <= P; ++iy)
          for (int ix = 0; ix <= P; ++ix) {
            const int e = entity_index(P, ix, iy, iz);
            if (e == 13) {
              conf_of_interior[m.off[k] + (iz * NP + iy) * NP + ix] = (int32_t)nC++;
              continue;
            }
            Master& mm = ms[ent_master[27 * k + e]];
            if (mm.first != -1 || entity_dim(e) != mm.dim) continue;
            if (mm.boundary) {
              mm.first = -2;
              continue;
            }
            int64_t cnt = 1;
            for (int d = 0; d < mm.dim; ++d) cnt *= (mm.p - 1);
            if (cnt == 0) {
              mm.first = -2;
              continue;
            }
            mm.first = nC;
            nC += cnt;
          }
    }
    DG_REQUIRE(nC < (1LL << 31), "too many conforming unknowns");
  }

  static void axpy(Row& out, const Row& in, double w) {
    for (const auto& e : in) out.push_back({e.first, w * e.second});
  }

  std::unordered_map<int64_t, Row> gmemo;   // (master, grid point) -> value

  // value of the conforming function on master `id` at lattice position pos
  Row value_at(int32_t id, const double pos[3]) {
    struct { BoxKey box; int dim, p; bool boundary; int64_t first; } mm = {
        ms[id].box, ms[id].dim, ms[id].p, ms[id].boundary, ms[id].first};   // copies: lookups may grow ms
    Row out;
    if (mm.boundary) return out;
    if (mm.dim == 0) {
      out.push_back({(int32_t)mm.first, 1.0});
      return out;
    }
    int span[3], ns = 0;
    for (int a = 0; a < 3; ++a)
      if (mm.box.v[3 + a] > mm.box.v[a]) span[ns++] = a;
    const int q = mm.p;
    const auto& g = basis1d(q).nodes;
    double l[3][kMaxN];
    for (int t = 0; t < ns; ++t) {
      const int a = span[t];
      lagrange_eval(g, (pos[a] - mm.box.v[a]) / (double)(mm.box.v[3 + a] - mm.box.v[a]), l[t]);
    }
    int gi[3] = {0, 0, 0};
    int total = 1;
    for (int t = 0; t < ns; ++t) total *= (q + 1);
    for (int c = 0; c < total; ++c) {
      int cc = c;
      double w = 1.0;
      bool interior = true;
      for (int t = 0; t < ns; ++t) {
        gi[t] = cc % (q + 1);
        cc /= (q + 1);
        w *= l[t][gi[t]];
        interior = interior && gi[t] > 0 && gi[t] < q;
      }
      if (w == 0.0) continue;
      if (interior) {
        int64_t li = 0, stride = 1;
        for (int t = 0; t < ns; ++t) {
          li += (gi[t] - 1) * stride;
          stride *= (q - 1);
        }
        out.push_back({(int32_t)(mm.first + li), w});
        continue;
      }
      int64_t key = (int64_t)id * 1000;
      for (int t = 0, sc = 100; t < ns; ++t, sc /= 10) key += gi[t] * sc;
      auto it = gmemo.find(key);
      if (it == gmemo.end()) {
        BoxKey z = mm.box;
        double y[3] = {(double)mm.box.v[0], (double)mm.box.v[1], (double)mm.box.v[2]};
        for (int t = 0; t < ns; ++t) {
          const int a = span[t];
          y[a] = mm.box.v[a] + (mm.box.v[3 + a] - mm.box.v[a]) * g[gi[t]];
          if (gi[t] == 0) z.v[3 + a] = z.v[a];
          else if (gi[t] == q) z.v[a] = z.v[3 + a];
        }
        it = gmemo.emplace(key, value_at(master_of(z), y)).first;
      }
      axpy(out, it->second, w);
    }
    return out;
  }

  Csr build_P() {
    std::vector<int64_t> r;
    std::vector<int32_t> c;
    std::vector<double> v;
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      const auto& g = basis1d(P).nodes;
      const int h = m.size[k];
      for (int iz = 0; iz <= P; ++iz)
        for (int iy = 0; iy <= P; ++iy)
          for (int ix = 0; ix <= P; ++ix) {
            const int64_t row = m.off[k] + (iz * NP + iy) * NP + ix;
            const int e = entity_index(P, ix, iy, iz);
            Row vals;
            if (e == 13) {
              vals.push_back({conf_of_interior[row], 1.0});
            } else {
              const double pos[3] = {m.lo[3 * k] + h * g[ix], m.lo[3 * k + 1] + h * g[iy],
                                     m.lo[3 * k + 2] + h * g[iz]};
              vals = value_at(ent_master[27 * k + e], pos);
            }
            for (auto& t : vals) {
              r.push_back(row);
              c.push_back(t.first);
              v.push_back(t.second);
            }
          }
    }
    Csr Pm = csr_from_triplets(m.off[m.n], nC, r, c, v);
    Csr out;
    out.rows = Pm.rows;
    out.cols = Pm.cols;
    out.ptr.assign(Pm.rows + 1, 0);
    for (int64_t i = 0; i < Pm.rows; ++i) {
      for (int64_t t = Pm.ptr[i]; t < Pm.ptr[i + 1]; ++t)
        if (Pm.val[t] != 0.0) {
          out.idx.push_back(Pm.idx[t]);
          out.val.push_back(Pm.val[t]);
        }
      out.ptr[i + 1] = (int64_t)out.idx.size();
    }
    return out;
  }

  // ---- classification
  std::unordered_map<int64_t, int8_t> hp_memo;
  bool is_hp_vertex(int x, int y, int z) {
    const int64_t key = ((int64_t)z * (m.extent[1] + 1) + y) * (m.extent[0] + 1) + x;
    auto it = hp_memo.find(key);
    if (it != hp_memo.end()) return it->second != 0;
    const int m2[3] = {2 * x, 2 * y, 2 * z};
    int32_t el[8];
    const int ne = touching(m2, el);
    bool corner = false, same = true;
    for (int i = 0; i < ne; ++i) {
      const int64_t k = el[i];
      bool c = true;
      for (int a = 0; a < 3; ++a) {
        const int lo = m.lo[3 * k + a], hi = lo + m.size[k];
        c = c && (m2[a] == 2 * lo || m2[a] == 2 * hi);
      }
      corner = corner || c;
      same = same && m.p[k] == m.p[el[0]];
    }
    bool hp = false;
    if (corner && !same) {
      BoxKey v{{x, y, z, x, y, z}};
      hp = ms[master_of(v)].dim > 0;
    }
    hp_memo.emplace(key, hp ? 1 : 0);
    return hp;
  }

  bool master_good(int32_t id) {
    const Master mm = ms[id];
    bool one_p = true;
    for (int32_t k : mm.elems) one_p = one_p && m.p[k] == m.p[mm.elems[0]];
    if (!mm.boundary && !mm.slaved && one_p) return true;
    if (remark && mm.slaved && !mm.owners.empty()) {
      int pc = 0, pf = 1 << 30;
      for (int32_t k : mm.owners) pc = std::max(pc, m.p[k]);
      for (int32_t k : mm.elems)
        if (std::find(mm.owners.begin(), mm.owners.end(), k) == mm.owners.end()) pf = std::min(pf, m.p[k]);
      if (pc <= pf) return true;
    }
    const BoxKey b = mm.box;
    for (int z = b.v[2]; z <= b.v[5]; ++z)
      for (int y = b.v[1]; y <= b.v[4]; ++y)
        for (int x = b.v[0]; x <= b.v[3]; ++x)
          if (is_hp_vertex(x, y, z)) return false;
    return true;
  }

  std::vector<int8_t> classify() {
    std::vector<int8_t> kind(m.off[m.n], 0);
    std::vector<int8_t> good(ms.size(), -1);
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      for (int iz = 0; iz <= P; ++iz)
        for (int iy = 0; iy <= P; ++iy)
          for (int ix = 0; ix <= P; ++ix) {
            const int e = entity_index(P, ix, iy, iz);
            if (e == 13) continue;
            const int32_t id = ent_master[27 * k + e];
            int8_t& gd = good[id];
            if (gd < 0) gd = (ms[id].dim == 0 || master_good(id)) ? 1 : 0;
            kind[m.off[k] + (iz * NP + iy) * NP + ix] = gd ? 1 : 2;
          }
    }
    return kind;
  }
};

// Diagonal of element k's rows on a cube mesh, in closed form: the volume
// diagonal plus, for every side holding the node, the sub-face terms of the
// node's own basis function (trace l_a l_b, outward normal derivative dv l_a l_b).
void host_element_diag3(const dg_mesh& M, int64_t k, double* d) {
  const HostMesh& m = M.host;
  const int P = m.p[k], NP = P + 1, N2 = NP * NP;
  const Basis1D& B = basis1d(P);
  const double hk = M.h_h[k], ak = m.coef[k];
  const double* T = M.h_tables.data();
  const bool br2 = M.opts.form == DG_FORM_BR2;
  for (int iz = 0; iz < NP; ++iz)
    for (int iy = 0; iy < NP; ++iy)
      for (int ix = 0; ix < NP; ++ix) {
        const double kx = B.K[ix * NP + ix], ky = B.K[iy * NP + iy], kz = B.K[iz * NP + iz];
        const double mx = B.M[ix * NP + ix], my = B.M[iy * NP + iy], mz = B.M[iz * NP + iz];
        d[(iz * NP + iy) * NP + ix] = (ak * hk) * (kx * my * mz + mx * ky * mz + mx * my * kz);
      }
  // quadratic form of a 1D table row against the inverse of a 1D mass matrix
  auto qform = [&](const double* row, int stride, int n, const std::vector<double>& Mi) {
    double v = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) v += row[a * stride] * Mi[a * n + b] * row[b * stride];
    return v;
  };
  for (int s = 0; s < 6; ++s) {
    int ax, ta, tb;
    side_axes3(s, ax, ta, tb);
    const int q = (s & 1) ? P : 0;
    const double dv = ((s & 1) ? B.d1[P] : -B.d0[0]) * (ak / hk);   // a times the normal derivative
    for (int j = 0; j < NP; ++j)
      for (int i = 0; i < NP; ++i) {
        int idx[3];
        idx[ax] = q;
        idx[ta] = i;
        idx[tb] = j;
        double add = 0.0;
        for (int f0 = m.sf_ptr[6 * k + s]; f0 < m.sf_ptr[6 * k + s + 1]; ++f0) {
          const SubFaceRec3& f = M.h_sf3[f0];
          const bool interior = f.nb >= 0;
          const double moo = T[f.tab_oo[0] + i * NP + i] * T[f.tab_oo[1] + j * NP + j];
          if (!br2) {
            add += f.area * moo * (f.sigma - (interior ? 1.0 : 2.0) * dv);
            continue;
          }
          add -= (interior ? 1.0 : 2.0) * f.area * moo * dv;
          // both sides' liftings carry the larger a of the sub-face
          const double w = interior ? std::max(ak, m.coef[f.nb]) : ak;
          const double so = w * (B.Minv[0] / (hk * hk * hk));
          double st = so * f.area * qform(T + f.tab_oo[0] + i, NP, NP, B.Minv) *
                      qform(T + f.tab_oo[1] + j, NP, NP, B.Minv);
          if (interior) {
            const int nn = f.pn + 1;
            const Basis1D& Bn = basis1d(f.pn);
            const double hn = M.h_h[f.nb];
            const double sn = w * (Bn.Minv[0] / (hn * hn * hn));
            st += sn * f.area * qform(T + f.tab_on[0] + i * nn, 1, nn, Bn.Minv) *
                  qform(T + f.tab_on[1] + j * nn, 1, nn, Bn.Minv);
          }
          add += M.eta * (interior ? 0.25 : 1.0) * f.area * st;
        }
        d[(idx[2] * NP + idx[1]) * NP + idx[0]] += add;
      }
  }
  (void)N2;
}

}  // namespace

HostPrecond build_host_precond3(const dg_mesh& M, const dg_options& o) {
  const HostMesh& m = M.host;
  HostPrecond H;
  const bool timing = std::getenv("DG_SETUP_TIMING") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!timing) return;
    auto t1 = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[setup3] %-12s %8.3f s\n", what, std::chrono::duration<double>(t1 - t0).count());
    t0 = t1;
  };
  Builder3 B(M, o.remark_cases != 0);
  B.build_masters();
  lap("masters");
  B.number();
  H.nC = B.nC;
  H.P = B.build_P();
  lap("P");
  H.kind = B.classify();
  lap("classify");
  if (o.smoother == DG_SMOOTHER_JACOBI_ONLY)
    for (auto& k : H.kind)
      if (k == 2) k = 1;
  const int64_t n = m.off[m.n];
  // ---- V_e: the E nodes of each master entity, blocks ordered by first node
  {
    std::unordered_map<int32_t, int32_t> blk_of;
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      for (int iz = 0; iz <= P; ++iz)
        for (int iy = 0; iy <= P; ++iy)
          for (int ix = 0; ix <= P; ++ix) {
            const int64_t r = m.off[k] + (iz * NP + iy) * NP + ix;
            if (H.kind[r] != 2) continue;
            const int32_t id = B.ent_master[27 * k + Builder3::entity_index(P, ix, iy, iz)];
            auto it = blk_of.find(id);
            if (it == blk_of.end()) {
              it = blk_of.emplace(id, (int32_t)H.blocks.size()).first;
              H.blocks.emplace_back();
            }
            H.blocks[it->second].push_back(r);
          }
    }
    for (auto& b : H.blocks) std::sort(b.begin(), b.end());
    std::sort(H.blocks.begin(), H.blocks.end(),
              [](const std::vector<int64_t>& a, const std::vector<int64_t>& b) { return a[0] < b[0]; });
  }
  lap("blocks-list");
  // ---- diagonal on V_J (closed form)
  H.dinv.assign(n, 0.0);
  {
    std::vector<double> y((size_t)kMaxN * kMaxN * kMaxN);
    for (int64_t k = 0; k < m.n; ++k) {
      const int NP = m.p[k] + 1, N3 = NP * NP * NP;
      host_element_diag3(M, k, y.data());
      for (int i = 0; i < N3; ++i) {
        const int64_t r = m.off[k] + i;
        if (H.kind[r] != 1) continue;
        if (!(y[i] > 0.0)) throw Error(DG_EINVAL, "non-positive diagonal");
        H.dinv[r] = 1.0 / y[i];
      }
    }
  }
  lap("diagonal");
  // ---- A_e read off element rows (unit columns), blocks spread over threads
  H.block_inv.resize(H.blocks.size());
  {
    auto elem_of = [&](int64_t r) {
      return (int64_t)(std::upper_bound(m.off.begin(), m.off.end(), r) - m.off.begin() - 1);
    };
    const int nth = std::max(1, std::min<int>((int)H.blocks.size(), setup_threads()));
    std::vector<std::thread> pool;
    std::vector<std::string> errs(nth);
    for (int t = 0; t < nth; ++t)
      pool.emplace_back([&, t] {
        try {
          SerialSetup serial;   // one block per thread already
          std::vector<double> x(n, 0.0), y((size_t)kMaxN * kMaxN * kMaxN);
          for (size_t bi = t; bi < H.blocks.size(); bi += nth) {
            const auto& blk = H.blocks[bi];
            const int d = (int)blk.size();
            std::vector<double> Ab((int64_t)d * d, 0.0);
            std::vector<int64_t> el(d);
            for (int a = 0; a < d; ++a) el[a] = elem_of(blk[a]);
            std::vector<int64_t> uel(el);
            std::sort(uel.begin(), uel.end());
            uel.erase(std::unique(uel.begin(), uel.end()), uel.end());
            for (int b = 0; b < d; ++b) {
              x[blk[b]] = 1.0;
              const int64_t kb = el[b];
              std::vector<int64_t> near{kb};
              for (int j = m.sf_ptr[6 * kb]; j < m.sf_ptr[6 * kb + 6]; ++j)
                if (m.sf3[j].nb >= 0) near.push_back(m.sf3[j].nb);
              std::sort(near.begin(), near.end());
              near.erase(std::unique(near.begin(), near.end()), near.end());
              for (int64_t k : near) {
                if (!std::binary_search(uel.begin(), uel.end(), k)) continue;
                host_element_residual3(M, k, x.data(), y.data(), kb);   // x = e_b lives in kb
                for (int a = 0; a < d; ++a)
                  if (el[a] == k) Ab[(int64_t)a * d + b] = y[blk[a] - m.off[k]];
              }
              x[blk[b]] = 0.0;
            }
            for (int a = 0; a < d; ++a)
              for (int b = a + 1; b < d; ++b) {
                const double s = 0.5 * (Ab[(int64_t)a * d + b] + Ab[(int64_t)b * d + a]);
                Ab[(int64_t)a * d + b] = Ab[(int64_t)b * d + a] = s;
              }
            dense_inverse_spd(d, Ab);
            H.block_inv[bi] = std::move(Ab);
          }
        } catch (const std::exception& e) {
          errs[t] = e.what();
        }
      });
    for (auto& th : pool) th.join();
    for (auto& e : errs)
      if (!e.empty()) throw Error(DG_EINVAL, e);
  }
  lap("blocks");
  // ---- LOR: trilinear stiffness on the Gauss-Lobatto sub-grid of each element
  {
    Csr At;
    At.rows = At.cols = n;
    At.ptr.assign(n + 1, 0);
    const double m1[2][2] = {{2.0 / 6.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 6.0}};
    const double k1[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      const double h = M.h_h[k];
      const auto& g = basis1d(P).nodes;
      for (int kz = 0; kz < NP; ++kz)
        for (int j = 0; j < NP; ++j)
          for (int i = 0; i < NP; ++i) {
            double row[3][3][3] = {};
            for (int cz = kz - 1; cz <= kz; ++cz)
              for (int cj = j - 1; cj <= j; ++cj)
                for (int ci = i - 1; ci <= i; ++ci) {
                  if (ci < 0 || cj < 0 || cz < 0 || ci >= P || cj >= P || cz >= P) continue;
                  const double a = h * (g[ci + 1] - g[ci]), b = h * (g[cj + 1] - g[cj]),
                               c = h * (g[cz + 1] - g[cz]);
                  const int px = i - ci, py = j - cj, pz = kz - cz;
                  for (int qz = 0; qz < 2; ++qz)
                    for (int qy = 0; qy < 2; ++qy)
                      for (int qx = 0; qx < 2; ++qx)
                        row[cz + qz - kz + 1][cj + qy - j + 1][ci + qx - i + 1] +=
                            (b * c / a) * k1[px][qx] * m1[py][qy] * m1[pz][qz] +
                            (a * c / b) * m1[px][qx] * k1[py][qy] * m1[pz][qz] +
                            (a * b / c) * m1[px][qx] * m1[py][qy] * k1[pz][qz];
                }
            for (int dz = 0; dz < 3; ++dz)
              for (int dj = 0; dj < 3; ++dj)
                for (int di = 0; di < 3; ++di) {
                  const int ii = i + di - 1, jj = j + dj - 1, zz = kz + dz - 1;
                  if (ii < 0 || jj < 0 || zz < 0 || ii > P || jj > P || zz > P) continue;
                  At.idx.push_back((int32_t)(m.off[k] + (zz * NP + jj) * NP + ii));
                  At.val.push_back(m.coef[k] * row[dz][dj][di]);   // weighted by a_k
                }
            At.ptr[m.off[k] + (kz * NP + j) * NP + i + 1] = (int64_t)At.idx.size();
          }
    }
    lap("lor-local");
    H.Ac = csr_multiply(csr_transpose(H.P), csr_multiply(At, H.P));
    lap("lor-spgemm");
  }
  return H;
}

}  // namespace dg
