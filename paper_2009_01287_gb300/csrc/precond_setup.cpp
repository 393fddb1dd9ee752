// Host setup of the preconditioner B = B_B + B_C (Sections 3.2-3.4, 4.1).
//
// Conforming space V_C = V_h cap H^1_0 (Section 3.2.1 nodal points): one
// unknown per regular interior vertex, p_S - 1 per interior master edge S at
// the Gauss-Lobatto points of degree p_S (the lowest degree of the elements
// containing S), (p-1)^2 per element interior.  Hanging vertices take the
// value of the master edge containing them, transitively.  P evaluates the
// conforming basis at the DG nodes (the natural injection of Section 3.4).
// Numbering: first touch over elements, nodes in local lexicographic order.
//
// V_J: nodes at regular vertices and nodes on / hanging in a master edge that
// is conforming with equal degrees, whose closed edge holds no hp-vertex, or
// (remark_cases) whose coarse degree is <= every fine degree.  The other
// element-boundary nodes are split into V_e = connected components under
// "traces nonzero on a common sub-face" (the growth process of Section 3.3).
#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include "dg_internal.h"
#include "host_state.h"
#include "precond_setup.h"

namespace dg {

namespace {

using Row = std::vector<std::pair<int32_t, double>>;

struct Builder {
  const dg_mesh& M;
  const HostMesh& m;
  bool remark;
  int64_t nC = 0;
  std::vector<int32_t> conf_of_interior;                  // per DG node or -1
  std::unordered_map<int64_t, int32_t> vertex_dof;
  std::vector<int64_t> master_first;                      // -1 none yet, -2 no unknowns
  std::unordered_map<int64_t, Row> vmemo;

  Builder(const dg_mesh& M_, bool remark_) : M(M_), m(M_.host), remark(remark_) {}

  int64_t vkey(int x, int y) const { return (int64_t)y * (m.extent[0] + 1) + x; }
  bool hanging(int x, int y) const { return m.containing_side(x, y, nullptr) >= 0; }

  void corner_xy(int64_t k, int ix, int iy, int& x, int& y) const {
    const int P = m.p[k];
    x = m.lo[2 * k] + (ix == P ? m.size[k] : 0);
    y = m.lo[2 * k + 1] + (iy == P ? m.size[k] : 0);
  }
  static int node_side(int P, int ix, int iy) {
    if (ix == 0) return 0;
    if (ix == P) return 1;
    if (iy == 0) return 2;
    return 3;
  }

  void number() {
    conf_of_interior.assign(m.off[m.n], -1);
    master_first.assign(m.masters.size(), -1);
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k];
      for (int iy = 0; iy <= P; ++iy)
        for (int ix = 0; ix <= P; ++ix) {
          const bool bx = (ix == 0 || ix == P), by = (iy == 0 || iy == P);
          if (!bx && !by) {
            conf_of_interior[m.off[k] + iy * (P + 1) + ix] = (int32_t)nC++;
          } else if (bx && by) {
            int x, y;
            corner_xy(k, ix, iy, x, y);
            if (!m.on_boundary(x, y) && !hanging(x, y) && !vertex_dof.count(vkey(x, y)))
              vertex_dof[vkey(x, y)] = (int32_t)nC++;
          } else {
            const int id = m.side_master[4 * k + node_side(P, ix, iy)];
            if (master_first[id] == -1) {
              const auto& S = m.masters[id];
              if (S.boundary) {
                master_first[id] = -2;
              } else {
                master_first[id] = nC;
                nC += S.p - 1;
              }
            }
          }
        }
    }
  }

  static void axpy(Row& out, const Row& in, double w) {
    for (const auto& e : in) out.push_back({e.first, w * e.second});
  }

  Row vertex_value(int x, int y) {
    const int64_t key = vkey(x, y);
    auto it = vmemo.find(key);
    if (it != vmemo.end()) return it->second;
    Row r;
    if (!m.on_boundary(x, y)) {
      auto v = vertex_dof.find(key);
      if (v != vertex_dof.end()) {
        r.push_back({v->second, 1.0});
      } else {
        int side = 0;
        const int e = m.containing_side(x, y, &side);
        if (e < 0) throw Error(DG_EINVAL, "vertex without unknown");
        const int id = m.side_master[4 * e + side];
        const auto& S = m.masters[id];
        r = edge_value(id, S.axis == 0 ? (double)y : (double)x);
      }
    }
    vmemo[key] = r;
    return r;
  }

  Row edge_value(int id, double tan) {
    const auto& S = m.masters[id];
    const double lam = (tan - S.t0) / (double)(S.t1 - S.t0);
    double l[kMaxN];
    lagrange_eval(basis1d(S.p).nodes, lam, l);
    Row out;
    if (l[0] != 0.0) {
      Row a = S.axis == 0 ? vertex_value(S.c, S.t0) : vertex_value(S.t0, S.c);
      axpy(out, a, l[0]);
    }
    if (l[S.p] != 0.0) {
      Row b = S.axis == 0 ? vertex_value(S.c, S.t1) : vertex_value(S.t1, S.c);
      axpy(out, b, l[S.p]);
    }
    if (master_first[id] >= 0)
      for (int j = 1; j < S.p; ++j) out.push_back({(int32_t)(master_first[id] + j - 1), l[j]});
    return out;
  }

  Csr build_P() {
    std::vector<int64_t> r;
    std::vector<int32_t> c;
    std::vector<double> v;
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k];
      const auto& g = basis1d(P).nodes;
      const int x0 = m.lo[2 * k], y0 = m.lo[2 * k + 1], h = m.size[k];
      for (int iy = 0; iy <= P; ++iy)
        for (int ix = 0; ix <= P; ++ix) {
          const int64_t row = m.off[k] + iy * (P + 1) + ix;
          const bool bx = (ix == 0 || ix == P), by = (iy == 0 || iy == P);
          Row vals;
          if (!bx && !by) {
            vals.push_back({conf_of_interior[row], 1.0});
          } else if (bx && by) {
            int x, y;
            corner_xy(k, ix, iy, x, y);
            vals = vertex_value(x, y);
          } else {
            const int s = node_side(P, ix, iy);
            const double tan = (s < 2) ? (y0 + h * g[iy]) : (x0 + h * g[ix]);
            vals = edge_value(m.side_master[4 * k + s], tan);
          }
          for (auto& e : vals) {
            r.push_back(row);
            c.push_back(e.first);
            v.push_back(e.second);
          }
        }
    }
    Csr Pm = csr_from_triplets(m.off[m.n], nC, r, c, v);
    // drop entries that summed to exactly zero
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

  bool master_good(int id) const {
    const auto& S = m.masters[id];
    if (S.owners.size() == 2 && m.p[S.owners[0]] == m.p[S.owners[1]]) return true;
    bool hp = false;
    for (const auto& v : S.hanging) hp = hp || m.is_hp_vertex(v.first, v.second);
    if (S.axis == 0) {
      hp = hp || m.is_hp_vertex(S.c, S.t0) || m.is_hp_vertex(S.c, S.t1);
    } else {
      hp = hp || m.is_hp_vertex(S.t0, S.c) || m.is_hp_vertex(S.t1, S.c);
    }
    if (!hp) return true;
    if (remark && !S.slaves.empty()) {
      int pc = 1 << 30;
      for (int k : S.owners) pc = std::min(pc, m.p[k]);
      bool ok = true;
      for (int k : S.slaves) ok = ok && pc <= m.p[k];
      if (ok) return true;
    }
    return false;
  }

  // 0 interior, 1 J, 2 E
  std::vector<int8_t> classify() {
    std::vector<int8_t> kind(m.off[m.n], 0);
    std::vector<int8_t> good(m.masters.size());
    for (size_t i = 0; i < m.masters.size(); ++i) good[i] = master_good((int)i) ? 1 : 0;
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k];
      for (int iy = 0; iy <= P; ++iy)
        for (int ix = 0; ix <= P; ++ix) {
          const int64_t row = m.off[k] + iy * (P + 1) + ix;
          const bool bx = (ix == 0 || ix == P), by = (iy == 0 || iy == P);
          if (!bx && !by) continue;
          if (bx && by) {
            int x, y, side = 0;
            corner_xy(k, ix, iy, x, y);
            const int e = m.containing_side(x, y, &side);
            kind[row] = (e < 0 || good[m.side_master[4 * e + side]]) ? 1 : 2;
          } else {
            kind[row] = good[m.side_master[4 * k + node_side(P, ix, iy)]] ? 1 : 2;
          }
        }
    }
    return kind;
  }
};

int64_t find_root(std::vector<int64_t>& parent, int64_t a) {
  while (parent[a] != a) {
    parent[a] = parent[parent[a]];
    a = parent[a];
  }
  return a;
}

}  // namespace

HostPrecond build_host_precond(const dg_mesh& M, const dg_options& o) {
  const HostMesh& m = M.host;
  HostPrecond H;
  const bool timing = std::getenv("DG_SETUP_TIMING") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!timing) return;
    auto t1 = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[setup] %-12s %8.3f s\n", what, std::chrono::duration<double>(t1 - t0).count());
    t0 = t1;
  };
  Builder B(M, o.remark_cases != 0);
  B.number();
  lap("number");
  H.nC = B.nC;
  H.P = B.build_P();
  lap("P");
  H.kind = B.classify();
  lap("classify");
  if (o.smoother == DG_SMOOTHER_JACOBI_ONLY)
    for (auto& k : H.kind)
      if (k == 2) k = 1;
  const int64_t n = m.off[m.n];
  // ---- V_e: union of E nodes sharing a sub-face
  std::vector<int64_t> parent(n);
  std::iota(parent.begin(), parent.end(), 0);
  auto side_nodes = [&](int64_t k, int s, std::vector<int64_t>& out) {
    const int P = m.p[k];
    for (int i = 0; i <= P; ++i) {
      int ix, iy;
      if (s < 2) { ix = (s == 1) ? P : 0; iy = i; }
      else { iy = (s == 3) ? P : 0; ix = i; }
      const int64_t r = m.off[k] + iy * (P + 1) + ix;
      if (H.kind[r] == 2) out.push_back(r);
    }
  };
  std::vector<int64_t> mem;
  for (int64_t k = 0; k < m.n; ++k)
    for (int s = 0; s < 4; ++s)
      for (int j = m.sf_ptr[4 * k + s]; j < m.sf_ptr[4 * k + s + 1]; ++j) {
        mem.clear();
        side_nodes(k, s, mem);
        const auto& f = m.sf[j];
        if (f.nb >= 0) side_nodes(f.nb, f.nb_side, mem);
        for (size_t t = 1; t < mem.size(); ++t) {
          int64_t a = find_root(parent, mem[0]), b = find_root(parent, mem[t]);
          if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
      }
  std::unordered_map<int64_t, int32_t> comp;
  for (int64_t r = 0; r < n; ++r) {
    if (H.kind[r] != 2) continue;
    const int64_t root = find_root(parent, r);
    auto it = comp.find(root);
    if (it == comp.end()) {
      it = comp.emplace(root, (int32_t)H.blocks.size()).first;
      H.blocks.emplace_back();
    }
    H.blocks[it->second].push_back(r);
  }
  lap("components");
  // ---- entries of A: diagonal on V_J and the V_e blocks, read off element rows
  H.dinv.assign(n, 0.0);
  std::vector<double> y((kMaxN) * (kMaxN));
  for (int64_t k = 0; k < m.n; ++k) {
    const int P = m.p[k], NN = (P + 1) * (P + 1);
    host_element_diag(M, k, y.data());
    for (int i = 0; i < NN; ++i) {
      const int64_t r = m.off[k] + i;
      if (H.kind[r] != 1) continue;
      if (!(y[i] > 0.0)) throw Error(DG_EINVAL, "non-positive diagonal");
      H.dinv[r] = 1.0 / y[i];
    }
  }
  lap("diagonal");
  auto elem_of = [&](int64_t r) {
    return (int64_t)(std::upper_bound(m.off.begin(), m.off.end(), r) - m.off.begin() - 1);
  };
  // one block at a time per thread (each block's entries and inverse are
  // computed the same way on any thread)
  H.block_inv.resize(H.blocks.size());
  auto block_range = [&](size_t first, size_t step) {
    SerialSetup serial;
    std::vector<double> xs(n, 0.0), ys((kMaxN) * (kMaxN));
    for (size_t bi = first; bi < H.blocks.size(); bi += step) {
      const auto& blk = H.blocks[bi];
      const int d = (int)blk.size();
      std::vector<double> Ab((int64_t)d * d, 0.0);
      std::vector<int64_t> el(d);
      for (int a = 0; a < d; ++a) el[a] = elem_of(blk[a]);
      std::vector<int64_t> uel(el);
      std::sort(uel.begin(), uel.end());
      uel.erase(std::unique(uel.begin(), uel.end()), uel.end());
      for (int b = 0; b < d; ++b) {
        xs[blk[b]] = 1.0;
        const int64_t kb = el[b];
        // rows that can see column b: its own element and the elements sharing a sub-face
        std::vector<int64_t> near{kb};
        for (int j = m.sf_ptr[4 * kb]; j < m.sf_ptr[4 * kb + 4]; ++j)
          if (m.sf[j].nb >= 0) near.push_back(m.sf[j].nb);
        std::sort(near.begin(), near.end());
        near.erase(std::unique(near.begin(), near.end()), near.end());
        for (int64_t k : near) {
          if (!std::binary_search(uel.begin(), uel.end(), k)) continue;
          host_element_residual(M, k, xs.data(), ys.data(), kb);   // x = e_b lives in kb
          for (int a = 0; a < d; ++a)
            if (el[a] == k) Ab[(int64_t)a * d + b] = ys[blk[a] - m.off[k]];
        }
        xs[blk[b]] = 0.0;
      }
      // symmetrise the round-off before the inverse
      for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) {
          const double s = 0.5 * (Ab[(int64_t)a * d + b] + Ab[(int64_t)b * d + a]);
          Ab[(int64_t)a * d + b] = Ab[(int64_t)b * d + a] = s;
        }
      dense_inverse_spd(d, Ab);
      H.block_inv[bi] = std::move(Ab);
    }
  };
  {
    const int nth = H.blocks.size() >= 64 ? std::min<int>((int)H.blocks.size(), setup_threads()) : 1;
    if (nth <= 1) {
      block_range(0, 1);
    } else {
      std::vector<std::thread> pool;
      std::vector<std::string> errs(nth);
      for (int t = 0; t < nth; ++t)
        pool.emplace_back([&, t] {
          try {
            block_range((size_t)t, (size_t)nth);
          } catch (const std::exception& e) {
            errs[t] = e.what();
          }
        });
      for (auto& th : pool) th.join();
      for (auto& e : errs)
        if (!e.empty()) throw Error(DG_EINVAL, e);
    }
  }
  lap("blocks");
  // ---- LOR: Q1 stiffness on the Gauss-Lobatto sub-grid of each element
  // (block diagonal A~ on the DG numbering), A~_C = P^T A~ P
  {
    Csr At;
    At.rows = At.cols = n;
    At.ptr.assign(n + 1, 0);
    const double m1[2][2] = {{2.0 / 6.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 6.0}};
    const double k1[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    std::vector<double> blk;
    for (int64_t k = 0; k < m.n; ++k) {
      const int P = m.p[k], NP = P + 1;
      const auto& g = basis1d(P).nodes;
      if (m.mapped) {   // Q1 on the mapped cells: the dense block, read in the same stencil
        blk.resize((size_t)NP * NP * NP * NP);
        host_lor_block_map(M, k, blk.data());
      }
      // local stencil: node (i, j) couples to (i+di, j+dj), |di|,|dj| <= 1
      for (int j = 0; j < NP; ++j)
        for (int i = 0; i < NP; ++i) {
          double row[3][3] = {{0}};
          if (m.mapped) {
            for (int dj = 0; dj < 3; ++dj)
              for (int di = 0; di < 3; ++di) {
                const int ii = i + di - 1, jj = j + dj - 1;
                if (ii < 0 || jj < 0 || ii > P || jj > P) continue;
                row[dj][di] = blk[(size_t)(j * NP + i) * NP * NP + jj * NP + ii];
              }
          }
          for (int cj = j - 1; cj <= j && !m.mapped; ++cj)
            for (int ci = i - 1; ci <= i; ++ci) {
              if (ci < 0 || cj < 0 || ci >= P || cj >= P) continue;
              const double a = g[ci + 1] - g[ci], b = g[cj + 1] - g[cj];
              const int px = i - ci, py = j - cj;   // this node's corner in the cell
              for (int qy = 0; qy < 2; ++qy)
                for (int qx = 0; qx < 2; ++qx)
                  row[cj + qy - j + 1][ci + qx - i + 1] +=
                      (b / a) * m1[py][qy] * k1[px][qx] + (a / b) * k1[py][qy] * m1[px][qx];
            }
          for (int dj = 0; dj < 3; ++dj)
            for (int di = 0; di < 3; ++di) {
              const int ii = i + di - 1, jj = j + dj - 1;
              if (ii < 0 || jj < 0 || ii > P || jj > P) continue;
              At.idx.push_back((int32_t)(m.off[k] + jj * NP + ii));
              At.val.push_back(m.coef[k] * row[dj][di]);   // weighted by a_k
            }
          At.ptr[m.off[k] + j * NP + i + 1] = (int64_t)At.idx.size();
        }
    }
    lap("lor-local");
    H.Ac = csr_multiply(csr_transpose(H.P), csr_multiply(At, H.P));
    lap("lor-spgemm");
  }
  return H;
}

}  // namespace dg
