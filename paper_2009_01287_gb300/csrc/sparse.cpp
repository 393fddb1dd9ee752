// Host CSR utilities and the smoothed-aggregation AMG setup used as the LOR
// conforming solver (Section 3.4 uses one AMG V-cycle on P^T A~ P).
//
// AMG algorithm (fixed so that it is deterministic):
//   strength   j != i strong for i  iff  a_ij^2 > theta^2 a_ii a_jj
//              (theta = 0.08 on squares, 0.02 on cubes)
//   pass 1     i unaggregated with >= 1 strong neighbour, all of them
//              unaggregated: new aggregate {i} + strong neighbours
//   pass 2     i unaggregated: joins the pass-1 aggregate of its
//              lowest-numbered strong neighbour that has one
//   pass 3     i still unaggregated: new aggregate {i} + its unaggregated
//              strong neighbours
//   smoothing  P = (I - omega D^-1 A) T, omega = 4/(3 rho),
//              rho = max_i sum_j |a_ij| / a_ii
//   coarse     A_c = P^T A P; stop at <= kAmgCoarseMax rows, when a level
//              does not shrink below 0.9 n, or at kAmgMaxLevels levels; the
//              last level is inverted densely.
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <chrono>
#include <thread>
#include <cmath>
#include <numeric>

#include "dg_internal.h"
#include "sparse.h"

namespace dg {

Csr csr_from_triplets(int64_t rows, int64_t cols, std::vector<int64_t>& r,
                      std::vector<int32_t>& c, std::vector<double>& v) {
  Csr A;
  A.rows = rows;
  A.cols = cols;
  std::vector<int64_t> order(r.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return r[a] != r[b] ? r[a] < r[b] : c[a] < c[b];
  });
  A.ptr.assign(rows + 1, 0);
  for (size_t t = 0; t < order.size();) {
    size_t u = t;
    double s = 0.0;
    while (u < order.size() && r[order[u]] == r[order[t]] && c[order[u]] == c[order[t]]) {
      s += v[order[u]];
      ++u;
    }
    A.idx.push_back(c[order[t]]);
    A.val.push_back(s);
    A.ptr[r[order[t]] + 1]++;
    t = u;
  }
  for (int64_t i = 0; i < rows; ++i) A.ptr[i + 1] += A.ptr[i];
  return A;
}

Csr csr_transpose(const Csr& A) {
  Csr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.ptr.assign(T.rows + 1, 0);
  for (int32_t c : A.idx) T.ptr[c + 1]++;
  for (int64_t i = 0; i < T.rows; ++i) T.ptr[i + 1] += T.ptr[i];
  T.idx.resize(A.idx.size());
  T.val.resize(A.val.size());
  std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.rows; ++i)
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
      int64_t d = pos[A.idx[t]]++;
      T.idx[d] = (int32_t)i;
      T.val[d] = A.val[t];
    }
  return T;
}

namespace {

// rows [r0, r1) of C = A B: per row the columns in increasing order and the
// sums in the order of A's row and B's rows (the same whatever the split)
void multiply_rows(const Csr& A, const Csr& B, int64_t r0, int64_t r1, std::vector<int64_t>& cnt,
                   std::vector<int32_t>& idx, std::vector<double>& val) {
  std::vector<int64_t> mark(B.cols, -1);
  std::vector<double> acc(B.cols, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = r0; i < r1; ++i) {
    cols.clear();
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
      const int32_t a = A.idx[t];
      const double av = A.val[t];
      for (int64_t u = B.ptr[a]; u < B.ptr[a + 1]; ++u) {
        const int32_t b = B.idx[u];
        if (mark[b] != i) {
          mark[b] = i;
          acc[b] = 0.0;
          cols.push_back(b);
        }
        acc[b] += av * B.val[u];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t b : cols) {
      idx.push_back(b);
      val.push_back(acc[b]);
    }
    cnt[i - r0] = (int64_t)cols.size();
  }
}

thread_local bool t_serial = false;

}  // namespace

SerialSetup::SerialSetup() : prev(t_serial) { t_serial = true; }
SerialSetup::~SerialSetup() { t_serial = prev; }

int setup_threads() {
  return t_serial ? 1 : (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
}

Csr csr_multiply(const Csr& A, const Csr& B) {
  Csr C;
  C.rows = A.rows;
  C.cols = B.cols;
  C.ptr.assign(A.rows + 1, 0);
  // large products are split into row ranges of about equal work (A's
  // nonzeros) computed by threads; every row is computed exactly as in one
  // pass, so the result does not depend on the split
  const int nth = A.nnz() > (1 << 16) ? setup_threads() : 1;
  if (nth <= 1) {
    std::vector<int64_t> cnt(A.rows);
    multiply_rows(A, B, 0, A.rows, cnt, C.idx, C.val);
    for (int64_t i = 0; i < A.rows; ++i) C.ptr[i + 1] = C.ptr[i] + cnt[i];
    return C;
  }
  std::vector<int64_t> cut(nth + 1, A.rows);
  cut[0] = 0;
  for (int t = 1; t < nth; ++t) {
    const int64_t target = A.nnz() * t / nth;
    cut[t] = std::upper_bound(A.ptr.begin(), A.ptr.end(), target) - A.ptr.begin() - 1;
    cut[t] = std::max(cut[t], cut[t - 1]);
  }
  std::vector<std::vector<int64_t>> cnt(nth);
  std::vector<std::vector<int32_t>> idx(nth);
  std::vector<std::vector<double>> val(nth);
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) {
    cnt[t].resize(cut[t + 1] - cut[t]);
    pool.emplace_back([&, t] { multiply_rows(A, B, cut[t], cut[t + 1], cnt[t], idx[t], val[t]); });
  }
  for (auto& th : pool) th.join();
  for (int t = 0; t < nth; ++t) {
    for (int64_t i = cut[t]; i < cut[t + 1]; ++i) C.ptr[i + 1] = C.ptr[i] + cnt[t][i - cut[t]];
    C.idx.insert(C.idx.end(), idx[t].begin(), idx[t].end());
    C.val.insert(C.val.end(), val[t].begin(), val[t].end());
  }
  return C;
}

void dense_inverse_spd(int n, std::vector<double>& a) {
  // Cholesky A = L L^T, then A^-1 = L^-T L^-1 column by column.  Every entry
  // is one fixed sequence of operations (sums in ascending k); rows of L are
  // formed four at a time and the columns of the inverse four at a time (on
  // several threads when n is large) only to overlap independent sums, so the
  // result does not depend on the grouping or the thread count.
  std::vector<double> L(a);
  for (int j = 0; j < n; ++j) {
    const double* Lj = &L[(int64_t)j * n];
    double d = Lj[j];
    for (int k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
    if (!(d > 0.0)) throw Error(DG_EINVAL, "matrix not positive definite");
    d = std::sqrt(d);
    L[(int64_t)j * n + j] = d;
    int i = j + 1;
    for (; i + 4 <= n; i += 4) {
      double* R0 = &L[(int64_t)i * n];
      double *R1 = R0 + n, *R2 = R1 + n, *R3 = R2 + n;
      double s0 = R0[j], s1 = R1[j], s2 = R2[j], s3 = R3[j];
      for (int k = 0; k < j; ++k) {
        const double l = Lj[k];
        s0 -= R0[k] * l;
        s1 -= R1[k] * l;
        s2 -= R2[k] * l;
        s3 -= R3[k] * l;
      }
      R0[j] = s0 / d;
      R1[j] = s1 / d;
      R2[j] = s2 / d;
      R3[j] = s3 / d;
    }
    for (; i < n; ++i) {
      double* Ri = &L[(int64_t)i * n];
      double s = Ri[j];
      for (int k = 0; k < j; ++k) s -= Ri[k] * Lj[k];
      Ri[j] = s / d;
    }
  }
  // L^T row by row, so that the backward solves read contiguous memory
  std::vector<double> Lt((int64_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = i; k < n; ++k) Lt[(int64_t)i * n + k] = L[(int64_t)k * n + i];
  constexpr int W = 4;
  auto solve_columns = [&](int c0, int c1) {
    std::vector<double> col((int64_t)n * W);   // col[i * W + r]: column c + r
    for (int c = c0; c < c1; c += W) {
      const int w = std::min(W, c1 - c);
      // L y = e_c
      for (int i = 0; i < n; ++i) {
        const double* Li = &L[(int64_t)i * n];
        double s[W];
        for (int r = 0; r < W; ++r) s[r] = (i == c + r) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) {
          const double l = Li[k];
          for (int r = 0; r < W; ++r) s[r] -= l * col[(int64_t)k * W + r];
        }
        for (int r = 0; r < W; ++r) col[(int64_t)i * W + r] = s[r] / Li[i];
      }
      // L^T z = y
      for (int i = n - 1; i >= 0; --i) {
        const double* Ti = &Lt[(int64_t)i * n];
        double s[W];
        for (int r = 0; r < W; ++r) s[r] = col[(int64_t)i * W + r];
        for (int k = i + 1; k < n; ++k) {
          const double l = Ti[k];
          for (int r = 0; r < W; ++r) s[r] -= l * col[(int64_t)k * W + r];
        }
        for (int r = 0; r < W; ++r) col[(int64_t)i * W + r] = s[r] / Ti[i];
      }
      for (int i = 0; i < n; ++i)
        for (int r = 0; r < w; ++r) a[(int64_t)i * n + c + r] = col[(int64_t)i * W + r];
    }
  };
  const int nth = n >= 256 ? setup_threads() : 1;
  const int nblk = (n + W - 1) / W;
  if (nth <= 1) {
    solve_columns(0, n);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) {
    const int c0 = (int)((int64_t)nblk * t / nth) * W;
    const int c1 = std::min(n, (int)((int64_t)nblk * (t + 1) / nth) * W);
    if (c0 < c1) pool.emplace_back(solve_columns, c0, c1);
  }
  for (auto& th : pool) th.join();
}

namespace {

std::vector<int32_t> aggregate(const Csr& A, double theta) {
  const int64_t n = A.rows;
  std::vector<double> diag(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t)
      if (A.idx[t] == i) diag[i] = A.val[t];
  // strong neighbour lists (columns ascending)
  std::vector<int64_t> sptr(n + 1, 0);
  std::vector<int32_t> sidx;
  const double th2 = theta * theta;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
      const int32_t j = A.idx[t];
      if (j == i) continue;
      const double v = A.val[t];
      if (v * v > th2 * diag[i] * diag[j]) sidx.push_back(j);
    }
    sptr[i + 1] = (int64_t)sidx.size();
  }
  std::vector<int32_t> agg(n, -1);
  int32_t na = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0 || sptr[i + 1] == sptr[i]) continue;
    bool free_all = true;
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t)
      if (agg[sidx[t]] >= 0) { free_all = false; break; }
    if (!free_all) continue;
    agg[i] = na;
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t) agg[sidx[t]] = na;
    ++na;
  }
  std::vector<int32_t> after1(agg);
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t)
      if (after1[sidx[t]] >= 0) { agg[i] = after1[sidx[t]]; break; }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t)
      if (agg[sidx[t]] < 0) agg[sidx[t]] = na;
    ++na;
  }
  return agg;
}

std::vector<double> l1_diag(const Csr& A) {
  std::vector<double> d(A.rows, 0.0);
  for (int64_t i = 0; i < A.rows; ++i)
    for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) d[i] += std::fabs(A.val[t]);
  return d;
}

}  // namespace

AmgHierarchy amg_setup(const Csr& A0, double theta) {
  const bool timing = std::getenv("DG_SETUP_TIMING") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!timing) return;
    auto t1 = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[amg]    %-12s %8.3f s\n", what, std::chrono::duration<double>(t1 - t0).count());
    t0 = t1;
  };
  AmgHierarchy H;
  H.levels.push_back({A0, l1_diag(A0), {}, {}});
  while (true) {
    AmgLevel& L = H.levels.back();
    const int64_t n = L.A.rows;
    if (n <= kAmgCoarseMax || (int)H.levels.size() >= kAmgMaxLevels) break;
    std::vector<int32_t> agg = aggregate(L.A, theta);
    lap("aggregate");
    int64_t nc = 0;
    for (int32_t a : agg) nc = std::max<int64_t>(nc, a + 1);
    if ((double)nc >= 0.9 * (double)n) break;
    std::vector<double> diag(n, 0.0);
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t t = L.A.ptr[i]; t < L.A.ptr[i + 1]; ++t) {
        if (L.A.idx[t] == i) diag[i] = L.A.val[t];
        s += std::fabs(L.A.val[t]);
      }
      rho = std::max(rho, s / diag[i]);
    }
    const double omega = 4.0 / (3.0 * rho);
    // P = (I - omega D^-1 A) T: row i, column agg[j] gets delta_ij - omega a_ij / a_ii
    std::vector<int64_t> r;
    std::vector<int32_t> c;
    std::vector<double> v;
    for (int64_t i = 0; i < n; ++i) {
      r.push_back(i);
      c.push_back(agg[i]);
      v.push_back(1.0);
      for (int64_t t = L.A.ptr[i]; t < L.A.ptr[i + 1]; ++t) {
        r.push_back(i);
        c.push_back(agg[L.A.idx[t]]);
        v.push_back(-omega * L.A.val[t] / diag[i]);
      }
    }
    Csr P = csr_from_triplets(n, nc, r, c, v);
    lap("P");
    Csr R = csr_transpose(P);
    Csr Ac = csr_multiply(R, csr_multiply(L.A, P));
    lap("RAP");
    L.P = std::move(P);
    L.R = std::move(R);
    AmgLevel next{std::move(Ac), {}, {}, {}};
    next.dl1 = l1_diag(next.A);
    H.levels.push_back(std::move(next));
  }
  // composite operators of every level that continues, except the levels
  // the device applies in the plain form anyway (more than kAmgPlainNnz
  // nonzeros: so many in any union of instances that holds this level)
  for (size_t l = 0; l + 1 < H.levels.size(); ++l) {
    AmgLevel& L = H.levels[l];
    const Csr& A = L.A;
    if (A.nnz() > kAmgPlainNnz) continue;
    const std::vector<double>& d = L.dl1;
    Csr M1 = A, M2 = A, Sb = A;   // I - A D^-1, I - D^-1 A, 2 D^-1 - D^-1 A D^-1
    for (int64_t i = 0; i < A.rows; ++i)
      for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
        const int32_t j = A.idx[t];
        const double a = A.val[t];
        M1.val[t] = (i == j ? 1.0 : 0.0) - a / d[j];
        M2.val[t] = (i == j ? 1.0 : 0.0) - a / d[i];
        Sb.val[t] = (i == j ? 2.0 / d[i] : 0.0) - a / (d[i] * d[j]);
      }
    L.Rpre = csr_multiply(L.R, M1);
    L.Sp = csr_multiply(M2, L.P);
    L.Sb = std::move(Sb);
  }
  lap("composite");
  const Csr& C = H.levels.back().A;
  if (C.rows > kAmgDenseMax)
    throw Error(DG_EUNSUPPORTED, "AMG coarsening stalled above the dense coarse-solve limit");
  const int nc = (int)C.rows;
  H.coarse_inv.assign((int64_t)nc * nc, 0.0);
  for (int64_t i = 0; i < nc; ++i)
    for (int64_t t = C.ptr[i]; t < C.ptr[i + 1]; ++t) H.coarse_inv[i * nc + C.idx[t]] = C.val[t];
  dense_inverse_spd(nc, H.coarse_inv);
  lap("coarse");
  return H;
}

}  // namespace dg
