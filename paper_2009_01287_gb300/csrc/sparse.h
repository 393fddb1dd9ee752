// Small host CSR toolkit for the preconditioner setup (LOR triple product and
// the smoothed-aggregation hierarchy).
#pragma once

#include <cstdint>
#include <vector>

namespace dg {

struct Csr {
  int64_t rows = 0, cols = 0;
  std::vector<int64_t> ptr;   // rows+1
  std::vector<int32_t> idx;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)idx.size(); }
};

// Triplets -> CSR with duplicates summed and columns sorted.
Csr csr_from_triplets(int64_t rows, int64_t cols, std::vector<int64_t>& r,
                      std::vector<int32_t>& c, std::vector<double>& v);
Csr csr_transpose(const Csr& A);
Csr csr_multiply(const Csr& A, const Csr& B);   // sorted columns, exact zeros kept
// While an instance lives, csr_multiply on this thread stays on it (callers
// that already run one setup per thread, like the batched solver's, keep the
// machine from being oversubscribed).  Results are the same either way.
struct SerialSetup {
  SerialSetup();
  ~SerialSetup();
  bool prev;
};
// Threads a setup step may use on this thread: 1 under SerialSetup, else the
// hardware threads (at most 16).
int setup_threads();

// Deterministic smoothed-aggregation AMG hierarchy (setup only).
struct AmgLevel {
  Csr A;
  std::vector<double> dl1;   // l1-Jacobi diagonal sum_j |a_ij|
  Csr P, R;                  // prolongator to this level from the next, R = P^T
  // The V-cycle of this level rewritten with composite operators (D = diag(dl1)):
  //   b_next = Rpre b,           Rpre = R (I - A D^-1)
  //   x_out  = Sb b + Sp x_next, Sb = 2 D^-1 - D^-1 A D^-1, Sp = (I - D^-1 A) P
  // which is pre-smoothing x = D^-1 b, restriction of b - A x, coarse
  // correction x += P x_next and post-smoothing x += D^-1 (b - A x) exactly.
  Csr Rpre, Sb, Sp;
};
struct AmgHierarchy {
  std::vector<AmgLevel> levels;
  std::vector<double> coarse_inv;  // dense inverse of the last level (row-major)
};

constexpr double kAmgTheta = 0.08;    // squares: the Q1 9-point stencil's links are strong
constexpr double kAmgTheta3 = 0.02;   // cubes: trilinear 27-point links are ~1/32 of the diagonal
constexpr int kAmgCoarseMax = 1024;
constexpr int kAmgMaxLevels = 12;
constexpr int kAmgDenseMax = 8192;    // largest coarsest level inverted densely
// A level whose continuing rows hold more nonzeros than this is applied in the
// plain form (A, R, P: about half the matrix bytes of the composite operators,
// which pays when the level is bandwidth-bound); smaller levels, bound by
// launch latency, keep the two-kernel composite form.
constexpr int64_t kAmgPlainNnz = 4000000;
// Largest product W = (coarsest inverse) Rpre (entries) that replaces the last
// composite restriction and the dense coarsest solve by one dense product.
constexpr int64_t kCoarseFuseMax = 4000000;

AmgHierarchy amg_setup(const Csr& A, double theta = kAmgTheta);
void dense_inverse_spd(int n, std::vector<double>& a);  // in place, Cholesky based

}  // namespace dg
