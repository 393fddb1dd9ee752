// Internal data structures of the hp-DG library (host + device).
#pragma once

#include <cmath>
#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dg.h"

namespace dg {

constexpr int kMaxP = 8;
constexpr int kMaxN = kMaxP + 1;
constexpr int kThreads = 256;   // threads per CTA of the operator kernel
// elements of degree p per operator CTA (one thread per node, at most 16)
constexpr int apply_epb(int p) {
  return (kThreads / ((p + 1) * (p + 1))) > 16 ? 16 : (kThreads / ((p + 1) * (p + 1)));
}

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  dg_status code;
  Error(dg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
void set_last_error(const std::string& msg);
#define DG_REQUIRE(cond, msg) \
  do { if (!(cond)) throw ::dg::Error(DG_EINVAL, msg); } while (0)
#define DG_CUDA(call)                                                            \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      throw ::dg::Error(e_ == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

// ------------------------------------------------------------------ basis (host)
// Gauss-Lobatto nodes on [0,1] (Section 2.2), Gauss-Legendre rules, Lagrange
// values by the barycentric formula.
std::vector<double> gll_nodes(int p);
void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w);
// values l_j(t), j = 0..n-1, of the Lagrange basis on `nodes` at t
void lagrange_eval(const std::vector<double>& nodes, double t, double* out);
void lagrange_deriv_eval(const std::vector<double>& nodes, double t, double* out);

// 1D reference matrices of degree p on [0,1] (exact Gauss integration)
struct Basis1D {
  int p;
  std::vector<double> nodes;   // p+1
  std::vector<double> M, K;    // (p+1)^2 row-major, exact mass / stiffness
  std::vector<double> Minv;    // inverse of M
  std::vector<double> d0, d1;  // l_k'(0), l_k'(1)
};
const Basis1D& basis1d(int p);

// ------------------------------------------------------------------ device records
// One sub-face seen from one of its sides (the "own" element).
struct SubFaceRec {
  int32_t nb;        // neighbour element, -1 on the boundary
  int32_t nb_side;   // neighbour side holding the sub-face
  int32_t pn;        // neighbour degree
  int32_t tab_oo;    // offset of the own-own face mass (ref, (p+1)^2)
  int32_t tab_on;    // offset of own-neighbour face mass ((p+1) x (pn+1))
  int32_t tab_nn;    // offset of neighbour-neighbour face mass ((pn+1)^2)
  double sigma;      // SIPG penalty
  double len;        // physical length of the sub-face
};

// BR2 lifting of one sub-face of a square mesh, multiplied out (beside the
// SubFaceRec of the same index): the stabilisation residual at own side node
// i is cz [(Z u-)_i - (V u+)_i] + cx [(X u-)_i - (Y u+)_i] with the products
// of the face tables and the 1D mass inverses Minv (own), Minv_n (neighbour)
//   Z = M_oo Minv M_oo, V = M_oo Minv M_on, X = M_on Minv_n M_no, Y = M_on Minv_n M_nn
// and cz, cx = eta coef len^2 a Minv_00 / h^2 of the own / neighbour element
// (coef 1/4 inside, 1 on the boundary; a the larger coefficient of the two
// sides).  On a sub-face that is the own element's whole side M_oo is the 1D
// mass matrix, so Z = M_oo and V = M_on; on the neighbour's whole side Y = M_on.
struct SubFaceBr2 {
  int32_t tab_z, tab_v, tab_x, tab_y;   // table offsets ((p+1) x (p+1) or (p+1) x (pn+1))
  int32_t full;                         // bit 0: own whole side, bit 1: neighbour's whole side
  int32_t pad;
  double cz, cx;
};

// One sub-face of a cube mesh seen from one of its sides.  The sub-face is a
// square; its face integrals factor into two 1D tables, one per tangential
// axis of the side (the lower-numbered axis first).
struct SubFaceRec3 {
  int32_t nb;        // neighbour element, -1 on the boundary
  int32_t nb_side;   // neighbour side holding the sub-face
  int32_t pn;        // neighbour degree
  int32_t full;      // bit 0: the sub-face is the own element's whole face, bit 1: the neighbour's
  int32_t tab_oo[2]; // own-own 1D face mass per tangential axis ((p+1)^2)
  int32_t tab_on[2]; // own-neighbour ((p+1) x (pn+1))
  int32_t tab_nn[2]; // neighbour-neighbour ((pn+1)^2)
  // BR2 lifting products per tangential axis (Minv: 1D mass inverse):
  //   Z = M_oo Minv M_oo, V = M_oo Minv M_on, X = M_on Minv_n M_no, Y = M_on Minv_n M_nn
  // (on a whole own face M_oo is the 1D mass matrix, so Z = M_oo and V = M_on;
  // on a whole neighbour face likewise Y = M_on)
  int32_t tab_z[2], tab_v[2], tab_x[2], tab_y[2];
  double sigma;      // SIPG penalty
  double area;       // physical area of the sub-face
  double cz, cx;     // BR2: a eta coef area^2 Minv_00 / h^3 of the own / neighbour element,
                     // a the larger coefficient of the sub-face's two sides
};

// Shared-memory budget (doubles) of one 3D operator tile; the host sizes the
// tiles and their sub-face item chunks so that every one fits.
constexpr int kApply3Budget = 9 * 1024;
constexpr int kApply3MinChunk = 12;   // sub-face items a tile keeps room for
// doubles of shared memory one element of degree p needs in a 3D tile (volume
// passes and the per-side residual and normal-derivative coefficients)
constexpr int apply3_elem_doubles(int p) {
  return 5 * (p + 1) * (p + 1) * (p + 1) + 12 * (p + 1) * (p + 1);
}
// doubles one sub-face item needs: first-pass scratch ((p+1) x nq per product,
// nq = max(p, pn) + 1) and its two partial side arrays
constexpr int apply3_item_doubles(int p, int nq, bool br2) {
  return (br2 ? 8 : 4) * (p + 1) * nq + 2 * (p + 1) * (p + 1);
}

// Offsets of the degree-p 1D matrices inside the device table buffer.
struct BasisOff {
  int M, K, Minv, d0, d1;
};

// Per-CTA work item of the operator kernel: a run of elements of one degree.
struct ApplyTile {
  int32_t p;
  int32_t first;     // index into the degree-sorted element order
  int32_t count;
  int32_t inst;      // batch instance of the tile's elements (0 for a single mesh)
  int32_t nq;        // 3D: max(p, neighbour degrees) + 1 over the tile
  int32_t chunk;     // 3D: sub-face items processed at a time
};

// ------------------------------------------------------------------ mapped squares
// The bilinear map of the lattice domain onto a quadrilateral (dg_mesh_desc
// corners c0..c3, the images of (0,0), (Lx,0), (0,Ly), (Lx,Ly)).  In the
// pre-image coordinates (X, Y) its Jacobian columns are
//   dPhi/dX = u1 + Y u3,  dPhi/dY = u2 + X u3,
// u1 = (c1 - c0) / Lx, u2 = (c2 - c0) / Ly, u3 = (c3 - c2 - c1 + c0) / (Lx Ly).
struct DomainMap {
  double u1x, u1y, u2x, u2y, u3x, u3y;
};
// the Jacobian of the domain map at the pre-image point (X, Y):
// j0 = dx/dX, j1 = dx/dY, j2 = dy/dX, j3 = dy/dY
struct Jac2 {
  double j0, j1, j2, j3;
};
__host__ __device__ inline Jac2 domain_jacobian(const DomainMap& D, double X, double Y) {
  return Jac2{D.u1x + Y * D.u3x, D.u2x + X * D.u3x, D.u1y + Y * D.u3y, D.u2y + X * D.u3y};
}
// Gauss points per direction of the mapped integrals: p + 2 on the volume,
// max(p-, p+) + 2 on a sub-face
constexpr int kMapQExtra = 1;
constexpr int kMapQMax = kMaxP + 1 + kMapQExtra;

// One sub-face of a mapped square mesh seen from one side (beside the
// SubFaceRec of the same index): its Gauss rule size, both sides' 1D basis
// values and derivatives at the rule's points, its geometric factors and its
// penalty.
struct SubFaceMap {
  int32_t qf;       // Gauss points, max(p, pn) + 2
  int32_t tab_bo;   // own side: l_i(s_g) (qf rows of p+1), then l_i'(s_g)
  int32_t tab_bn;   // the neighbour's side, the same with pn (boundary: tab_bo)
  int32_t geo;      // offset of the point factors in the face geometry: qf values of
                    // w = w_g |J t| dt, then w m_t, then w m_n s (m = J^-1 n in the
                    // pre-image axes, s = +1 / -1 for an upper / lower side)
  double sigma;     // SIPG penalty with h_kappa = sqrt(area of kappa)
  double cbr2;      // BR2: eta coef a (coef 1/4 inside, 1 on the boundary; a the
                    // larger coefficient of the two sides), 0 for SIPG
};

// Offsets of the degree-p volume tables of mapped meshes: the (p+2)-point
// Gauss rule (points, weights) and l_j, l_j' at its points ((p+2) x (p+1)).
struct MapOff {
  int gx, gw, B, D;
};

// ------------------------------------------------------------------ mesh (host topology)
// a_kappa of every element from a mesh description (all 1 when coeff is NULL)
inline void copy_coeff(const dg_mesh_desc* d, std::vector<double>& coef) {
  coef.assign(d->n_elems, 1.0);
  if (!d->coeff) return;
  for (int64_t k = 0; k < d->n_elems; ++k) {
    const double a = d->coeff[k];
    if (!(a > 0.0) || !std::isfinite(a)) throw Error(DG_EINVAL, "coefficient must be positive and finite");
    coef[k] = a;
  }
}

struct HostMesh {
  int dim = 2;
  int64_t n = 0;
  std::vector<int32_t> lo;      // n*dim
  std::vector<int32_t> size;    // n
  std::vector<int32_t> p;       // n
  int32_t extent[3] = {0, 0, 1};
  double lh = 1.0;
  std::vector<double> coef;     // n coefficients a (1 when none given)
  bool mapped = false;          // squares carried by the bilinear map of `corners`
  double corners[8] = {0.0};    // images of (0,0), (Lx,0), (0,Ly), (Lx,Ly), (x, y) each
  std::vector<int64_t> off;     // n+1 DOF offsets
  std::vector<int32_t> cellmap; // lattice cell (x fastest) -> element

  // 3D: sub-faces seen from every element side, sf_ptr[6k+s] .. sf_ptr[6k+s+1];
  // a sub-face is the square [a0, a0+len] x [b0, b0+len] in the side's
  // (first, second) tangential lattice coordinates
  struct SF3 { int32_t nb, nb_side, a0, b0, len; };
  std::vector<SF3> sf3;
  int32_t elem_at3(int x, int y, int z) const {
    return cellmap[((int64_t)z * extent[1] + y) * extent[0] + x];
  }

  // sub-faces seen from each element side: sf_ptr[4k+s] .. sf_ptr[4k+s+1]
  std::vector<int32_t> sf_ptr;
  struct SF { int32_t nb, nb_side, t0, t1; };
  std::vector<SF> sf;

  // master edges
  struct Master {
    int axis, c, t0, t1;
    bool boundary;
    int p;                          // min degree of owners and slaves
    std::vector<int32_t> owners, slaves;
    std::vector<std::pair<int,int>> hanging;  // interior hanging vertices
  };
  std::vector<Master> masters;
  std::vector<int32_t> side_master;  // 4n

  int32_t elem_at(int x, int y) const { return cellmap[(int64_t)y * extent[0] + x]; }
  void side_segment(int k, int s, int& axis, int& c, int& t0, int& t1) const;
  bool corner_of(int k, int x, int y) const;
  // element + side containing (x,y) in the relative interior of the side, or -1
  int containing_side(int x, int y, int* side) const;
  // a vertex of the domain boundary: one of the four cells around it is
  // outside the lattice or a hole (no element covers it)
  bool on_boundary(int x, int y) const {
    for (int cy = y - 1; cy <= y; ++cy)
      for (int cx = x - 1; cx <= x; ++cx)
        if (cx < 0 || cy < 0 || cx >= extent[0] || cy >= extent[1] || elem_at(cx, cy) < 0) return true;
    return false;
  }
  bool is_hp_vertex(int x, int y) const;
};

void build_topology(HostMesh& m);   // fills sf, masters, side_master
void build_topology3(HostMesh& m);  // fills sf_ptr (6 per element), sf3

// side s of a cube: normal axis s / 2, upper face if s is odd; tangential axes
// in increasing order
inline void side_axes3(int s, int& ax, int& t0, int& t1) {
  ax = s >> 1;
  t0 = (ax == 0) ? 1 : 0;
  t1 = (ax == 2) ? 1 : 2;
}

// Face-mass tables (Section 2: exact face integrals on sub-faces).
struct FaceTables {
  std::vector<double> data;
  std::map<std::tuple<int,int,int,int,int,int>, int> index;
  int get(int p, int L, int off, int pn, int Ln, int offn);
};

}  // namespace dg

