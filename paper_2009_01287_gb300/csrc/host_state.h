// Definitions of the opaque handles and the device-side views used by the
// kernels.
#pragma once

#include <vector>

#include "dg_internal.h"
#include "sparse.h"

namespace dg {

// device allocation tracked by its owner
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;   // total requested
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    DG_CUDA(cudaMalloc(&p, n * sizeof(T)));
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return (T*)p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* d = alloc<T>(v.size());
    if (!v.empty()) DG_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

// CSR on the device: int32 indices, values of the preconditioner precision
struct DevCsr {
  int64_t rows = 0, nnz = 0;
  int32_t* ptr = nullptr;
  int32_t* idx = nullptr;
  void* val = nullptr;
  int group = 1;       // lanes per row in the group tier (power of two <= 32)
  int group_all = 1;   // lanes per row of the fused AMG up-sweep (set per level from the mean row length)
  // rows read by a whole CTA (more than kCsrCtaRow entries) and by a whole
  // warp (more than long_min entries); the group tier skips both
  int32_t* cta_rows = nullptr;
  int32_t* warp_rows = nullptr;
  int n_cta = 0, n_warp = 0;
  int long_min = 0x7fffffff;
};

// lanes per row for a CSR with the given average row length
inline int csr_group_for(double avg) {
  int g = 1;
  while (g < 32 && g * 2 <= avg) g *= 2;
  return g;
}

// rows with more entries than this are read by a whole CTA in the row kernels
constexpr int kCsrCtaRow = 1024;
// threads resident on the whole GPU at full occupancy (152 SMs x 2048)
constexpr int64_t kResidentThreads = 152 * 2048;

// the CTA and warp tiers of a CSR row kernel launch (see DevCsr)
struct CsrTiers {
  const int32_t* cta_rows;
  const int32_t* warp_rows;
  int n_cta, n_warp;
  int long_min;
};

struct DevLevel {
  int64_t n = 0;
  int64_t n_cont = 0;  // rows [0, n_cont) continue to the next level (smoothed,
                       // restricted); rows [n_cont, n) are coarsest levels of
                       // their problem and are solved densely (blocks below)
  DevCsr Rpre, Sb, Sp;  // composite V-cycle operators on the continuing rows (see AmgLevel)
  // large levels take the plain form instead (fewer matrix bytes, two more
  // launches): A on the continuing rows, R = P^T, P, the l1 diagonal inverse
  // and two work vectors
  bool plain = false;
  DevCsr A, R, P;
  void* dinv = nullptr;
  void* t1 = nullptr;
  void* t2 = nullptr;
  int n_end = 0;                   // dense coarse blocks
  int max_end = 0;                 // largest of them
  int32_t* end_row = nullptr;      // n_end+1 row offsets (level numbering)
  int64_t* end_inv_off = nullptr;  // offsets of the row-major inverses
  void* end_inv = nullptr;
  int64_t end_inv_entries = 0;
  void* b = nullptr;     // right-hand side of this level
  void* xo = nullptr;    // the level's output (after post-smoothing)
  // Coarse fusion (single problem, composite level next to the dense
  // coarsest level): W = (coarsest inverse) Rpre, row-major n_next x n, so the
  // restriction and the coarse solve are one dense product xo_next = W b.
  void* coarse_w = nullptr;
  int64_t coarse_w_rows = 0;
};

}  // namespace dg

struct dg_mesh {
  dg::HostMesh host;
  int device = 0;          // CUDA device current at dg_mesh_create (holds the handle's memory)
  dg_options opts{};
  double eta = 0.0;
  int64_t n_dofs = 0;
  dg_mesh_stats stats{};
  // host copies of what the device holds
  std::vector<double> h_h;
  std::vector<dg::SubFaceRec> h_sf;
  std::vector<dg::SubFaceBr2> h_sfb;    // square meshes, BR2: one per h_sf record
  std::vector<dg::SubFaceRec3> h_sf3;   // cube meshes
  // mapped squares: one record per h_sf record, the volume tables of each
  // degree, the map; the geometric factors at the Gauss points - per element
  // (offset h_goff[k]) the volume factors a w_g w_h G of its (p+2)^2 points as
  // three planes G11, G12, G22; per sub-face record its face factors
  std::vector<dg::SubFaceMap> h_sfm;
  dg::MapOff moff[dg::kMaxP + 1];
  dg::DomainMap dmap{};
  std::vector<double> h_gvol, h_gface;
  std::vector<int64_t> h_goff;
  // BR2 on mapped squares: per element side the block of the element's mass
  // inverse on that side's nodes ((p+1)^2 row-major, four per element, from
  // h_g2off[k])
  std::vector<double> h_gbr2;
  std::vector<int64_t> h_g2off;
  // host only: per element the images of its (p+1)^2 Gauss-Lobatto nodes (the
  // LOR cells' vertices) and, at the (p+3)^2 points of the load-vector rule,
  // the image and det J (x, y, det per point; offsets h_roff), so that no
  // later call needs the caller's map
  std::vector<double> h_xnode, h_xrhs;
  std::vector<int64_t> h_roff;
  // host only: per boundary sub-face record j (h_boff[j] >= 0) at the p+3
  // Gauss points of the element's degree along it: the image (x, y), the
  // weight w |J t| dt and m = J^-1 n of the outward physical normal n (five
  // values per point), for weakly imposed Dirichlet data on mapped meshes
  std::vector<double> h_xbnd;
  std::vector<int64_t> h_boff;
  int64_t apply3_smem = 0;              // dynamic shared memory of the 3D operator kernel
  std::vector<double> h_tables;
  dg::BasisOff boff[dg::kMaxP + 1];
  std::vector<dg::ApplyTile> h_tiles;
  std::vector<int32_t> h_order;      // degree-sorted element order
  // square meshes, SIPG: the sub-face work of every tile as a flat list of
  // (record, tile-local side) items, and per element side (in tile order) the
  // first item and the item count
  std::vector<int32_t> h_items;       // 2 per item: record index, and (e_local * 4 + s, cubes
                                      // e_local * 6 + s) | (position in sub-face order << 16)
  std::vector<int32_t> h_item_ptr;    // n_tiles + 1
  std::vector<int32_t> h_side_items;  // 2 per (order position, side): first item, count
  int64_t apply_smem = 0;             // dynamic shared memory of the 2D operator kernel
  // tile shapes: squares, elements per operator tile of each degree (at most
  // apply_epb(p), the compiled capacity); cubes, the shared-memory budget of a
  // tile in doubles.  Fixed rules unless the tile tuner chose them.
  int tile_epb[dg::kMaxP + 1];
  int64_t apply3_budget = dg::kApply3Budget;
  dg::DevArena tile_arena;            // device copies of the tile lists (rebuilt when tuned)
  // device
  dg::DevArena arena;
  int32_t* d_p = nullptr;
  int64_t* d_off = nullptr;
  double* d_ih = nullptr;       // 1 / h
  double* d_aih = nullptr;      // a / h (normal derivatives of traces and test functions)
  double* d_ahk = nullptr;      // a h (volume term on cubes)
  double* d_ak = nullptr;       // a
  int64_t* d_toff = nullptr;    // side-trace offsets (8 (p+1) doubles per element)
  double* d_tr = nullptr;       // side traces written by each apply
  int32_t* d_sf_ptr = nullptr;
  dg::SubFaceRec* d_sf = nullptr;
  dg::SubFaceBr2* d_sfb = nullptr;
  dg::SubFaceRec3* d_sf3 = nullptr;
  dg::SubFaceMap* d_sfm = nullptr;   // mapped squares
  double* d_gvol = nullptr;          // mapped squares: geometric factors (h_gvol, h_goff, h_gface)
  int64_t* d_goff = nullptr;
  double* d_gface = nullptr;
  double* d_gbr2 = nullptr;          // mapped squares, BR2 (h_gbr2, h_g2off)
  int64_t* d_g2off = nullptr;
  double* d_tables = nullptr;
  int32_t* d_order = nullptr;
  dg::ApplyTile* d_tiles = nullptr;
  int32_t* d_items = nullptr;
  int32_t* d_item_ptr = nullptr;
  int32_t* d_side_items = nullptr;
  int n_tiles = 0;
  unsigned* d_sched = nullptr;  // operator tile counter + exit ticket
  int apply_grid = 1;           // resident CTAs of the persistent operator kernel
  // batch only: per-instance stop flags; tiles of stopped instances are skipped
  const double* skip_status = nullptr;
  int skip_stride = 0;
  dg_mesh() {
    for (int p = 0; p <= dg::kMaxP; ++p) tile_epb[p] = p >= 1 ? dg::apply_epb(p) : 1;
  }
  ~dg_mesh() {
    tile_arena.release();
    arena.release();
  }
};

struct dg_precond {
  const dg_mesh* mesh = nullptr;
  int precision = DG_PREC_FP64;
  int lor = DG_LOR_AMG;
  int64_t n_dofs = 0, n_c = 0;
  dg_precond_stats stats{};
  dg::DevArena arena;
  dg::DevCsr P, PT;          // P: n_dofs x n_c (rows = DG nodes), PT = P^T
  void* dinv = nullptr;      // n_dofs, 1/A_jj on V_J and 0 elsewhere
  int32_t* e_pos = nullptr;     // n_dofs, slot of the node's result in zE, or -1 outside the V_e
  // block-solve work units, largest blocks first: one per 32-row panel of a
  // large V_e block, {slot of the block's first node in zE, d, first row, 0},
  // with the offset of the panel's first row in blk_inv
  int32_t* blk_unit = nullptr;   // 4 per unit
  int64_t* blk_ubase = nullptr;
  // small blocks, packed several to a unit {first block, count, 0, W}: per block
  // {slot of its first node, d, inverse offset low / high 32 bits}
  int32_t* blk_rec = nullptr;
  int32_t* blk_dofs = nullptr;   // DG node of every slot, block by block
  void* blk_inv = nullptr;   // dense inverses, column-major
  void* lor_inv = nullptr;   // exact LOR solve: dense inverse n_c x n_c
  std::vector<dg::DevLevel> levels;  // AMG (level 0 = LOR matrix)
  void* rc = nullptr;        // n_c restriction of r
  void* ec = nullptr;        // n_c LOR correction
  void* zE = nullptr;        // block-solve results, one per V_e node (block order)
  int64_t n_blocks = 0, max_block = 0, n_units = 0;
  int64_t blk_inv_entries = 0, blk_slots = 0;   // sizes of blk_inv and blk_dofs
  cudaStream_t side = nullptr;   // the block solves run here, beside the V-cycle
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // PCG workspace and captured solve graph, built by dg_precond_setup
  void* pcg_cache = nullptr;
  void (*pcg_cache_free)(void*) = nullptr;
  ~dg_precond() {
    if (pcg_cache_free) pcg_cache_free(pcg_cache);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    arena.release();
  }
};

namespace dg {
// validate the description and build everything the device needs, on the host
void build_mesh_host(dg_mesh* M, const dg_mesh_desc* desc, const dg_options* opts);
// degree-sorted element order and operator tiles from M->host.p
void build_tiles(dg_mesh* M);
// flat sub-face item lists of the tiles (square meshes; after the tiles)
void build_face_items(dg_mesh* M);
// cube meshes: degree-sorted order, tiles and their item lists
void build_tiles3(dg_mesh* M);
// upload the host-built operator data (M->host.p/off/sf_ptr, h_* arrays)
void upload_mesh(dg_mesh* M, cudaStream_t s);
// (re)upload the tile lists and size the operator launch (tile_arena)
void upload_tiles(dg_mesh* M, cudaStream_t s);
// Time the operator kernel over candidate tile shapes and keep the fastest:
// squares, for each degree present (highest first) the elements per tile in
// {apply_epb(p), 3/4, 1/2 of it}; cubes, shared-memory budgets for 4, 3 and 2
// tiles per SM.  retile rebuilds the host tile lists from the tile shapes.
// Records the choice and the times in M->stats.
void tune_tiles(dg_mesh* M, cudaStream_t s, void (*retile)(dg_mesh*, void*), void* ctx);
// cube meshes: topology, records, tables, tiles, stats (opts already validated)
void build_mesh_host3(dg_mesh* M, const dg_mesh_desc* desc, const dg_options& opts);
// mapped squares: records, tables and geometry (after the SIPG records), and
// the flop and byte counts of the mapped operator (after the box counts)
void build_mesh_map(dg_mesh* M, const dg_mesh_desc* desc);
void map_stats(dg_mesh* M);
// rows of element k of y = A x on a mapped mesh, and their diagonal, and the
// LOR block of element k (dense (p+1)^2 x (p+1)^2, row-major)
void host_element_residual_map(const dg_mesh& M, int64_t k, const double* x, double* y);
void host_element_diag_map(const dg_mesh& M, int64_t k, double* d);
void host_lor_block_map(const dg_mesh& M, int64_t k, double* A);
// rows of element k of y = A x (x: full host vector), same formulation as the kernel
void host_element_residual(const dg_mesh& M, int64_t k, const double* x, double* y, int64_t source = -1);
// (source >= 0: x vanishes outside element `source`, and the terms that are
// exact zeros then are skipped; the result is the same)
void host_element_residual3(const dg_mesh& M, int64_t k, const double* x, double* y, int64_t source = -1);
// load vector of caller-supplied f (volume) and boundary data g (SIPG, weak)
// into hb (n_dofs doubles); either may be null
void host_load(const dg_mesh& M, dg_field_fn f, dg_field_fn g, void* ctx, double* hb);
// load vector of the sine right-hand side into hb (n_dofs doubles, zeroed)
void host_rhs_sine(const dg_mesh& mesh, int n_modes, const double* amps, const int32_t* waves,
                   double* hb);
// diagonal of element k's rows of A (closed form of the same terms)
void host_element_diag(const dg_mesh& M, int64_t k, double* d);
}  // namespace dg
