// Host-only inspection library (libdgsc_inspect.so): runs the library's own
// host setup - topology, conforming prolongation, V_J / V_e split, LOR matrix,
// AMG hierarchy - and the host mirror of the operator, without a GPU, so that
// they can be compared with an independent implementation on a CPU machine.
// Not part of the solver ABI (include/dg.h); every call is synchronous.
#include <cstring>
#include <memory>

#include "dg_internal.h"
#include "host_state.h"
#include "precond_setup.h"
#include "work_units.h"

using namespace dg;

namespace {
struct Inspect {
  dg_mesh mesh;
  HostPrecond pc;
  AmgHierarchy amg;
  std::string err;
};
thread_local std::string g_err;
thread_local int g_status = DG_OK;
}  // namespace

namespace dg {
void set_last_error(const std::string& msg) { g_err = msg; }
}

extern "C" {

const char* dginspect_last_error(void) { return g_err.c_str(); }
// the dg_status of the last failed dginspect_create (DG_EINVAL for other errors)
int dginspect_last_status(void) { return g_status; }

// Work units of the block solves for blocks of the given sizes, slots and
// inverse offsets (see plan_block_units).  unit: 4 * cap ints, ubase: cap,
// brec: 4 * nb ints.  Returns the number of units, -1 on error or when cap is
// too small.
int64_t dginspect_block_units(int64_t nb, const int32_t* dims, const int32_t* slot, const int64_t* inv_off,
                              int32_t* unit, int64_t* ubase, int32_t* brec, int64_t cap) {
  try {
    std::vector<int32_t> d(dims, dims + nb), sl(slot, slot + nb), u, br;
    std::vector<int64_t> io(inv_off, inv_off + nb), ub;
    plan_block_units(d, sl, io, u, ub, br);
    const int64_t n = (int64_t)ub.size();
    if (n > cap) return -1;
    std::memcpy(unit, u.data(), u.size() * sizeof(int32_t));
    std::memcpy(ubase, ub.data(), ub.size() * sizeof(int64_t));
    if (!br.empty()) std::memcpy(brec, br.data(), br.size() * sizeof(int32_t));
    return n;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -1;
  }
}

// Row tiers of the CSR row kernel for a matrix with the given row pointers
// (see plan_csr_tiers): out2 = {group, long_min}, counts = {n_cta, n_warp},
// cta and warp: rows ints each.
int dginspect_csr_tiers(int64_t rows, const int64_t* ptr, int32_t* out2, int64_t* counts, int32_t* cta,
                        int32_t* warp) {
  try {
    Csr C;
    C.rows = rows;
    C.ptr.assign(ptr, ptr + rows + 1);
    const CsrTierPlan T = plan_csr_tiers(C);
    out2[0] = T.group;
    out2[1] = T.long_min;
    counts[0] = (int64_t)T.cta.size();
    counts[1] = (int64_t)T.warp.size();
    if (!T.cta.empty()) std::memcpy(cta, T.cta.data(), T.cta.size() * sizeof(int32_t));
    if (!T.warp.empty()) std::memcpy(warp, T.warp.data(), T.warp.size() * sizeof(int32_t));
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -1;
  }
}

void* dginspect_create(const dg_mesh_desc* desc, const dg_options* opts, int with_amg) {
  try {
    std::unique_ptr<Inspect> I(new Inspect());
    build_mesh_host(&I->mesh, desc, opts);
    dg_options o = I->mesh.opts;
    if (opts) {
      o.smoother = opts->smoother;
      o.remark_cases = opts->remark_cases;
    }
    I->pc = (I->mesh.host.dim == 3) ? build_host_precond3(I->mesh, o) : build_host_precond(I->mesh, o);
    if (with_amg && I->pc.nC > 0)
      I->amg = amg_setup(I->pc.Ac, I->mesh.host.dim == 3 ? kAmgTheta3 : kAmgTheta);
    g_status = DG_OK;
    return I.release();
  } catch (const Error& e) {
    g_err = e.what();
    g_status = e.code;
    return nullptr;
  } catch (const std::exception& e) {
    g_err = e.what();
    g_status = DG_EINVAL;
    return nullptr;
  }
}

void dginspect_destroy(void* h) { delete (Inspect*)h; }

// the operator's tiles and sub-face items: out = [n_tiles, n_items, dim]
void dginspect_item_sizes(void* h, int64_t* out) {
  const dg_mesh& M = ((Inspect*)h)->mesh;
  out[0] = M.n_tiles;
  out[1] = (int64_t)M.h_items.size() / 2;
  out[2] = M.host.dim;
}

// item_ptr (n_tiles + 1), items (2 per item, as the kernels read them), per
// tile its chunk length (cubes; squares: the tile's item count), and per item
// the fields its branches depend on: interior (0/1), neighbour degree, the
// whole-side flags (BR2 records; 0 without them)
void dginspect_items(void* h, int32_t* item_ptr, int32_t* items, int32_t* chunk, int32_t* info) {
  const dg_mesh& M = ((Inspect*)h)->mesh;
  std::memcpy(item_ptr, M.h_item_ptr.data(), M.h_item_ptr.size() * sizeof(int32_t));
  std::memcpy(items, M.h_items.data(), M.h_items.size() * sizeof(int32_t));
  for (int t = 0; t < M.n_tiles; ++t)
    chunk[t] = M.host.dim == 3 ? M.h_tiles[t].chunk : M.h_item_ptr[t + 1] - M.h_item_ptr[t];
  const int64_t n = (int64_t)M.h_items.size() / 2;
  for (int64_t g = 0; g < n; ++g) {
    const int32_t r = M.h_items[2 * g];
    if (M.host.dim == 3) {
      const SubFaceRec3& f = M.h_sf3[r];
      info[3 * g] = f.nb >= 0 ? 1 : 0;
      info[3 * g + 1] = f.pn;
      info[3 * g + 2] = f.full;
    } else {
      const SubFaceRec& f = M.h_sf[r];
      info[3 * g] = f.nb >= 0 ? 1 : 0;
      info[3 * g + 1] = f.pn;
      info[3 * g + 2] = M.h_sfb.empty() ? 0 : M.h_sfb[r].full;
    }
  }
}

// sizes: [n_dofs, n_c, nnz(P), nnz(Ac), n_blocks, total block dofs, n_levels,
//         eta*1e6, sum of squared block dims]
void dginspect_sizes(void* h, int64_t* out) {
  Inspect* I = (Inspect*)h;
  out[0] = I->mesh.n_dofs;
  out[1] = I->pc.nC;
  out[2] = I->pc.P.nnz();
  out[3] = I->pc.Ac.nnz();
  out[4] = (int64_t)I->pc.blocks.size();
  int64_t t = 0;
  for (auto& b : I->pc.blocks) t += (int64_t)b.size();
  out[5] = t;
  out[6] = (int64_t)I->amg.levels.size();
  out[7] = (int64_t)(I->mesh.eta * 1e6);
  int64_t q = 0;
  for (auto& b : I->pc.blocks) q += (int64_t)b.size() * (int64_t)b.size();
  out[8] = q;
}

static void copy_csr(const Csr& C, int64_t* ptr, int32_t* idx, double* val) {
  std::memcpy(ptr, C.ptr.data(), C.ptr.size() * sizeof(int64_t));
  std::memcpy(idx, C.idx.data(), C.idx.size() * sizeof(int32_t));
  std::memcpy(val, C.val.data(), C.val.size() * sizeof(double));
}

void dginspect_P(void* h, int64_t* ptr, int32_t* idx, double* val) { copy_csr(((Inspect*)h)->pc.P, ptr, idx, val); }
void dginspect_lor(void* h, int64_t* ptr, int32_t* idx, double* val) { copy_csr(((Inspect*)h)->pc.Ac, ptr, idx, val); }

void dginspect_kind(void* h, int8_t* kind) {
  Inspect* I = (Inspect*)h;
  std::memcpy(kind, I->pc.kind.data(), I->pc.kind.size());
}

void dginspect_dinv(void* h, double* dinv) {
  Inspect* I = (Inspect*)h;
  std::memcpy(dinv, I->pc.dinv.data(), I->pc.dinv.size() * sizeof(double));
}

// blocks: offsets (n_blocks+1) and node lists; inverse entries concatenated
void dginspect_blocks(void* h, int64_t* offsets, int64_t* nodes, double* inv) {
  Inspect* I = (Inspect*)h;
  int64_t o = 0, q = 0;
  offsets[0] = 0;
  for (size_t b = 0; b < I->pc.blocks.size(); ++b) {
    for (int64_t r : I->pc.blocks[b]) nodes[o++] = r;
    offsets[b + 1] = o;
    for (double v : I->pc.block_inv[b]) inv[q++] = v;
  }
}

int64_t dginspect_level_rows(void* h, int l) {
  Inspect* I = (Inspect*)h;
  return I->amg.levels[l].A.rows;
}
int64_t dginspect_level_nnz(void* h, int l) {
  Inspect* I = (Inspect*)h;
  return I->amg.levels[l].A.nnz();
}
void dginspect_level_A(void* h, int l, int64_t* ptr, int32_t* idx, double* val) {
  copy_csr(((Inspect*)h)->amg.levels[l].A, ptr, idx, val);
}

// the load vector of caller-supplied f and boundary data g (host_load) into
// b (n_dofs doubles); 0, or -1 with the message in dginspect_last_error
int dginspect_rhs_eval(void* h, dg_field_fn f, dg_field_fn g, void* ctx, double* b) {
  try {
    host_load(((Inspect*)h)->mesh, f, g, ctx, b);
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -1;
  }
}

// y = A x with the host mirror of the operator kernel
void dginspect_apply(void* h, const double* x, double* y) {
  Inspect* I = (Inspect*)h;
  const HostMesh& m = I->mesh.host;
  for (int64_t k = 0; k < m.n; ++k) {
    if (m.dim == 3) host_element_residual3(I->mesh, k, x, y + m.off[k]);
    else host_element_residual(I->mesh, k, x, y + m.off[k]);
  }
}

}  // extern "C"
