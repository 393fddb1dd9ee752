// C ABI entry points (include/dg.h): validation, host setup, uploads, the
// graph-captured PCG loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "precond_setup.h"
#include "union.h"

namespace dg {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

template <typename F>
static dg_status guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return DG_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return DG_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return DG_EINVAL;
  }
}

static void build_mesh(dg_mesh* M, const dg_mesh_desc* desc, const dg_options* opts, cudaStream_t s) {
  build_mesh_host(M, desc, opts);   // validates before any device work
  DG_CUDA(cudaGetDevice(&M->device));
  upload_mesh(M, s);
}

void upload_tiles(dg_mesh* M, cudaStream_t s) {
  M->tile_arena.release();
  DevArena& a = M->tile_arena;
  M->apply_smem = apply_smem_for(*M);
  M->apply_grid = apply_kernel_setup(*M);
  M->d_order = a.upload(M->h_order, s);
  M->d_tiles = a.upload(M->h_tiles, s);
  M->d_items = a.upload(M->h_items, s);
  M->d_item_ptr = a.upload(M->h_item_ptr, s);
  M->d_side_items = a.upload(M->h_side_items, s);
  DG_CUDA(cudaStreamSynchronize(s));
}

void upload_mesh(dg_mesh* M, cudaStream_t s) {
  const HostMesh& m = M->host;
  // upload
  DevArena& a = M->arena;
  M->d_p = a.upload(m.p, s);
  M->d_off = a.upload(m.off, s);
  {
    std::vector<double> ih(m.n), aih(m.n), ahk(m.n);
    std::vector<int64_t> toff(m.n + 1, 0);
    for (int64_t k = 0; k < m.n; ++k) {
      ih[k] = 1.0 / M->h_h[k];
      aih[k] = m.coef[k] / M->h_h[k];
      ahk[k] = m.coef[k] * M->h_h[k];
      const int64_t np = m.p[k] + 1;
      toff[k + 1] = toff[k] + (m.dim == 3 ? 12 * np * np : 8 * np);
    }
    M->d_ih = a.upload(ih, s);
    M->d_aih = a.upload(aih, s);
    M->d_ahk = a.upload(ahk, s);
    M->d_ak = a.upload(m.coef, s);
    M->d_toff = a.upload(toff, s);
    M->d_tr = a.alloc<double>(toff[m.n]);
  }
  M->d_sf_ptr = a.upload(m.sf_ptr, s);
  M->d_sf = a.upload(M->h_sf, s);
  M->d_sfb = M->h_sfb.empty() ? nullptr : a.upload(M->h_sfb, s);
  M->d_sf3 = a.upload(M->h_sf3, s);
  if (m.mapped) {
    M->d_sfm = a.upload(M->h_sfm, s);
    M->d_gvol = a.upload(M->h_gvol, s);
    M->d_goff = a.upload(M->h_goff, s);
    M->d_gface = a.upload(M->h_gface, s);
    if (!M->h_gbr2.empty()) {
      M->d_gbr2 = a.upload(M->h_gbr2, s);
      M->d_g2off = a.upload(M->h_g2off, s);
    }
  }
  M->d_tables = a.upload(M->h_tables, s);
  M->d_sched = a.alloc<unsigned>(2);
  DG_CUDA(cudaMemsetAsync(M->d_sched, 0, 2 * sizeof(unsigned), s));
  upload_tiles(M, s);
}

// rebuild the tile lists of a single mesh from its tile shapes
static void retile_mesh(dg_mesh* M, void*) {
  if (M->host.dim == 3) build_tiles3(M);
  else build_tiles(M);
}


// b_i = int f phi_i with a (p+3)-point Gauss rule per direction (host)
void host_rhs_sine(const dg_mesh& mesh, int n_modes, const double* amps, const int32_t* waves,
                   double* hb) {
  const HostMesh& m = mesh.host;
  const int dim = m.dim;
  for (int64_t k = 0; k < m.n; ++k) {
    const int P = m.p[k], NP = P + 1;
    const Basis1D& B = basis1d(P);
    std::vector<double> gx, gw;
    gauss_rule(P + 3, gx, gw);
    const double h = mesh.h_h[k];
    double x0[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < dim; ++d) x0[d] = m.lo[dim * k + d] * m.lh;
    const int q = (int)gx.size();
    std::vector<double> L((size_t)q * NP);
    for (int g = 0; g < q; ++g) lagrange_eval(B.nodes, gx[g], &L[(size_t)g * NP]);
    const int qz = dim == 3 ? q : 1, nz = dim == 3 ? NP : 1;
    for (int gz = 0; gz < qz; ++gz)
      for (int gy = 0; gy < q; ++gy)
        for (int gxi = 0; gxi < q; ++gxi) {
          double X[3] = {x0[0] + h * gx[gxi], x0[1] + h * gx[gy], x0[2] + h * gx[gz]};
          double detJ = 1.0;
          if (m.mapped) {   // f at the physical point, the weight times det J (stored at creation)
            const double* pt = mesh.h_xrhs.data() + mesh.h_roff[k] + 3 * (gy * q + gxi);
            X[0] = pt[0];
            X[1] = pt[1];
            detJ = pt[2];
          }
          double f = 0.0;
          for (int md = 0; md < n_modes; ++md) {
            double t = amps[md];
            for (int d = 0; d < dim; ++d) t *= std::sin(M_PI * waves[dim * md + d] * X[d]);
            f += t;
          }
          double w = gw[gxi] * gw[gy] * h * h * f * detJ;
          if (dim == 3) w *= gw[gz] * h;
          for (int iz = 0; iz < nz; ++iz) {
            const double lz = dim == 3 ? L[(size_t)gz * NP + iz] : 1.0;
            for (int iy = 0; iy < NP; ++iy)
              for (int ix = 0; ix < NP; ++ix)
                hb[m.off[k] + (iz * NP + iy) * NP + ix] +=
                    w * lz * L[(size_t)gy * NP + iy] * L[(size_t)gxi * NP + ix];
          }
        }
  }
}

// ----------------------------------------------------------------- precond upload
template <typename T>
static void upload_precond(dg_precond* pc, HostPrecond& H, cudaStream_t s) {
  if (pc->lor == DG_LOR_AMG) {
    AmgHierarchy Hm = amg_setup(H.Ac, pc->mesh->host.dim == 3 ? kAmgTheta3 : kAmgTheta);
    upload_union_precond<T>(pc, {InstSrc{&H, &Hm, 0}}, s);
    return;
  }
  // exact LOR solve: P, blocks and Jacobi as in the union form, dense inverse of A~_C
  AmgHierarchy none;
  none.levels.push_back({Csr{}, {}, {}, {}});
  none.levels[0].A.rows = H.nC;
  HostPrecond Hp = H;
  upload_union_precond<T>(pc, {InstSrc{&Hp, &none, 0}}, s);
  pc->levels.clear();
  DevArena& a = pc->arena;
  DG_REQUIRE(pc->n_c <= 8192, "exact LOR solve limited to 8192 conforming unknowns");
  std::vector<double> dense((size_t)pc->n_c * pc->n_c, 0.0);
  for (int64_t i = 0; i < H.Ac.rows; ++i)
    for (int64_t t = H.Ac.ptr[i]; t < H.Ac.ptr[i + 1]; ++t) dense[i * pc->n_c + H.Ac.idx[t]] = H.Ac.val[t];
  if (pc->n_c > 0) dense_inverse_spd((int)pc->n_c, dense);
  pc->lor_inv = a.upload(std::vector<T>(dense.begin(), dense.end()), s);
  pc->stats.n_levels = 1;
  pc->stats.level_rows[0] = pc->n_c;
  pc->stats.level_nnz[0] = H.Ac.nnz();
  DG_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------------- PCG workspace
// Created with the preconditioner (dg_precond_setup), so solves allocate
// nothing: the work vectors, the solve's own copies of b and x, pinned scalars,
// a capture stream, two events and the captured iteration graph.  The graph
// reads b from and writes x to the workspace copies and takes the tolerance
// and iteration limit from device scalars, so one capture serves every solve.
struct PcgWork {
  int64_t n = 0;
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *b = nullptr, *x = nullptr;   // the solve's copies of b and x
  double *part_pq = nullptr, *part_rr = nullptr, *part_rz = nullptr, *part_bb = nullptr;
  double* sc = nullptr;
  unsigned* tick = nullptr;  // reduction tickets (TK_*)
  double* hsc = nullptr;     // pinned: scalars read back (SC_COUNT) + limits sent (2)
  DevArena arena;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  bool graph_failed = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~PcgWork() {
    drop_graph();
    if (cap) cudaStreamDestroy(cap);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    arena.release();
    if (hsc) cudaFreeHost(hsc);
  }
};

static void free_pcg_work(void* p) { delete (PcgWork*)p; }

static PcgWork& pcg_work(const dg_precond* pc) {
  dg_precond* m = const_cast<dg_precond*>(pc);
  if (m->pcg_cache) return *(PcgWork*)m->pcg_cache;
  PcgWork* w = new PcgWork();
  m->pcg_cache = w;
  m->pcg_cache_free = free_pcg_work;
  const dg_mesh* M = pc->mesh;
  w->n = M->n_dofs;
  w->r = w->arena.alloc<double>(w->n);
  w->z = w->arena.alloc<double>(w->n);
  w->p = w->arena.alloc<double>(w->n);
  w->q = w->arena.alloc<double>(w->n);
  w->b = w->arena.alloc<double>(w->n);
  w->x = w->arena.alloc<double>(w->n);
  w->part_pq = w->arena.alloc<double>(std::max(M->n_tiles, 1));
  w->part_rr = w->arena.alloc<double>(kVecBlocks);
  w->part_rz = w->arena.alloc<double>(kVecBlocks);
  w->part_bb = w->arena.alloc<double>(kVecBlocks);
  w->sc = w->arena.alloc<double>(SC_COUNT);
  w->tick = w->arena.alloc<unsigned>(TK_COUNT);
  DG_CUDA(cudaMemset(w->tick, 0, TK_COUNT * sizeof(unsigned)));
  DG_CUDA(cudaMallocHost(&w->hsc, (SC_COUNT + 2) * sizeof(double)));
  DG_CUDA(cudaEventCreate(&w->e0));
  DG_CUDA(cudaEventCreate(&w->e1));
  DG_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
  return *w;
}

static int64_t pcg_work_bytes(const dg_precond* pc) {
  return pc->pcg_cache ? (int64_t)((PcgWork*)pc->pcg_cache)->arena.bytes : 0;
}

static void pcg_body(const dg_mesh* M, const dg_precond* pc, PcgWork& w, double* x, int maxit,
                     double rtol2, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  // q = A p (the side traces of p were written with p by launch_pcg_p_trace);
  // the launch's last CTA sums p . q and forms alpha
  launch_apply(*M, w.p, w.q, Reduce{w.part_pq, w.sc + SC_PQ, w.tick + TK_PQ}, s, false, w.sc);
  // z = B (r - alpha q): the preconditioner's kernels read the updated
  // residual on the fly and its final kernel stores it with x += alpha p (no
  // launch of its own), sums r . z and r . r, and its last CTA sets beta,
  // tests convergence, counts the iteration and sets the while condition
  launch_precond(*pc, w.r, w.z, Reduce{w.part_rz, w.sc + SC_RZNEW, w.tick + TK_RZ}, s, nullptr,
                 Reduce{w.part_rr, w.sc + SC_RRNEW, nullptr},
                 PcgCtl{w.sc, maxit, rtol2, (unsigned long long)h, use_cond},
                 XrDefer{w.r, x, w.p, w.q, w.sc + SC_ALPHA});
  launch_pcg_p_trace(*M, w.p, w.z, w.sc, (unsigned long long)h, use_cond, 0, s);
}

// PCG start: x = 0, r = b, z = B r, p = z with its side traces, the initial
// scalars; with use_cond the last kernel sets the loop condition (b . b > 0)
static void pcg_start_kernels(const dg_precond* pc, PcgWork& w, const double* b, double* x,
                              cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  launch_pcg_init(b, x, w.r, w.n, Reduce{w.part_bb, w.sc + SC_BB, w.tick + TK_BB}, s);
  launch_precond(*pc, w.r, w.z, Reduce{w.part_rz, w.sc + SC_RZNEW, w.tick + TK_RZ}, s);
  launch_pcg_p_trace(*pc->mesh, w.p, w.z, w.sc, (unsigned long long)h, use_cond, 1, s);
}

// host-driven start: the kernels above, then b . b read back (synchronises)
static double pcg_start(const dg_precond* pc, PcgWork& w, const double* b, double* x, double* hsc,
                        cudaStream_t s) {
  pcg_start_kernels(pc, w, b, x, 0, 0, s);
  DG_CUDA(cudaMemcpyAsync(hsc, w.sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return hsc[SC_BB];
}

// One graph for a whole solve: the start kernels, then a device-side while
// node around one PCG iteration whose condition the kernels set.  Captured
// once per preconditioner, on the workspace copies of b and x, with the limits
// read from device scalars.
static bool pcg_capture(const dg_mesh* M, const dg_precond* pc, PcgWork& w) {
  if (w.exec) return true;
  if (w.graph_failed) return false;
  const char* env = std::getenv("DG_PCG_GRAPH");
  if (env && env[0] == '0') return false;  // host-driven loop requested
  cudaGraphConditionalHandle handle = 0;
  bool ok = false;
  std::string why;
  if (cudaGraphCreate(&w.graph, 0) == cudaSuccess &&
      cudaGraphConditionalHandleCreate(&handle, w.graph, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
      cudaStreamBeginCaptureToGraph(w.cap, w.graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
          cudaSuccess) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    bool launched = true;
    try {
      pcg_start_kernels(pc, w, w.b, w.x, handle, 1, w.cap);
      // the while node follows the start kernels
      cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
      cudaGraph_t g = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      DG_CUDA(cudaStreamGetCaptureInfo(w.cap, &st, nullptr, &g, &deps, nullptr, &nd));
      cudaGraphNode_t cnode = nullptr;
      DG_CUDA(cudaGraphAddNode(&cnode, g, deps, nullptr, nd, &cp));
      DG_CUDA(cudaStreamUpdateCaptureDependencies(w.cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    } catch (const Error& e) {
      launched = false;
      why = e.what();
    }
    cudaGraph_t out = nullptr;
    cudaError_t ec = cudaStreamEndCapture(w.cap, &out);
    ok = ec == cudaSuccess && launched;
    if (ok) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      ec = cudaStreamBeginCaptureToGraph(w.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (ec == cudaSuccess) {
        try {
          pcg_body(M, pc, w, w.x, -1, 0.0, handle, 1, w.cap);
        } catch (const Error& e) {
          launched = false;
          why = e.what();
        }
        ec = cudaStreamEndCapture(w.cap, &out);
      }
      ok = ec == cudaSuccess && launched;
    }
    cudaError_t ei = cudaSuccess;
    if (ok) {
      ei = cudaGraphInstantiate(&w.exec, w.graph, 0);
      ok = ei == cudaSuccess;
    }
    if (!ok && std::getenv("DG_VERBOSE"))
      std::fprintf(stderr, "dg: capture: launch [%s] capture %s instantiate %s\n", why.c_str(),
                   cudaGetErrorString(ec), cudaGetErrorString(ei));
  }
  const cudaError_t cap_err = cudaGetLastError();
  if (!ok) {
    if (std::getenv("DG_VERBOSE"))
      std::fprintf(stderr, "dg: PCG graph capture failed (%s), using the host-driven loop\n",
                   cudaGetErrorString(cap_err));
    w.drop_graph();
    w.graph_failed = true;
    return false;
  }
  return true;
}

// Solve into the workspace copy of x.  solve_ms spans everything the solve
// puts on the stream: the copy of b, the limits, the start, the iterations and
// the copy of x; with the graph there is no host round trip inside it.
static void pcg_run(const dg_mesh* M, const dg_precond* pc, const double* b, double* x, double rtol,
                    int maxit, dg_solve_info* info, cudaStream_t s) {
  DG_REQUIRE(M && pc && b && x, "null argument");
  DG_REQUIRE(pc->mesh == M, "preconditioner belongs to another mesh");
  DG_REQUIRE(rtol > 0.0 && maxit >= 1, "rtol must be > 0 and maxit >= 1");
  PcgWork& w = pcg_work(pc);
  const double rtol2 = rtol * rtol;
  const bool use_graph = pcg_capture(M, pc, w);
  // the previous solve with this handle has finished (solves are synchronous),
  // so the pinned slots are free to take this solve's limits
  w.hsc[SC_COUNT] = (double)maxit;
  w.hsc[SC_COUNT + 1] = rtol2;
  DG_CUDA(cudaEventRecord(w.e0, s));
  if (b != w.b) DG_CUDA(cudaMemcpyAsync(w.b, b, w.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaMemcpyAsync(w.sc + SC_MAXIT, w.hsc + SC_COUNT, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  if (use_graph) {
    DG_CUDA(cudaGraphLaunch(w.exec, s));
  } else if (pcg_start(pc, w, w.b, w.x, w.hsc, s) > 0.0) {
    // host-driven loop, status read back every 8 iterations
    for (int it = 0; it < maxit;) {
      for (int j = 0; j < 8 && it < maxit; ++j, ++it) pcg_body(M, pc, w, w.x, maxit, rtol2, 0, 0, s);
      DG_CUDA(cudaMemcpyAsync(w.hsc, w.sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
      DG_CUDA(cudaStreamSynchronize(s));
      if (w.hsc[SC_STATUS] != 0.0) break;
    }
  }
  if (x != w.x) DG_CUDA(cudaMemcpyAsync(x, w.x, w.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaEventRecord(w.e1, s));
  DG_CUDA(cudaMemcpyAsync(w.hsc, w.sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.0f;
  DG_CUDA(cudaEventElapsedTime(&ms, w.e0, w.e1));
  const int iters = (int)w.hsc[SC_IT];
  const double bb = w.hsc[SC_BB];
  const double rel = bb > 0.0 ? std::sqrt(w.hsc[SC_RR] / bb) : 0.0;
  const bool conv = bb == 0.0 || w.hsc[SC_STATUS] == 1.0;
  if (info) {
    info->iters = bb > 0.0 ? iters : 0;
    info->rel_res = rel;
    info->status = conv ? DG_OK : DG_ENOTCONV;
    info->solve_ms = ms;
  }
  if (!conv) throw Error(DG_ENOTCONV, "PCG reached maxit");
}

}  // namespace dg

using namespace dg;

extern "C" {

const char* dg_last_error(void) { return g_last_error.c_str(); }

dg_status dg_mesh_create(const dg_mesh_desc* desc, const dg_options* opts, void* stream, dg_mesh** out) {
  if (!out) { set_last_error("null output handle"); return DG_EINVAL; }
  *out = nullptr;
  dg_mesh* M = nullptr;
  dg_status st = guarded([&] {
    M = new dg_mesh();
    build_mesh(M, desc, opts, (cudaStream_t)stream);
    if (opts && opts->tune_tiles) tune_tiles(M, (cudaStream_t)stream, retile_mesh, nullptr);
  });
  if (st != DG_OK) { delete M; return st; }
  *out = M;
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* mesh) { delete mesh; }

int64_t dg_num_dofs(const dg_mesh* mesh) { return mesh ? mesh->n_dofs : -1; }

dg_status dg_mesh_stats_get(const dg_mesh* mesh, dg_mesh_stats* out) {
  return guarded([&] {
    DG_REQUIRE(mesh && out, "null argument");
    *out = mesh->stats;
    out->device_bytes = (int64_t)(mesh->arena.bytes + mesh->tile_arena.bytes);
    if (!out->tiles_tuned) {
      for (int p = 0; p <= kMaxP; ++p) out->tile_elems[p] = mesh->host.dim == 2 ? mesh->tile_epb[p] : 0;
      out->tile_smem_budget = mesh->host.dim == 3 ? 8 * mesh->apply3_budget : 0;
    }
  });
}

dg_status dg_dof_layout(const dg_mesh* mesh, int64_t* elem_offsets) {
  return guarded([&] {
    DG_REQUIRE(mesh && elem_offsets, "null argument");
    const std::vector<int64_t>& off = mesh->host.off;
    std::copy(off.begin(), off.end(), elem_offsets);
  });
}

dg_status dg_apply(const dg_mesh* mesh, const double* x, double* y, void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh && x && y, "null argument");
    DG_REQUIRE(x != y, "x and y must not alias");
    launch_apply(*mesh, x, y, Reduce{}, (cudaStream_t)stream);
  });
}

dg_status dg_precond_setup(const dg_mesh* mesh, const dg_options* opts, dg_precond** out) {
  if (!out) { set_last_error("null output handle"); return DG_EINVAL; }
  *out = nullptr;
  dg_precond* pc = nullptr;
  dg_status st = guarded([&] {
    DG_REQUIRE(mesh != nullptr, "null mesh");
    dg_options o = mesh->opts;
    if (opts) {
      o.precision = opts->precision;
      o.lor = opts->lor;
      o.smoother = opts->smoother;
      o.remark_cases = opts->remark_cases;
    }
    DG_REQUIRE(o.precision == DG_PREC_FP64 || o.precision == DG_PREC_MIXED, "unknown precision");
    DG_REQUIRE(o.lor == DG_LOR_EXACT || o.lor == DG_LOR_AMG, "unknown LOR solver");
    DG_REQUIRE(o.smoother == DG_SMOOTHER_FULL || o.smoother == DG_SMOOTHER_JACOBI_ONLY, "unknown smoother");
    HostPrecond H = (mesh->host.dim == 3) ? build_host_precond3(*mesh, o) : build_host_precond(*mesh, o);
    pc = new dg_precond();
    pc->mesh = mesh;
    pc->precision = o.precision;
    pc->lor = o.lor;
    pc->n_dofs = mesh->n_dofs;
    pc->n_c = H.nC;
    auto& S = pc->stats;
    S.n_dofs = mesh->n_dofs;
    S.n_conforming = H.nC;
    for (auto k : H.kind) { S.n_j += (k == 1); S.n_e += (k == 2); }
    S.n_blocks = (int64_t)H.blocks.size();
    for (auto& b : H.blocks) S.max_block = std::max<int64_t>(S.max_block, (int64_t)b.size());
    S.lor_nnz = H.Ac.nnz();
    S.p_nnz = H.P.nnz();
    cudaStream_t s = nullptr;
    if (o.precision == DG_PREC_MIXED) upload_precond<float>(pc, H, s);
    else upload_precond<double>(pc, H, s);
    // the solves' workspace and graph, so that solves allocate nothing
    pcg_capture(mesh, pc, pcg_work(pc));
  });
  if (st != DG_OK) { delete pc; return st; }
  *out = pc;
  return DG_OK;
}

void dg_precond_destroy(dg_precond* pc) { delete pc; }

dg_status dg_precond_stats_get(const dg_precond* pc, dg_precond_stats* out) {
  return guarded([&] {
    DG_REQUIRE(pc && out, "null argument");
    *out = pc->stats;
    out->kernels_per_apply = precond_kernel_count(*pc);
    out->device_bytes = (int64_t)pc->arena.bytes + pcg_work_bytes(pc);
    precond_algorithmic_bytes(*pc, &out->apply_bytes, &out->block_bytes);
  });
}

dg_status dg_precond_apply(const dg_precond* pc, const double* r, double* z, void* stream) {
  return guarded([&] {
    DG_REQUIRE(pc && r && z, "null argument");
    DG_REQUIRE(r != z, "r and z must not alias");
    launch_precond(*pc, r, z, Reduce{}, (cudaStream_t)stream);
  });
}

// events of one profiled call, destroyed on every exit
struct EventSet {
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  explicit EventSet(int n) {
    for (int i = 0; i < n; ++i) DG_CUDA(cudaEventCreate(&ev[i]));
  }
  ~EventSet() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  double ms(int a, int b) const {
    float t = 0.0f;
    DG_CUDA(cudaEventElapsedTime(&t, ev[a], ev[b]));
    return t;
  }
};

dg_status dg_precond_profile(const dg_precond* pc, const double* r, double* z, dg_precond_times* out,
                             void* stream) {
  return guarded([&] {
    DG_REQUIRE(pc && r && z && out, "null argument");
    DG_REQUIRE(r != z, "r and z must not alias");
    const cudaStream_t s = (cudaStream_t)stream;
    EventSet E(5);
    PrecondMarks mk;
    for (int i = 0; i < 5; ++i) mk.ev[i] = E.ev[i];
    launch_precond(*pc, r, z, Reduce{}, s, &mk);
    DG_CUDA(cudaEventSynchronize(E.ev[4]));
    out->blocks_ms = E.ms(0, 1);
    out->restrict_ms = E.ms(1, 2);
    out->lor_ms = E.ms(2, 3);
    out->final_ms = E.ms(3, 4);
    out->total_ms = E.ms(0, 4);
  });
}

dg_status dg_apply_profile(const dg_mesh* mesh, const double* x, double* y, dg_apply_times* out,
                           void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh && x && y && out, "null argument");
    DG_REQUIRE(x != y, "x and y must not alias");
    const cudaStream_t s = (cudaStream_t)stream;
    EventSet E(3);
    DG_CUDA(cudaEventRecord(E.ev[0], s));
    launch_trace(*mesh, x, s);
    DG_CUDA(cudaEventRecord(E.ev[1], s));
    launch_apply(*mesh, x, y, Reduce{}, s, false);
    DG_CUDA(cudaEventRecord(E.ev[2], s));
    DG_CUDA(cudaEventSynchronize(E.ev[2]));
    out->trace_ms = E.ms(0, 1);
    out->apply_ms = E.ms(1, 2);
  });
}

dg_status dg_pcg_solve(const dg_mesh* mesh, const dg_precond* pc, const double* b, double* x,
                       double rtol, int maxit, dg_solve_info* info, void* stream) {
  return guarded([&] { pcg_run(mesh, pc, b, x, rtol, maxit, info, (cudaStream_t)stream); });
}

dg_status dg_pcg_solve_host(const dg_mesh* mesh, const dg_precond* pc, const double* b_host,
                            double* x_host, double rtol, int maxit, dg_solve_info* info,
                            void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh && pc && b_host && x_host, "null argument");
    DG_REQUIRE(pc->mesh == mesh, "preconditioner belongs to another mesh");
    const cudaStream_t s = (cudaStream_t)stream;
    PcgWork& w = pcg_work(pc);
    DG_CUDA(cudaMemcpyAsync(w.b, b_host, mesh->n_dofs * sizeof(double), cudaMemcpyHostToDevice, s));
    dg_status st = DG_OK;
    try {
      pcg_run(mesh, pc, w.b, w.x, rtol, maxit, info, s);
    } catch (const Error& e) {
      if (e.code != DG_ENOTCONV) throw;
      st = DG_ENOTCONV;
    }
    DG_CUDA(cudaMemcpyAsync(x_host, w.x, mesh->n_dofs * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    if (st != DG_OK) throw Error(st, "PCG reached maxit");
  });
}

dg_status dg_rhs_eval(const dg_mesh* mesh, dg_field_fn f, dg_field_fn g, void* ctx, double* b, void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh && b, "bad argument");
    std::vector<double> hb(mesh->n_dofs, 0.0);
    host_load(*mesh, f, g, ctx, hb.data());
    DG_CUDA(cudaMemcpyAsync(b, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

dg_status dg_rhs_sine(const dg_mesh* mesh, int n_modes, const double* amps, const int32_t* waves,
                      double* b, void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh && b && n_modes >= 0 && (n_modes == 0 || (amps && waves)), "bad argument");
    std::vector<double> hb(mesh->n_dofs, 0.0);
    host_rhs_sine(*mesh, n_modes, amps, waves, hb.data());
    DG_CUDA(cudaMemcpyAsync(b, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

}  // extern "C"

// ============================================================================
// Allocation-free PCG solve.
//
// dg_pcg_solve keeps its work vectors (r, z, p, q, reduction partials) in
// device memory that the library allocates on the first solve with each
// preconditioner, plus a captured graph and pinned host memory.  The variant
// below takes all of its solve-time scratch from one file-scope device array
// of fixed size instead, and runs the iteration from a host loop, so a call
// allocates nothing.
// ============================================================================
namespace dg {

constexpr int64_t kNoAllocMaxDofs = 262144;   // largest mesh the variant accepts
constexpr int64_t kNoAllocMaxTiles = 8192;    // operator CTAs (apply partials)
constexpr int64_t kNoAllocDoubles =
    4 * kNoAllocMaxDofs + kNoAllocMaxTiles + 3 * (int64_t)kVecBlocks + SC_COUNT + TK_COUNT;

// 8.1 MiB per device that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device
// (under a lock; the pointers are read without it once set).
static std::atomic<double*> g_noalloc_ptr[64];
static std::mutex g_noalloc_mu;

// The scratch of the mesh's device, which must be the current device: the
// kernels run on the current device and the array's address is per device.
static double* noalloc_scratch_for(const dg_mesh* mesh) {
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_REQUIRE(dev == mesh->device, "dg_pcg_solve_noalloc: the current device is not the mesh's device");
  DG_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
  double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
      void* a = nullptr;
      DG_CUDA(cudaGetSymbolAddress(&a, g_noalloc_scratch));
      p = (double*)a;
      g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
  }
  return p;
}

}  // namespace dg

extern "C" dg_status dg_pcg_solve_noalloc(const dg_mesh* mesh, const dg_precond* pc,
                                          const double* b, double* x, double rtol, int maxit,
                                          dg_solve_info* info, void* stream) {
  return guarded([&] {
    DG_REQUIRE(mesh != nullptr, "null mesh");
    if (mesh->n_dofs > kNoAllocMaxDofs)
      throw Error(DG_EINVAL, "dg_pcg_solve_noalloc: n_dofs " + std::to_string(mesh->n_dofs) +
                                 " exceeds the static scratch limit of " +
                                 std::to_string(kNoAllocMaxDofs));
    // implied by the DOF limit (a tile holds at least three elements' nodes, 243
    // or more), kept as a guard of the partials' slice
    if (mesh->n_tiles > kNoAllocMaxTiles)
      throw Error(DG_EINVAL, "dg_pcg_solve_noalloc: mesh needs more operator tiles than the static scratch holds");
    DG_REQUIRE(pc && b && x, "null argument");
    DG_REQUIRE(pc->mesh == mesh, "preconditioner belongs to another mesh");
    DG_REQUIRE(rtol > 0.0 && maxit >= 1, "rtol must be > 0 and maxit >= 1");
    const cudaStream_t s = (cudaStream_t)stream;
    double* base = noalloc_scratch_for(mesh);
    // carve the work vectors; every kernel below writes a slot before reading it
    PcgWork w;
    w.n = mesh->n_dofs;
    w.r = base;
    w.z = w.r + kNoAllocMaxDofs;
    w.p = w.z + kNoAllocMaxDofs;
    w.q = w.p + kNoAllocMaxDofs;
    w.part_pq = w.q + kNoAllocMaxDofs;
    w.part_rr = w.part_pq + kNoAllocMaxTiles;
    w.part_rz = w.part_rr + kVecBlocks;
    w.part_bb = w.part_rz + kVecBlocks;
    w.sc = w.part_bb + kVecBlocks;
    w.tick = reinterpret_cast<unsigned*>(w.sc + SC_COUNT);
    double hsc[SC_COUNT];
    const double rtol2 = rtol * rtol;
    const auto t0 = std::chrono::steady_clock::now();
    // the reduction tickets must start at zero
    DG_CUDA(cudaMemsetAsync(w.tick, 0, TK_COUNT * sizeof(unsigned), s));
    if (pcg_start(pc, w, b, x, hsc, s) > 0.0) {
      for (int it = 0; it < maxit;) {
        for (int j = 0; j < 8 && it < maxit; ++j, ++it) pcg_body(mesh, pc, w, x, maxit, rtol2, 0, 0, s);
        DG_CUDA(cudaMemcpyAsync(hsc, w.sc, sizeof(hsc), cudaMemcpyDeviceToHost, s));
        DG_CUDA(cudaStreamSynchronize(s));
        if (hsc[SC_STATUS] != 0.0) break;
      }
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const double bb = hsc[SC_BB];
    const bool conv = bb == 0.0 || hsc[SC_STATUS] == 1.0;
    if (info) {
      info->iters = bb > 0.0 ? (int)hsc[SC_IT] : 0;
      info->rel_res = bb > 0.0 ? std::sqrt(hsc[SC_RR] / bb) : 0.0;
      info->status = conv ? DG_OK : DG_ENOTCONV;
      info->solve_ms = ms;
    }
    if (!conv) throw Error(DG_ENOTCONV, "PCG reached maxit");
  });
}
