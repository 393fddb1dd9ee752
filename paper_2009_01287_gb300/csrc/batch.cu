// Batched solver: many independent hp-DG problems, each with several
// right-hand sides, solved together by one graph launch.
//
// Every (problem, right-hand side) pair is an "instance".  The union of all
// instances is one block-diagonal system: the operator kernel runs over all
// elements of all instances at once, the preconditioner is the union of the
// instances' preconditioners (union.cu), and PCG keeps its scalars per
// instance: the dot products are segmented reductions over fixed chunks of
// each instance's DOF range, alpha, beta and the stopping test are per
// instance, and an instance that has converged stops updating its x, r, p.
// Each instance therefore follows exactly the iteration it would follow
// alone.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <thread>

#include "kernels.cuh"
#include "precond_setup.h"
#include "union.h"

namespace dg {

constexpr int kChunk = 2048;       // DOFs per reduction chunk
constexpr int kSegThreads = 256;

enum { BS_RZ = 0, BS_BB = 1, BS_RR = 2, BS_IT = 3, BS_STATUS = 4, BS_RZNEW = 5, BS_PQ = 6, BS_N = 8 };

struct SegView {
  const int32_t* c_inst;    // chunk -> instance
  const int64_t* c_beg;     // chunk DOF range [beg, end)
  const int64_t* c_end;
  const int32_t* i_cfirst;  // instance -> first chunk (n_inst + 1)
  int nchunks;
  int ninst;
};

// sum of an instance's chunk partials, in chunk order, by the whole CTA
__device__ __forceinline__ double inst_sum(const SegView& v, const double* part, int inst, double* red) {
  const int c0 = v.i_cfirst[inst], c1 = v.i_cfirst[inst + 1];
  double s = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += kSegThreads) s += __ldcg(part + c);
  return block_sum<kSegThreads>(s, red);
}

__global__ void __launch_bounds__(kSegThreads)
seg_dot_kernel(SegView v, const double* __restrict__ a, const double* __restrict__ b,
               double* __restrict__ part) {
  pdl_entry();
  __shared__ double red[kSegThreads];
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    double s = 0.0;
    for (int64_t i = v.c_beg[c] + threadIdx.x; i < v.c_end[c]; i += kSegThreads) s += a[i] * b[i];
    s = block_sum<kSegThreads>(s, red);
    if (threadIdx.x == 0) part[c] = s;
  }
}

__global__ void __launch_bounds__(kSegThreads)
seg_init_kernel(SegView v, const double* __restrict__ b, double* __restrict__ x,
                double* __restrict__ r, double* __restrict__ part) {
  pdl_entry();
  __shared__ double red[kSegThreads];
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    double s = 0.0;
    for (int64_t i = v.c_beg[c] + threadIdx.x; i < v.c_end[c]; i += kSegThreads) {
      const double bi = b[i];
      x[i] = 0.0;
      r[i] = bi;
      s += bi * bi;
    }
    s = block_sum<kSegThreads>(s, red);
    if (threadIdx.x == 0) part[c] = s;
  }
}

// per-instance start: rz, bb from the chunk partials; status 1 for b = 0
__global__ void __launch_bounds__(kSegThreads)
seg_start_kernel(SegView v, const double* part_rz, const double* part_bb, double* sc,
                 unsigned* n_done) {
  pdl_entry();
  __shared__ double red[kSegThreads];
  for (int i = blockIdx.x; i < v.ninst; i += gridDim.x) {
    const double rz = inst_sum(v, part_rz, i, red);
    const double bb = inst_sum(v, part_bb, i, red);
    if (threadIdx.x == 0) {
      double* s = sc + BS_N * i;
      s[BS_RZ] = rz;
      s[BS_BB] = bb;
      s[BS_RR] = bb;
      s[BS_IT] = 0.0;
      s[BS_STATUS] = (bb == 0.0) ? 1.0 : 0.0;
      if (bb == 0.0) atomicAdd(n_done, 1u);
    }
  }
}

__global__ void __launch_bounds__(kSegThreads)
seg_copy_kernel(SegView v, const double* __restrict__ z, double* __restrict__ p) {
  pdl_entry();
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x)
    for (int64_t i = v.c_beg[c] + threadIdx.x; i < v.c_end[c]; i += kSegThreads) p[i] = z[i];
}

__global__ void __launch_bounds__(kSegThreads)
seg_update_xr_kernel(SegView v, double* __restrict__ x, double* __restrict__ r,
                     const double* __restrict__ p, const double* __restrict__ q, const double* sc,
                     const double* part_pq, double* part_rr) {
  pdl_entry();
  __shared__ double red[kSegThreads];
  __shared__ double s_q;
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int inst = v.c_inst[c];
    const double* s = sc + BS_N * inst;
    if (s[BS_STATUS] != 0.0) {
      if (threadIdx.x == 0) part_rr[c] = 0.0;
      continue;
    }
    const double pq = inst_sum(v, part_pq, inst, red);
    if (threadIdx.x == 0) s_q = s[BS_RZ] / pq;   // one FP64 division per chunk
    __syncthreads();
    const double alpha = s_q;
    double acc = 0.0;
    for (int64_t i = v.c_beg[c] + threadIdx.x; i < v.c_end[c]; i += kSegThreads) {
      x[i] = fma(alpha, p[i], x[i]);
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      acc += ri * ri;
    }
    acc = block_sum<kSegThreads>(acc, red);
    if (threadIdx.x == 0) part_rr[c] = acc;
  }
}

// p = z + beta p per instance; the last chunk of an instance advances its
// scalars and tests convergence; the last CTA sets the graph's while condition
__global__ void __launch_bounds__(kSegThreads)
seg_update_p_kernel(SegView v, double* __restrict__ p, const double* __restrict__ z, double* sc,
                    const double* part_rz, const double* part_rr, unsigned* inst_ticket,
                    unsigned* grid_ticket, unsigned* n_done, int maxit, double rtol2,
                    cudaGraphConditionalHandle h, int use_cond) {
  pdl_entry();
  __shared__ double red[kSegThreads];
  __shared__ unsigned s_last;
  __shared__ double s_q;
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int inst = v.c_inst[c];
    double* s = sc + BS_N * inst;
    if (s[BS_STATUS] != 0.0) continue;
    const double rz_new = inst_sum(v, part_rz, inst, red);
    if (threadIdx.x == 0) s_q = rz_new / s[BS_RZ];   // one FP64 division per chunk
    __syncthreads();
    const double beta = s_q;
    for (int64_t i = v.c_beg[c] + threadIdx.x; i < v.c_end[c]; i += kSegThreads)
      p[i] = fma(beta, p[i], z[i]);
    const double rr = inst_sum(v, part_rr, inst, red);   // every CTA reads rz before its ticket
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned nch = (unsigned)(v.i_cfirst[inst + 1] - v.i_cfirst[inst]);
      s_last = (atomicAdd(inst_ticket + inst, 1u) == nch - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      const double it = s[BS_IT] + 1.0;
      s[BS_IT] = it;
      s[BS_RR] = rr;
      s[BS_RZ] = rz_new;
      double st = 0.0;
      if (rr <= rtol2 * s[BS_BB]) st = 1.0;
      else if (it >= (double)maxit) st = 2.0;
      inst_ticket[inst] = 0u;
      if (st != 0.0) {
        __threadfence();
        s[BS_STATUS] = st;
        atomicAdd(n_done, 1u);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(grid_ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    *grid_ticket = 0u;
    __threadfence();
    const unsigned done = atomicAdd(n_done, 0u);
    if (use_cond) cudaGraphSetConditional(h, done < (unsigned)v.ninst ? 1u : 0u);
  }
}

}  // namespace dg

using namespace dg;

struct dg_batch {
  int n_problems = 0, n_rhs = 0, n_inst = 0;
  std::vector<std::unique_ptr<dg_mesh>> meshes;      // per problem, host data only
  std::vector<HostPrecond> hpc;
  std::vector<AmgHierarchy> amg;
  std::vector<int64_t> inst_off;                      // n_inst + 1
  dg_mesh U;                                          // union operator (device)
  dg_precond UP;                                      // union preconditioner (device)
  // segmented PCG
  DevArena arena;
  SegView seg{};
  int grid = 1;
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *part_pq = nullptr, *part_rz = nullptr, *part_rr = nullptr, *part_bb = nullptr;
  double* sc = nullptr;
  unsigned *inst_ticket = nullptr, *grid_ticket = nullptr, *n_done = nullptr;
  std::vector<double> hsc;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* g_x = nullptr;
  int g_maxit = -1;
  double g_rtol2 = -1.0;
  ~dg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    arena.release();
  }
};

namespace dg {

// operator tiles of the union: per instance, degree-sorted runs of at most
// U.tile_epb[p] elements; tiles never span two instances, so a converged
// instance's tiles can be skipped
static void build_batch_tiles(dg_batch* B) {
  dg_mesh& U = B->U;
  const HostMesh& um = U.host;
  std::vector<int32_t> order;
  U.h_tiles.clear();
  int64_t e0 = 0;
  for (int i = 0; i < B->n_inst; ++i) {
    const int64_t ne = B->meshes[i / B->n_rhs]->host.n;
    std::vector<int32_t> loc(ne);
    for (int64_t e = 0; e < ne; ++e) loc[e] = (int32_t)(e0 + e);
    std::stable_sort(loc.begin(), loc.end(), [&](int32_t a, int32_t b) { return um.p[a] > um.p[b]; });
    for (int64_t j = 0; j < ne;) {
      const int P = um.p[loc[j]];
      int64_t l = j;
      while (l < ne && um.p[loc[l]] == P && l - j < U.tile_epb[P]) ++l;
      U.h_tiles.push_back({P, (int32_t)(order.size() + j), (int32_t)(l - j), i});
      j = l;
    }
    order.insert(order.end(), loc.begin(), loc.end());
    e0 += ne;
  }
  U.h_order = order;
  U.n_tiles = (int)U.h_tiles.size();
  build_face_items(&U);
}

static void retile_batch(dg_mesh*, void* ctx) { build_batch_tiles((dg_batch*)ctx); }

// union of the instances' operator data (host side), then upload
static void build_union_mesh(dg_batch* B, cudaStream_t s) {
  dg_mesh& U = B->U;
  const dg_mesh& first = *B->meshes[0];
  U.opts = first.opts;
  U.eta = first.eta;
  for (int p = 0; p <= kMaxP; ++p) U.boff[p] = first.boff[p];
  // basis tables are identical in every mesh: take the first mesh's prefix
  const int basis_len = first.boff[kMaxP].d1 + kMaxP + 1;
  U.h_tables.assign(first.h_tables.begin(), first.h_tables.begin() + basis_len);
  std::vector<int64_t> tshift(B->n_problems);
  for (int k = 0; k < B->n_problems; ++k) {
    const dg_mesh& M = *B->meshes[k];
    tshift[k] = (int64_t)U.h_tables.size() - basis_len;
    U.h_tables.insert(U.h_tables.end(), M.h_tables.begin() + basis_len, M.h_tables.end());
  }
  DG_REQUIRE(U.h_tables.size() < (1ULL << 31), "face tables too large");
  HostMesh& um = U.host;
  um.n = 0;
  um.off.assign(1, 0);
  um.sf_ptr.assign(1, 0);
  U.stats = dg_mesh_stats{};
  for (int i = 0; i < B->n_inst; ++i) {
    const int k = i / B->n_rhs;
    const dg_mesh& M = *B->meshes[k];
    const HostMesh& m = M.host;
    const int64_t e0 = um.n, d0 = um.off.back();
    const int32_t s0 = (int32_t)U.h_sf.size();
    um.p.insert(um.p.end(), m.p.begin(), m.p.end());
    um.coef.insert(um.coef.end(), m.coef.begin(), m.coef.end());
    for (int64_t e = 0; e < m.n; ++e) um.off.push_back(d0 + m.off[e + 1]);
    for (int64_t j = 1; j <= 4 * m.n; ++j) um.sf_ptr.push_back(s0 + m.sf_ptr[j]);
    U.h_h.insert(U.h_h.end(), M.h_h.begin(), M.h_h.end());
    for (const SubFaceRec& f : M.h_sf) {
      SubFaceRec g = f;
      if (g.nb >= 0) g.nb += (int32_t)e0;
      g.tab_oo += (int32_t)tshift[k];
      g.tab_on += (int32_t)tshift[k];
      g.tab_nn += (int32_t)tshift[k];
      U.h_sf.push_back(g);
    }
    for (const SubFaceBr2& b : M.h_sfb) {   // BR2: one per record, in the same order
      SubFaceBr2 g = b;
      g.tab_z += (int32_t)tshift[k];
      g.tab_v += (int32_t)tshift[k];
      g.tab_x += (int32_t)tshift[k];
      g.tab_y += (int32_t)tshift[k];
      U.h_sfb.push_back(g);
    }
    um.n += m.n;
    U.stats.n_elems += M.stats.n_elems;
    U.stats.n_subfaces += M.stats.n_subfaces;
    U.stats.apply_flops += M.stats.apply_flops;
    U.stats.apply_bytes += M.stats.apply_bytes;
    U.stats.max_level_gap = std::max(U.stats.max_level_gap, M.stats.max_level_gap);
  }
  U.n_dofs = um.off.back();
  U.stats.n_dofs = U.n_dofs;
  DG_REQUIRE(U.n_dofs < (1LL << 31) && um.n < (1LL << 31), "batch too large for 32-bit indices");
  build_batch_tiles(B);
  upload_mesh(&U, s);
}

static void batch_alloc(dg_batch* B) {
  const int64_t n = B->U.n_dofs;
  std::vector<int32_t> c_inst, i_cfirst;
  std::vector<int64_t> c_beg, c_end;
  for (int i = 0; i < B->n_inst; ++i) {
    i_cfirst.push_back((int32_t)c_inst.size());
    for (int64_t a = B->inst_off[i]; a < B->inst_off[i + 1]; a += kChunk) {
      c_inst.push_back(i);
      c_beg.push_back(a);
      c_end.push_back(std::min(a + kChunk, B->inst_off[i + 1]));
    }
  }
  i_cfirst.push_back((int32_t)c_inst.size());
  DevArena& a = B->arena;
  B->seg.c_inst = a.upload(c_inst, nullptr);
  B->seg.c_beg = a.upload(c_beg, nullptr);
  B->seg.c_end = a.upload(c_end, nullptr);
  B->seg.i_cfirst = a.upload(i_cfirst, nullptr);
  B->seg.nchunks = (int)c_inst.size();
  B->seg.ninst = B->n_inst;
  B->grid = std::max(1, std::min(B->seg.nchunks, 8 * 152));
  B->r = a.alloc<double>(n);
  B->z = a.alloc<double>(n);
  B->p = a.alloc<double>(n);
  B->q = a.alloc<double>(n);
  const int nc = std::max(1, B->seg.nchunks);
  B->part_pq = a.alloc<double>(nc);
  B->part_rz = a.alloc<double>(nc);
  B->part_rr = a.alloc<double>(nc);
  B->part_bb = a.alloc<double>(nc);
  B->sc = a.alloc<double>((size_t)BS_N * B->n_inst);
  B->inst_ticket = a.alloc<unsigned>(B->n_inst);
  B->grid_ticket = a.alloc<unsigned>(1);
  B->n_done = a.alloc<unsigned>(1);
  DG_CUDA(cudaMemset(B->inst_ticket, 0, B->n_inst * sizeof(unsigned)));
  DG_CUDA(cudaMemset(B->grid_ticket, 0, sizeof(unsigned)));
  B->hsc.resize((size_t)BS_N * B->n_inst);
  DG_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  DG_CUDA(cudaEventCreate(&B->e0));
  DG_CUDA(cudaEventCreate(&B->e1));
  DG_CUDA(cudaDeviceSynchronize());
}

static void batch_body(dg_batch* B, double* x, int maxit, double rtol2,
                       cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  launch_apply(B->U, B->p, B->q, Reduce{}, s);
  launch_k(seg_dot_kernel, B->grid, kSegThreads, 0, s, B->seg, B->p, B->q, B->part_pq);
  launch_k(seg_update_xr_kernel, B->grid, kSegThreads, 0, s, B->seg, x, B->r, B->p, B->q, B->sc,
                                                        B->part_pq, B->part_rr);
  launch_precond(B->UP, B->r, B->z, Reduce{}, s);
  launch_k(seg_dot_kernel, B->grid, kSegThreads, 0, s, B->seg, B->r, B->z, B->part_rz);
  launch_k(seg_update_p_kernel, B->grid, kSegThreads, 0, s, B->seg, B->p, B->z, B->sc, B->part_rz,
                                                       B->part_rr, B->inst_ticket, B->grid_ticket,
                                                       B->n_done, maxit, rtol2, h, use_cond);
  DG_CUDA(cudaGetLastError());
}

static bool batch_capture(dg_batch* B, double* x, int maxit, double rtol2) {
  if (B->exec && B->g_x == x && B->g_maxit == maxit && B->g_rtol2 == rtol2) return true;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
  const char* env = std::getenv("DG_PCG_GRAPH");
  if (env && env[0] == '0') return false;
  cudaGraphConditionalHandle handle = 0;
  bool ok = false;
  if (cudaGraphCreate(&B->graph, 0) == cudaSuccess &&
      cudaGraphConditionalHandleCreate(&handle, B->graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, B->graph, nullptr, nullptr, 0, &cp) == cudaSuccess &&
        cudaStreamBeginCaptureToGraph(B->cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      bool launched = true;
      try {
        batch_body(B, x, maxit, rtol2, handle, 1, B->cap);
      } catch (const Error&) {
        launched = false;
      }
      cudaGraph_t out = nullptr;
      if (cudaStreamEndCapture(B->cap, &out) == cudaSuccess && launched &&
          cudaGraphInstantiate(&B->exec, B->graph, 0) == cudaSuccess)
        ok = true;
    }
  }
  cudaGetLastError();
  if (!ok) {
    if (B->graph) cudaGraphDestroy(B->graph);
    B->graph = nullptr;
    B->exec = nullptr;
    return false;
  }
  B->g_x = x;
  B->g_maxit = maxit;
  B->g_rtol2 = rtol2;
  return true;
}

}  // namespace dg

extern "C" {

dg_status dg_batch_create(const dg_mesh_desc* descs, int n_problems, int n_rhs,
                          const dg_options* opts, void* stream, dg_batch** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  std::unique_ptr<dg_batch> B(new dg_batch());
  try {
    DG_REQUIRE(descs && n_problems >= 1 && n_rhs >= 1, "bad batch size");
    for (int k = 0; k < n_problems; ++k)
      if (descs[k].dim != 2 || descs[k].corners || descs[k].map)
        throw Error(DG_EUNSUPPORTED, "the batched solver takes unmapped square meshes only");
    dg_options o{};
    o.form = DG_FORM_SIPG;
    o.precision = DG_PREC_MIXED;
    o.lor = DG_LOR_AMG;
    if (opts) o = *opts;
    DG_REQUIRE(o.lor == DG_LOR_AMG, "the batched solver uses the AMG LOR solve");
    DG_REQUIRE(o.form == DG_FORM_SIPG || o.eta > 0.0, "batched BR2 needs an explicit eta");
    B->n_problems = n_problems;
    B->n_rhs = n_rhs;
    B->n_inst = n_problems * n_rhs;
    B->meshes.resize(n_problems);
    B->hpc.resize(n_problems);
    B->amg.resize(n_problems);
    // host setup per problem, in parallel
    std::vector<std::string> errs(n_problems);
    std::vector<dg_status> codes(n_problems, DG_OK);
    const int nth = std::max(1, std::min<int>(n_problems, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t)
      pool.emplace_back([&, t] {
        SerialSetup serial;   // one problem per thread already
        for (int k = t; k < n_problems; k += nth) {
          try {
            B->meshes[k].reset(new dg_mesh());
            build_mesh_host(B->meshes[k].get(), &descs[k], &o);
            B->hpc[k] = build_host_precond(*B->meshes[k], o);
            B->amg[k] = amg_setup(B->hpc[k].Ac);
          } catch (const Error& e) {
            codes[k] = e.code;
            errs[k] = e.what();
          } catch (const std::exception& e) {
            codes[k] = DG_EINVAL;
            errs[k] = e.what();
          }
        }
      });
    for (auto& th : pool) th.join();
    for (int k = 0; k < n_problems; ++k)
      if (codes[k] != DG_OK) throw Error(codes[k], "problem " + std::to_string(k) + ": " + errs[k]);
    const cudaStream_t s = (cudaStream_t)stream;
    B->inst_off.assign(1, 0);
    for (int i = 0; i < B->n_inst; ++i)
      B->inst_off.push_back(B->inst_off.back() + B->meshes[i / n_rhs]->n_dofs);
    build_union_mesh(B.get(), s);
    if (o.tune_tiles) tune_tiles(&B->U, s, retile_batch, B.get());
    // union preconditioner
    B->UP.mesh = &B->U;
    B->UP.precision = o.precision;
    B->UP.lor = DG_LOR_AMG;
    B->UP.n_dofs = B->U.n_dofs;
    std::vector<InstSrc> inst;
    for (int i = 0; i < B->n_inst; ++i) inst.push_back({&B->hpc[i / n_rhs], &B->amg[i / n_rhs], B->inst_off[i]});
    if (o.precision == DG_PREC_MIXED) upload_union_precond<float>(&B->UP, inst, s);
    else upload_union_precond<double>(&B->UP, inst, s);
    batch_alloc(B.get());
    B->U.skip_status = B->sc + BS_STATUS;
    B->U.skip_stride = BS_N;
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
  *out = B.release();
  return DG_OK;
}

void dg_batch_destroy(dg_batch* b) { delete b; }

int64_t dg_batch_num_dofs(const dg_batch* b) { return b ? b->U.n_dofs : -1; }

dg_status dg_batch_offsets(const dg_batch* b, int64_t* offsets) {
  if (!b || !offsets) { set_last_error("null argument"); return DG_EINVAL; }
  std::copy(b->inst_off.begin(), b->inst_off.end(), offsets);
  return DG_OK;
}

dg_status dg_batch_stats_get(const dg_batch* b, dg_mesh_stats* out) {
  if (!b || !out) { set_last_error("null argument"); return DG_EINVAL; }
  *out = b->U.stats;
  out->device_bytes = (int64_t)(b->U.arena.bytes + b->U.tile_arena.bytes);
  if (!out->tiles_tuned)
    for (int p = 0; p <= kMaxP; ++p) out->tile_elems[p] = b->U.tile_epb[p];
  return DG_OK;
}

dg_status dg_batch_rhs_sine(const dg_batch* B, int n_modes, const double* amps,
                            const int32_t* waves, double* b, void* stream) {
  try {
    DG_REQUIRE(B && b && n_modes >= 0 && (n_modes == 0 || (amps && waves)), "bad argument");
    std::vector<double> hb(B->U.n_dofs, 0.0);
    std::vector<std::thread> pool;
    const int nth = std::max(1, std::min<int>(B->n_inst, (int)std::thread::hardware_concurrency()));
    for (int t = 0; t < nth; ++t)
      pool.emplace_back([&, t] {
        for (int i = t; i < B->n_inst; i += nth)
          host_rhs_sine(*B->meshes[i / B->n_rhs], n_modes, amps + (size_t)i * n_modes,
                        waves + (size_t)i * n_modes * 2, hb.data() + B->inst_off[i]);
      });
    for (auto& th : pool) th.join();
    DG_CUDA(cudaMemcpyAsync(b, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
  return DG_OK;
}

dg_status dg_batch_solve(dg_batch* B, const double* b, double* x, double rtol, int maxit,
                         dg_solve_info* results, double* solve_ms, void* stream) {
  try {
    DG_REQUIRE(B && b && x && results, "null argument");
    DG_REQUIRE(rtol > 0.0 && maxit >= 1, "rtol must be > 0 and maxit >= 1");
    const cudaStream_t s = (cudaStream_t)stream;
    const double rtol2 = rtol * rtol;
    const bool use_graph = batch_capture(B, x, maxit, rtol2);
    DG_CUDA(cudaEventRecord(B->e0, s));
    DG_CUDA(cudaMemsetAsync(B->n_done, 0, sizeof(unsigned), s));
    launch_k(seg_init_kernel, B->grid, kSegThreads, 0, s, B->seg, b, x, B->r, B->part_bb);
    launch_precond(B->UP, B->r, B->z, Reduce{}, s);
    launch_k(seg_dot_kernel, B->grid, kSegThreads, 0, s, B->seg, B->r, B->z, B->part_rz);
    launch_k(seg_start_kernel, std::max(1, std::min(B->n_inst, 8 * 152)), kSegThreads, 0, s, 
        B->seg, B->part_rz, B->part_bb, B->sc, B->n_done);
    launch_k(seg_copy_kernel, B->grid, kSegThreads, 0, s, B->seg, B->z, B->p);
    DG_CUDA(cudaGetLastError());
    if (use_graph) {
      DG_CUDA(cudaGraphLaunch(B->exec, s));
    } else {
      unsigned done = 0;
      for (int it = 0; it < maxit;) {
        for (int j = 0; j < 8 && it < maxit; ++j, ++it) batch_body(B, x, maxit, rtol2, 0, 0, s);
        DG_CUDA(cudaMemcpyAsync(&done, B->n_done, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        DG_CUDA(cudaStreamSynchronize(s));
        if ((int)done >= B->n_inst) break;
      }
    }
    DG_CUDA(cudaEventRecord(B->e1, s));
    DG_CUDA(cudaMemcpyAsync(B->hsc.data(), B->sc, B->hsc.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    DG_CUDA(cudaEventElapsedTime(&ms, B->e0, B->e1));
    if (solve_ms) *solve_ms = ms;
    bool all = true;
    for (int i = 0; i < B->n_inst; ++i) {
      const double* sc = B->hsc.data() + (size_t)BS_N * i;
      results[i].iters = (int)sc[BS_IT];
      results[i].rel_res = sc[BS_BB] > 0.0 ? std::sqrt(sc[BS_RR] / sc[BS_BB]) : 0.0;
      results[i].status = sc[BS_STATUS] == 1.0 ? DG_OK : DG_ENOTCONV;
      results[i].solve_ms = ms;
      all = all && sc[BS_STATUS] == 1.0;
    }
    if (!all) throw Error(DG_ENOTCONV, "some instances reached maxit");
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return DG_EINVAL;
  }
  return DG_OK;
}

}  // extern "C"
