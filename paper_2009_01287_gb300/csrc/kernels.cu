// Device kernels: preconditioner pieces (Section 4.1: P^T, LOR solve, P, point
// Jacobi, block solves) and the PCG vector work.  The operator's launch code
// is in apply_launch.cu.
#include <cstdio>
#include <type_traits>

#include "kernels.cuh"

namespace dg {

// ============================================================== preconditioner

// ---- CSR row kernels in three tiers (the rows of P^T and of the AMG levels
// are very uneven): rows longer than kCsrCtaRow entries take one CTA each
// (entries strided over the CTA, fixed block tree), rows longer than
// long_min take one warp each (fixed shuffle tree), and the rest are read by
// G lanes per row (fixed shuffle tree over G).  The grid holds the CTA-tier
// CTAs first, then the warp tier (8 rows per CTA), then the group tier, whose
// row loop advances by whole warps so that every lane reaches the shuffles.
// Every sum has a fixed order, so the results are deterministic.
template <typename T, int G, class Op>
__global__ void __launch_bounds__(kVecThreads)
csr_rows_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                const T* __restrict__ val, int64_t rows, CsrTiers tiers, const Op op_arg) {
  pdl_entry();
  const Op op = op_arg.bind();   // per-thread values an operation loads once (after the wait)
  int bid = blockIdx.x;
  if (bid < tiers.n_cta) {
    __shared__ double sred[kVecThreads];
    const int row = __ldg(tiers.cta_rows + bid);
    const int e = ptr[row + 1];
    T s = 0;
    for (int t = ptr[row] + threadIdx.x; t < e; t += kVecThreads) s += __ldg(val + t) * op.x(__ldg(idx + t));
    pdl_trigger();
    const double tot = block_sum<kVecThreads>((double)s, sred);
    if (threadIdx.x == 0) op.store(row, (T)tot);
    return;
  }
  bid -= tiers.n_cta;
  const int warp_ctas = (tiers.n_warp + 7) >> 3;
  if (bid < warp_ctas) {
    const int w = bid * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= tiers.n_warp) return;   // whole warps leave together
    const int row = __ldg(tiers.warp_rows + w);
    const int e = ptr[row + 1];
    T s = 0;
    for (int t = ptr[row] + lane; t < e; t += 32) s += __ldg(val + t) * op.x(__ldg(idx + t));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) op.store(row, s);
    return;
  }
  bid -= warp_ctas;
  const int nb = gridDim.x - tiers.n_cta - warp_ctas;
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)nb * blockDim.x) / G;
  const int64_t g0 = (bid * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (rows + groups_per_grid - 1) / groups_per_grid;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t row = g0 + rd * groups_per_grid;
    T s = 0;
    bool mine = false;
    if (row < rows) {
      const int b = ptr[row], e = ptr[row + 1];
      mine = e - b <= tiers.long_min;
      if (mine)
        for (int t = b + lane; t < e; t += G) s += __ldg(val + t) * op.x(__ldg(idx + t));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (mine && lane == 0) op.store(row, s);
  }
}

// Entry j of the residual a preconditioner kernel reads: r_j, or with a
// deferred PCG update (XrDefer) r_j - alpha q_j, by the same FMA in every
// kernel and in the final kernel that stores it.  r is not written while the
// readers run (the final kernel stores it after they end).
__device__ __forceinline__ double resid_in(const double* r, const double* q, double alpha, int64_t j) {
  const double rj = __ldg(r + j);
  return q ? fma(-alpha, __ldg(q + j), rj) : rj;
}

template <typename T>
struct OpSpmv {  // y = A v
  const T* v;
  T* y;
  __device__ OpSpmv bind() const { return *this; }
  __device__ T x(int j) const { return __ldg(v + j); }
  __device__ void store(int64_t i, T s) const { y[i] = s; }
};
template <typename T>
struct OpRestrict {  // out = P^T r, r in FP64 (with q: r - alpha q, see XrDefer)
  const double* r;
  T* out;
  const double* q = nullptr;
  const double* alpha = nullptr;
  double a = 0.0;   // *alpha, loaded once per thread by bind()
  __device__ OpRestrict bind() const {
    OpRestrict o = *this;
    if (q) o.a = __ldg(alpha);
    return o;
  }
  __device__ T x(int j) const { return (T)resid_in(r, q, a, j); }
  __device__ void store(int64_t i, T s) const { out[i] = s; }
};
// plain V-cycle level (D = diag(l1 row sums)):
template <typename T>
struct OpResid {  // out = b - A D^-1 b (pre-smoothing from zero, then the residual)
  const T* b;
  const T* dinv;
  T* out;
  __device__ OpResid bind() const { return *this; }
  __device__ T x(int j) const { return __ldg(b + j) * __ldg(dinv + j); }
  __device__ void store(int64_t i, T s) const { out[i] = b[i] - s; }
};
template <typename T>
struct OpCorr {  // out = D^-1 b + P xc (pre-smoothed iterate plus coarse correction)
  const T* b;
  const T* dinv;
  const T* xc;
  T* out;
  __device__ OpCorr bind() const { return *this; }
  __device__ T x(int j) const { return __ldg(xc + j); }
  __device__ void store(int64_t i, T s) const { out[i] = fma(b[i], dinv[i], s); }
};
template <typename T>
struct OpPost {  // out = xp + D^-1 (b - A xp) (post-smoothing)
  const T* xp;
  const T* b;
  const T* dinv;
  T* out;
  __device__ OpPost bind() const { return *this; }
  __device__ T x(int j) const { return __ldg(xp + j); }
  __device__ void store(int64_t i, T s) const { out[i] = fma(dinv[i], b[i] - s, xp[i]); }
};

template <typename T, class Op>
static void launch_rows(const DevCsr& A, const Op& op, cudaStream_t s) {
  if (A.rows == 0) return;
  int64_t threads = A.rows * (int64_t)A.group;
  int64_t blocks = (threads + kVecThreads - 1) / kVecThreads;
  if (blocks > 8 * 152) blocks = 8 * 152;
  const int32_t* p = A.ptr;
  const int32_t* ix = A.idx;
  const T* v = (const T*)A.val;
  const CsrTiers tr{A.cta_rows, A.warp_rows, A.n_cta, A.n_warp, A.long_min};
  const int g = (int)blocks + A.n_cta + (A.n_warp + 7) / 8;
#define DG_ROWS(G) launch_k(csr_rows_kernel<T, G, Op>, g, kVecThreads, 0, s, p, ix, v, A.rows, tr, op)
  switch (A.group) {
    case 1: DG_ROWS(1); break;
    case 2: DG_ROWS(2); break;
    case 4: DG_ROWS(4); break;
    case 8: DG_ROWS(8); break;
    case 16: DG_ROWS(16); break;
    default: DG_ROWS(32); break;
  }
#undef DG_ROWS
}

// dense y = Ainv x, one warp per row
template <typename T>
__global__ void dense_mv_kernel(const T* __restrict__ Ainv, const T* __restrict__ x,
                                T* __restrict__ y, int64_t n) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += warps) {
    T s = 0;
    for (int64_t j = lane; j < n; j += 32) s += __ldg(Ainv + row * n + j) * __ldg(x + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
  }
}

// Small V_e blocks packed into one warp: segment g of W lanes (W a power of
// two >= the block sizes) takes the g-th block of the unit, lane rr of the
// segment forms row rr.  Same column order and four accumulators (by column
// mod 4) as the panel path, so a block's result does not depend on the path.
template <typename T, int W>
__device__ __forceinline__ void block_solve_packed(const int4 h, const int4* __restrict__ brec,
                                                   const int32_t* __restrict__ dofs,
                                                   const T* __restrict__ inv, const double* __restrict__ r,
                                                   const double* __restrict__ q, double alpha,
                                                   T* __restrict__ zE, int lane) {
  const int seg = lane / W, rr = lane % W;
  const bool has = seg < h.y;   // h = {first block (sorted order), block count, 0, W}
  const int4 br = has ? __ldg(brec + h.x + seg) : make_int4(0, 0, 0, 0);   // {slot, d, inverse offset}
  const int d = br.y;
  const bool act = rr < d;
  const T* At = inv + ((int64_t)(unsigned)br.z | ((int64_t)br.w << 32)) + rr;
  const T rv = act ? (T)resid_in(r, q, alpha, __ldg(dofs + br.x + rr)) : (T)0;
  T v[W];
#pragma unroll
  for (int c = 0; c < W; ++c) v[c] = (act && c < d) ? __ldg(At + (int64_t)c * d) : (T)0;
  T a[4] = {0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < W; ++c) a[c & 3] = fma(v[c], __shfl_sync(0xffffffffu, rv, c, W), a[c & 3]);
  if (act) zE[br.x + rr] = (a[0] + a[1]) + (a[2] + a[3]);
}

// V_e block solves (Section 3.3, T_E = sum_e P_e): z_e = A_e^-1 r_e.  A work
// unit is taken by one warp: either a panel of 32 consecutive rows of one
// block (lane l forms row row0 + l over all d columns), or up to 32 / W small
// blocks of at most W rows side by side (block_solve_packed).  The inverses
// are stored column-major, so every step reads consecutive entries of one
// column; the block's residual entries are gathered 32 at a time, one per
// lane, and reach the other lanes by shuffles.  No shared memory and no block
// barrier; a warp issues a whole chunk of column loads before its first FMA.
// Units are sorted by work (largest blocks first) and dealt round-robin over
// the grid's warps.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 3)
block_solve_kernel(const int4* __restrict__ unit, const int64_t* __restrict__ ubase,
                   const int4* __restrict__ brec, const int32_t* __restrict__ dofs,
                   const T* __restrict__ inv, const double* __restrict__ r,
                   const double* __restrict__ q, const double* alpha_p, T* __restrict__ zE, int nunits) {
  pdl_entry();
  const double alpha = q ? __ldg(alpha_p) : 0.0;   // deferred PCG step (XrDefer)
  constexpr int H = 16;   // column loads per lane in one batch
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
    const int4 h = __ldg(unit + u);   // panel: {slot of the block's first node, d, row0, 0}
    if (h.w == 4) { block_solve_packed<T, 4>(h, brec, dofs, inv, r, q, alpha, zE, lane); continue; }
    if (h.w == 8) { block_solve_packed<T, 8>(h, brec, dofs, inv, r, q, alpha, zE, lane); continue; }
    if (h.w == 16) { block_solve_packed<T, 16>(h, brec, dofs, inv, r, q, alpha, zE, lane); continue; }
    const int d = h.y, row = h.z + lane;
    const bool act = row < d;
    const T* At = inv + __ldg(ubase + u) + lane;   // column 0 of this lane's row
    const int32_t* ds = dofs + h.x;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int c0 = 0; c0 < d; c0 += 32) {
      const T rv = c0 + lane < d ? (T)resid_in(r, q, alpha, __ldg(ds + c0 + lane)) : (T)0;
#pragma unroll
      for (int hh = 0; hh < 32; hh += H) {
        const int cnt = d - c0 - hh;   // columns left from this half on
        const T* Ac = At + (int64_t)(c0 + hh) * d;
        T v[H];
#pragma unroll
        for (int j = 0; j < H; ++j) v[j] = (act && j < cnt) ? __ldg(Ac + (int64_t)j * d) : (T)0;
#pragma unroll
        for (int j = 0; j < H; j += 4) {
          a0 = fma(v[j], __shfl_sync(0xffffffffu, rv, hh + j), a0);
          a1 = fma(v[j + 1], __shfl_sync(0xffffffffu, rv, hh + j + 1), a1);
          a2 = fma(v[j + 2], __shfl_sync(0xffffffffu, rv, hh + j + 2), a2);
          a3 = fma(v[j + 3], __shfl_sync(0xffffffffu, rv, hh + j + 3), a3);
        }
      }
    }
    if (act) zE[h.x + row] = (a0 + a1) + (a2 + a3);
  }
}

// CTAs of the final kernel resident per SM: its launch bound (48 registers,
// no spills; 8 per SM would cap it at 32 registers and spill) and its grid
// cap (one wave on 152 SMs)
constexpr int kFinalCtasPerSm = 5;

// z = P e_C + D_J^-1 r + (block result on V_e nodes), the r . z reduction and,
// when rr is given, the r . r reduction beside it (the PCG residual norm).
// With a deferred PCG update (xr.q) r is r - alpha q, stored here with
// x += alpha p: every other reader of r has finished when this kernel runs.
// G lanes per DG row share its P entries; the row's own terms (r, D_J^-1, the
// block result) are loaded before the P entries so that both chains of loads
// are in flight together.
template <typename T, int G>
__global__ void __launch_bounds__(kVecThreads, kFinalCtasPerSm)
precond_final_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                     const T* __restrict__ val, const T* __restrict__ ec,
                     const T* __restrict__ dinv, const int32_t* __restrict__ e_pos,
                     const T* __restrict__ zE, const double* r,
                     double* __restrict__ z, int64_t n, Reduce red, Reduce rr, PcgCtl ctl, XrDefer xr) {
  pdl_entry();
  __shared__ double sred[kVecThreads];
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (n + groups_per_grid - 1) / groups_per_grid;
  double dot = 0.0, dot_rr = 0.0;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t i = g0 + rd * groups_per_grid;
    T s = 0, tj = 0, te = 0;
    double ri = 0.0;
    bool has_e = false;
    if (i < n) {
      if (lane == 0) {
        if (xr.q) {   // r is rewritten below: plain loads
          const double a = *xr.alpha;
          ri = fma(-a, xr.q[i], r[i]);
          xr.r_out[i] = ri;
          xr.x[i] = fma(a, xr.p[i], xr.x[i]);
        } else {
          ri = __ldg(r + i);
        }
        tj = __ldg(dinv + i) * (T)ri;
        const int ep = __ldg(e_pos + i);
        has_e = ep >= 0;
        if (has_e) te = __ldg(zE + ep);
      }
      for (int t = ptr[i] + lane; t < ptr[i + 1]; t += G) s += __ldg(val + t) * __ldg(ec + __ldg(idx + t));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (i < n && lane == 0) {
      s += tj;
      if (has_e) s += te;
      const double zi = (double)s;
      z[i] = zi;
      dot += zi * ri;
      dot_rr += ri * ri;
    }
  }
  pdl_trigger();   // rows done: the next kernel launches during the reductions
  if (rr.partial) {
    // the scalars the controller reads, loaded by thread 0 of every CTA before
    // the reductions (their latency overlaps them; only the last CTA uses
    // them, and no CTA writes them before every CTA has passed this point)
    double c_status = 0.0, c_it = 0.0, c_rz = 0.0, c_bb = 0.0, c_lim = 0.0, c_tol2 = 0.0;
    if (ctl.sc && threadIdx.x == 0) {
      const double* sc = ctl.sc;
      c_status = sc[SC_STATUS];
      c_it = sc[SC_IT];
      c_rz = sc[SC_RZ];
      c_bb = sc[SC_BB];
      c_lim = ctl.maxit < 0 ? sc[SC_MAXIT] : (double)ctl.maxit;
      c_tol2 = ctl.maxit < 0 ? sc[SC_RTOL2] : ctl.rtol2;
    }
    const double t1 = block_sum<kVecThreads>(dot, sred);
    const double t2 = block_sum<kVecThreads>(dot_rr, sred);
    double rz_new = 0.0, rr_new = 0.0;
    if (reduce_finalize2<kVecThreads>(t1, t2, red, rr, sred, &rz_new, &rr_new) && ctl.sc &&
        threadIdx.x == 0 && c_status == 0.0) {
      // iteration control (PcgCtl): this iteration's r . z and r . r are final
      // here; an iteration queued after a stop (host-driven loop) changes nothing
      double* sc = ctl.sc;
      const double it = c_it + 1.0;
      sc[SC_IT] = it;
      sc[SC_RR] = rr_new;
      sc[SC_BETA] = rz_new / c_rz;
      sc[SC_RZ] = rz_new;
      int cont = 1;
      if (rr_new <= c_tol2 * c_bb) { sc[SC_STATUS] = 1.0; cont = 0; }
      else if (it >= c_lim) { sc[SC_STATUS] = 2.0; cont = 0; }
      if (ctl.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)ctl.cond, cont ? 1u : 0u);
    }
  } else if (red.partial) {
    const double tot = block_sum<kVecThreads>(dot, sred);
    reduce_finalize<kVecThreads>(tot, red, sred);
  }
}

static int grid_for(int64_t n, int threads = kVecThreads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > kVecBlocks) b = kVecBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

int precond_final_blocks(const dg_precond& pc) {
  int64_t b = (pc.n_dofs + kVecThreads - 1) / kVecThreads;   // one lane per row
  if (b > kFinalCtasPerSm * 152) b = kFinalCtasPerSm * 152;   // one resident wave
  return (int)(b < 1 ? 1 : b);
}

// fused up-sweep of one AMG level: xo = Sb b + Sp xc (G lanes per row share
// both rows; fixed shuffle tree)
template <typename T, int G>
__global__ void __launch_bounds__(kVecThreads)
amg_up_kernel(const int32_t* __restrict__ bp, const int32_t* __restrict__ bi, const T* __restrict__ bv,
              const int32_t* __restrict__ pp, const int32_t* __restrict__ pi, const T* __restrict__ pv,
              const T* __restrict__ b, const T* __restrict__ xc, T* __restrict__ xo, int64_t rows) {
  pdl_entry();
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (rows + groups_per_grid - 1) / groups_per_grid;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t row = g0 + rd * groups_per_grid;
    T s = 0;
    if (row < rows) {
      for (int t = bp[row] + lane; t < bp[row + 1]; t += G) s += __ldg(bv + t) * __ldg(b + __ldg(bi + t));
      for (int t = pp[row] + lane; t < pp[row + 1]; t += G) s += __ldg(pv + t) * __ldg(xc + __ldg(pi + t));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (row < rows && lane == 0) xo[row] = s;
  }
}

template <typename T>
static void launch_up(const DevLevel& L, const T* b, const T* xc, T* xo, cudaStream_t s) {
  if (L.n_cont == 0) return;
  int64_t blocks = (L.n_cont * (int64_t)L.Sb.group_all + kVecThreads - 1) / kVecThreads;
  if (blocks > 8 * 152) blocks = 8 * 152;
#define DG_UP(G)                                                                                  \
  launch_k(amg_up_kernel<T, G>, (int)blocks, kVecThreads, 0, s, L.Sb.ptr, L.Sb.idx,              \
           (const T*)L.Sb.val, L.Sp.ptr, L.Sp.idx, (const T*)L.Sp.val, b, xc, xo, L.n_cont)
  switch (L.Sb.group_all) {
    case 1: DG_UP(1); break;
    case 2: DG_UP(2); break;
    case 4: DG_UP(4); break;
    case 8: DG_UP(8); break;
    case 16: DG_UP(16); break;
    default: DG_UP(32); break;
  }
#undef DG_UP
}

// y = W x for a dense row-major m x n matrix, one CTA per row (fixed block
// tree): the fused last restriction and coarsest solve of the V-cycle
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
dense_rect_kernel(const T* __restrict__ W, const T* __restrict__ x, T* __restrict__ y, int64_t m, int64_t n) {
  pdl_entry();
  __shared__ double sred[kVecThreads];
  // 16-byte loads when W and x start 16-byte aligned and a row holds a whole
  // number of them (every row then starts aligned too)
  constexpr int V = 16 / sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const bool vec = n % V == 0 && ((reinterpret_cast<uintptr_t>(W) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
  for (int64_t row = blockIdx.x; row < m; row += gridDim.x) {
    const T* w = W + row * n;
    T s = 0;
    if (vec) {
      const Vec* w4 = reinterpret_cast<const Vec*>(w);
      const Vec* x4 = reinterpret_cast<const Vec*>(x);
      for (int64_t j = threadIdx.x; j < n / V; j += kVecThreads) {
        const Vec a = __ldg(w4 + j), b = __ldg(x4 + j);
        const T* av = reinterpret_cast<const T*>(&a);
        const T* bv = reinterpret_cast<const T*>(&b);
#pragma unroll
        for (int u = 0; u < V; ++u) s += av[u] * bv[u];
      }
    } else {
      for (int64_t j = threadIdx.x; j < n; j += kVecThreads) s += __ldg(w + j) * __ldg(x + j);
    }
    const double tot = block_sum<kVecThreads>((double)s, sred);
    if (threadIdx.x == 0) y[row] = (T)tot;
  }
}

// dense solves of the coarsest blocks of a level: block j covers level rows
// [row[j], row[j+1]); blockIdx.y picks 8 rows of it (one per warp)
template <typename T>
__global__ void __launch_bounds__(256)
dense_blocks_kernel(const int32_t* __restrict__ row, const int64_t* __restrict__ inv_off,
                    const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ xo,
                    int nblocks) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y * 8 + (threadIdx.x >> 5);
  for (int j = blockIdx.x; j < nblocks; j += gridDim.x) {
    const int r0 = __ldg(row + j);
    const int d = __ldg(row + j + 1) - r0;
    if (l >= d) continue;
    const T* A = inv + __ldg(inv_off + j) + (int64_t)l * d;
    T s = 0;
    for (int m = lane; m < d; m += 32) s += __ldg(A + m) * __ldg(b + r0 + m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) xo[r0 + l] = s;
  }
}

template <typename T>
static void vcycle(const dg_precond& pc, size_t l, cudaStream_t s) {
  const DevLevel& L = pc.levels[l];
  if (L.n_cont > 0 && L.plain) {
    const DevLevel& C = pc.levels[l + 1];
    const T* b = (const T*)L.b;
    const T* dinv = (const T*)L.dinv;
    launch_rows<T>(L.A, OpResid<T>{b, dinv, (T*)L.t1}, s);                  // b - A D^-1 b
    launch_rows<T>(L.R, OpSpmv<T>{(const T*)L.t1, (T*)C.b}, s);             // restrict
    vcycle<T>(pc, l + 1, s);
    launch_rows<T>(L.P, OpCorr<T>{b, dinv, (const T*)C.xo, (T*)L.t2}, s);   // D^-1 b + P xc
    launch_rows<T>(L.A, OpPost<T>{(const T*)L.t2, b, dinv, (T*)L.xo}, s);   // post-smoothing
  } else if (L.n_cont > 0 && L.coarse_w) {
    // restriction and the dense coarsest solve in one product: C.xo = W b
    const DevLevel& C = pc.levels[l + 1];
    const int g = (int)std::min<int64_t>(L.coarse_w_rows, 8 * 152);
    launch_k(dense_rect_kernel<T>, g, kVecThreads, 0, s, (const T*)L.coarse_w, (const T*)L.b, (T*)C.xo,
             L.coarse_w_rows, L.n);
    launch_up<T>(L, (const T*)L.b, (const T*)C.xo, (T*)L.xo, s);    // correction + smoothing
  } else if (L.n_cont > 0) {
    const DevLevel& C = pc.levels[l + 1];
    launch_rows<T>(L.Rpre, OpSpmv<T>{(const T*)L.b, (T*)C.b}, s);   // restrict b - A D^-1 b
    vcycle<T>(pc, l + 1, s);
    launch_up<T>(L, (const T*)L.b, (const T*)C.xo, (T*)L.xo, s);    // correction + smoothing
  }
  if (L.n_end > 0 && L.max_end > 0) {
    const int gx = L.n_end < 8 * 152 ? L.n_end : 8 * 152;
    launch_k(dense_blocks_kernel<T>, dim3(gx, (L.max_end + 7) / 8), 256, 0, s, 
        L.end_row, L.end_inv_off, (const T*)L.end_inv, (const T*)L.b, (T*)L.xo, L.n_end);
  }
}

template <typename T>
static void precond_impl(const dg_precond& pc, const double* r, double* z, Reduce red,
                         cudaStream_t s, const PrecondMarks* mk, Reduce rr, PcgCtl ctl, XrDefer xr) {
  // fork: the block solves depend only on r (profiling: run them first, alone)
  if (mk) DG_CUDA(cudaEventRecord(mk->ev[0], s));
  if (pc.n_blocks > 0) {
    cudaStream_t bs = mk ? s : pc.side;
    if (!mk) {
      DG_CUDA(cudaEventRecord(pc.ev_fork, s));
      DG_CUDA(cudaStreamWaitEvent(pc.side, pc.ev_fork, 0));
    }
    // 8 warps per CTA; as many CTAs as the launch bounds keep resident on 152 SMs
    const int64_t gc = (pc.n_units + 7) / 8, gmax = (sizeof(T) == 8 ? 2 : 3) * 152;
    const int g = (int)(gc < gmax ? gc : gmax);
    launch_k(block_solve_kernel<T>, g, 256, 0, bs, (const int4*)pc.blk_unit, pc.blk_ubase,
        (const int4*)pc.blk_rec, pc.blk_dofs, (const T*)pc.blk_inv, r, xr.q, xr.alpha, (T*)pc.zE,
        (int)pc.n_units);
    DG_CUDA(cudaGetLastError());
    if (!mk) DG_CUDA(cudaEventRecord(pc.ev_join, pc.side));
  }
  if (mk) DG_CUDA(cudaEventRecord(mk->ev[1], s));
  const void* ec = nullptr;
  if (pc.n_c > 0) {
    if (pc.lor == DG_LOR_EXACT) {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.rc, xr.q, xr.alpha}, s);
      if (mk) DG_CUDA(cudaEventRecord(mk->ev[2], s));
      launch_k(dense_mv_kernel<T>, grid_for(pc.n_c * 32), kVecThreads, 0, s, 
          (const T*)pc.lor_inv, (const T*)pc.rc, (T*)pc.ec, pc.n_c);
      ec = pc.ec;
    } else {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.levels[0].b, xr.q, xr.alpha}, s);
      if (mk) DG_CUDA(cudaEventRecord(mk->ev[2], s));
      vcycle<T>(pc, 0, s);
      ec = pc.levels[0].xo;
    }
  } else if (mk) {
    DG_CUDA(cudaEventRecord(mk->ev[2], s));
  }
  if (mk) DG_CUDA(cudaEventRecord(mk->ev[3], s));
  if (pc.n_blocks > 0 && !mk) DG_CUDA(cudaStreamWaitEvent(s, pc.ev_join, 0));
  const int nb = precond_final_blocks(pc);
#define DG_FINAL(G)                                                                          \
  launch_k(precond_final_kernel<T, G>, nb, kVecThreads, 0, s,                                      \
      pc.P.ptr, pc.P.idx, (const T*)pc.P.val, (const T*)ec, (const T*)pc.dinv, pc.e_pos,     \
      (const T*)pc.zE, r, z, pc.n_dofs, red, rr, ctl, xr)
  // one lane per DG row: measured faster than 2 or 4 lanes (P has about five
  // entries per row; fewer rounds of dependent loads per thread count more)
  DG_FINAL(1);
#undef DG_FINAL
  DG_CUDA(cudaGetLastError());
  if (mk) DG_CUDA(cudaEventRecord(mk->ev[4], s));
}

// bytes of a CSR matrix read once: values, column indices, row pointers
static double csr_bytes(const DevCsr& A, size_t tsz) {
  return (double)A.nnz * (4.0 + (double)tsz) + 4.0 * (double)(A.rows + 1);
}

void precond_algorithmic_bytes(const dg_precond& pc, double* total, double* blocks) {
  const double T = pc.precision == DG_PREC_MIXED ? 4.0 : 8.0;
  const double n = (double)pc.n_dofs;
  // block solves: the inverses, the block node lists, r gathered, results written, the units
  double blk = 0.0;
  if (pc.n_blocks > 0)
    blk = (double)pc.blk_inv_entries * T + (double)pc.blk_slots * (4.0 + 8.0 + T) + 16.0 * (double)pc.n_units;
  double tot = blk;
  if (pc.n_c > 0) {
    tot += csr_bytes(pc.PT, (size_t)T) + 8.0 * n + T * (double)pc.n_c;   // restriction
    if (pc.lor == DG_LOR_EXACT) {
      tot += T * (double)pc.n_c * (double)pc.n_c + 2.0 * T * (double)pc.n_c;
    } else {
      for (size_t l = 0; l < pc.levels.size(); ++l) {
        const DevLevel& L = pc.levels[l];
        const double nc = (double)L.n_cont, ncn = l + 1 < pc.levels.size() ? (double)pc.levels[l + 1].n : 0.0;
        if (L.n_cont > 0 && L.plain)   // A twice, R, P; b, D^-1, two work vectors, the coarse vectors
          tot += 2.0 * csr_bytes(L.A, (size_t)T) + csr_bytes(L.R, (size_t)T) + csr_bytes(L.P, (size_t)T) +
                 T * (6.0 * nc + 2.0 * ncn);
        else if (L.n_cont > 0 && L.coarse_w)   // W (dense), Sb, Sp; b read twice, xo, the coarse output
          tot += T * (double)L.coarse_w_rows * (double)L.n + csr_bytes(L.Sb, (size_t)T) +
                 csr_bytes(L.Sp, (size_t)T) + T * (3.0 * nc + ncn);
        else if (L.n_cont > 0)         // Rpre, Sb, Sp; b read twice, xo, the coarse vectors
          tot += csr_bytes(L.Rpre, (size_t)T) + csr_bytes(L.Sb, (size_t)T) + csr_bytes(L.Sp, (size_t)T) +
                 T * (3.0 * nc + 2.0 * ncn);
        const bool fused_here = l > 0 && pc.levels[l - 1].coarse_w;
        if (!fused_here)   // dense coarse blocks
          tot += T * (double)L.end_inv_entries + 2.0 * T * (double)(L.n - L.n_cont);
      }
    }
  }
  // final combination: P, e_C, D_J^-1, the slot of each node, block results, r, z
  tot += csr_bytes(pc.P, (size_t)T) + T * (double)pc.n_c + n * (T + 4.0 + 8.0 + 8.0) + T * (double)pc.blk_slots;
  *total = tot;
  *blocks = blk;
}

int precond_kernel_count(const dg_precond& pc) {
  int k = (pc.n_blocks > 0 ? 1 : 0) + 1;   // block solves, final combination
  if (pc.n_c > 0) {
    k += 1;                                // restriction
    if (pc.lor == DG_LOR_EXACT) return k + 1;
    for (size_t l = 0; l < pc.levels.size(); ++l) {
      const DevLevel& L = pc.levels[l];
      if (L.n_cont > 0) k += L.plain ? 4 : 2;
      // a fused coarse product replaces the next level's dense solve
      const bool skipped = l > 0 && pc.levels[l - 1].coarse_w;
      if (L.n_end > 0 && L.max_end > 0 && !skipped) k += 1;
    }
  }
  return k;
}

void launch_precond(const dg_precond& pc, const double* r, double* z, Reduce red, cudaStream_t s,
                    const PrecondMarks* marks, Reduce rr, PcgCtl ctl, XrDefer xr) {
  DG_REQUIRE(!rr.partial || red.partial, "the r . r reduction rides on the r . z reduction");
  DG_REQUIRE(!ctl.sc || rr.partial, "the iteration control needs the r . r reduction");
  DG_REQUIRE(!xr.q || (xr.r_out == r && xr.x && xr.p && xr.alpha && !marks),
             "a deferred PCG update needs r_out = r, x, p, alpha, and no profiling marks");
  if (pc.precision == DG_PREC_MIXED) precond_impl<float>(pc, r, z, red, s, marks, rr, ctl, xr);
  else precond_impl<double>(pc, r, z, red, s, marks, rr, ctl, xr);
}

// ============================================================== PCG
__global__ void __launch_bounds__(kVecThreads)
pcg_init_kernel(const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                int64_t n, Reduce bb) {
  pdl_entry();
  __shared__ double red[kVecThreads];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    s += bi * bi;
  }
  pdl_trigger();
  reduce_finalize<kVecThreads>(block_sum<kVecThreads>(s, red), bb, red);
}

void launch_pcg_init(const double* b, double* x, double* r, int64_t n, Reduce bb, cudaStream_t s) {
  launch_k(pcg_init_kernel, grid_for(n), kVecThreads, 0, s, b, x, r, n, bb);
  DG_CUDA(cudaGetLastError());
}

// p = z + beta p (first: p = z) tile by tile, and the side traces of the new p
// for the next operator apply, so the apply needs no trace launch of its own.
// The last CTA to finish advances the iteration count and the scalars, tests
// convergence and sets the graph's while condition (first: the initial
// scalars, from the preconditioner's r . z and b . b).
template <bool CUBE>
__global__ void __launch_bounds__(kThreads)
pcg_p_trace_kernel(const ApplyArgs A, double* __restrict__ p, const double* __restrict__ z, double* sc,
                   cudaGraphConditionalHandle h, int use_cond, int first) {
  pdl_entry();
  if (!first && sc[SC_STATUS] != 0.0) return;   // stopped: the loop condition is already clear
  const double beta = first ? 0.0 : sc[SC_BETA];
  const ApplyTile T = A.tiles[blockIdx.x];
  const int np = T.p + 1;
  const int nn = CUBE ? np * np * np : np * np;
  for (int t = threadIdx.x; t < T.count * nn; t += blockDim.x) {
    const int e = t / nn;
    const int64_t i = A.off[A.order[T.first + e]] + (t - e * nn);
    p[i] = first ? z[i] : fma(beta, p[i], z[i]);
  }
  __syncthreads();
  switch (T.p) {
#define DG_TRACE_CASE(PP) \
    case PP: if (CUBE) trace3_tile<PP, false>(A, T); else trace_tile<PP, false>(A, T); break;
    DG_TRACE_CASE(1) DG_TRACE_CASE(2) DG_TRACE_CASE(3) DG_TRACE_CASE(4)
    DG_TRACE_CASE(5) DG_TRACE_CASE(6) DG_TRACE_CASE(7) DG_TRACE_CASE(8)
#undef DG_TRACE_CASE
    default: break;
  }
  if (first && blockIdx.x == 0 && threadIdx.x == 0) {
    sc[SC_RZ] = sc[SC_RZNEW];
    sc[SC_RR] = sc[SC_BB];
    sc[SC_IT] = 0.0;
    sc[SC_STATUS] = 0.0;
    // a zero right-hand side needs no iteration (x = 0 is exact)
    if (use_cond) cudaGraphSetConditional(h, sc[SC_BB] > 0.0 ? 1u : 0u);
  }
}

void launch_pcg_p_trace(const dg_mesh& M, double* p, const double* z, double* sc,
                        unsigned long long cond_handle, int use_cond, int first, cudaStream_t s) {
  if (M.n_tiles == 0) return;
  const ApplyArgs A = make_apply_args(M, p, nullptr, Reduce{});
  if (M.host.dim == 3)
    launch_k(pcg_p_trace_kernel<true>, M.n_tiles, kThreads, 0, s, A, p, z, sc,
             (cudaGraphConditionalHandle)cond_handle, use_cond, first);
  else
    launch_k(pcg_p_trace_kernel<false>, M.n_tiles, kThreads, 0, s, A, p, z, sc,
             (cudaGraphConditionalHandle)cond_handle, use_cond, first);
  DG_CUDA(cudaGetLastError());
}

}  // namespace dg
