// Device kernels: operator apply launch, preconditioner pieces (Section 4.1:
// P^T, LOR solve, P, point Jacobi, block solves) and the PCG vector work.
#include <cstdio>

#include "kernels.cuh"

namespace dg {

// ============================================================== operator
__global__ void __launch_bounds__(kThreads) trace_kernel(const ApplyArgs A) {
  pdl_entry();
  const ApplyTile T = A.tiles[blockIdx.x];
  switch (T.p) {
    case 1: trace_tile<1>(A, T); break;
    case 2: trace_tile<2>(A, T); break;
    case 3: trace_tile<3>(A, T); break;
    case 4: trace_tile<4>(A, T); break;
    case 5: trace_tile<5>(A, T); break;
    case 6: trace_tile<6>(A, T); break;
    case 7: trace_tile<7>(A, T); break;
    case 8: trace_tile<8>(A, T); break;
    default: break;
  }
}

// End of a persistent operator launch: the last CTA to leave resets the tile
// counter and sums the tile partials of x . y in tile order.
__device__ __forceinline__ void apply_exit(const ApplyArgs& A, double* red) {
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(A.sched + 1, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (A.dot_partial) {
      double v = 0.0;
      for (int i = threadIdx.x; i < A.n_tiles; i += kThreads) v += __ldcg(A.dot_partial + i);
      v = block_sum<kThreads>(v, red);
      if (threadIdx.x == 0) *A.dot_out = v;
    }
    if (threadIdx.x == 0) {
      A.sched[0] = 0u;
      A.sched[1] = 0u;
    }
  }
}

// Persistent operator kernel: a grid sized to the resident capacity takes
// tiles from an atomic counter, heaviest first (tiles are degree-sorted), so
// the uneven tiles balance across SMs.  The last CTA to leave resets the
// counter and, when a dot product is requested, sums the tile partials in
// tile order (deterministic whichever CTA ran which tile).
template <bool BR2>
__global__ void __launch_bounds__(kThreads) apply_kernel(const ApplyArgs A) {
  pdl_entry();
  extern __shared__ __align__(16) double smem[];
  __shared__ double red[kThreads];
  __shared__ int s_tile;
  while (true) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(A.sched, 1u);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= A.n_tiles) break;
    const ApplyTile T = A.tiles[t];
    switch (T.p) {
      case 1: apply_tile<1, BR2>(A, T, t, smem, red); break;
      case 2: apply_tile<2, BR2>(A, T, t, smem, red); break;
      case 3: apply_tile<3, BR2>(A, T, t, smem, red); break;
      case 4: apply_tile<4, BR2>(A, T, t, smem, red); break;
      case 5: apply_tile<5, BR2>(A, T, t, smem, red); break;
      case 6: apply_tile<6, BR2>(A, T, t, smem, red); break;
      case 7: apply_tile<7, BR2>(A, T, t, smem, red); break;
      case 8: apply_tile<8, BR2>(A, T, t, smem, red); break;
      default: break;
    }
    __syncthreads();
  }
  apply_exit(A, red);
}

__global__ void __launch_bounds__(kThreads) trace3_kernel(const ApplyArgs A) {
  pdl_entry();
  const ApplyTile T = A.tiles[blockIdx.x];
  switch (T.p) {
    case 1: trace3_tile<1>(A, T); break;
    case 2: trace3_tile<2>(A, T); break;
    case 3: trace3_tile<3>(A, T); break;
    case 4: trace3_tile<4>(A, T); break;
    case 5: trace3_tile<5>(A, T); break;
    case 6: trace3_tile<6>(A, T); break;
    case 7: trace3_tile<7>(A, T); break;
    case 8: trace3_tile<8>(A, T); break;
    default: break;
  }
}

// Persistent operator kernel of cube meshes (same scheduling as on squares).
template <bool BR2>
__global__ void __launch_bounds__(kThreads) apply3_kernel(const ApplyArgs A) {
  pdl_entry();
  extern __shared__ __align__(16) double smem[];
  __shared__ double red[kThreads];
  __shared__ int s_tile;
  while (true) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(A.sched, 1u);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= A.n_tiles) break;
    const ApplyTile T = A.tiles[t];
    switch (T.p) {
      case 1: apply3_tile<1, BR2>(A, T, t, smem, red); break;
      case 2: apply3_tile<2, BR2>(A, T, t, smem, red); break;
      case 3: apply3_tile<3, BR2>(A, T, t, smem, red); break;
      case 4: apply3_tile<4, BR2>(A, T, t, smem, red); break;
      case 5: apply3_tile<5, BR2>(A, T, t, smem, red); break;
      case 6: apply3_tile<6, BR2>(A, T, t, smem, red); break;
      case 7: apply3_tile<7, BR2>(A, T, t, smem, red); break;
      case 8: apply3_tile<8, BR2>(A, T, t, smem, red); break;
      default: break;
    }
    __syncthreads();
  }
  apply_exit(A, red);
}

// static shared-memory layout of a degree-p tile up to the item partials (doubles)
static int apply_shape_smem(int p) {
  switch (p) {
    case 1: return ApplyShape<1>::PART;
    case 2: return ApplyShape<2>::PART;
    case 3: return ApplyShape<3>::PART;
    case 4: return ApplyShape<4>::PART;
    case 5: return ApplyShape<5>::PART;
    case 6: return ApplyShape<6>::PART;
    case 7: return ApplyShape<7>::PART;
    default: return ApplyShape<8>::PART;
  }
}

int64_t apply_smem_for(const dg_mesh& M) {
  if (M.host.dim == 3) return M.apply3_smem;
  // the layout of the tile's degree plus its sub-face item partials
  int64_t mx = 0;
  for (int t = 0; t < M.n_tiles; ++t) {
    const ApplyTile& T = M.h_tiles[t];
    const int64_t nit = M.h_item_ptr.empty() ? 0 : M.h_item_ptr[t + 1] - M.h_item_ptr[t];
    mx = std::max<int64_t>(mx, apply_shape_smem(T.p) + 2 * nit * (T.p + 1));
  }
  return 8 * mx;
}

ApplyArgs make_apply_args(const dg_mesh& M, const double* x, double* y, Reduce red) {
  ApplyArgs A;
  A.x = x;
  A.y = y;
  A.off = M.d_off;
  A.ih = M.d_ih;
  A.toff = M.d_toff;
  A.tr = M.d_tr;
  A.sf_ptr = M.d_sf_ptr;
  A.sf = M.d_sf;
  A.sf3 = M.d_sf3;
  A.hk = M.d_h;
  A.tab = M.d_tables;
  A.order = M.d_order;
  A.tiles = M.d_tiles;
  A.items = reinterpret_cast<const int2*>(M.d_items);
  A.item_ptr = M.d_item_ptr;
  A.side_items = reinterpret_cast<const int2*>(M.d_side_items);
  A.eta = M.eta;
  A.dot_partial = red.partial;
  A.dot_out = red.out;
  A.dot_ticket = red.ticket;
  A.skip = M.skip_status;
  A.skip_stride = M.skip_stride;
  A.n_tiles = M.n_tiles;
  A.sched = M.d_sched;
  for (int p = 0; p <= kMaxP; ++p) A.boff[p] = M.boff[p];
  return A;
}

int apply_kernel_setup(const dg_mesh& M) {
  // The shared-memory opt-in is an attribute of the kernel function on the
  // current device, shared by every mesh: raise it to the device limit (a
  // mesh's own size could lower it under an earlier mesh's needs), and size the
  // resident grid of this mesh's persistent launch from its own tile layout.
  int dev = 0, sms = 0, per = 0, optin = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  optin -= 4 * 1024;   // room for the kernels' static shared memory
  const bool br2 = M.opts.form == DG_FORM_BR2;
  if (M.host.dim == 3) {
    const int smem = (int)M.apply3_smem;
    DG_REQUIRE(smem <= optin, "operator tile needs too much shared memory");
    DG_CUDA(cudaFuncSetAttribute(apply3_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    DG_CUDA(cudaFuncSetAttribute(apply3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    if (br2) DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply3_kernel<true>, kThreads, smem));
    else DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply3_kernel<false>, kThreads, smem));
    return sms * (per > 0 ? per : 1);
  }
  const int smem = (int)M.apply_smem;
  DG_REQUIRE(smem <= optin, "operator tile needs too much shared memory");
  DG_CUDA(cudaFuncSetAttribute(apply_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  DG_CUDA(cudaFuncSetAttribute(apply_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  if (br2)
    DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_kernel<true>, kThreads, smem));
  else
    DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_kernel<false>, kThreads, smem));
  return sms * (per > 0 ? per : 1);
}

void launch_apply(const dg_mesh& M, const double* x, double* y, Reduce red, cudaStream_t s,
                  bool with_trace) {
  if (M.n_tiles == 0) return;
  const ApplyArgs A = make_apply_args(M, x, y, red);
  const int grid = M.n_tiles < M.apply_grid ? M.n_tiles : M.apply_grid;
  if (M.host.dim == 3) {
    if (with_trace) launch_k(trace3_kernel, M.n_tiles, kThreads, 0, s, A);
    const int smem3 = (int)M.apply3_smem;
    if (M.opts.form == DG_FORM_BR2) launch_k(apply3_kernel<true>, grid, kThreads, smem3, s, A);
    else launch_k(apply3_kernel<false>, grid, kThreads, smem3, s, A);
    DG_CUDA(cudaGetLastError());
    return;
  }
  const int smem = (int)M.apply_smem;
  if (with_trace) launch_k(trace_kernel, M.n_tiles, kThreads, 0, s, A);
  if (M.opts.form == DG_FORM_BR2) launch_k(apply_kernel<true>, grid, kThreads, smem, s, A);
  else launch_k(apply_kernel<false>, grid, kThreads, smem, s, A);
  DG_CUDA(cudaGetLastError());
}

template <int NT>
__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) s += part[i];
  return block_sum<NT>(s, red);
}

// ============================================================== preconditioner

// ---- group-per-row CSR kernels: G lanes of a warp share one row, strided
// over its entries, then a fixed shuffle tree (deterministic for a fixed G).
// The row loop advances by whole warps so that every lane of a warp reaches
// the shuffles together.
template <typename T, int G, class Op>
__global__ void __launch_bounds__(kVecThreads)
csr_rows_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                const T* __restrict__ val, int64_t rows, Op op) {
  pdl_entry();
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (rows + groups_per_grid - 1) / groups_per_grid;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t row = g0 + rd * groups_per_grid;
    T s = 0;
    if (row < rows) {
      const int e = ptr[row + 1];
      for (int t = ptr[row] + lane; t < e; t += G) s += __ldg(val + t) * op.x(__ldg(idx + t));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (row < rows && lane == 0) op.store(row, s);
  }
}

template <typename T>
struct OpSpmv {  // y = A v
  const T* v;
  T* y;
  __device__ T x(int j) const { return __ldg(v + j); }
  __device__ void store(int64_t i, T s) const { y[i] = s; }
};
template <typename T>
struct OpRestrict {  // out = P^T r, r in FP64
  const double* r;
  T* out;
  __device__ T x(int j) const { return (T)__ldg(r + j); }
  __device__ void store(int64_t i, T s) const { out[i] = s; }
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
  switch (A.group) {
    case 1: launch_k(csr_rows_kernel<T, 1, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
    case 2: launch_k(csr_rows_kernel<T, 2, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
    case 4: launch_k(csr_rows_kernel<T, 4, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
    case 8: launch_k(csr_rows_kernel<T, 8, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
    case 16: launch_k(csr_rows_kernel<T, 16, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
    default: launch_k(csr_rows_kernel<T, 32, Op>, (int)blocks, kVecThreads, 0, s, p, ix, v, A.rows, op); break;
  }
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

// V_e block solves, one CTA per block (Section 3.3, T_E = sum_e P_e): the
// block's residual entries are gathered into shared memory once, then thread l
// forms row l of A_e^-1 r_e.  The inverse is stored column-major, so at every
// step the threads of a warp read consecutive entries of one column, and each
// thread's loads are independent of its running sum (unrolled, in flight
// together).
template <typename T>
__global__ void __launch_bounds__(128)
block_solve_kernel(const int64_t* __restrict__ inv_off, const int32_t* __restrict__ dofs_off,
                   const int32_t* __restrict__ dim, const int32_t* __restrict__ dofs,
                   const T* __restrict__ inv, const double* __restrict__ r, T* __restrict__ zE,
                   int nblocks) {
  pdl_entry();
  extern __shared__ unsigned char smem_raw[];
  T* sr = reinterpret_cast<T*>(smem_raw);
  for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int d = __ldg(dim + b);
    const int32_t* ds = dofs + __ldg(dofs_off + b);
    for (int m = threadIdx.x; m < d; m += blockDim.x) sr[m] = (T)__ldg(r + __ldg(ds + m));
    __syncthreads();
    // thread l: row l of A_e^-1 (stored column-major: step m reads a contiguous column)
    const T* At = inv + __ldg(inv_off + b);
    for (int l = threadIdx.x; l < d; l += blockDim.x) {
      T acc = 0;
#pragma unroll 8
      for (int m = 0; m < d; ++m) acc = fma(__ldg(At + (int64_t)m * d + l), sr[m], acc);
      zE[__ldg(dofs_off + b) + l] = acc;
    }
    __syncthreads();
  }
}

// z = P e_C + D_J^-1 r + (block result on V_e nodes), and the r . z reduction.
// G lanes per DG row share its P entries.
template <typename T, int G>
__global__ void __launch_bounds__(kVecThreads)
precond_final_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                     const T* __restrict__ val, const T* __restrict__ ec,
                     const T* __restrict__ dinv, const int32_t* __restrict__ e_block,
                     const int32_t* __restrict__ e_local, const int32_t* __restrict__ dofs_off,
                     const T* __restrict__ zE, const double* __restrict__ r,
                     double* __restrict__ z, int64_t n, Reduce red) {
  pdl_entry();
  __shared__ double sred[kVecThreads];
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (n + groups_per_grid - 1) / groups_per_grid;
  double dot = 0.0;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t i = g0 + rd * groups_per_grid;
    T s = 0;
    if (i < n)
      for (int t = ptr[i] + lane; t < ptr[i + 1]; t += G) s += __ldg(val + t) * __ldg(ec + __ldg(idx + t));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (i < n && lane == 0) {
      const double ri = __ldg(r + i);
      s += __ldg(dinv + i) * (T)ri;
      const int b = __ldg(e_block + i);
      if (b >= 0) s += __ldg(zE + __ldg(dofs_off + b) + __ldg(e_local + i));
      const double zi = (double)s;
      z[i] = zi;
      dot += zi * ri;
    }
  }
  if (red.partial) {
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
  int64_t b = (pc.n_dofs * pc.P.group + kVecThreads - 1) / kVecThreads;
  if (b > kVecBlocks) b = kVecBlocks;
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
  int64_t blocks = (L.n_cont * (int64_t)L.Sb.group + kVecThreads - 1) / kVecThreads;
  if (blocks > 8 * 152) blocks = 8 * 152;
#define DG_UP(G)                                                                                  \
  launch_k(amg_up_kernel<T, G>, (int)blocks, kVecThreads, 0, s, L.Sb.ptr, L.Sb.idx,              \
           (const T*)L.Sb.val, L.Sp.ptr, L.Sp.idx, (const T*)L.Sp.val, b, xc, xo, L.n_cont)
  switch (L.Sb.group) {
    case 1: DG_UP(1); break;
    case 2: DG_UP(2); break;
    case 4: DG_UP(4); break;
    case 8: DG_UP(8); break;
    case 16: DG_UP(16); break;
    default: DG_UP(32); break;
  }
#undef DG_UP
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
  if (L.n_cont > 0) {
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
                         cudaStream_t s) {
  // fork: the block solves depend only on r
  if (pc.n_blocks > 0) {
    DG_CUDA(cudaEventRecord(pc.ev_fork, s));
    DG_CUDA(cudaStreamWaitEvent(pc.side, pc.ev_fork, 0));
    int g = (int)(pc.n_blocks < 16 * 152 ? pc.n_blocks : 16 * 152);
    launch_k(block_solve_kernel<T>, g, 128, (size_t)pc.max_block * sizeof(T), pc.side, 
        pc.blk_inv_off, pc.blk_dofs_off, pc.blk_dim, pc.blk_dofs, (const T*)pc.blk_inv, r,
        (T*)pc.zE, (int)pc.n_blocks);
    DG_CUDA(cudaGetLastError());
    DG_CUDA(cudaEventRecord(pc.ev_join, pc.side));
  }
  const void* ec = nullptr;
  if (pc.n_c > 0) {
    if (pc.lor == DG_LOR_EXACT) {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.rc}, s);
      launch_k(dense_mv_kernel<T>, grid_for(pc.n_c * 32), kVecThreads, 0, s, 
          (const T*)pc.lor_inv, (const T*)pc.rc, (T*)pc.ec, pc.n_c);
      ec = pc.ec;
    } else {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.levels[0].b}, s);
      vcycle<T>(pc, 0, s);
      ec = pc.levels[0].xo;
    }
  }
  if (pc.n_blocks > 0) DG_CUDA(cudaStreamWaitEvent(s, pc.ev_join, 0));
  const int nb = precond_final_blocks(pc);
#define DG_FINAL(G)                                                                          \
  launch_k(precond_final_kernel<T, G>, nb, kVecThreads, 0, s,                                      \
      pc.P.ptr, pc.P.idx, (const T*)pc.P.val, (const T*)ec, (const T*)pc.dinv, pc.e_block,   \
      pc.e_local, pc.blk_dofs_off, (const T*)pc.zE, r, z, pc.n_dofs, red)
  if (pc.P.group <= 1) DG_FINAL(1);
  else if (pc.P.group == 2) DG_FINAL(2);
  else DG_FINAL(4);
#undef DG_FINAL
  DG_CUDA(cudaGetLastError());
}

void launch_precond(const dg_precond& pc, const double* r, double* z, Reduce red, cudaStream_t s) {
  if (pc.precision == DG_PREC_MIXED) precond_impl<float>(pc, r, z, red, s);
  else precond_impl<double>(pc, r, z, red, s);
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
  reduce_finalize<kVecThreads>(block_sum<kVecThreads>(s, red), bb, red);
}

void launch_pcg_init(const double* b, double* x, double* r, int64_t n, Reduce bb, cudaStream_t s) {
  launch_k(pcg_init_kernel, grid_for(n), kVecThreads, 0, s, b, x, r, n, bb);
  DG_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(kVecThreads)
pcg_update_xr_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                     const double* __restrict__ q, int64_t n, double* sc, Reduce rr) {
  pdl_entry();
  __shared__ double red[kVecThreads];
  if (sc[SC_STATUS] != 0.0) return;  // converged or stopped: iterations queued after it are no-ops
  const double alpha = sc[SC_RZ] / sc[SC_PQ];
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_ALPHA] = alpha;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s += ri * ri;
  }
  reduce_finalize<kVecThreads>(block_sum<kVecThreads>(s, red), rr, red);
}

void launch_pcg_update_xr(double* x, double* r, const double* p, const double* q, int64_t n,
                          double* sc, Reduce rr, cudaStream_t s) {
  launch_k(pcg_update_xr_kernel, grid_for(n), kVecThreads, 0, s, x, r, p, q, n, sc, rr);
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
                   unsigned* ticket, int maxit, double rtol2, cudaGraphConditionalHandle h, int use_cond,
                   int first) {
  pdl_entry();
  __shared__ unsigned s_last;
  if (!first && sc[SC_STATUS] != 0.0) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double beta = first ? 0.0 : sc[SC_RZNEW] / sc[SC_RZ];
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
  if (first) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc[SC_RZ] = sc[SC_RZNEW];
      sc[SC_RR] = sc[SC_BB];
      sc[SC_IT] = 0.0;
      sc[SC_STATUS] = 0.0;
    }
    return;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    const double it = sc[SC_IT] + 1.0;
    const double rr = sc[SC_RRNEW];
    sc[SC_IT] = it;
    sc[SC_RR] = rr;
    sc[SC_RZ] = sc[SC_RZNEW];
    int cont = 1;
    if (rr <= rtol2 * sc[SC_BB]) { sc[SC_STATUS] = 1.0; cont = 0; }
    else if (it >= (double)maxit) { sc[SC_STATUS] = 2.0; cont = 0; }
    *ticket = 0u;
    if (use_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
  }
}

void launch_pcg_p_trace(const dg_mesh& M, double* p, const double* z, double* sc, unsigned* ticket,
                        int maxit, double rtol2, unsigned long long cond_handle, int use_cond, int first,
                        cudaStream_t s) {
  if (M.n_tiles == 0) return;
  const ApplyArgs A = make_apply_args(M, p, nullptr, Reduce{});
  if (M.host.dim == 3)
    launch_k(pcg_p_trace_kernel<true>, M.n_tiles, kThreads, 0, s, A, p, z, sc, ticket, maxit, rtol2,
             (cudaGraphConditionalHandle)cond_handle, use_cond, first);
  else
    launch_k(pcg_p_trace_kernel<false>, M.n_tiles, kThreads, 0, s, A, p, z, sc, ticket, maxit, rtol2,
             (cudaGraphConditionalHandle)cond_handle, use_cond, first);
  DG_CUDA(cudaGetLastError());
}

}  // namespace dg
