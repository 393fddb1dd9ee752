// Device kernels: operator apply launch, preconditioner pieces (Section 4.1:
// P^T, LOR solve, P, point Jacobi, block solves) and the PCG vector work.
#include <cstdio>

#include "kernels.cuh"

namespace dg {

// ============================================================== operator
__global__ void __launch_bounds__(kThreads) trace_kernel(const ApplyArgs A) {
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

template <bool BR2>
__global__ void __launch_bounds__(kThreads) apply_kernel(const ApplyArgs A) {
  extern __shared__ double smem[];
  const ApplyTile T = A.tiles[blockIdx.x];
  switch (T.p) {
    case 1: apply_tile<1, BR2>(A, T, smem); break;
    case 2: apply_tile<2, BR2>(A, T, smem); break;
    case 3: apply_tile<3, BR2>(A, T, smem); break;
    case 4: apply_tile<4, BR2>(A, T, smem); break;
    case 5: apply_tile<5, BR2>(A, T, smem); break;
    case 6: apply_tile<6, BR2>(A, T, smem); break;
    case 7: apply_tile<7, BR2>(A, T, smem); break;
    case 8: apply_tile<8, BR2>(A, T, smem); break;
    default: break;
  }
}

static int apply_smem_bytes() {
  int m = ApplyShape<1>::SMEM;
  m = m > ApplyShape<2>::SMEM ? m : ApplyShape<2>::SMEM;
  m = m > ApplyShape<3>::SMEM ? m : ApplyShape<3>::SMEM;
  m = m > ApplyShape<4>::SMEM ? m : ApplyShape<4>::SMEM;
  m = m > ApplyShape<5>::SMEM ? m : ApplyShape<5>::SMEM;
  m = m > ApplyShape<6>::SMEM ? m : ApplyShape<6>::SMEM;
  m = m > ApplyShape<7>::SMEM ? m : ApplyShape<7>::SMEM;
  m = m > ApplyShape<8>::SMEM ? m : ApplyShape<8>::SMEM;
  return m * (int)sizeof(double);
}

ApplyArgs make_apply_args(const dg_mesh& M, const double* x, double* y, double* dot_partial) {
  ApplyArgs A;
  A.x = x;
  A.y = y;
  A.off = M.d_off;
  A.ih = M.d_ih;
  A.toff = M.d_toff;
  A.tr = M.d_tr;
  A.sf_ptr = M.d_sf_ptr;
  A.sf = M.d_sf;
  A.tab = M.d_tables;
  A.order = M.d_order;
  A.tiles = M.d_tiles;
  A.eta = M.eta;
  A.dot_partial = dot_partial;
  for (int p = 0; p <= kMaxP; ++p) A.boff[p] = M.boff[p];
  return A;
}

void apply_kernel_setup() {
  // the shared-memory opt-in is per device: set it on the current one
  const int smem = apply_smem_bytes();
  DG_CUDA(cudaFuncSetAttribute(apply_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  DG_CUDA(cudaFuncSetAttribute(apply_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
}

void launch_apply(const dg_mesh& M, const double* x, double* y, double* dot_partial, cudaStream_t s) {
  if (M.n_tiles == 0) return;
  const ApplyArgs A = make_apply_args(M, x, y, dot_partial);
  const int smem = apply_smem_bytes();
  trace_kernel<<<M.n_tiles, kThreads, 0, s>>>(A);
  if (M.opts.form == DG_FORM_BR2) apply_kernel<true><<<M.n_tiles, kThreads, smem, s>>>(A);
  else apply_kernel<false><<<M.n_tiles, kThreads, smem, s>>>(A);
  DG_CUDA(cudaGetLastError());
}

// ============================================================== reductions
// Deterministic block sum: fixed strided assignment + fixed tree.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
#pragma unroll
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) s += part[i];
  return block_sum<NT>(s, red);
}

// ============================================================== preconditioner
template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// ---- group-per-row CSR kernels: G lanes of a warp share one row, strided
// over its entries, then a fixed shuffle tree (deterministic for a fixed G).
// The row loop advances by whole warps so that every lane of a warp reaches
// the shuffles together.
template <typename T, int G, class Op>
__global__ void __launch_bounds__(kVecThreads)
csr_rows_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                const T* __restrict__ val, int64_t rows, Op op) {
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
template <typename T>
struct OpPre {  // x = b d ; r = b - A (b d)
  const T* b;
  const T* dinv;
  T* xo;
  T* r;
  __device__ T x(int j) const { return __ldg(b + j) * __ldg(dinv + j); }
  __device__ void store(int64_t i, T s) const {
    const T bi = b[i];
    xo[i] = bi * dinv[i];
    r[i] = bi - s;
  }
};
template <typename T>
struct OpProlong {  // x += P xc
  const T* xc;
  T* xo;
  __device__ T x(int j) const { return __ldg(xc + j); }
  __device__ void store(int64_t i, T s) const { xo[i] += s; }
};
template <typename T>
struct OpPost {  // xo = x + d (b - A x)
  const T* xin;
  const T* b;
  const T* dinv;
  T* xo;
  __device__ T x(int j) const { return __ldg(xin + j); }
  __device__ void store(int64_t i, T s) const { xo[i] = xin[i] + dinv[i] * (b[i] - s); }
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
    case 1: csr_rows_kernel<T, 1, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
    case 2: csr_rows_kernel<T, 2, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
    case 4: csr_rows_kernel<T, 4, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
    case 8: csr_rows_kernel<T, 8, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
    case 16: csr_rows_kernel<T, 16, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
    default: csr_rows_kernel<T, 32, Op><<<(int)blocks, kVecThreads, 0, s>>>(p, ix, v, A.rows, op); break;
  }
}

// dense y = Ainv x, one warp per row
template <typename T>
__global__ void dense_mv_kernel(const T* __restrict__ Ainv, const T* __restrict__ x,
                                T* __restrict__ y, int64_t n) {
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

// z = P e_C + D_J^-1 r + sum_e R_e^T A_e^-1 R_e r, and a partial of r . z.
// kFinalG lanes per DG row: they share the P entries and the block row.
constexpr int kFinalG = 8;
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
precond_final_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                     const T* __restrict__ val, const T* __restrict__ ec,
                     const T* __restrict__ dinv, const int32_t* __restrict__ e_block,
                     const int32_t* __restrict__ e_local, const int64_t* __restrict__ inv_off,
                     const int32_t* __restrict__ dofs_off, const int32_t* __restrict__ dim,
                     const int32_t* __restrict__ dofs, const T* __restrict__ inv,
                     const double* __restrict__ r, double* __restrict__ z, int64_t n,
                     double* __restrict__ dot_partial) {
  __shared__ double red[kVecThreads];
  constexpr int G = kFinalG;
  const int lane = threadIdx.x % G;
  const int64_t groups_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t rounds = (n + groups_per_grid - 1) / groups_per_grid;
  double dot = 0.0;
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t i = g0 + rd * groups_per_grid;
    T s = 0;
    if (i < n) {
      for (int t = ptr[i] + lane; t < ptr[i + 1]; t += G) s += __ldg(val + t) * __ldg(ec + __ldg(idx + t));
      const int b = __ldg(e_block + i);
      if (b >= 0) {
        const int d = __ldg(dim + b);
        const T* row = inv + __ldg(inv_off + b) + (int64_t)__ldg(e_local + i) * d;
        const int32_t* ds = dofs + __ldg(dofs_off + b);
        for (int m = lane; m < d; m += G) s += __ldg(row + m) * (T)__ldg(r + __ldg(ds + m));
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (i < n && lane == 0) {
      const double ri = __ldg(r + i);
      const double zi = (double)(s + __ldg(dinv + i) * (T)ri);
      z[i] = zi;
      dot += zi * ri;
    }
  }
  const double tot = block_sum<kVecThreads>(dot, red);
  if (dot_partial && threadIdx.x == 0) dot_partial[blockIdx.x] = tot;
}

static int grid_for(int64_t n, int threads = kVecThreads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > kVecBlocks) b = kVecBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

int precond_final_blocks(const dg_precond& pc) {
  int64_t b = (pc.n_dofs * kFinalG + kVecThreads - 1) / kVecThreads;
  if (b > kVecBlocks) b = kVecBlocks;
  return (int)(b < 1 ? 1 : b);
}

template <typename T>
static void vcycle(const dg_precond& pc, size_t l, cudaStream_t s) {
  const DevLevel& L = pc.levels[l];
  if (l + 1 == pc.levels.size()) {
    dense_mv_kernel<T><<<grid_for(L.n * 32), kVecThreads, 0, s>>>(
        (const T*)pc.coarse_inv, (const T*)L.b, (T*)L.xo, L.n);
    return;
  }
  const DevLevel& C = pc.levels[l + 1];
  launch_rows<T>(L.A, OpPre<T>{(const T*)L.b, (const T*)L.dinv, (T*)L.x, (T*)L.r}, s);
  launch_rows<T>(L.R, OpSpmv<T>{(const T*)L.r, (T*)C.b}, s);
  vcycle<T>(pc, l + 1, s);
  launch_rows<T>(L.P, OpProlong<T>{(const T*)C.xo, (T*)L.x}, s);
  launch_rows<T>(L.A, OpPost<T>{(const T*)L.x, (const T*)L.b, (const T*)L.dinv, (T*)L.xo}, s);
}

template <typename T>
static void precond_impl(const dg_precond& pc, const double* r, double* z, double* dot_partial,
                         cudaStream_t s) {
  const void* ec = nullptr;
  if (pc.n_c > 0) {
    if (pc.lor == DG_LOR_EXACT) {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.rc}, s);
      dense_mv_kernel<T><<<grid_for(pc.n_c * 32), kVecThreads, 0, s>>>(
          (const T*)pc.lor_inv, (const T*)pc.rc, (T*)pc.ec, pc.n_c);
      ec = pc.ec;
    } else {
      launch_rows<T>(pc.PT, OpRestrict<T>{r, (T*)pc.levels[0].b}, s);
      vcycle<T>(pc, 0, s);
      ec = pc.levels[0].xo;
    }
  }
  precond_final_kernel<T><<<precond_final_blocks(pc), kVecThreads, 0, s>>>(
      pc.P.ptr, pc.P.idx, (const T*)pc.P.val, (const T*)ec, (const T*)pc.dinv, pc.e_block,
      pc.e_local, pc.blk_inv_off, pc.blk_dofs_off, pc.blk_dim, pc.blk_dofs,
      (const T*)pc.blk_inv, r, z, pc.n_dofs, dot_partial);
  DG_CUDA(cudaGetLastError());
}

void launch_precond(const dg_precond& pc, const double* r, double* z, double* dot_partial,
                    cudaStream_t s) {
  if (pc.precision == DG_PREC_MIXED) precond_impl<float>(pc, r, z, dot_partial, s);
  else precond_impl<double>(pc, r, z, dot_partial, s);
}

// ============================================================== PCG

__global__ void pcg_init_kernel(const double* __restrict__ b, double* __restrict__ x,
                                double* __restrict__ r, int64_t n, double* part_bb) {
  __shared__ double red[kVecThreads];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    s += bi * bi;
  }
  const double t = block_sum<kVecThreads>(s, red);
  if (threadIdx.x == 0) part_bb[blockIdx.x] = t;
}

void launch_pcg_init(const double* b, double* x, double* r, int64_t n, double* partial_bb,
                     cudaStream_t s) {
  pcg_init_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(b, x, r, n, partial_bb);
  DG_CUDA(cudaGetLastError());
}

__global__ void copy_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

void launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s) {
  copy_kernel<<<grid_for(n), kVecThreads, 0, s>>>(src, dst, n);
  DG_CUDA(cudaGetLastError());
}

__global__ void pcg_first_kernel(const double* part_rz, int n_rz, const double* part_bb,
                                 double* sc) {
  __shared__ double red[kVecThreads];
  const double rz = sum_partials<kVecThreads>(part_rz, n_rz, red);
  const double bb = sum_partials<kVecThreads>(part_bb, kVecBlocks, red);
  if (threadIdx.x == 0) {
    sc[SC_RZ] = rz;
    sc[SC_BB] = bb;
    sc[SC_RR] = bb;
    sc[SC_IT] = 0.0;
    sc[SC_STATUS] = 0.0;
  }
}

void launch_pcg_first(const double* part_rz, int n_rz, const double* part_bb, double* sc,
                      cudaStream_t s) {
  pcg_first_kernel<<<1, kVecThreads, 0, s>>>(part_rz, n_rz, part_bb, sc);
  DG_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(kVecThreads)
pcg_update_xr_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                     const double* __restrict__ q, int64_t n, const double* part_pq, int n_pq,
                     double* sc, double* part_rr) {
  __shared__ double red[kVecThreads];
  if (sc[SC_STATUS] != 0.0) return;  // converged or stopped: iterations queued after it are no-ops
  const double pq = sum_partials<kVecThreads>(part_pq, n_pq, red);
  const double alpha = sc[SC_RZ] / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_ALPHA] = alpha;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s += ri * ri;
  }
  const double t = block_sum<kVecThreads>(s, red);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = t;
}

void launch_pcg_update_xr(double* x, double* r, const double* p, const double* q, int64_t n,
                          const double* part_pq, int n_pq, double* sc, double* part_rr,
                          cudaStream_t s) {
  pcg_update_xr_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(x, r, p, q, n, part_pq, n_pq, sc, part_rr);
  DG_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(kVecThreads)
pcg_update_p_kernel(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                    const double* part_rz, int n_rz, const double* sc) {
  __shared__ double red[kVecThreads];
  if (sc[SC_STATUS] != 0.0) return;
  const double rz_new = sum_partials<kVecThreads>(part_rz, n_rz, red);
  const double beta = rz_new / sc[SC_RZ];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

void launch_pcg_update_p(double* p, const double* z, int64_t n, const double* part_rz, int n_rz,
                         double* sc, cudaStream_t s) {
  pcg_update_p_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(p, z, n, part_rz, n_rz, sc);
  DG_CUDA(cudaGetLastError());
}

__global__ void pcg_check_kernel(const double* part_rr, int n_rr, const double* part_rz, int n_rz,
                                 double* sc, int maxit, double rtol2,
                                 cudaGraphConditionalHandle h, int use_cond) {
  __shared__ double red[kVecThreads];
  if (sc[SC_STATUS] != 0.0) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double rr = sum_partials<kVecThreads>(part_rr, n_rr, red);
  const double rz = sum_partials<kVecThreads>(part_rz, n_rz, red);
  if (threadIdx.x == 0) {
    const double it = sc[SC_IT] + 1.0;
    sc[SC_IT] = it;
    sc[SC_RR] = rr;
    sc[SC_RZ] = rz;
    int cont = 1;
    if (rr <= rtol2 * sc[SC_BB]) { sc[SC_STATUS] = 1.0; cont = 0; }
    else if (it >= (double)maxit) { sc[SC_STATUS] = 2.0; cont = 0; }
    if (use_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
  }
}

void launch_pcg_check(const double* part_rr, int n_rr, const double* part_rz, int n_rz,
                      double* sc, int maxit, double rtol2, unsigned long long cond_handle,
                      int use_cond, cudaStream_t s) {
  pcg_check_kernel<<<1, kVecThreads, 0, s>>>(part_rr, n_rr, part_rz, n_rz, sc, maxit, rtol2,
                                             (cudaGraphConditionalHandle)cond_handle, use_cond);
  DG_CUDA(cudaGetLastError());
}

}  // namespace dg
