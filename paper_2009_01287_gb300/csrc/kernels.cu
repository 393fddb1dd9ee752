// Device kernels: operator apply launch, preconditioner pieces (Section 4.1:
// P^T, LOR solve, P, point Jacobi, block solves) and the PCG vector work.
#include <cstdio>

#include "kernels.cuh"

namespace dg {

// ============================================================== operator
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
  A.p = M.d_p;
  A.off = M.d_off;
  A.h = M.d_h;
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

// rc = P^T r  (rows of P^T)
template <typename T>
__global__ void restrict_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                const T* __restrict__ val, const double* __restrict__ r,
                                T* __restrict__ out, int64_t rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) s += ld(val + t) * (T)__ldg(r + ld(idx + t));
    out[i] = s;
  }
}

// y = A x for a CSR of precision T
template <typename T>
__global__ void spmv_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                            const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y,
                            int64_t rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) s += ld(val + t) * ld(x + ld(idx + t));
    y[i] = s;
  }
}

// dense y = Ainv x, one warp per row
template <typename T>
__global__ void dense_mv_kernel(const T* __restrict__ Ainv, const T* __restrict__ x,
                                T* __restrict__ y, int64_t n) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    T s = 0;
    for (int64_t j = lane; j < n; j += 32) s += ld(Ainv + row * n + j) * ld(x + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
  }
}

// pre-smoothing from zero and residual: x = b d, r = b - A (b d)
template <typename T>
__global__ void amg_pre_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                               const T* __restrict__ val, const T* __restrict__ dinv,
                               const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) {
      const int j = ld(idx + t);
      s += ld(val + t) * (ld(b + j) * ld(dinv + j));
    }
    const T bi = ld(b + i);
    x[i] = bi * ld(dinv + i);
    r[i] = bi - s;
  }
}

// coarse-grid correction: x += P xc
template <typename T>
__global__ void amg_prolong_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                   const T* __restrict__ val, const T* __restrict__ xc,
                                   T* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) s += ld(val + t) * ld(xc + ld(idx + t));
    x[i] += s;
  }
}

// post-smoothing: xo = x + d (b - A x)
template <typename T>
__global__ void amg_post_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                const T* __restrict__ val, const T* __restrict__ dinv,
                                const T* __restrict__ b, const T* __restrict__ x,
                                T* __restrict__ xo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) s += ld(val + t) * ld(x + ld(idx + t));
    xo[i] = ld(x + i) + ld(dinv + i) * (ld(b + i) - s);
  }
}

// z = P e_C + D_J^-1 r + sum_e R_e^T A_e^-1 R_e r, and a partial of r . z
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
  double dot = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int t = ptr[i]; t < ptr[i + 1]; ++t) s += ld(val + t) * ld(ec + ld(idx + t));
    const double ri = __ldg(r + i);
    s += ld(dinv + i) * (T)ri;
    const int b = __ldg(e_block + i);
    if (b >= 0) {
      const int d = __ldg(dim + b);
      const T* row = inv + __ldg(inv_off + b) + (int64_t)__ldg(e_local + i) * d;
      const int32_t* ds = dofs + __ldg(dofs_off + b);
      T acc = 0;
      for (int m = 0; m < d; ++m) acc += ld(row + m) * (T)__ldg(r + __ldg(ds + m));
      s += acc;
    }
    const double zi = (double)s;
    z[i] = zi;
    dot += zi * ri;
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

int precond_final_blocks(const dg_precond& pc) { return grid_for(pc.n_dofs); }

template <typename T>
static void vcycle(const dg_precond& pc, size_t l, cudaStream_t s) {
  const DevLevel& L = pc.levels[l];
  if (l + 1 == pc.levels.size()) {
    dense_mv_kernel<T><<<grid_for(L.n * 32), kVecThreads, 0, s>>>(
        (const T*)pc.coarse_inv, (const T*)L.b, (T*)L.xo, L.n);
    return;
  }
  const DevLevel& C = pc.levels[l + 1];
  amg_pre_kernel<T><<<grid_for(L.n), kVecThreads, 0, s>>>(L.A.ptr, L.A.idx, (const T*)L.A.val,
      (const T*)L.dinv, (const T*)L.b, (T*)L.x, (T*)L.r, L.n);
  spmv_kernel<T><<<grid_for(C.n), kVecThreads, 0, s>>>(L.R.ptr, L.R.idx, (const T*)L.R.val,
      (const T*)L.r, (T*)C.b, C.n);
  vcycle<T>(pc, l + 1, s);
  amg_prolong_kernel<T><<<grid_for(L.n), kVecThreads, 0, s>>>(L.P.ptr, L.P.idx, (const T*)L.P.val,
      (const T*)C.xo, (T*)L.x, L.n);
  amg_post_kernel<T><<<grid_for(L.n), kVecThreads, 0, s>>>(L.A.ptr, L.A.idx, (const T*)L.A.val,
      (const T*)L.dinv, (const T*)L.b, (const T*)L.x, (T*)L.xo, L.n);
}

template <typename T>
static void precond_impl(const dg_precond& pc, const double* r, double* z, double* dot_partial,
                         cudaStream_t s) {
  const void* ec = nullptr;
  if (pc.n_c > 0) {
    if (pc.lor == DG_LOR_EXACT) {
      restrict_kernel<T><<<grid_for(pc.n_c), kVecThreads, 0, s>>>(pc.PT.ptr, pc.PT.idx,
          (const T*)pc.PT.val, r, (T*)pc.rc, pc.n_c);
      dense_mv_kernel<T><<<grid_for(pc.n_c * 32), kVecThreads, 0, s>>>(
          (const T*)pc.lor_inv, (const T*)pc.rc, (T*)pc.ec, pc.n_c);
      ec = pc.ec;
    } else {
      restrict_kernel<T><<<grid_for(pc.n_c), kVecThreads, 0, s>>>(pc.PT.ptr, pc.PT.idx,
          (const T*)pc.PT.val, r, (T*)pc.levels[0].b, pc.n_c);
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
