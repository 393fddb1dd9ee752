// Matrix-free SIPG / BR2 operator y = A x on 2D leaf squares (Section 2,
// Eq. fe-problem; BR2 stabilisation of Section 4.4), FP64.
//
// Two kernels per apply:
//  trace_kernel  for every element side: the side values u and the outward
//                normal derivative dn at the p+1 side nodes (GLL nodes include
//                the ends, so the side trace is a row of x; dn contracts the
//                normal direction with l_k'(0 or 1) / h);
//  apply_kernel  one CTA per tile of EPB elements of one degree P:
//    volume  y = (K (x) M + M (x) K) x, sum factorised through shared memory
//            (Section 4.1: O(p^{d+1}) work per element);
//    faces   one thread per (sub-face item, side node) of the tile - the
//            tile's sub-faces are a flat list, so a side with many hanging
//            sub-faces does not hold the whole CTA at the next barrier - then
//            one thread per side node sums its sub-faces in order.
//            With the exact face mass matrices of the sub-face, M_oo (own-own)
//            and M_on (own-neighbour), an item forms
//              a = M_oo u-, c = M_oo dn-, b = M_on u+, d = M_on dn+
//            (dn+ along this element's outward normal), and accumulates the
//            residual of this element's test functions:
//              side nodes:  -1/2 (c + d) + sigma (a - b)   (interior)
//                           -c + sigma a                   (boundary)
//              all nodes:   dn(v) * (-1/2 (a - b))         (interior)
//                           dn(v) * (-a)                   (boundary)
//            For BR2 the sigma term becomes
//              eta/4 [M_oo G_o (a - b) + M_on G_n (M_no u- - M_nn u+)]
//            (eta [M_oo G_o a] on the boundary), G = edge block of the
//            element mass inverse = h^-2 Minv_00 Minv, times the larger
//            coefficient a of the sub-face's two sides.  Multiplied out it is
//            cz (Z u- - V u+) + cx (X u- - Y u+) with the product tables and
//            scalars of SubFaceBr2, so an item forms up to four more 1D
//            products in the same pass (none of the lifting's solves and
//            barriers per sub-face); on whole sides Z, V, Y are M_oo or M_on,
//            taken from a and b.
// Every sub-face is evaluated from both of its sides (no atomics): applies are
// bit-reproducible.
#pragma once

#include <utility>

#include "dg_internal.h"

namespace dg {

// Programmatic dependent launch.  Every kernel waits at entry until the
// kernels it depends on have completed with their memory visible
// (pdl_entry), and lets its dependents start launching once each of its CTAs
// has done its main work (pdl_trigger, or the CTA's exit): the next kernel's
// launch and CTA dispatch then overlap this kernel's stores and its
// reduction tail.  The wait alone orders the data, wherever the trigger is.
// Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kernel launch with programmatic stream serialisation allowed (captured into
// a graph, it becomes a programmatic edge from the kernel before it)
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

// A grid-wide deterministic dot product: each CTA writes its partial, the last
// CTA to finish (atomic ticket) sums the partials in CTA order into *out and
// resets the ticket.  All-null = no reduction.
struct Reduce {
  double* partial = nullptr;
  double* out = nullptr;
  unsigned* ticket = nullptr;
};

// ============================================================== reductions
// Deterministic block sum (blockDim.x == NT, a multiple of 32): a fixed
// shuffle tree inside each warp, then the warp sums, in warp order, by a fixed
// shuffle tree in warp 0.  Three barriers instead of the log2(NT) + 2 of a
// shared-memory tree (about 1 us less per reducing kernel on GB300).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block_sum: NT must be a multiple of 32, at most 1024");
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double r = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (lane == 0) red[NT / 32] = r;
  }
  __syncthreads();
  const double r = red[NT / 32];
  __syncthreads();
  return r;
}

// Last-CTA finalisation of a grid-wide sum (see Reduce): deterministic, the
// partials are summed in CTA order whichever CTA finishes last.
template <int NT>
__device__ __forceinline__ void reduce_finalize(double tot, const Reduce& R, double* red) {
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    R.partial[blockIdx.x] = tot;
    __threadfence();
    s_last = (atomicAdd(R.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) v += __ldcg(R.partial + i);
    v = block_sum<NT>(v, red);
    if (threadIdx.x == 0) {
      *R.out = v;
      *R.ticket = 0u;
    }
  }
}

// Two sums finalised together: the ticket of R1 counts the CTAs; the last one
// sums both partial arrays in CTA order into R1.out and R2.out, returns true
// (in every thread of that CTA) and leaves the sums in *v1_out, *v2_out.
template <int NT>
__device__ __forceinline__ bool reduce_finalize2(double t1, double t2, const Reduce& R1, const Reduce& R2,
                                                 double* red, double* v1_out, double* v2_out) {
  __shared__ unsigned s_last2;
  if (threadIdx.x == 0) {
    R1.partial[blockIdx.x] = t1;
    R2.partial[blockIdx.x] = t2;
    __threadfence();
    s_last2 = (atomicAdd(R1.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last2) {
    __threadfence();
    double v1 = 0.0, v2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) {
      v1 += __ldcg(R1.partial + i);
      v2 += __ldcg(R2.partial + i);
    }
    v1 = block_sum<NT>(v1, red);
    v2 = block_sum<NT>(v2, red);
    if (threadIdx.x == 0) {
      *R1.out = v1;
      *R2.out = v2;
      *R1.ticket = 0u;
    }
    *v1_out = v1;
    *v2_out = v2;
    return true;
  }
  return false;
}

struct ApplyArgs {
  const double* x;
  double* y;
  const int64_t* off;
  const double* ih;           // 1 / h per element
  const double* aih;          // a / h per element (a: the diffusion coefficient)
  const double* ahk;          // a h per element (cube meshes)
  const double* ak;           // a per element
  const int64_t* toff;        // offset of the element's side traces in tr
  double* tr;                 // side traces: [side][node][u, dn]
  const int32_t* sf_ptr;
  const SubFaceRec* sf;
  const SubFaceBr2* sfb;      // square meshes, BR2: the multiplied-out liftings
  const SubFaceRec3* sf3;     // cube meshes
  const double* tab;          // basis + face tables
  const int32_t* order;       // degree-sorted element order
  const ApplyTile* tiles;
  const int2* items;          // square meshes, SIPG: (record, e_local * 4 + s) per sub-face item
  const int32_t* item_ptr;    // items of tile t: [item_ptr[t], item_ptr[t + 1])
  const int2* side_items;     // per (order position, side): first item, count
  double eta;                 // BR2 penalty
  double* dot_partial;        // optional reduction of x . y (see Reduce)
  double* dot_out;
  unsigned* dot_ticket;
  double* pcg_sc;             // PCG scalars: with the x . y sum, alpha = (r.z) / (p.q)
  const double* skip;         // batch: tiles whose instance has skip[inst * skip_stride] != 0 are idle
  int skip_stride;
  int n_tiles;
  unsigned* sched;            // [0] next tile, [1] exit ticket (both zero between launches)
  BasisOff boff[kMaxP + 1];
  // mapped squares: per sub-face record its rule size, tables, factors and
  // penalty; the geometric factors at the Gauss points (volume per element,
  // faces per record); the volume tables
  const SubFaceMap* sfm;
  const double* gvol;
  const int64_t* goff;
  const double* gface;
  const double* gbr2;         // BR2: mass-inverse side blocks, per element from g2off[k]
  const int64_t* g2off;
  MapOff moff[kMaxP + 1];
};

template <int P>
struct ApplyShape {
  static constexpr int NP = P + 1;
  static constexpr int NN = NP * NP;
  static constexpr int EPB = apply_epb(P);
  // shared doubles: M, K (2 NN) + x, T1, T2 (3 EPB NN) + r, c2 (8 EPB NP)
  static constexpr int SMEM = 2 * NN + 3 * EPB * NN + 8 * EPB * NP;
  // start (doubles) of the sub-face item partials: double2, so 16-byte aligned
  static constexpr int PART = (SMEM + 1) & ~1;
};

__device__ __forceinline__ int side_node(int s, int i, int k, int np) {
  // node on side s at tangential index i, normal index k (k = 0 / np-1 is the
  // side itself for s = 0,2 / 1,3)
  return (s < 2) ? (i * np + k) : (k * np + i);
}

// load through the read-only path, or a plain load when the data may have been
// written earlier in the same kernel
template <bool RO>
__device__ __forceinline__ double ld_x(const double* p) {
  if (RO) return __ldg(p);
  return *p;
}

// Side traces of one tile: task = (element, side, node), packed.
template <int P, bool RO = true>
__device__ __forceinline__ void trace_tile(const ApplyArgs& A, const ApplyTile& T) {
  constexpr int NP = P + 1;
  const BasisOff bo = A.boff[P];
  if (A.skip && A.skip[(int64_t)T.inst * A.skip_stride] != 0.0) return;
  const int ntask = T.count * 4 * NP;
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    const int e = t / (4 * NP);
    const int s = (t / NP) & 3;
    const int i = t % NP;
    const int k = A.order[T.first + e];
    const double* xk = A.x + A.off[k];
    const double* dv = A.tab + ((s & 1) ? bo.d1 : bo.d0);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) acc = fma(__ldg(dv + q), ld_x<RO>(xk + side_node(s, i, q, NP)), acc);
    const double sg = (s & 1) ? A.aih[k] : -A.aih[k];   // a grad u . n
    double2 v;
    v.x = ld_x<RO>(xk + side_node(s, i, (s & 1) ? P : 0, NP));
    v.y = sg * acc;
    reinterpret_cast<double2*>(A.tr + A.toff[k])[s * NP + i] = v;
  }
}

template <int P, bool BR2>
__device__ __forceinline__ void apply_tile(const ApplyArgs& A, const ApplyTile& T, int tile,
                                           double* sm, double* red) {
  using S = ApplyShape<P>;
  constexpr int NP = S::NP, NN = S::NN, EPB = S::EPB;
  double* sM = sm;
  double* sK = sM + NN;
  double* sx = sK + NN;
  double* sT1 = sx + EPB * NN;
  double* sT2 = sT1 + EPB * NN;
  double* sr = sT2 + EPB * NN;           // [EPB][4][NP]
  double* sc2 = sr + EPB * 4 * NP;       // [EPB][4][NP]

  const int tid = threadIdx.x;
  if (A.skip && A.skip[(int64_t)T.inst * A.skip_stride] != 0.0) {   // CTA-uniform
    if (A.dot_partial && tid == 0) A.dot_partial[tile] = 0.0;
    return;
  }
  const int count = T.count;
  const int nnode = count * NN;           // volume / gather tasks
  const int nside = count * 4 * NP;       // face tasks
  const BasisOff bo = A.boff[P];

  for (int i = tid; i < NN; i += blockDim.x) {
    sM[i] = __ldg(A.tab + bo.M + i);
    sK[i] = __ldg(A.tab + bo.K + i);
  }
  for (int t = tid; t < nnode; t += blockDim.x) {
    const int e = t / NN;
    sx[t] = A.x[A.off[A.order[T.first + e]] + (t - e * NN)];
  }
  __syncthreads();
  // ---- volume pass 1: contract along x
  for (int t = tid; t < nnode; t += blockDim.x) {
    const int e = t / NN, node = t - e * NN;
    const int ix = node % NP, iy = node / NP;
    const double* xr = sx + e * NN + iy * NP;
    double t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      t1 = fma(sK[ix * NP + j], xr[j], t1);
      t2 = fma(sM[ix * NP + j], xr[j], t2);
    }
    sT1[t] = t1;
    sT2[t] = t2;
  }
  // ---- faces: one thread per (sub-face item, side node) forms that
  // sub-face's contribution to the node, then one thread per side node sums
  // its sub-faces' contributions in sub-face order (deterministic)
  {
    const int ib = A.item_ptr[tile];
    const int nit = A.item_ptr[tile + 1] - ib;
    double2* part = reinterpret_cast<double2*>(sm + S::PART);   // [nit][NP]
    for (int t = tid; t < nit * NP; t += blockDim.x) {
      const int it = t / NP, i = t - it * NP;
      const int2 item = A.items[ib + it];   // sorted by branch; item.y >> 16: sub-face order
      const SubFaceRec f = A.sf[item.x];
      const int e = (item.y & 0xffff) >> 2, s = item.y & 3;
      const int k = A.order[T.first + e];
      const double2* trk = reinterpret_cast<const double2*>(A.tr + A.toff[k]) + s * NP;
      const double* Moo = A.tab + f.tab_oo + i * NP;
      double a = 0.0, c = 0.0;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const double w = __ldg(Moo + m);
        const double2 v = trk[m];
        a = fma(w, v.x, a);
        c = fma(w, v.y, c);
      }
      double r, c2;
      if (f.nb < 0) {
        if (BR2) {   // eta [M_oo G_o a]: cz (Z u-)_i, Z = M_oo on the whole side
          const SubFaceBr2 g = A.sfb[item.x];
          double z = a;
          if (!(g.full & 1)) {
            const double* Z = A.tab + g.tab_z + i * NP;
            z = 0.0;
#pragma unroll
            for (int m = 0; m < NP; ++m) z = fma(__ldg(Z + m), trk[m].x, z);
          }
          r = fma(g.cz, z, -f.len * c);
        } else {
          r = f.len * (f.sigma * a - c);
        }
        c2 = -f.len * a;
      } else {
        const int np = f.pn + 1;
        const double* Mon = A.tab + f.tab_on + i * np;
        const double2* trn = reinterpret_cast<const double2*>(A.tr + A.toff[f.nb]) + f.nb_side * np;
        double b = 0.0, d = 0.0;
        for (int m = 0; m < np; ++m) {
          const double w = __ldg(Mon + m);
          const double2 v = trn[m];
          b = fma(w, v.x, b);
          d = fma(w, v.y, d);   // neighbour's outward dn: this side's dn+ is -v.y
        }
        const double jmp = a - b;
        if (BR2) {   // eta/4 [M_oo G_o jo + M_on G_n jn] = cz (Z u- - V u+) + cx (X u- - Y u+)
          const SubFaceBr2 g = A.sfb[item.x];
          const double* X = A.tab + g.tab_x + i * NP;
          double xx = 0.0;
#pragma unroll
          for (int m = 0; m < NP; ++m) xx = fma(__ldg(X + m), trk[m].x, xx);
          double z = a, v = b, y = b;   // whole own side: Z = M_oo, V = M_on; whole neighbour side: Y = M_on
          if (!(g.full & 1)) {
            const double* Z = A.tab + g.tab_z + i * NP;
            const double* V = A.tab + g.tab_v + i * np;
            z = 0.0;
            v = 0.0;
#pragma unroll
            for (int m = 0; m < NP; ++m) z = fma(__ldg(Z + m), trk[m].x, z);
            for (int m = 0; m < np; ++m) v = fma(__ldg(V + m), trn[m].x, v);
          }
          if (!(g.full & 2)) {
            const double* Y = A.tab + g.tab_y + i * np;
            y = 0.0;
            for (int m = 0; m < np; ++m) y = fma(__ldg(Y + m), trn[m].x, y);
          }
          r = fma(g.cz, z - v, fma(g.cx, xx - y, -0.5 * f.len * (c - d)));
        } else {
          r = f.len * (f.sigma * jmp - 0.5 * (c - d));
        }
        c2 = -0.5 * f.len * jmp;
      }
      part[(item.y >> 16) * NP + i] = make_double2(r, c2);
    }
    __syncthreads();
    for (int t = tid; t < nside; t += blockDim.x) {
      const int e = t / (4 * NP);
      const int s = (t / NP) & 3;
      const int i = t % NP;
      const int2 si = A.side_items[(int64_t)(T.first + e) * 4 + s];
      double r = 0.0, c2 = 0.0;
      for (int j = 0; j < si.y; ++j) {
        const double2 v = part[(si.x - ib + j) * NP + i];
        r += v.x;
        c2 += v.y;
      }
      sr[t] = r;
      sc2[t] = c2;
    }
  }
  __syncthreads();
  // ---- gather: volume pass 2 + side residuals + normal-derivative terms
  double part = 0.0;
  for (int t = tid; t < nnode; t += blockDim.x) {
    const int e = t / NN, node = t - e * NN;
    const int ix = node % NP, iy = node / NP;
    const int k = A.order[T.first + e];
    double y = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      y = fma(sM[iy * NP + q], sT1[e * NN + q * NP + ix], y);
      y = fma(sK[iy * NP + q], sT2[e * NN + q * NP + ix], y);
    }
    const double* d0 = A.tab + bo.d0;
    const double* d1 = A.tab + bo.d1;
    const double aih = A.aih[k];
    y *= A.ak[k];
    const double* c2 = sc2 + e * 4 * NP;
    const double* r = sr + e * 4 * NP;
    double g = -__ldg(d0 + ix) * c2[0 * NP + iy];
    g = fma(__ldg(d1 + ix), c2[1 * NP + iy], g);
    g = fma(-__ldg(d0 + iy), c2[2 * NP + ix], g);
    g = fma(__ldg(d1 + iy), c2[3 * NP + ix], g);
    y = fma(g, aih, y);
    if (ix == 0) y += r[0 * NP + iy];
    if (ix == P) y += r[1 * NP + iy];
    if (iy == 0) y += r[2 * NP + ix];
    if (iy == P) y += r[3 * NP + ix];
    A.y[A.off[k] + node] = y;
    part = fma(y, sx[t], part);
  }
  if (A.dot_partial) {
    // tile partial of x . y (summed in tile order when the launch ends)
    const double tot = block_sum<kThreads>(part, red);
    if (tid == 0) A.dot_partial[tile] = tot;
  }
}

}  // namespace dg
