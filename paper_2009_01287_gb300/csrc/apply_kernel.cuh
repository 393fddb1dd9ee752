// Matrix-free SIPG / BR2 operator y = A x on 2D leaf squares (Section 2,
// Eq. fe-problem; BR2 stabilisation of Section 4.4), FP64.
//
// One CTA of kThreads threads processes a tile of EPB elements of one degree
// P, one thread per Gauss-Lobatto node.  Per element:
//   volume  y = (K (x) M + M (x) K) x       sum factorised, two passes through
//           shared memory (Section 4.1: O(p^{d+1}) work per element);
//   faces   every sub-face of every side is computed from this element's
//           side (so no atomics, deterministic): own / neighbour traces and
//           outward normal derivatives at the side nodes, then the exact face
//           mass matrices M_oo (own-own) and M_on (own-neighbour) of the
//           sub-face give the four projections
//             a = M_oo u-, b = M_on u+, c = M_oo dn-, d = M_on dn+,
//           and the residual of the test functions of this element is
//             edge nodes:   -1/2 (c + d) + stab        (interior)
//                           -c + sigma a               (boundary)
//             all nodes:    dn(v) * (-1/2 (a - b))     (interior)
//                           dn(v) * (-a)               (boundary)
//           with stab = sigma (a - b) for SIPG and, for BR2,
//             stab = eta/4 [M_oo G_o (a - b) + M_on G_n (M_no u- - M_nn u+)],
//           G = edge block of the element mass inverse = h^-2 Minv_00 Minv.
#pragma once

#include "dg_internal.h"

namespace dg {

struct ApplyArgs {
  const double* x;
  double* y;
  const int32_t* p;
  const int64_t* off;
  const double* h;
  const int32_t* sf_ptr;
  const SubFaceRec* sf;
  const double* tab;          // basis + face tables
  const int32_t* order;       // degree-sorted element order
  const ApplyTile* tiles;
  double eta;                 // BR2 penalty
  double* dot_partial;        // optional per-CTA partial of x . y
  BasisOff boff[kMaxP + 1];
};

template <int P>
struct ApplyShape {
  static constexpr int NP = P + 1;
  static constexpr int NN = NP * NP;
  static constexpr int EPB = apply_epb(P);
  // shared doubles: M,K (2 NN) + x,T1,T2 (3 EPB NN) + dn own (4 EPB NP)
  // + nb u,dn (8 EPB kMaxN) + r,c2 (8 EPB NP) + BR2: jo,go,cd (12 EPB NP), jn,gn (8 EPB kMaxN)
  static constexpr int SMEM = 2 * NN + 3 * EPB * NN + 4 * EPB * NP + 8 * EPB * kMaxN +
                              8 * EPB * NP + 12 * EPB * NP + 8 * EPB * kMaxN;
};

__device__ __forceinline__ int side_node(int s, int i, int k, int np) {
  // node on side s at tangential index i, normal index k (k = 0 / np-1 is the
  // side itself for s = 0,2 / 1,3)
  return (s < 2) ? (i * np + k) : (k * np + i);
}

template <int P, bool BR2>
__device__ __forceinline__ void apply_tile(const ApplyArgs& A, const ApplyTile& T, double* sm) {
  using S = ApplyShape<P>;
  constexpr int NP = S::NP, NN = S::NN, EPB = S::EPB;
  double* sM = sm;
  double* sK = sM + NN;
  double* sx = sK + NN;
  double* sT1 = sx + EPB * NN;
  double* sT2 = sT1 + EPB * NN;
  double* sdn = sT2 + EPB * NN;          // [EPB][4][NP]
  double* sun = sdn + EPB * 4 * NP;      // [EPB][4][kMaxN]
  double* sdnn = sun + EPB * 4 * kMaxN;  // [EPB][4][kMaxN]
  double* sr = sdnn + EPB * 4 * kMaxN;   // [EPB][4][NP]
  double* sc2 = sr + EPB * 4 * NP;       // [EPB][4][NP]
  double* sjo = sc2 + EPB * 4 * NP;      // BR2 [EPB][4][NP]
  double* sgo = sjo + EPB * 4 * NP;
  double* scd = sgo + EPB * 4 * NP;
  double* sjn = scd + EPB * 4 * NP;      // [EPB][4][kMaxN]
  double* sgn = sjn + EPB * 4 * kMaxN;

  __shared__ int s_maxsub;
  const int tid = threadIdx.x;
  const int e = tid / NN;
  const int node = tid - e * NN;
  const bool active = (e < EPB) && (e < T.count);
  const int k = active ? A.order[T.first + e] : 0;
  const int64_t base = active ? A.off[k] : 0;
  const double hk = active ? A.h[k] : 1.0;
  const BasisOff bo = A.boff[P];

  if (tid == 0) s_maxsub = 0;
  for (int i = tid; i < NN; i += blockDim.x) {
    sM[i] = __ldg(A.tab + bo.M + i);
    sK[i] = __ldg(A.tab + bo.K + i);
  }
  if (active) sx[e * NN + node] = A.x[base + node];
  __syncthreads();
  if (active && node < 4) {
    int cnt = A.sf_ptr[4 * k + node + 1] - A.sf_ptr[4 * k + node];
    atomicMax(&s_maxsub, cnt);
  }
  // ---- volume pass 1 (thread = (ix, row k)): contract along x
  const int ix = node % NP, iy = node / NP;
  if (active) {
    const double* xr = sx + e * NN + iy * NP;
    double t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      t1 = fma(sK[ix * NP + j], xr[j], t1);
      t2 = fma(sM[ix * NP + j], xr[j], t2);
    }
    sT1[e * NN + iy * NP + ix] = t1;
    sT2[e * NN + iy * NP + ix] = t2;
  }
  // own outward normal derivatives at the side nodes; zero the accumulators
  if (active) {
    for (int task = node; task < 4 * NP; task += NN) {
      const int s = task / NP, i = task - s * NP;
      const double* dv = A.tab + ((s & 1) ? bo.d1 : bo.d0);
      const double sg = ((s & 1) ? 1.0 : -1.0) / hk;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NP; ++q) acc = fma(__ldg(dv + q), sx[e * NN + side_node(s, i, q, NP)], acc);
      sdn[(e * 4 + s) * NP + i] = sg * acc;
      sr[(e * 4 + s) * NP + i] = 0.0;
      sc2[(e * 4 + s) * NP + i] = 0.0;
    }
  }
  __syncthreads();
  // ---- volume pass 2: contract along y
  double yv = 0.0;
  if (active) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      yv = fma(sM[iy * NP + q], sT1[e * NN + q * NP + ix], yv);
      yv = fma(sK[iy * NP + q], sT2[e * NN + q * NP + ix], yv);
    }
  }
  const int maxsub = s_maxsub;
  // ---- faces
  for (int j = 0; j < maxsub; ++j) {
    // stage neighbour traces / normal derivatives (along this element's
    // outward normal) at the neighbour's side nodes
    if (active) {
      for (int task = node; task < 4 * kMaxN; task += NN) {
        const int s = task / kMaxN, m = task - s * kMaxN;
        const int b = A.sf_ptr[4 * k + s];
        if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
        const SubFaceRec f = A.sf[b + j];
        if (f.nb < 0 || m > f.pn) continue;
        const int np = f.pn + 1;
        const int64_t nbase = A.off[f.nb];
        const int kedge = (f.nb_side & 1) ? f.pn : 0;
        const BasisOff bn = A.boff[f.pn];
        const double* dv = A.tab + ((f.nb_side & 1) ? bn.d1 : bn.d0);
        const double sg = ((f.nb_side & 1) ? -1.0 : 1.0) / A.h[f.nb];  // minus nb outward
        double acc = 0.0;
        for (int q = 0; q < np; ++q)
          acc = fma(__ldg(dv + q), __ldg(A.x + nbase + side_node(f.nb_side, m, q, np)), acc);
        sun[(e * 4 + s) * kMaxN + m] = __ldg(A.x + nbase + side_node(f.nb_side, m, kedge, np));
        sdnn[(e * 4 + s) * kMaxN + m] = sg * acc;
      }
    }
    __syncthreads();
    if (active) {
      for (int task = node; task < 4 * NP; task += NN) {
        const int s = task / NP, i = task - s * NP;
        const int b = A.sf_ptr[4 * k + s];
        if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
        const SubFaceRec f = A.sf[b + j];
        const double* Moo = A.tab + f.tab_oo + i * NP;
        const int kedge = (s & 1) ? P : 0;
        double a = 0.0, c = 0.0;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const double w = __ldg(Moo + m);
          a = fma(w, sx[e * NN + side_node(s, m, kedge, NP)], a);
          c = fma(w, sdn[(e * 4 + s) * NP + m], c);
        }
        a *= f.len;
        c *= f.len;
        const int o = (e * 4 + s) * NP + i;
        if (f.nb < 0) {
          sc2[o] -= a;
          if (BR2) { sjo[o] = a; scd[o] = -c; }
          else sr[o] += -c + f.sigma * a;
        } else {
          const int np = f.pn + 1;
          const double* Mon = A.tab + f.tab_on + i * np;
          double bb = 0.0, d = 0.0;
          for (int m = 0; m < np; ++m) {
            const double w = __ldg(Mon + m);
            bb = fma(w, sun[(e * 4 + s) * kMaxN + m], bb);
            d = fma(w, sdnn[(e * 4 + s) * kMaxN + m], d);
          }
          bb *= f.len;
          d *= f.len;
          sc2[o] -= 0.5 * (a - bb);
          if (BR2) { sjo[o] = a - bb; scd[o] = -0.5 * (c + d); }
          else sr[o] += -0.5 * (c + d) + f.sigma * (a - bb);
        }
      }
      if (BR2) {
        // neighbour-indexed jump projection jn = M_no u- - M_nn u+
        for (int task = node; task < 4 * kMaxN; task += NN) {
          const int s = task / kMaxN, m = task - s * kMaxN;
          const int b = A.sf_ptr[4 * k + s];
          if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
          const SubFaceRec f = A.sf[b + j];
          if (f.nb < 0 || m > f.pn) continue;
          const int np = f.pn + 1;
          const int kedge = (s & 1) ? P : 0;
          double v = 0.0;
          for (int i = 0; i < NP; ++i)
            v = fma(__ldg(A.tab + f.tab_on + i * np + m), sx[e * NN + side_node(s, i, kedge, NP)], v);
          for (int q = 0; q < np; ++q)
            v = fma(-__ldg(A.tab + f.tab_nn + m * np + q), sun[(e * 4 + s) * kMaxN + q], v);
          sjn[(e * 4 + s) * kMaxN + m] = v * f.len;
        }
      }
    }
    if (BR2) {
      __syncthreads();
      if (active) {
        // G applied on both sides
        for (int task = node; task < 4 * NP; task += NN) {
          const int s = task / NP, i = task - s * NP;
          const int b = A.sf_ptr[4 * k + s];
          if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
          const double* Mi = A.tab + bo.Minv;
          double g = 0.0;
#pragma unroll
          for (int m = 0; m < NP; ++m) g = fma(__ldg(Mi + i * NP + m), sjo[(e * 4 + s) * NP + m], g);
          sgo[(e * 4 + s) * NP + i] = g * __ldg(Mi) / (hk * hk);
        }
        for (int task = node; task < 4 * kMaxN; task += NN) {
          const int s = task / kMaxN, m = task - s * kMaxN;
          const int b = A.sf_ptr[4 * k + s];
          if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
          const SubFaceRec f = A.sf[b + j];
          if (f.nb < 0 || m > f.pn) continue;
          const int np = f.pn + 1;
          const double* Mi = A.tab + A.boff[f.pn].Minv;
          double g = 0.0;
          for (int q = 0; q < np; ++q) g = fma(__ldg(Mi + m * np + q), sjn[(e * 4 + s) * kMaxN + q], g);
          const double hn = A.h[f.nb];
          sgn[(e * 4 + s) * kMaxN + m] = g * __ldg(Mi) / (hn * hn);
        }
      }
      __syncthreads();
      if (active) {
        for (int task = node; task < 4 * NP; task += NN) {
          const int s = task / NP, i = task - s * NP;
          const int b = A.sf_ptr[4 * k + s];
          if (j >= A.sf_ptr[4 * k + s + 1] - b) continue;
          const SubFaceRec f = A.sf[b + j];
          const int o = (e * 4 + s) * NP + i;
          double st = 0.0;
#pragma unroll
          for (int m = 0; m < NP; ++m) st = fma(__ldg(A.tab + f.tab_oo + i * NP + m), sgo[(e * 4 + s) * NP + m], st);
          double coef = 1.0;
          if (f.nb >= 0) {
            const int np = f.pn + 1;
            for (int m = 0; m < np; ++m)
              st = fma(__ldg(A.tab + f.tab_on + i * np + m), sgn[(e * 4 + s) * kMaxN + m], st);
            coef = 0.25;
          }
          sr[o] += scd[o] + A.eta * coef * f.len * st;
        }
      }
    }
    __syncthreads();
  }
  // ---- gather: volume + edge residuals + normal-derivative terms
  if (active) {
    double y = yv;
    const int ixn = node % NP, iyn = node / NP;
    const double* d0 = A.tab + bo.d0;
    const double* d1 = A.tab + bo.d1;
    const double ih = 1.0 / hk;
    // side 0/1 (x = 0 / 1): tangential index iy, normal index ix
    y = fma(-__ldg(d0 + ixn) * ih, sc2[(e * 4 + 0) * NP + iyn], y);
    y = fma(__ldg(d1 + ixn) * ih, sc2[(e * 4 + 1) * NP + iyn], y);
    y = fma(-__ldg(d0 + iyn) * ih, sc2[(e * 4 + 2) * NP + ixn], y);
    y = fma(__ldg(d1 + iyn) * ih, sc2[(e * 4 + 3) * NP + ixn], y);
    if (ixn == 0) y += sr[(e * 4 + 0) * NP + iyn];
    if (ixn == P) y += sr[(e * 4 + 1) * NP + iyn];
    if (iyn == 0) y += sr[(e * 4 + 2) * NP + ixn];
    if (iyn == P) y += sr[(e * 4 + 3) * NP + ixn];
    A.y[base + node] = y;
    sT1[e * NN + node] = y * sx[e * NN + node];
  }
  if (A.dot_partial) {
    __syncthreads();
    // deterministic tile partial of x . y
    if (tid == 0) {
      double s = 0.0;
      const int nact = (T.count < EPB ? T.count : EPB) * NN;
      for (int i = 0; i < nact; ++i) s += sT1[i];
      A.dot_partial[blockIdx.x] = s;
    }
  }
}

}  // namespace dg
