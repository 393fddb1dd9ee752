// Matrix-free SIPG / BR2 operator y = A x on mapped squares (Section 2:
// element maps T_kappa onto general quadrilaterals; Eq. fe-problem; BR2 of
// Section 4.4), FP64.
//
// The elements are the images of the leaf boxes under the bilinear map of the
// lattice domain (DomainMap), so the geometric factors vary inside every
// element and the separable M / K contractions of boxes no longer apply.  The
// kernel works at Gauss points instead, with the same tiles, side traces and
// flat sub-face item lists as the box kernel:
//   volume  u at the (p+2)^2 Gauss points by sum factorisation (B = l_j(x_g),
//           D = l_j'(x_g)): grad_xi u = ((B (x) D) u, (D (x) B) u); at every
//           point the flux a w_g w_h G grad_xi u with G = det(J) J^-1 J^-T of
//           the map there (three factors per point, stored at setup); back to
//           the nodes with the transposed products: four passes of
//           O((p+1)(p+2)^2) work per element instead of two;
//   faces   one thread per (sub-face item, Gauss point) evaluates both sides'
//           traces there (values and a-weighted normal derivatives from the
//           trace array, tangential derivatives from the trace values) and,
//           with the point's stored factors (the arc-length weight w and w m
//           for m = J^-1 n, n = J^-T nu / |J^-T nu| the physical normal),
//           writes three adjoint weights: of the test function's value, of its
//           tangential derivative and of its normal derivative; one thread per
//           side node then sums them over its sub-faces in sub-face order
//           (deterministic) with the side's basis tables, and the gather adds
//           the normal-derivative weights through l_k'(0 or 1) / h as on boxes.
//   BR2     the mass matrix of a mapped element is not a Kronecker product, so
//           the lifting takes the block of each element's mass inverse on a
//           side's nodes (stored at setup): per item the jump projected onto
//           both sides' nodes, the two blocks applied, and the lifted values
//           at the item's points added to the value weights (three more
//           passes of the tile's items).
// Every sub-face is evaluated from both of its sides (no atomics): applies are
// bit-reproducible.
#pragma once

#include "apply_kernel.cuh"

namespace dg {

template <int P>
struct MapShape {
  static constexpr int NP = P + 1;
  static constexpr int NN = NP * NP;
  static constexpr int Q = P + 1 + kMapQExtra;
  static constexpr int QQ = Q * Q;
  static constexpr int EPB = apply_epb(P);
  // shared doubles: B, D (2 Q NP), x (EPB NN), stage 1 / 3 (2 EPB NP Q),
  // point fluxes (2 EPB QQ), side sums r, c2 (8 EPB NP)
  static constexpr int SMEM = 2 * Q * NP + EPB * NN + 2 * EPB * NP * Q + 2 * EPB * QQ + 8 * EPB * NP;
  // then the sub-face item weights: [item][kMapQMax][3]; BR2 adds per item
  // the weighted jumps at its points and both sides' lifting vectors
  static constexpr int PART = SMEM;
};
constexpr int kMapItemDoubles = 3 * kMapQMax;
constexpr int kMapItemBr2 = kMapQMax + 4 * kMaxN;   // w [[u]] per point; j-, j+, z-, z+

template <int P, bool BR2>
__device__ __forceinline__ void apply_map_tile(const ApplyArgs& A, const ApplyTile& T, int tile, double* sm,
                                               double* red) {
  using S = MapShape<P>;
  constexpr int NP = S::NP, NN = S::NN, Q = S::Q, QQ = S::QQ, EPB = S::EPB;
  double* sB = sm;                    // [Q][NP]
  double* sD = sB + Q * NP;
  double* sx = sD + Q * NP;           // [EPB][NN]
  double* sA1 = sx + EPB * NN;        // [EPB][NP][Q]; stage 3 reuses it
  double* sA2 = sA1 + EPB * NP * Q;
  double* sF1 = sA2 + EPB * NP * Q;   // [EPB][Q][Q]
  double* sF2 = sF1 + EPB * QQ;
  double* sr = sF2 + EPB * QQ;        // [EPB][4][NP]
  double* sc2 = sr + EPB * 4 * NP;
  double* part = sm + S::PART;        // [item][kMapQMax][3]

  const int tid = threadIdx.x;
  const int count = T.count;
  const MapOff mo = A.moff[P];
  for (int i = tid; i < Q * NP; i += blockDim.x) {
    sB[i] = __ldg(A.tab + mo.B + i);
    sD[i] = __ldg(A.tab + mo.D + i);
  }
  for (int t = tid; t < count * NN; t += blockDim.x) {
    const int e = t / NN;
    sx[t] = A.x[A.off[A.order[T.first + e]] + (t - e * NN)];
  }
  __syncthreads();
  // ---- volume stage 1: contract along x at the Gauss points (derivative and value)
  for (int t = tid; t < count * NP * Q; t += blockDim.x) {
    const int e = t / (NP * Q), rem = t - e * NP * Q;
    const int jy = rem / Q, g = rem - jy * Q;
    const double* xr = sx + e * NN + jy * NP;
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      a = fma(sD[g * NP + j], xr[j], a);
      b = fma(sB[g * NP + j], xr[j], b);
    }
    sA1[t] = a;
    sA2[t] = b;
  }
  // ---- faces, pass 1: one thread per (sub-face item, Gauss point)
  const int ib = A.item_ptr[tile];
  const int nit = A.item_ptr[tile + 1] - ib;
  double* br2 = part + kMapItemDoubles * nit;   // BR2: [item][kMapItemBr2]
  for (int t = tid; t < nit * kMapQMax; t += blockDim.x) {
    const int it = t / kMapQMax, g = t - it * kMapQMax;
    const int2 item = A.items[ib + it];
    const SubFaceMap fm = A.sfm[item.x];
    const int qf = fm.qf;
    if (g >= qf) continue;
    const SubFaceRec f = A.sf[item.x];
    const int e = (item.y & 0xffff) >> 2, s = item.y & 3;
    const int k = A.order[T.first + e];
    const double2* trk = reinterpret_cast<const double2*>(A.tr + A.toff[k]) + s * NP;
    const double* Bo = A.tab + fm.tab_bo + g * NP;
    const double* Do = A.tab + fm.tab_bo + (qf + g) * NP;
    double u0 = 0.0, du0 = 0.0, f0 = 0.0;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const double2 v = trk[m];
      const double b = __ldg(Bo + m);
      u0 = fma(b, v.x, u0);
      du0 = fma(__ldg(Do + m), v.x, du0);
      f0 = fma(b, v.y, f0);
    }
    du0 *= A.ih[k];
    // the point's factors: w = w_g |J t| dt, w m_t, w m_n s (m = J^-1 n)
    const double* gf = A.gface + fm.geo;
    const double w = __ldg(gf + g), wmt = __ldg(gf + qf + g), wmn = __ldg(gf + 2 * qf + g);
    const double Fo = fma(f0, wmn, A.ak[k] * du0 * wmt);   // w (a grad u-) . n
    double jmp, flux, cc;
    if (f.nb >= 0) {
      const int npn = f.pn + 1;
      const double2* trn = reinterpret_cast<const double2*>(A.tr + A.toff[f.nb]) + f.nb_side * npn;
      const double* Bn = A.tab + fm.tab_bn + g * npn;
      const double* Dn = A.tab + fm.tab_bn + (qf + g) * npn;
      double u1 = 0.0, du1 = 0.0, f1 = 0.0;
      for (int m = 0; m < npn; ++m) {
        const double2 v = trn[m];
        const double b = __ldg(Bn + m);
        u1 = fma(b, v.x, u1);
        du1 = fma(__ldg(Dn + m), v.x, du1);
        f1 = fma(b, v.y, f1);
      }
      du1 *= A.ih[f.nb];
      const double Fn = fma(-f1, wmn, A.ak[f.nb] * du1 * wmt);   // w (a grad u+) . n
      jmp = u0 - u1;
      flux = 0.5 * (Fo + Fn);
      cc = 0.5;
    } else {
      jmp = u0;
      flux = Fo;
      cc = 1.0;
    }
    double* pp = part + ((item.y >> 16) * kMapQMax + g) * 3;
    if (BR2) {
      pp[0] = -flux;                                    // the lifting term is added below
      br2[(item.y >> 16) * kMapItemBr2 + g] = w * jmp;
    } else {
      pp[0] = fma(fm.sigma * jmp, w, -flux);   // weight of v-
    }
    pp[1] = -cc * jmp * wmt;                 // of d v- / d t (times a / h and l' at the side sums)
    pp[2] = -cc * jmp * wmn;                 // of a times the outward normal derivative of v-
  }
  __syncthreads();
  if (BR2) {
    // BR2 liftings (Section 4.4) of every sub-face on both of its sides:
    // j = int phi_j [[u]] ds on each side's nodes, z = (block of that
    // element's mass inverse on the side) j, and at every point the weight
    // eta coef a w (z-(x_g) + z+(x_g)) of the own test function's value.
    // One thread per (item, side node) for j and z, per (item, point) after.
    for (int t = tid; t < nit * kMaxN; t += blockDim.x) {
      const int it = t / kMaxN, j = t - it * kMaxN;
      const int2 item = A.items[ib + it];
      const SubFaceMap fm = A.sfm[item.x];
      const SubFaceRec f = A.sf[item.x];
      double* b = br2 + (item.y >> 16) * kMapItemBr2;
      if (j < NP) {
        double a = 0.0;
        for (int g = 0; g < fm.qf; ++g) a = fma(__ldg(A.tab + fm.tab_bo + g * NP + j), b[g], a);
        b[kMapQMax + j] = a;
      }
      if (f.nb >= 0 && j <= f.pn) {
        const int npn = f.pn + 1;
        double a = 0.0;
        for (int g = 0; g < fm.qf; ++g) a = fma(__ldg(A.tab + fm.tab_bn + g * npn + j), b[g], a);
        b[kMapQMax + kMaxN + j] = a;
      }
    }
    __syncthreads();
    for (int t = tid; t < nit * kMaxN; t += blockDim.x) {
      const int it = t / kMaxN, j = t - it * kMaxN;
      const int2 item = A.items[ib + it];
      const SubFaceRec f = A.sf[item.x];
      const int e = (item.y & 0xffff) >> 2, s = item.y & 3;
      double* b = br2 + (item.y >> 16) * kMapItemBr2;
      if (j < NP) {
        const int k = A.order[T.first + e];
        const double* Go = A.gbr2 + A.g2off[k] + s * NP * NP + j * NP;
        double z = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) z = fma(__ldg(Go + i), b[kMapQMax + i], z);
        b[kMapQMax + 2 * kMaxN + j] = z;
      }
      if (f.nb >= 0 && j <= f.pn) {
        const int npn = f.pn + 1;
        const double* Gn = A.gbr2 + A.g2off[f.nb] + f.nb_side * npn * npn + j * npn;
        double z = 0.0;
        for (int i = 0; i < npn; ++i) z = fma(__ldg(Gn + i), b[kMapQMax + kMaxN + i], z);
        b[kMapQMax + 3 * kMaxN + j] = z;
      }
    }
    __syncthreads();
    for (int t = tid; t < nit * kMapQMax; t += blockDim.x) {
      const int it = t / kMapQMax, g = t - it * kMapQMax;
      const int2 item = A.items[ib + it];
      const SubFaceMap fm = A.sfm[item.x];
      if (g >= fm.qf) continue;
      const SubFaceRec f = A.sf[item.x];
      const double* b = br2 + (item.y >> 16) * kMapItemBr2;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) v = fma(__ldg(A.tab + fm.tab_bo + g * NP + i), b[kMapQMax + 2 * kMaxN + i], v);
      if (f.nb >= 0) {
        const int npn = f.pn + 1;
        for (int i = 0; i < npn; ++i)
          v = fma(__ldg(A.tab + fm.tab_bn + g * npn + i), b[kMapQMax + 3 * kMaxN + i], v);
      }
      part[((item.y >> 16) * kMapQMax + g) * 3] += fm.cbr2 * __ldg(A.gface + fm.geo + g) * v;
    }
    __syncthreads();
  }
  // ---- volume stage 2 and the flux at every Gauss point
  for (int t = tid; t < count * QQ; t += blockDim.x) {
    const int e = t / QQ, rem = t - e * QQ;
    const int gy = rem / Q, gxi = rem - gy * Q;
    const double* a1 = sA1 + e * NP * Q + gxi;
    const double* a2 = sA2 + e * NP * Q + gxi;
    double ux = 0.0, uy = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      ux = fma(sB[gy * NP + j], a1[j * Q], ux);
      uy = fma(sD[gy * NP + j], a2[j * Q], uy);
    }
    // the point's factors a w_g w_h G (three planes per element)
    const double* G = A.gvol + A.goff[A.order[T.first + e]] + rem;
    const double g11 = __ldg(G), g12 = __ldg(G + QQ), g22 = __ldg(G + 2 * QQ);
    sF1[t] = fma(g11, ux, g12 * uy);
    sF2[t] = fma(g12, ux, g22 * uy);
  }
  // ---- faces, pass 2: one thread per side node sums its sub-faces' weights
  // in sub-face order with the side's basis tables
  for (int t = tid; t < count * 4 * NP; t += blockDim.x) {
    const int e = t / (4 * NP);
    const int s = (t / NP) & 3;
    const int i = t % NP;
    const int k = A.order[T.first + e];
    const int2 si = A.side_items[(int64_t)(T.first + e) * 4 + s];
    const int rec0 = A.sf_ptr[4 * k + s];
    const double aih = A.aih[k];
    double r = 0.0, c2 = 0.0;
    for (int j = 0; j < si.y; ++j) {
      const SubFaceMap fm = A.sfm[rec0 + j];
      const double* pp = part + (si.x - ib + j) * kMapQMax * 3;
      const double* Bo = A.tab + fm.tab_bo + i;
      const double* Do = Bo + fm.qf * NP;
      for (int g = 0; g < fm.qf; ++g) {
        const double b = __ldg(Bo + g * NP);
        r = fma(b, pp[3 * g], r);
        r = fma(aih * __ldg(Do + g * NP), pp[3 * g + 1], r);
        c2 = fma(b, pp[3 * g + 2], c2);
      }
    }
    sr[t] = r;
    sc2[t] = c2;
  }
  __syncthreads();
  // ---- volume stage 3: back along y (into the stage-1 arrays)
  for (int t = tid; t < count * NP * Q; t += blockDim.x) {
    const int e = t / (NP * Q), rem = t - e * NP * Q;
    const int iy = rem / Q, g = rem - iy * Q;
    const double* f1 = sF1 + e * QQ + g;
    const double* f2 = sF2 + e * QQ + g;
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int gy = 0; gy < Q; ++gy) {
      a = fma(sB[gy * NP + iy], f1[gy * Q], a);
      b = fma(sD[gy * NP + iy], f2[gy * Q], b);
    }
    sA1[t] = a;
    sA2[t] = b;
  }
  __syncthreads();
  // ---- gather: volume stage 4 + side residuals + normal-derivative terms
  const BasisOff bo = A.boff[P];
  double part_dot = 0.0;
  for (int t = tid; t < count * NN; t += blockDim.x) {
    const int e = t / NN, node = t - e * NN;
    const int ix = node % NP, iy = node / NP;
    const int k = A.order[T.first + e];
    const double* c1 = sA1 + e * NP * Q + iy * Q;
    const double* c2v = sA2 + e * NP * Q + iy * Q;
    double y = 0.0;
#pragma unroll
    for (int g = 0; g < Q; ++g) {
      y = fma(sD[g * NP + ix], c1[g], y);
      y = fma(sB[g * NP + ix], c2v[g], y);
    }
    const double* d0 = A.tab + bo.d0;
    const double* d1 = A.tab + bo.d1;
    const double* c2 = sc2 + e * 4 * NP;
    const double* r = sr + e * 4 * NP;
    double gg = -__ldg(d0 + ix) * c2[0 * NP + iy];
    gg = fma(__ldg(d1 + ix), c2[1 * NP + iy], gg);
    gg = fma(-__ldg(d0 + iy), c2[2 * NP + ix], gg);
    gg = fma(__ldg(d1 + iy), c2[3 * NP + ix], gg);
    y = fma(gg, A.aih[k], y);
    if (ix == 0) y += r[0 * NP + iy];
    if (ix == P) y += r[1 * NP + iy];
    if (iy == 0) y += r[2 * NP + ix];
    if (iy == P) y += r[3 * NP + ix];
    A.y[A.off[k] + node] = y;
    part_dot = fma(y, sx[t], part_dot);
  }
  if (A.dot_partial) {
    // tile partial of x . y (summed in tile order when the launch ends)
    const double tot = block_sum<kThreads>(part_dot, red);
    if (tid == 0) A.dot_partial[tile] = tot;
  }
}

}  // namespace dg
