// Matrix-free SIPG / BR2 operator y = A x on cube meshes (the method of
// Section 2 on hexahedra; BR2 stabilisation of Section 4.4), FP64.
//
// The same two kernels as on squares:
//  trace3  for every element side, the value u and outward normal derivative
//          dn at its (p+1)^2 side nodes (one contraction along the normal);
//  apply3  one CTA per tile of elements of one degree P:
//    volume  y = h (K x M x M + M x K x M + M x M x K) x, sum factorised in
//            three passes through shared memory (7 (p+1)^4 FMAs per element):
//              along z: A = M x, B = K x;  along y: C = M A, D = K A + M B;
//              along x: y = h (K C + M D);
//    faces   the tile's sub-faces are a flat list of (record, side) items,
//            taken in chunks that fit shared memory.  A sub-face is a square
//            whose face-mass matrices are Kronecker products of 1D tables (first
//            tangential axis a, second b), so every face product is two 1D
//            contractions, one pass over all items of the chunk each, with a
//            barrier between them (a chunk's items sorted by the branches they
//            take, so that warps split less); a third pass adds each item's
//            partials to its side nodes in sub-face order (deterministic):
//              a = M_oo u-, c = M_oo dn-, b = M_on u+, d = M_on dn+
//            and, for SIPG, side residual += area (sigma (a - b) - (c - d) / 2)
//            and normal-derivative coefficient c2 -= area (a - b) / 2
//            (boundary: area (sigma a - c) and -area a).  For BR2 the sigma term
//            becomes eta/4 area [M_oo G_o jo + M_on G_n jn] with the jump
//            projections jo = area (a - b), jn = area (M_no u- - M_nn u+) and
//            G = h^-3 Minv_00 (Minv x Minv), the side block of the element mass
//            inverse (boundary: eta area M_oo G_o jo).  Multiplied out per axis
//            it is cz [(Z x Z) u- - (V x V) u+] + cx [(X x X) u- - (Y x Y) u+]
//            with the 1D products Z = M_oo Minv M_oo, V = M_oo Minv M_on,
//            X = M_on Minv_n M_no, Y = M_on Minv_n M_nn and the scalars
//            cz, cx = eta/4 area^2 Minv_00 / h^3 of the two elements, so BR2
//            takes the same two passes as SIPG.  On a sub-face that is the
//            whole own face Z = M_oo and V = M_on (M_oo is then the 1D mass
//            matrix), on the whole neighbour face Y = M_on: those products are
//            taken from a and b, their loops skipped as a whole;
//    gather  volume pass along x, side residuals and the normal-derivative
//            terms c2 (x) dn(v) of all six sides.
// Each sub-face is evaluated from both of its sides (no atomics): applies are
// bit-reproducible.
#pragma once

#include "apply_kernel.cuh"

namespace dg {

// volume index of side node (i, j) at normal index q on side s
template <int NP>
__device__ __forceinline__ int side_node3(int s, int i, int j, int q) {
  const int ax = s >> 1;
  return ax == 0 ? q + NP * (i + NP * j) : (ax == 1 ? i + NP * (q + NP * j) : i + NP * (j + NP * q));
}

template <int P, bool RO = true>
__device__ __forceinline__ void trace3_tile(const ApplyArgs& A, const ApplyTile& T) {
  constexpr int NP = P + 1, N2 = NP * NP;
  const BasisOff bo = A.boff[P];
  const int ntask = T.count * 6 * N2;
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    const int e = t / (6 * N2);
    const int rem = t - e * 6 * N2;
    const int s = rem / N2;
    const int ij = rem - s * N2;
    const int i = ij % NP, j = ij / NP;
    const int k = A.order[T.first + e];
    const double* xk = A.x + A.off[k];
    const double* dv = A.tab + ((s & 1) ? bo.d1 : bo.d0);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) acc = fma(__ldg(dv + q), ld_x<RO>(xk + side_node3<NP>(s, i, j, q)), acc);
    const double sg = (s & 1) ? A.aih[k] : -A.aih[k];   // a grad u . n
    double2 v;
    v.x = ld_x<RO>(xk + side_node3<NP>(s, i, j, (s & 1) ? P : 0));
    v.y = sg * acc;
    reinterpret_cast<double2*>(A.tr + A.toff[k])[s * N2 + ij] = v;
  }
}

template <int P, bool BR2>
__device__ __forceinline__ void apply3_tile(const ApplyArgs& A, const ApplyTile& T, int tile,
                                            double* sm, double* red) {
  constexpr int NP = P + 1, N2 = NP * NP, N3 = N2 * NP;
  constexpr int S = BR2 ? 8 : 4;          // first-pass products per sub-face item
  const int cnt = T.count, NQ = T.nq, WQ = NP * NQ;
  double* sM = sm;
  double* sK = sM + N2;
  double* sx = sK + N2;
  double* sA = sx + cnt * N3;
  double* sB = sA + cnt * N3;
  double* sC = sB + cnt * N3;
  double* sD = sC + cnt * N3;
  double* sr = sD + cnt * N3;             // [cnt][6][N2] side residuals
  double* sc2 = sr + cnt * 6 * N2;        // [cnt][6][N2] normal-derivative coefficients
  double* sw = sc2 + cnt * 6 * N2;        // [chunk][S][NP x NQ] first-pass scratch
  double* sp = sw + T.chunk * S * WQ;     // [chunk][2][N2] item partials (residual, c2)

  const int tid = threadIdx.x;
  if (A.skip && A.skip[(int64_t)T.inst * A.skip_stride] != 0.0) {   // CTA-uniform
    if (A.dot_partial && tid == 0) A.dot_partial[tile] = 0.0;
    return;
  }
  const BasisOff bo = A.boff[P];
  const int nvol = cnt * N3;
  for (int i = tid; i < N2; i += blockDim.x) {
    sM[i] = __ldg(A.tab + bo.M + i);
    sK[i] = __ldg(A.tab + bo.K + i);
  }
  for (int t = tid; t < nvol; t += blockDim.x) {
    const int e = t / N3;
    sx[t] = A.x[A.off[A.order[T.first + e]] + (t - e * N3)];
  }
  for (int t = tid; t < cnt * 6 * N2; t += blockDim.x) {
    sr[t] = 0.0;
    sc2[t] = 0.0;
  }
  __syncthreads();
  // ---- volume pass along z
  for (int t = tid; t < nvol; t += blockDim.x) {
    const int e = t / N3, node = t - e * N3;
    const int ixy = node % N2, iz = node / N2;
    const double* xc = sx + e * N3 + ixy;
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const double v = xc[q * N2];
      a = fma(sM[iz * NP + q], v, a);
      b = fma(sK[iz * NP + q], v, b);
    }
    sA[t] = a;
    sB[t] = b;
  }
  __syncthreads();
  // ---- volume pass along y
  for (int t = tid; t < nvol; t += blockDim.x) {
    const int e = t / N3, node = t - e * N3;
    const int ix = node % NP, iy = (node / NP) % NP, iz = node / N2;
    const double* ac = sA + e * N3 + iz * N2 + ix;
    const double* bc = sB + e * N3 + iz * N2 + ix;
    double c = 0.0, d = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const double m = sM[iy * NP + q], kk = sK[iy * NP + q];
      c = fma(m, ac[q * NP], c);
      d = fma(kk, ac[q * NP], d);
      d = fma(m, bc[q * NP], d);
    }
    sC[t] = c;
    sD[t] = d;
  }
  // ---- faces: the tile's sub-face items in chunks; per chunk two passes
  // (one per tangential axis) over all items at once, then every side node
  // adds its items' partials in sub-face order
  const double* tab = A.tab;
  const int ib = A.item_ptr[tile];
  const int nit = A.item_ptr[tile + 1] - ib;
  for (int c0 = 0; c0 < nit; c0 += T.chunk) {
    const int nc = min(T.chunk, nit - c0);
    // P1: contractions along the first tangential axis
    for (int t = tid; t < nc * WQ; t += blockDim.x) {
      const int it = t / WQ, q = t - it * WQ;
      const int i = q % NP, n = q / NP;
      const int2 item = A.items[ib + c0 + it];   // chunk-sorted (see the tile build)
      const SubFaceRec3& f = A.sf3[item.x];
      const int es = item.y & 0xffff, e = es / 6, s = es - e * 6;
      const int k = A.order[T.first + e];
      const int np = f.pn + 1;
      const bool in = f.nb >= 0;
      double* W = sw + it * S * WQ;
      // on a whole own face Z = M_oo, V = M_on; on a whole neighbour face Y = M_on:
      // those products are not formed (their loops skipped as a whole)
      const bool zv = BR2 && !(f.full & 1), yy_ = BR2 && !(f.full & 2);
      if (n < NP) {
        const double2* trk = reinterpret_cast<const double2*>(A.tr + A.toff[k]) + s * N2;
        const double* Ma = tab + f.tab_oo[0] + i * NP;
        double wa = 0.0, wc = 0.0, wx = 0.0;
        if (BR2 && in) {
          const double* Xa = tab + f.tab_x[0] + i * NP;
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            const double2 v = trk[n * NP + m];
            const double w = __ldg(Ma + m);
            wa = fma(w, v.x, wa);
            wc = fma(w, v.y, wc);
            wx = fma(__ldg(Xa + m), v.x, wx);
          }
        } else {
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            const double2 v = trk[n * NP + m];
            const double w = __ldg(Ma + m);
            wa = fma(w, v.x, wa);
            wc = fma(w, v.y, wc);
          }
        }
        W[0 * WQ + i * NQ + n] = wa;
        W[1 * WQ + i * NQ + n] = wc;
        if (BR2) W[5 * WQ + i * NQ + n] = wx;
        if (zv) {
          const double* Za = tab + f.tab_z[0] + i * NP;
          double wz = 0.0;
#pragma unroll
          for (int m = 0; m < NP; ++m) wz = fma(__ldg(Za + m), trk[n * NP + m].x, wz);
          W[4 * WQ + i * NQ + n] = wz;
        }
      }
      if (in && n < np) {
        const double2* trn = reinterpret_cast<const double2*>(A.tr + A.toff[f.nb]) + f.nb_side * np * np;
        const double* Ma = tab + f.tab_on[0] + i * np;
        double wb = 0.0, wd = 0.0;
        for (int m = 0; m < np; ++m) {
          const double2 v = trn[n * np + m];
          const double w = __ldg(Ma + m);
          wb = fma(w, v.x, wb);
          wd = fma(w, v.y, wd);
        }
        W[2 * WQ + i * NQ + n] = wb;
        W[3 * WQ + i * NQ + n] = wd;
        if (zv) {
          const double* Va = tab + f.tab_v[0] + i * np;
          double wv = 0.0;
          for (int m = 0; m < np; ++m) wv = fma(__ldg(Va + m), trn[n * np + m].x, wv);
          W[6 * WQ + i * NQ + n] = wv;
        }
        if (yy_) {
          const double* Ya = tab + f.tab_y[0] + i * np;
          double wy = 0.0;
          for (int m = 0; m < np; ++m) wy = fma(__ldg(Ya + m), trn[n * np + m].x, wy);
          W[7 * WQ + i * NQ + n] = wy;
        }
      }
    }
    __syncthreads();
    // P2: contractions along the second tangential axis: the item's partials
    for (int t = tid; t < nc * N2; t += blockDim.x) {
      const int it = t / N2, q = t - it * N2;
      const int i = q % NP, jj = q / NP;
      const int2 item = A.items[ib + c0 + it];
      const SubFaceRec3& f = A.sf3[item.x];
      const int np = f.pn + 1;
      const bool in = f.nb >= 0;
      const double* W = sw + it * S * WQ;
      const double ar = f.area;
      const double* Mb = tab + f.tab_oo[1] + jj * NP;
      const bool zv = BR2 && !(f.full & 1), yy_ = BR2 && !(f.full & 2);
      double a = 0.0, c = 0.0, b = 0.0, d = 0.0, zz = 0.0, xx = 0.0, vv = 0.0, yy = 0.0;
      if (BR2 && in) {
        const double* Xb = tab + f.tab_x[1] + jj * NP;
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          const double w = __ldg(Mb + n);
          a = fma(w, W[0 * WQ + i * NQ + n], a);
          c = fma(w, W[1 * WQ + i * NQ + n], c);
          xx = fma(__ldg(Xb + n), W[5 * WQ + i * NQ + n], xx);
        }
      } else {
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          const double w = __ldg(Mb + n);
          a = fma(w, W[0 * WQ + i * NQ + n], a);
          c = fma(w, W[1 * WQ + i * NQ + n], c);
        }
      }
      if (zv) {
        const double* Zb = tab + f.tab_z[1] + jj * NP;
#pragma unroll
        for (int n = 0; n < NP; ++n) zz = fma(__ldg(Zb + n), W[4 * WQ + i * NQ + n], zz);
      }
      if (in) {
        const double* Mbn = tab + f.tab_on[1] + jj * np;
        for (int n = 0; n < np; ++n) {
          const double w = __ldg(Mbn + n);
          b = fma(w, W[2 * WQ + i * NQ + n], b);
          d = fma(w, W[3 * WQ + i * NQ + n], d);
        }
        if (zv) {
          const double* Vb = tab + f.tab_v[1] + jj * np;
          for (int n = 0; n < np; ++n) vv = fma(__ldg(Vb + n), W[6 * WQ + i * NQ + n], vv);
        }
        if (yy_) {
          const double* Yb = tab + f.tab_y[1] + jj * np;
          for (int n = 0; n < np; ++n) yy = fma(__ldg(Yb + n), W[7 * WQ + i * NQ + n], yy);
        }
      }
      if (BR2 && !zv) {   // whole own face: Z = M_oo, V = M_on
        zz = a;
        vv = b;
      }
      if (BR2 && !yy_) yy = b;   // whole neighbour face: Y = M_on
      const double jmp = a - b;
      double rr, cc;
      if (in) {
        rr = -0.5 * ar * (c - d);
        cc = -0.5 * ar * jmp;
      } else {
        rr = -ar * c;
        cc = -ar * a;
      }
      if (BR2) rr += f.cz * (zz - vv) + f.cx * (xx - yy);
      else rr = fma(f.sigma * ar, jmp, rr);
      const int pos = item.y >> 16;   // the item's position in sub-face order
      sp[pos * 2 * N2 + q] = rr;
      sp[pos * 2 * N2 + N2 + q] = cc;
    }
    __syncthreads();
    // P3: every side node adds the partials of its items in this chunk, in order
    for (int t = tid; t < cnt * 6 * N2; t += blockDim.x) {
      const int es = t / N2, q = t - es * N2;
      const int e = es / 6, s = es - e * 6;
      const int2 si = A.side_items[(int64_t)(T.first + e) * 6 + s];
      const int lo = max(si.x - ib, c0), hi = min(si.x - ib + si.y, c0 + nc);
      double rr = 0.0, cc = 0.0;
      for (int g = lo; g < hi; ++g) {
        rr += sp[(g - c0) * 2 * N2 + q];
        cc += sp[(g - c0) * 2 * N2 + N2 + q];
      }
      if (hi > lo) {
        sr[t] += rr;
        sc2[t] += cc;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // ---- gather: pass along x, side residuals, normal-derivative terms
  double part = 0.0;
  const double* d0 = A.tab + bo.d0;
  const double* d1 = A.tab + bo.d1;
  for (int t = tid; t < nvol; t += blockDim.x) {
    const int e = t / N3, node = t - e * N3;
    const int ix = node % NP, iy = (node / NP) % NP, iz = node / N2;
    const int k = A.order[T.first + e];
    const double* cr = sC + e * N3 + iz * N2 + iy * NP;
    const double* dr = sD + e * N3 + iz * N2 + iy * NP;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      v = fma(sK[ix * NP + q], cr[q], v);
      v = fma(sM[ix * NP + q], dr[q], v);
    }
    double y = A.ahk[k] * v;
    const double* c2 = sc2 + e * 6 * N2;
    const double* r = sr + e * 6 * N2;
    double g = -__ldg(d0 + ix) * c2[0 * N2 + iz * NP + iy];
    g = fma(__ldg(d1 + ix), c2[1 * N2 + iz * NP + iy], g);
    g = fma(-__ldg(d0 + iy), c2[2 * N2 + iz * NP + ix], g);
    g = fma(__ldg(d1 + iy), c2[3 * N2 + iz * NP + ix], g);
    g = fma(-__ldg(d0 + iz), c2[4 * N2 + iy * NP + ix], g);
    g = fma(__ldg(d1 + iz), c2[5 * N2 + iy * NP + ix], g);
    y = fma(g, A.aih[k], y);
    if (ix == 0) y += r[0 * N2 + iz * NP + iy];
    if (ix == P) y += r[1 * N2 + iz * NP + iy];
    if (iy == 0) y += r[2 * N2 + iz * NP + ix];
    if (iy == P) y += r[3 * N2 + iz * NP + ix];
    if (iz == 0) y += r[4 * N2 + iy * NP + ix];
    if (iz == P) y += r[5 * N2 + iy * NP + ix];
    A.y[A.off[k] + node] = y;
    part = fma(y, sx[t], part);
  }
  if (A.dot_partial) {
    const double tot = block_sum<kThreads>(part, red);
    if (tid == 0) A.dot_partial[tile] = tot;
  }
}

}  // namespace dg
