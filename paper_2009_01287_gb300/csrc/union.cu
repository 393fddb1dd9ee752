// Device images of one or many problems ("instances") side by side.
//
// A single solve is the one-instance case.  With several instances (the
// batched solver) every operator is block diagonal: the meshes are concatenated
// (element and DOF numbers shifted, sub-face neighbours and table offsets
// remapped), and the preconditioner's pieces are concatenated per instance.
// The AMG hierarchies of the instances are built independently (each exactly
// as it would be alone) and stacked level by level: at level l the instances
// that continue to level l+1 come first (their rows are smoothed and
// restricted), the instances whose coarsest level is l follow and are solved
// with their own dense inverse.  Each instance therefore sees exactly the
// preconditioner it would have alone.
#include <algorithm>
#include <cstring>

#include "kernels.cuh"
#include "precond_setup.h"
#include "union.h"
#include "work_units.h"

namespace dg {

namespace {

void append_rows(Csr& out, const Csr& in, int64_t col_shift) {
  if (out.ptr.empty()) out.ptr.push_back(0);
  for (int64_t i = 0; i < in.rows; ++i) {
    for (int64_t t = in.ptr[i]; t < in.ptr[i + 1]; ++t) {
      out.idx.push_back((int32_t)(in.idx[t] + col_shift));
      out.val.push_back(in.val[t]);
    }
    out.ptr.push_back((int64_t)out.idx.size());
  }
  out.rows += in.rows;
}

template <typename T>
void upload_csr_t(DevArena& a, const Csr& C, DevCsr& D, cudaStream_t s) {
  DG_REQUIRE(C.nnz() < (1LL << 31), "matrix too large for 32-bit indices");
  std::vector<int32_t> ptr(C.ptr.begin(), C.ptr.end());
  if (ptr.empty()) ptr.push_back(0);
  std::vector<T> val(C.val.begin(), C.val.end());
  D.rows = C.rows;
  D.nnz = C.nnz();
  D.group_all = csr_group_for(C.rows ? (double)C.nnz() / (double)C.rows : 1.0);
  const CsrTierPlan tp = plan_csr_tiers(C);
  D.group = tp.group;
  D.long_min = tp.long_min;
  D.n_cta = (int)tp.cta.size();
  D.n_warp = (int)tp.warp.size();
  if (!tp.cta.empty()) D.cta_rows = a.upload(tp.cta, s);
  if (!tp.warp.empty()) D.warp_rows = a.upload(tp.warp, s);
  D.ptr = a.upload(ptr, s);
  D.idx = a.upload(C.idx, s);
  D.val = a.upload(val, s);
}

}  // namespace

template <typename T>
void upload_union_precond(dg_precond* pc, const std::vector<InstSrc>& inst, cudaStream_t s) {
  DevArena& a = pc->arena;
  const size_t ni = inst.size();
  // ---- AMG level layout
  size_t nlev = 0;
  for (const auto& I : inst) nlev = std::max(nlev, I.A->levels.size());
  DG_REQUIRE(nlev <= 16, "too many AMG levels");
  // row offset of every instance at every level (-1: absent)
  std::vector<std::vector<int64_t>> row_off(nlev, std::vector<int64_t>(ni, -1));
  std::vector<std::vector<size_t>> order(nlev);   // level row order of instances
  std::vector<int64_t> nrows(nlev, 0), ncont(nlev, 0);
  for (size_t l = 0; l < nlev; ++l) {
    for (int pass = 0; pass < 2; ++pass)
      for (size_t i = 0; i < ni; ++i) {
        const size_t L = inst[i].A->levels.size();
        const bool cont = L > l + 1, end = L == l + 1;
        if ((pass == 0 && cont) || (pass == 1 && end)) {
          row_off[l][i] = nrows[l];
          order[l].push_back(i);
          nrows[l] += inst[i].A->levels[l].A.rows;
          if (cont) ncont[l] = nrows[l];
        }
      }
  }
  // ---- DG-level pieces: P (columns = level-0 rows), D_J^-1, V_e blocks
  Csr P;
  std::vector<double> dinv;
  std::vector<int32_t> eb, dofs_off, dims, dofs;
  std::vector<int64_t> inv_off;
  std::vector<T> inv;
  int64_t nb = 0;
  for (size_t i = 0; i < ni; ++i) {
    const HostPrecond& H = *inst[i].H;
    append_rows(P, H.P, nlev ? row_off[0][i] : 0);
    dinv.insert(dinv.end(), H.dinv.begin(), H.dinv.end());
    const size_t base = eb.size();
    eb.resize(base + H.dinv.size(), -1);
    // largest blocks first: the block-solve CTAs take blocks in this order
    std::vector<size_t> border(H.blocks.size());
    for (size_t b = 0; b < border.size(); ++b) border[b] = b;
    std::stable_sort(border.begin(), border.end(),
                     [&](size_t x, size_t y) { return H.blocks[x].size() > H.blocks[y].size(); });
    for (size_t b : border) {
      const auto& blk = H.blocks[b];
      dofs_off.push_back((int32_t)dofs.size());
      dims.push_back((int32_t)blk.size());
      inv_off.push_back((int64_t)inv.size());
      for (size_t j = 0; j < blk.size(); ++j) {
        eb[base + blk[j]] = (int32_t)dofs.size();   // the node's slot in the block results
        dofs.push_back((int32_t)(inst[i].dof_off + blk[j]));
      }
      // stored transposed (column-major) so that the block-solve threads,
      // one per output row, read consecutive addresses at every step
      const size_t d = blk.size(), o = inv.size();
      inv.resize(o + d * d);
      for (size_t r = 0; r < d; ++r)
        for (size_t c = 0; c < d; ++c) inv[o + c * d + r] = (T)H.block_inv[b][r * d + c];
      pc->max_block = std::max<int64_t>(pc->max_block, (int64_t)blk.size());
    }
    nb += (int64_t)H.blocks.size();
  }
  P.cols = nlev ? nrows[0] : 0;
  DG_REQUIRE((int64_t)dinv.size() == pc->n_dofs, "instance sizes do not add up");
  upload_csr_t<T>(a, P, pc->P, s);
  upload_csr_t<T>(a, csr_transpose(P), pc->PT, s);
  pc->dinv = a.upload(std::vector<T>(dinv.begin(), dinv.end()), s);
  pc->e_pos = a.upload(eb, s);
  // block-solve units over all instances, largest blocks first
  std::vector<int32_t> unit, brec;
  std::vector<int64_t> ubase;
  plan_block_units(dims, dofs_off, inv_off, unit, ubase, brec);
  pc->blk_unit = a.upload(unit, s);
  pc->blk_ubase = a.upload(ubase, s);
  pc->blk_rec = a.upload(brec, s);
  pc->blk_dofs = a.upload(dofs, s);
  pc->blk_inv = a.upload(inv, s);
  pc->blk_inv_entries = (int64_t)inv.size();
  pc->blk_slots = (int64_t)dofs.size();
  pc->zE = a.alloc<T>(dofs.size());
  pc->n_blocks = nb;
  pc->n_units = (int64_t)ubase.size();
  pc->n_c = nlev ? nrows[0] : 0;
  // ---- AMG levels
  pc->levels.resize(nlev);
  for (size_t l = 0; l < nlev; ++l) {
    DevLevel& D = pc->levels[l];
    D.n = nrows[l];
    D.n_cont = ncont[l];
    Csr Sb, Sp, Rp;
    std::vector<int32_t> end_row{(int32_t)ncont[l]};
    std::vector<int64_t> end_off;
    std::vector<T> end_inv;
    int64_t nnz_all = 0, nnz_cont = 0;
    for (size_t i : order[l])
      if (row_off[l][i] < ncont[l]) nnz_cont += inst[i].A->levels[l].A.nnz();
    D.plain = nnz_cont > kAmgPlainNnz;
    Csr Ac, Pc, Rc;
    std::vector<T> dinv_c;
    for (size_t i : order[l]) {
      const AmgLevel& L = inst[i].A->levels[l];
      nnz_all += L.A.nnz();
      if (row_off[l][i] < ncont[l]) {
        if (D.plain) {
          append_rows(Ac, L.A, row_off[l][i]);
          append_rows(Pc, L.P, row_off[l + 1][i]);
          for (double d : L.dl1) dinv_c.push_back((T)(1.0 / d));
        } else {
          append_rows(Sb, L.Sb, row_off[l][i]);
          append_rows(Sp, L.Sp, row_off[l + 1][i]);
        }
      } else {
        end_off.push_back((int64_t)end_inv.size());
        end_inv.insert(end_inv.end(), inst[i].A->coarse_inv.begin(), inst[i].A->coarse_inv.end());
        end_row.push_back((int32_t)(row_off[l][i] + L.A.rows));
        D.max_end = std::max<int>(D.max_end, (int)L.A.rows);
      }
    }
    if (l + 1 < nlev)
      for (size_t i : order[l + 1]) {
        if (D.plain) append_rows(Rc, inst[i].A->levels[l].R, row_off[l][i]);
        else append_rows(Rp, inst[i].A->levels[l].Rpre, row_off[l][i]);
      }
    if (D.plain) {
      Ac.cols = ncont[l];
      Pc.cols = (l + 1 < nlev) ? nrows[l + 1] : 0;
      Rc.cols = ncont[l];
      upload_csr_t<T>(a, Ac, D.A, s);
      upload_csr_t<T>(a, Pc, D.P, s);
      upload_csr_t<T>(a, Rc, D.R, s);
      D.dinv = a.upload(dinv_c, s);
      D.t1 = a.alloc<T>(ncont[l]);
      D.t2 = a.alloc<T>(ncont[l]);
    } else {
      Sb.cols = ncont[l];
      Sp.cols = (l + 1 < nlev) ? nrows[l + 1] : 0;
      Rp.cols = ncont[l];
      upload_csr_t<T>(a, Sb, D.Sb, s);
      upload_csr_t<T>(a, Sp, D.Sp, s);
      upload_csr_t<T>(a, Rp, D.Rpre, s);
      // lanes per row of the fused up-sweep: half the power of two below the
      // mean length of both operators' rows together (measured faster), and
      // on a level too small to fill the GPU at that width (rows x lanes under
      // the resident threads of 152 SMs) twice that, up to a warp per row
      int g = std::max(1, csr_group_for(ncont[l] ? (double)(Sb.nnz() + Sp.nnz()) / (double)ncont[l] : 1.0) / 2);
      while (g < 32 && ncont[l] * (int64_t)g < kResidentThreads) g *= 2;
      D.Sb.group_all = g;
    }
    D.n_end = (int)end_off.size();
    D.end_row = a.upload(end_row, s);
    D.end_inv_off = a.upload(end_off, s);
    D.end_inv = a.upload(end_inv, s);
    D.end_inv_entries = (int64_t)end_inv.size();
    D.b = a.alloc<T>(D.n);
    D.xo = a.alloc<T>(D.n);
    pc->stats.level_rows[l] = D.n;
    pc->stats.level_nnz[l] = nnz_all;
    pc->stats.level_plain[l] = D.plain ? 1 : 0;
  }
  pc->stats.n_levels = (int)nlev;
  // coarse fusion: the last composite restriction and the dense coarsest solve
  // as one dense product (one launch fewer per V-cycle), when W is modest
  if (inst.size() == 1 && nlev >= 2) {
    const size_t l = nlev - 2;
    DevLevel& D = pc->levels[l];
    const DevLevel& C = pc->levels[nlev - 1];
    const AmgHierarchy& H = *inst[0].A;
    const Csr& R = H.levels[l].Rpre;   // C.n x D.n
    if (!D.plain && D.n_cont == D.n && C.n_cont == 0 && C.n_end == 1 && R.rows == C.n && R.cols == D.n &&
        (int64_t)H.coarse_inv.size() == C.n * C.n && C.n * D.n <= kCoarseFuseMax) {
      const int64_t m = C.n, n = D.n;
      std::vector<double> W((size_t)(m * n), 0.0);
      for (int64_t i = 0; i < m; ++i) {
        double* wi = W.data() + i * n;
        for (int64_t k = 0; k < m; ++k) {
          const double g = H.coarse_inv[(size_t)(i * m + k)];
          if (g == 0.0) continue;
          for (int64_t t = R.ptr[k]; t < R.ptr[k + 1]; ++t) wi[R.idx[t]] += g * R.val[t];
        }
      }
      D.coarse_w = a.upload(std::vector<T>(W.begin(), W.end()), s);
      D.coarse_w_rows = m;
    }
  }
  DG_CUDA(cudaStreamCreateWithFlags(&pc->side, cudaStreamNonBlocking));
  DG_CUDA(cudaEventCreateWithFlags(&pc->ev_fork, cudaEventDisableTiming));
  DG_CUDA(cudaEventCreateWithFlags(&pc->ev_join, cudaEventDisableTiming));
  pc->rc = a.alloc<T>(pc->n_c);
  pc->ec = a.alloc<T>(pc->n_c);
  DG_CUDA(cudaStreamSynchronize(s));
}

template void upload_union_precond<float>(dg_precond*, const std::vector<InstSrc>&, cudaStream_t);
template void upload_union_precond<double>(dg_precond*, const std::vector<InstSrc>&, cudaStream_t);

}  // namespace dg
