// Host planning of the work lists of the CSR row kernel and the block-solve
// kernel (see work_units.h).
#include "work_units.h"

#include <algorithm>

#include "host_state.h"

namespace dg {

CsrTierPlan plan_csr_tiers(const Csr& C) {
  CsrTierPlan T;
  // the group width follows the rows of at most 64 entries: half the power of
  // two below their mean (measured faster than the mean itself: each lane
  // keeps about twice as many entries in flight, a warp takes twice the rows)
  double ssum = 0.0;
  int64_t scnt = 0;
  for (int64_t i = 0; i < C.rows; ++i) {
    const int64_t len = C.ptr[i + 1] - C.ptr[i];
    if (len <= 64) ssum += (double)len, ++scnt;
  }
  T.group = std::max(1, csr_group_for(scnt ? ssum / (double)scnt : 64.0) / 2);
  // rows longer than 8 group rounds go to a warp each, rows longer than
  // kCsrCtaRow to a CTA each
  T.long_min = T.group >= 32 ? kCsrCtaRow : std::max(8 * T.group, 16);
  for (int64_t i = 0; i < C.rows; ++i) {
    const int64_t len = C.ptr[i + 1] - C.ptr[i];
    if (len > kCsrCtaRow) T.cta.push_back((int32_t)i);
    else if (len > T.long_min) T.warp.push_back((int32_t)i);
  }
  auto longer = [&](int32_t x, int32_t y) {
    return C.ptr[x + 1] - C.ptr[x] > C.ptr[y + 1] - C.ptr[y];
  };
  std::stable_sort(T.cta.begin(), T.cta.end(), longer);
  std::stable_sort(T.warp.begin(), T.warp.end(), longer);
  return T;
}

void plan_block_units(const std::vector<int32_t>& dims, const std::vector<int32_t>& slot,
                      const std::vector<int64_t>& inv_off, std::vector<int32_t>& unit,
                      std::vector<int64_t>& ubase, std::vector<int32_t>& brec) {
  const int64_t nb = (int64_t)dims.size();
  for (int64_t b = 0; b < nb; ++b)
    DG_REQUIRE(dims[b] >= 1 && dims[b] <= 32 * 256, "a V_e block must have 1 to 8192 nodes");
  std::vector<int64_t> bsort(nb);
  for (int64_t b = 0; b < nb; ++b) bsort[b] = b;
  std::stable_sort(bsort.begin(), bsort.end(), [&](int64_t x, int64_t y) { return dims[x] > dims[y]; });
  unit.clear();
  ubase.clear();
  brec.clear();
  for (int64_t k = 0; k < nb;) {
    const int64_t b = bsort[k];
    const int32_t d = dims[b];
    if (d > 16) {
      for (int32_t r0 = 0; r0 < d; r0 += 32) {
        unit.insert(unit.end(), {slot[b], d, r0, 0});
        ubase.push_back(inv_off[b] + r0);
      }
      ++k;
      continue;
    }
    const int32_t W = d > 8 ? 16 : (d > 4 ? 8 : 4);
    int32_t cnt = 0;
    const int64_t first = (int64_t)brec.size() / 4;
    while (k < nb && cnt < 32 / W && dims[bsort[k]] <= W && (W == 4 || dims[bsort[k]] > W / 2)) {
      const int64_t bb = bsort[k];
      brec.insert(brec.end(), {slot[bb], dims[bb], (int32_t)(uint32_t)(inv_off[bb] & 0xffffffffu),
                               (int32_t)(inv_off[bb] >> 32)});
      ++cnt;
      ++k;
    }
    unit.insert(unit.end(), {(int32_t)first, cnt, 0, W});
    ubase.push_back(0);
  }
}

}  // namespace dg
