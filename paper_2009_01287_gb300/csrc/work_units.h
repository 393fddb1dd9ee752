// Work lists of the preconditioner's CSR row kernel and block-solve kernel,
// planned on the host from the matrix structure and the V_e block sizes.
#pragma once

#include <cstdint>
#include <vector>

#include "sparse.h"

namespace dg {

// Row tiers of the CSR row kernel for one matrix: rows of more than
// kCsrCtaRow entries take a CTA each, rows of more than long_min entries a
// warp each (both lists longest first, ties in row order), the rest `group`
// lanes each.
struct CsrTierPlan {
  int group = 1;
  int long_min = 0;
  std::vector<int32_t> cta, warp;
};
CsrTierPlan plan_csr_tiers(const Csr& C);

// Work units of the V_e block solves (4 ints per unit), largest blocks first:
// blocks of more than 16 nodes give one unit per 32-row panel,
// {slot of the block's first node, d, first row, 0}, with ubase = the offset
// of the panel's first row in the inverses; blocks of at most W = 4, 8 or 16
// nodes (W the smallest of these that holds d) are packed 32 / W to a unit,
// {index of the first packed block, count, 0, W}, and listed in brec as
// {slot, d, inverse offset low 32 bits, high 32 bits} (ubase = 0).
void plan_block_units(const std::vector<int32_t>& dims, const std::vector<int32_t>& slot,
                      const std::vector<int64_t>& inv_off, std::vector<int32_t>& unit,
                      std::vector<int64_t>& ubase, std::vector<int32_t>& brec);

}  // namespace dg
