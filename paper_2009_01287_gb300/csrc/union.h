// Building the device image of one or many problems side by side.
#pragma once

#include <vector>

#include "host_state.h"
#include "precond_setup.h"
#include "sparse.h"

namespace dg {

// One instance of the union: host preconditioner data, its AMG hierarchy and
// where its DOFs start in the union vectors.
struct InstSrc {
  const HostPrecond* H;
  const AmgHierarchy* A;
  int64_t dof_off;
};

// Upload the union preconditioner (AMG LOR solver) into pc; pc->n_dofs and
// pc->precision must be set.
template <typename T>
void upload_union_precond(dg_precond* pc, const std::vector<InstSrc>& inst, cudaStream_t s);

}  // namespace dg
