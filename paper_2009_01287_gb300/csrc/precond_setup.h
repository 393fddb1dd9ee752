// Host-side preconditioner data before upload.
#pragma once

#include <vector>

#include "dg_internal.h"
#include "sparse.h"

struct dg_mesh;

namespace dg {

struct HostPrecond {
  int64_t nC = 0;
  Csr P;                                 // n_dofs x nC
  Csr Ac;                                // LOR conforming matrix P^T A~ P
  std::vector<int8_t> kind;              // per DG node: 0 interior, 1 J, 2 E
  std::vector<double> dinv;              // 1/A_jj on J, 0 elsewhere
  std::vector<std::vector<int64_t>> blocks;      // V_e node lists (ascending)
  std::vector<std::vector<double>> block_inv;    // dense A_e^-1 (row-major)
};

HostPrecond build_host_precond(const dg_mesh& M, const dg_options& o);
// the same on cube meshes (master-entity construction)
HostPrecond build_host_precond3(const dg_mesh& M, const dg_options& o);

}  // namespace dg
