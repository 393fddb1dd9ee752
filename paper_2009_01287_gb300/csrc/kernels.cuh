// Launch wrappers of the device kernels.
#pragma once

#include "apply_kernel.cuh"
#include "host_state.h"

namespace dg {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 608;   // 4 x 152 SMs: fixed so reductions are deterministic

void apply_kernel_setup();
ApplyArgs make_apply_args(const dg_mesh& M, const double* x, double* y, double* dot_partial);
void launch_apply(const dg_mesh& M, const double* x, double* y, double* dot_partial, cudaStream_t s);

// z = B r (FP64 or mixed); optional per-CTA partial of r . z
void launch_precond(const dg_precond& pc, const double* r, double* z, double* dot_partial,
                    cudaStream_t s);
int precond_final_blocks(const dg_precond& pc);

// PCG pieces.  Scalars live in `sc` (device): see capi.cu for the layout.
void launch_pcg_init(const double* b, double* x, double* r, int64_t n, double* partial_bb,
                     cudaStream_t s);
void launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s);
void launch_pcg_update_xr(double* x, double* r, const double* p, const double* q, int64_t n,
                          const double* part_pq, int n_pq, double* sc, double* part_rr,
                          cudaStream_t s);
void launch_pcg_update_p(double* p, const double* z, int64_t n, const double* part_rz,
                         int n_rz, double* sc, cudaStream_t s);
void launch_pcg_first(const double* part_rz, int n_rz, const double* part_bb, double* sc,
                      cudaStream_t s);
void launch_pcg_check(const double* part_rr, int n_rr, const double* part_rz, int n_rz,
                      double* sc, int maxit, double rtol2, unsigned long long cond_handle,
                      int use_cond, cudaStream_t s);
enum { SC_RZ = 0, SC_BB = 1, SC_RR = 2, SC_IT = 3, SC_ALPHA = 4, SC_STATUS = 5, SC_COUNT = 8 };

}  // namespace dg
