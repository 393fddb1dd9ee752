// Launch wrappers of the device kernels.
#pragma once

#include "apply_kernel.cuh"
#include "apply3_kernel.cuh"
#include "host_state.h"

namespace dg {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 1216;   // 8 x 152 SMs: fixed so reductions are deterministic

// resident CTAs of the persistent operator kernel of this mesh (sets the
// kernel's shared-memory opt-in on the current device)
int apply_kernel_setup(const dg_mesh& M);
// dynamic shared memory of the operator kernel of this mesh (bytes)
int64_t apply_smem_for(const dg_mesh& M);

ApplyArgs make_apply_args(const dg_mesh& M, const double* x, double* y, Reduce red);
// y = A x; with_trace = false when the side traces of x are already in place
// (written by launch_pcg_p_trace).  pcg_sc (PCG scalars, needs red): the
// launch's last CTA also sets sc[SC_ALPHA] = sc[SC_RZ] / (x . y), or 0 once
// sc[SC_STATUS] is set.
void launch_apply(const dg_mesh& M, const double* x, double* y, Reduce red, cudaStream_t s,
                  bool with_trace = true, double* pcg_sc = nullptr);
// the side traces of x alone (the first of the two kernels of launch_apply)
void launch_trace(const dg_mesh& M, const double* x, cudaStream_t s);

// PCG scalar slots (doubles) and reduction tickets
enum {
  SC_RZ = 0, SC_BB = 1, SC_RR = 2, SC_IT = 3, SC_ALPHA = 4, SC_STATUS = 5,
  SC_PQ = 6, SC_RZNEW = 7, SC_RRNEW = 8,
  SC_MAXIT = 9, SC_RTOL2 = 10,   // iteration limit and tol^2, read when the launch passes maxit < 0
  SC_BETA = 11,                  // beta of the p update, set with the convergence test
  SC_COUNT = 16
};

// PCG iteration control run by the last CTA of the preconditioner's final
// kernel once r . z and r . r are summed: beta = (r.z)_new / (r.z)_old, the
// convergence test ||r|| <= tol ||b|| or the iteration limit, the iteration
// count and the graph's while condition.  sc null: no control.
struct PcgCtl {
  double* sc = nullptr;
  int maxit = 0;                    // < 0: limit and tol^2 from sc[SC_MAXIT], sc[SC_RTOL2]
  double rtol2 = 0.0;
  unsigned long long cond = 0;      // cudaGraphConditionalHandle
  int use_cond = 0;
};
// Events recorded between the parts of a preconditioner apply: ev[0] start,
// ev[1] after the block solves, ev[2] after the restriction, ev[3] after the
// LOR solve, ev[4] after the final combination.  With marks the block solves
// run on the calling stream before the other parts (serial, for timing).
struct PrecondMarks {
  cudaEvent_t ev[5];
};
// The PCG update of this iteration, deferred into the preconditioner: its
// kernels read the residual as r - alpha q (formed on the fly, the same FMA
// everywhere), and the final kernel, which runs after every other reader of
// r, stores it to r_out (the vector r itself) and sets x += alpha p.  alpha is
// the device scalar written by the operator launch (launch_apply with pcg_sc).
// q null: r as given.
struct XrDefer {
  double* r_out = nullptr;
  double* x = nullptr;
  const double* p = nullptr;
  const double* q = nullptr;
  const double* alpha = nullptr;
};
// z = B r (FP64 or mixed); optional reduction of r . z
// (with rr: the r . r reduction as well, in the final kernel; needs red; with
// ctl.sc also the iteration control, see PcgCtl; with xr.q the residual is
// r - alpha q and is written back, see XrDefer)
void launch_precond(const dg_precond& pc, const double* r, double* z, Reduce red, cudaStream_t s,
                    const PrecondMarks* marks = nullptr, Reduce rr = Reduce{}, PcgCtl ctl = PcgCtl{},
                    XrDefer xr = XrDefer{});
// algorithmic bytes of one preconditioner apply (every matrix entry and vector
// the kernels touch, read or written once) and of its block-solve kernel
void precond_algorithmic_bytes(const dg_precond& pc, double* total, double* blocks);
int precond_final_blocks(const dg_precond& pc);
// device kernel launches of one preconditioner apply
int precond_kernel_count(const dg_precond& pc);

enum { TK_PQ = 0, TK_RR = 1, TK_RZ = 2, TK_P = 3, TK_BB = 4, TK_COUNT = 8 };

void launch_pcg_init(const double* b, double* x, double* r, int64_t n, Reduce bb, cudaStream_t s);
// p = z + beta p (first: p = z and the initial scalars) tile by tile, writing
// the side traces of the new p for the next operator apply.  beta comes from
// sc[SC_BETA], set with the convergence test by the preconditioner's final
// kernel (PcgCtl); after a stop the kernel does nothing.  First: the initial
// scalars and, with use_cond, the loop condition b . b > 0.
void launch_pcg_p_trace(const dg_mesh& M, double* p, const double* z, double* sc,
                        unsigned long long cond_handle, int use_cond, int first, cudaStream_t s);

}  // namespace dg
