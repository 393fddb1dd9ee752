/*
 * dg.h - C ABI of the GB300 hp-DG subspace-correction solver.
 *
 * Problem (Section 2, Eq. poisson / fe-problem): -Laplace(u) = f on a box
 * domain with u = 0 on the boundary, or -div(a grad u) = f with a
 * piecewise-constant coefficient a (Section 4.3; dg_mesh_desc.coeff),
 * discretised by the symmetric interior penalty (SIPG) or BR2 (Section 4.4)
 * DG method on a mesh of axis-aligned leaf squares (2D) or cubes (3D) of
 * variable size (hanging nodes, arbitrary irregularity) and variable degree p
 * in 1..8, with the Gauss-Lobatto nodal basis of Section 2.2.  Solved by conjugate gradients (Section 4.1) preconditioned by
 * B = B_B + B_C (Section 3.1, 3.3, 3.4): variational restriction P^T, a
 * low-order-refined (LOR) conforming solve (exact or one AMG V-cycle), the
 * prolongation P, point Jacobi on V_J and exact block solves on the V_e.
 *
 * Conventions shared by every entry point
 *   - Vectors are DEVICE pointers to double, owned by the caller, in the
 *     element-major DG layout: element k (in the order given to
 *     dg_mesh_create) owns (p_k+1)^d consecutive entries; inside an element
 *     the node (ix, iy[, iz]) is entry (iz*(p_k+1) + iy)*(p_k+1) + ix, nodes
 *     at the Gauss-Lobatto points of [0,1] mapped to the element.  Unless a
 *     name ends in _host.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is stream-ordered and returns once its work is enqueued, except where
 *     stated.  A handle is not thread-safe; distinct handles are.
 *   - Handles are allocated and owned by the library; free them with the
 *     matching *_destroy.  Device memory for the handle's state is allocated
 *     by the library (cudaMalloc) at creation time.
 *   - Errors: a non-zero dg_status; dg_last_error() returns a message for the
 *     calling thread.  DG_EINVAL leaves no side effects.
 */
#ifndef DG_H_
#define DG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,        /* invalid argument or mesh                         */
  DG_ENOMEM = 2,        /* host or device allocation failed                 */
  DG_ECUDA = 3,         /* a CUDA call failed                               */
  DG_ENOTCONV = 4,      /* PCG reached maxit; x holds the last iterate      */
  DG_ETIMEOUT = 5,      /* a bounded device-side wait gave up               */
  DG_EUNSUPPORTED = 6   /* valid but not supported by this build            */
} dg_status;

typedef struct dg_mesh dg_mesh;
typedef struct dg_precond dg_precond;

/* Leaf boxes on an integer lattice (Section 2: mesh T, degrees p_kappa).
 * dim is 2 (squares) or 3 (cubes).  lo: n_elems*dim lower corners (lattice
 * units); size: n_elems edge lengths (powers of two); p: n_elems degrees in
 * 1..8; extent: dim domain lengths in lattice units; the physical domain is
 * [0, extent_0*lattice_h] x ... .  The boxes must not overlap; cubes must
 * tile the lattice exactly, while on squares lattice cells that no box covers
 * are holes of the domain (an L-shaped domain, say: the domain is the union of
 * the boxes), whose edges are boundary like the lattice's own; an element
 * side must then border a hole along its whole length or not at all
 * (DG_EINVAL otherwise).
 * coeff: NULL (a = 1) or n_elems values a_kappa > 0 of the piecewise-constant
 * coefficient of -div(a grad u) = f (Section 4.3, random refinement): a_kappa
 * weights element kappa's volume term and its share of the face averages
 * {a grad u}; the SIPG penalty of a sub-face and both sides' BR2 lifting
 * energies take the larger a of its two sides; the LOR blocks are weighted by
 * a_kappa.
 * A value that is not positive and finite is DG_EINVAL.
 * corners: NULL (the boxes themselves), or, squares only, 8 doubles: the
 * physical (x, y) images of the lattice domain's corners (0, 0), (X, 0),
 * (0, Y), (X, Y) (X, Y = extent * lattice_h), in that order.  The boxes are
 * then pre-images: the bilinear map of the domain onto the quadrilateral with
 * these corners carries every leaf box to its element, so T_kappa of
 * Section 2 is that map after the box's own affine map (parallelograms when
 * the corners form one, general convex quadrilaterals otherwise; straight
 * sub-faces, the same hanging structure).  Integrals on such elements use
 * p+2 Gauss points per direction on the volume and max(p-, p+)+2 on a
 * sub-face, the SIPG penalty takes h_kappa = sqrt(area of kappa), the BR2
 * liftings the element's own (mapped) mass matrix, and the LOR blocks are the
 * Q1 stiffness on the mapped Gauss-Lobatto cells.  Corners (or a map) in a
 * batch are DG_EUNSUPPORTED.
 * Corners that do not bound a convex, counter-clockwise quadrilateral (det
 * of the map's Jacobian not positive at a corner) are DG_EINVAL.
 * map, map_ctx: NULL (the boxes, or the corners' bilinear map), or, squares
 * only and with corners NULL, a smooth map of the lattice domain chosen by
 * the caller (curved elements): for n pre-image points X (n x 2, row-major)
 * it writes their images x (n x 2) and the map's Jacobian there, J (n x 4:
 * dx/dX, dx/dY, dy/dX, dy/dY).  The element maps are then T_kappa = map o
 * (box map) and the sub-faces the images of the lattice segments (curved
 * faces, the same hanging structure); the map is evaluated at every
 * quadrature point, Gauss-Lobatto node and load-vector point during
 * dg_mesh_create only, on the calling thread (never afterwards), and the
 * geometric factors are stored.  The same forms, rules and penalty size as
 * for corners.  A map whose Jacobian determinant is not positive, or whose
 * values are not finite, at any of those points is DG_EINVAL.
 * All pointers are HOST pointers, read during the call. */
typedef void (*dg_map_fn)(int64_t n, const double* X, double* x, double* J, void* ctx);
typedef struct {
  int dim;
  int64_t n_elems;
  const int32_t* lo;
  const int32_t* size;
  const int32_t* p;
  const int32_t* extent;
  double lattice_h;
  const double* coeff;
  const double* corners;
  dg_map_fn map;
  void* map_ctx;
} dg_mesh_desc;

enum { DG_FORM_SIPG = 0, DG_FORM_BR2 = 1 };
/* SIPG penalty (Section 2.1): sigma = eta p_e^2 / h_e (PAPER) or
 * eta (p_e+1)^2 / h_e (P1SQ); p_e = max, h_e = min over the two sides. */
enum { DG_PENALTY_PAPER = 0, DG_PENALTY_P1SQ = 1 };
enum { DG_PREC_FP64 = 0, DG_PREC_MIXED = 1 };   /* preconditioner arithmetic */
enum { DG_LOR_EXACT = 0, DG_LOR_AMG = 1 };      /* LOR conforming solve      */
enum { DG_SMOOTHER_FULL = 0, DG_SMOOTHER_JACOBI_ONLY = 1 }; /* B or B~ (4.1) */

typedef struct {
  int form;          /* DG_FORM_*                                           */
  double eta;        /* penalty; <= 0 selects the default (SIPG 100, BR2:
                        the largest number of sub-faces of one element)     */
  int penalty_form;  /* DG_PENALTY_*                                        */
  int precision;     /* DG_PREC_*                                           */
  int lor;           /* DG_LOR_*                                            */
  int smoother;      /* DG_SMOOTHER_*                                       */
  int remark_cases;  /* 1: add the further V_J cases of the remark in
                        Section 3.2 (coarse degree <= every fine degree)    */
  int tune_tiles;    /* 1: dg_mesh_create / dg_batch_create time the
                        operator kernel over candidate tile shapes and keep
                        the fastest (squares: elements per tile of each
                        degree; cubes: the tile's shared-memory budget);
                        the choice is in dg_mesh_stats.  No counterpart in
                        the paper (a launch-shape choice).                  */
} dg_options;

typedef struct {
  int iters;         /* PCG iterations performed                            */
  double rel_res;    /* ||r||_2 / ||b||_2 at exit                           */
  int status;        /* DG_OK or DG_ENOTCONV                                */
  double solve_ms;   /* device time of the iteration loop (CUDA events)     */
} dg_solve_info;

typedef struct {
  int64_t n_dofs;        /* DG unknowns                                     */
  int64_t n_conforming;  /* dim V_C (LOR unknowns)                          */
  int64_t n_j;           /* nodes in V_J                                    */
  int64_t n_e;           /* nodes in the union of the V_e                   */
  int64_t n_blocks;      /* number of V_e                                   */
  int64_t max_block;     /* largest dim V_e                                 */
  int64_t lor_nnz;       /* nonzeros of the LOR conforming matrix           */
  int64_t p_nnz;         /* nonzeros of P                                   */
  int n_levels;          /* AMG levels (1 = exact dense solve)              */
  int64_t level_rows[16];
  int64_t level_nnz[16];
  int level_plain[16];   /* 1: level applied in the plain form (A, R, P),
                            0: composite operators (see dg_precond_setup)   */
  int kernels_per_apply; /* device kernel launches of one dg_precond_apply  */
  int64_t device_bytes;  /* device memory held by the handle: the
                            preconditioner and the PCG workspace of its
                            solves (the mesh's own memory not included)     */
  double apply_bytes;    /* algorithmic bytes of one dg_precond_apply: every
                            matrix entry (value + index), row pointer and
                            vector entry its kernels touch, counted once    */
  double block_bytes;    /* the same for its block solves (the V_e inverses,
                            node lists, gathered residual, results)         */
} dg_precond_stats;

typedef struct {
  int64_t n_elems;
  int64_t n_dofs;
  int64_t n_subfaces;     /* sub-faces counted once per side (interior ones twice) */
  int64_t max_level_gap;  /* largest log2 size ratio across a sub-face            */
  double apply_flops;     /* FP64 flops of one dg_apply as formulated (FMA = 2)  */
  double apply_bytes;     /* algorithmic bytes of one dg_apply: x read, y write,
                             per-element and per-sub-face records read once     */
  int64_t device_bytes;   /* device memory held by the mesh handle              */
  int32_t tile_elems[9];  /* squares: elements per operator tile of degree p
                             (index p), fixed rule min(16, 256/(p+1)^2) unless
                             tuned                                               */
  int64_t tile_smem_budget; /* cubes: shared-memory budget of an operator tile
                               (bytes)                                           */
  int32_t tiles_tuned;    /* 1: chosen by timing (dg_options.tune_tiles)        */
  double apply_ms_fixed;  /* when tuned: the operator kernel's time with the
                             fixed rule ...                                      */
  double apply_ms_tuned;  /* ... and with the chosen tiles (CUDA events around
                             a graph of 20 launches, as a solve runs them,
                             warm, best of 3, per launch)                       */
} dg_mesh_stats;

/* Build the mesh topology (sub-faces, hanging vertices, master edges) and
 * upload the operator data.  Section 2 (mesh, DG space) and 2.1 (sigma).
 * opts: only form, eta and penalty_form are used here.  stream: for uploads. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, const dg_options* opts,
                         void* stream, dg_mesh** out);
void dg_mesh_destroy(dg_mesh* mesh);
int64_t dg_num_dofs(const dg_mesh* mesh);
dg_status dg_mesh_stats_get(const dg_mesh* mesh, dg_mesh_stats* out);
/* DOF layout (Section 2: V_h is the direct sum of the Q_{p_k} spaces of the
 * elements): elem_offsets (HOST, n_elems + 1 entries) receives the offset of
 * each element's first entry in a DG vector, in the element order given to
 * dg_mesh_create; elem_offsets[n_elems] = n_dofs.  Inside an element the
 * entries follow the node order stated at the top of this header. */
dg_status dg_dof_layout(const dg_mesh* mesh, int64_t* elem_offsets);

/* y = A x, the matrix-free DG operator of Eq. fe-problem (SIPG) or of the
 * BR2 form (Section 4.4), FP64.  x and y: device, n_dofs doubles, must not
 * overlap. */
dg_status dg_apply(const dg_mesh* mesh, const double* x, double* y, void* stream);

/* Set up B = B_B + B_C (Sections 3.3, 3.4, 4.1): V_J / V_e classification,
 * the V_e generation (connected components by jump overlap; on cube meshes the
 * E nodes of each master entity), dense block inverses, diag(A) on V_J, P,
 * the LOR matrix P^T A~ P and its solver.  An AMG level is applied either
 * through composite operators (two kernels) or, when its matrix is large, in
 * the plain form (four kernels, about half the bytes); both are the same
 * V-cycle.  Host work, then uploads; synchronous. */
dg_status dg_precond_setup(const dg_mesh* mesh, const dg_options* opts, dg_precond** out);
/* (dg_precond_setup also creates the workspace and the captured graph of the
 * PCG solves with this handle, so that dg_pcg_solve allocates nothing.) */
void dg_precond_destroy(dg_precond* pc);
dg_status dg_precond_stats_get(const dg_precond* pc, dg_precond_stats* out);

/* z = B r (Section 4.1).  r, z: device, n_dofs doubles, must not overlap. */
dg_status dg_precond_apply(const dg_precond* pc, const double* r, double* z, void* stream);

/* ---- Profiling (CUDA events; stream-ordered, synchronous on `stream`).
 * dg_precond_profile runs one z = B r with its parts one after another on
 * `stream` (the block solves first, alone, instead of beside the V-cycle) and
 * returns the time of each part: the block solves on the V_e (Section 3.3),
 * the restriction P^T r, the LOR solve (Section 3.4), and the final
 * combination z = P e_C + D_J^-1 r + block results.  z is the same as from
 * dg_precond_apply.  dg_apply_profile times the two kernels of one y = A x:
 * the side traces of x, then the operator kernel. */
typedef struct {
  double blocks_ms, restrict_ms, lor_ms, final_ms, total_ms;
} dg_precond_times;
dg_status dg_precond_profile(const dg_precond* pc, const double* r, double* z, dg_precond_times* out,
                             void* stream);
typedef struct {
  double trace_ms, apply_ms;
} dg_apply_times;
dg_status dg_apply_profile(const dg_mesh* mesh, const double* x, double* y, dg_apply_times* out,
                           void* stream);
/* FP64 FMA throughput of the current device: 8 independent FMA chains per
 * thread, 8 CTAs of 256 threads per SM, `iters` steps each, timed with CUDA
 * events after one shorter warm-up launch.  The operator kernels are bound by
 * FP64 arithmetic, so this is the peak their roofline is reported against.
 * No counterpart in the paper (a measurement aid).  Synchronous. */
dg_status dg_fp64_fma_probe(int64_t iters, double* tflops, double* ms, void* stream);

/* PCG (Section 4.1) from x0 = 0 until ||r||_2 <= rtol ||b||_2 or maxit.
 * b, x: device, n_dofs doubles; x receives the solution (the last iterate on
 * DG_ENOTCONV).  A solve is one CUDA graph launch: the start (x = 0, r = b,
 * z = B r, p = z) and a device-side while loop of PCG iterations, captured
 * once per preconditioner on the handle's own copies of b and x (copied in
 * and out inside the call) with rtol and maxit read from device memory, so
 * any b, x, rtol and maxit reuse it.  The call waits for the solve
 * (synchronous on `stream`); info->solve_ms is the CUDA-event time of
 * everything the solve enqueues, from the copy of b to the copy of x, with no
 * host round trip inside. */
dg_status dg_pcg_solve(const dg_mesh* mesh, const dg_precond* pc, const double* b,
                       double* x, double rtol, int maxit, dg_solve_info* info,
                       void* stream);

/* The same solve with HOST b and x (copied in and out by the call). */
dg_status dg_pcg_solve_host(const dg_mesh* mesh, const dg_precond* pc, const double* b_host,
                            double* x_host, double rtol, int maxit, dg_solve_info* info,
                            void* stream);

/* The same PCG solve as dg_pcg_solve, but one that allocates nothing: the
 * paper has no counterpart; this is an interface for callers that must not
 * have the library allocate device or pinned memory, or build CUDA graphs,
 * while they solve.  Examples: a service that reserves all device memory at
 * start-up and forbids cudaMalloc/cudaFree afterwards (they can synchronise
 * the whole device and stall other streams), or a caller that runs the solve
 * from a context where new allocations would fail its memory budget.
 * dg_pcg_solve allocates its work vectors, a graph and pinned memory on its
 * first call per preconditioner; this entry point instead takes its work
 * vectors (r, z, p, q and the reduction partials) from one fixed array in
 * device memory that every GPU which loads the library holds until exit
 * (about 8.1 MiB), and iterates from a host loop.  The caller still passes b
 * and x (device, n_dofs doubles) and the handles (made beforehand by
 * dg_mesh_create / dg_precond_setup, which do allocate).
 *   - n_dofs is limited to 262144; larger meshes get DG_EINVAL and a message.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before starting any stream capture.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and give wrong results.  Each
 *     call overwrites every part of the array it reads, so nothing has to be
 *     cleared between calls.
 *   - info->solve_ms is host wall time of the call's iteration loop.
 * Synchronous on `stream`. */
dg_status dg_pcg_solve_noalloc(const dg_mesh* mesh, const dg_precond* pc, const double* b,
                               double* x, double rtol, int maxit, dg_solve_info* info,
                               void* stream);

/* b_i = int f phi_i for f(x) = sum_m amps[m] prod_d sin(pi waves[m*dim+d] x_d)
 * ((p+3)-point Gauss rule per direction); b: device.  Host arithmetic. */
dg_status dg_rhs_sine(const dg_mesh* mesh, int n_modes, const double* amps,
                      const int32_t* waves, double* b, void* stream);

/* Load vector of caller-supplied data (Section 2, Eq. fe-problem, right-hand
 * side; the adaptive-refinement problems of Section 4.2 have inhomogeneous
 * Dirichlet data): b_i = int f phi_i, plus, when g is given, the terms of the
 * boundary condition u = g imposed weakly by SIPG,
 *   sum over boundary sub-faces of int g (sigma phi_i - a grad phi_i . n) ds.
 * f and g are host callbacks (dg_field_fn: n physical points x, n x 2
 * row-major, into out, n values), called on the calling thread during the
 * call; either may be NULL (no volume term / homogeneous data).  Quadrature:
 * p+3 Gauss points per direction on the volume and on each boundary
 * sub-face, at physical points (on mapped meshes the points, weights and
 * normals were stored by dg_mesh_create, so the map is not called again).
 * Square meshes, mapped or not; g needs the SIPG form (otherwise, and on
 * cube meshes, DG_EUNSUPPORTED).  A non-finite value from a callback is
 * DG_EINVAL.  b: device; host arithmetic, synchronous on `stream`. */
typedef void (*dg_field_fn)(int64_t n, const double* x, double* out, void* ctx);
dg_status dg_rhs_eval(const dg_mesh* mesh, dg_field_fn f, dg_field_fn g, void* ctx, double* b,
                      void* stream);

/* ---- Batched solver: many problems x several right-hand sides, one launch.
 * Each (problem k, right-hand side r) pair is an instance, numbered
 * k*n_rhs + r; the batch's vectors hold all instances one after another
 * (offsets from dg_batch_offsets).  The problems are independent: the batch
 * is one block-diagonal system whose PCG keeps alpha, beta and the stopping
 * test per instance (Section 4.1's PCG for every instance), so every
 * instance follows the iteration it would follow alone.  opts: form, eta,
 * penalty_form, precision, smoother and remark_cases apply to every problem;
 * the LOR solve is one AMG V-cycle; BR2 needs an explicit eta.  The host
 * setup of the problems runs on all host threads. */
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(const dg_mesh_desc* descs, int n_problems, int n_rhs,
                          const dg_options* opts, void* stream, dg_batch** out);
void dg_batch_destroy(dg_batch* batch);
int64_t dg_batch_num_dofs(const dg_batch* batch);
/* offsets: n_problems*n_rhs + 1 entries (host). */
dg_status dg_batch_offsets(const dg_batch* batch, int64_t* offsets);
/* Statistics of the batch's concatenated operator (all instances), with its
 * tile shapes (tuned when opts->tune_tiles was set at creation). */
dg_status dg_batch_stats_get(const dg_batch* batch, dg_mesh_stats* out);
/* Sine right-hand sides for every instance (as dg_rhs_sine): amps holds
 * n_modes values per instance, waves 2*n_modes per instance; b: device. */
dg_status dg_batch_rhs_sine(const dg_batch* batch, int n_modes, const double* amps,
                            const int32_t* waves, double* b, void* stream);
/* Solve all instances from x0 = 0 to ||r_i|| <= rtol ||b_i|| (or maxit each).
 * b, x: device, dg_batch_num_dofs doubles.  results: host array of
 * n_problems*n_rhs entries (iters, rel_res, status per instance);
 * solve_ms: device time of the whole batch.  One CUDA graph with a device
 * while loop that runs until every instance has stopped; synchronous.
 * Returns DG_ENOTCONV if any instance reached maxit. */
dg_status dg_batch_solve(dg_batch* batch, const double* b, double* x, double rtol, int maxit,
                         dg_solve_info* results, double* solve_ms, void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H_ */
