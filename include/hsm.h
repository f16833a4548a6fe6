/*
 * hsm.h -- C ABI of libhsm, the GB300 (sm_103a) implementation of the hybrid
 * scattered-regular meshless operators of Jancic, Rot and Kosec,
 * "Spatially-varying meshless approximation method for enhanced computational
 * efficiency" (arXiv:2303.01760).
 *
 * The library takes a node set with a regular/scattered flag per node
 * (Section 2: regular nodes fill the domain, scattered nodes fill the layers
 * near irregular boundaries), builds one stencil per node, computes the
 * weights of Eq. 1 for the operators d/dx, d/dy, d/dz and the Laplacian --
 * monomial-only (MON) weights on regular nodes, PHS r^3 + monomials (RBF-FD)
 * on scattered nodes -- applies them to fields, and runs the explicit
 * Boussinesq natural-convection step of Section 3 on top of them.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA device (or managed) memory owned by the
 *     caller; the library never frees them.  Objects returned through handles
 *     (hsm_plan, hsm_stepper, hsm_mlp) own their internal device memory and
 *     release it in the matching *_destroy call.
 *   - Coordinates and fields are structure-of-arrays: coords[k * n_nodes + i]
 *     is coordinate k of node i.  Operator outputs are [n_ops][n_nodes] with the
 *     operators in bit order of hsm_op (DX, DY, DZ, LAP).
 *   - All device work is enqueued on the stream given at creation and is
 *     asynchronous unless the comment says the call synchronises.
 *   - Errors: the return value is an hsm_status; no exception crosses the ABI.
 *     Argument errors are detected before any work is enqueued.  A CUDA error
 *     is reported as HSM_ECUDA and its text is kept for hsm_last_error.
 *   - Handles are not thread safe: use one handle per host thread.
 */
#ifndef HSM_H
#define HSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSM_OK = 0,
  HSM_EINVAL = 1,     /* invalid argument (null pointer, size, flag)            */
  HSM_ENOMEM = 2,     /* device allocation failed                               */
  HSM_ECUDA = 3,      /* a CUDA call failed; see hsm_last_error                 */
  HSM_ESINGULAR = 4,  /* at least one node has no valid weights                 */
  HSM_ENOTCONV = 5,   /* an iterative solve did not reach its tolerance         */
  HSM_ETIMEOUT = 6,   /* a bounded device wait gave up                          */
  HSM_EBOUNDS = 7,    /* a stencil index or size lies outside its range         */
  HSM_ESTATE = 8      /* call out of order (e.g. weights before stencils)       */
} hsm_status;

/* Operators of Eq. 1 (bit flags; several may be or-ed into an op mask). */
typedef enum { HSM_DX = 1, HSM_DY = 2, HSM_DZ = 4, HSM_LAP = 8 } hsm_op;

/* How the weights of scattered (RBF-FD) nodes are obtained. */
typedef enum {
  HSM_PREC_FP64 = 0,         /* direct solve in FP64                               */
  HSM_PREC_FP32_REFINE = 1,  /* FP32 LU with FP64-residual iterative refinement    */
  HSM_PREC_LEARNED = 2       /* MLP prediction + exact FP64 consistency projection,
                                direct FP64 solve as fallback (needs hsm_mlp_attach) */
} hsm_prec;

/* Storage type of an input field. */
typedef enum { HSM_F32 = 0, HSM_F64 = 1 } hsm_dtype;

/* Per-node status codes written by hsm_plan_compute_weights. */
enum {
  HSM_NODE_OK = 0,
  HSM_NODE_DEMOTED = 1,      /* regular-flagged node that had to use RBF-FD        */
  HSM_NODE_REFINE_FP64 = 2,  /* FP32 refinement did not converge; FP64 solve used  */
  HSM_NODE_LEARNED_SOLVE = 3,/* learned weights rejected; FP64 solve used          */
  HSM_NODE_REDUCED_DEGREE = 4,/* the degree-m monomials are not unisolvent on the
                                stencil: FP64 solve with the largest lower degree
                                m' >= 1 that is, on the same n nodes             */
  HSM_NODE_SINGULAR = 255    /* no valid weights                                    */
};

typedef struct hsm_plan_s* hsm_plan;
typedef struct hsm_stepper_s* hsm_stepper;
typedef struct hsm_mlp_s* hsm_mlp;

/* ------------------------------------------------------------------------ */
/* Status                                                                    */
/* ------------------------------------------------------------------------ */

/* Static text for a status code (never NULL). */
const char* hsm_status_string(hsm_status s);

/* Copies the text of the last error seen by this plan (or by the library when
 * plan is NULL) into buf (always NUL-terminated when len > 0).               */
hsm_status hsm_last_error(hsm_plan plan, char* buf, size_t len);

/* ------------------------------------------------------------------------ */
/* Plan: node set -> stencils -> weights (Section 2, Eq. 1)                  */
/* ------------------------------------------------------------------------ */

/* Creates a plan for a node set (Section 2: nodes x_i, a regular/scattered
 * flag per node, stencil size n, augmentation order m).
 *   dim         2 or 3
 *   n_nodes     N >= 1 (and < 2^31)
 *   coords      device f64 [dim][N]; must stay valid while the plan is used
 *   is_regular  device u8 [N]; 1 = regular lattice node (MON candidate)
 *   is_boundary device u8 [N] or NULL; 1 = boundary node (always RBF-FD; its
 *               stencil is itself plus the n-1 interior nodes nearest to the
 *               point one lattice spacing inside, x_c - h_regular * n_c)
 *   normals     device f64 [dim][N] outward unit normals of boundary nodes, or
 *               NULL (then the search point is x_c itself)
 *   h_regular   spacing of the regular lattice; lattice points are integer
 *               multiples of h_regular along every axis
 *   aug_m       monomial augmentation degree m of the RBF-FD basis, 1..6
 *   stencil_n   RBF-FD stencil size; 0 selects n = 2 * C(m+d, m) (Section 1);
 *               otherwise C(m+d, m) < stencil_n <= 128
 *   op_mask     operators to compute weights for (or of hsm_op; DZ needs dim 3)
 *   cuda_stream cudaStream_t the plan enqueues on (NULL = legacy default)
 * Allocates nothing on the device until hsm_plan_build_stencils.            */
hsm_status hsm_plan_create(hsm_plan* out, int dim, int64_t n_nodes, const double* coords,
                           const uint8_t* is_regular, const uint8_t* is_boundary,
                           const double* normals, double h_regular, int aug_m, int stencil_n,
                           unsigned op_mask, void* cuda_stream);

/* Sets the local internodal distance h(x_i) of an h-refined node set (Section
 * 4.2: the spacing decreases linearly from h_r on the regular nodes to h_s at
 * the irregular boundary; Section 4.3 likewise in 3D).  It only moves the
 * search point of boundary stencils, which becomes x_c - h(x_c) * n_c: one
 * LOCAL spacing inside, so that a boundary node in a refined layer keeps the
 * nodes around it in its stencil.
 *   spacing  device f64 [N], every entry > 0, or NULL to restore h_regular;
 *            caller-owned, must stay valid while the plan is used
 * Takes effect at the next hsm_plan_build_stencils; stencils and weights
 * built before must be rebuilt.  Nothing is checked on the device; returns
 * HSM_EINVAL only for a NULL plan.                                           */
hsm_status hsm_plan_set_spacing(hsm_plan plan, const double* spacing);

/* Builds every stencil (Section 2, "a set of n neighbouring nodes"):
 *   MON nodes: {c, c-e1, c+e1, c-e2, c+e2[, c-e3, c+e3]} through the lattice;
 *   RBF-FD nodes: the n nodes of smallest (squared distance, node id), the
 *   squared distance summed in coordinate order in FP64 without fused
 *   multiply-add; boundary nodes: the node, then the n-1 interior nodes of
 *   smallest (squared distance to x_c - h n_c, node id), h = h_regular or the
 *   node's entry of hsm_plan_set_spacing.  A regular-flagged
 *   node that is a boundary node, is not on the lattice, or misses a lattice
 *   neighbour is demoted to RBF-FD.
 * In weights arrangement 2 (hsm_plan_set_tuning) the build also solves the
 * FP64 weights of both groups (see hsm_plan_compute_weights).
 * Synchronises the plan's stream (the group sizes are read back).           */
hsm_status hsm_plan_build_stencils(hsm_plan plan);

/* Computes the weights of all nodes for the plan's operators (Eq. 1):
 * MON weights solve P^T w = L p over {1, x_k, x_k^2}; RBF-FD weights solve the
 * augmented system [A P; P^T 0][w; lambda] = [L phi; L p] with phi = r^3
 * (Section 2.1, Section 4), by the method selected with prec.  With
 * HSM_PREC_FP64 the systems of both groups -- MON (2d+1 unknowns) and RBF-FD
 * (n + C(m+d,m)) -- are solved in one persistent launch whose blocks draw
 * batches of either kind from one work queue, or as MON weights beside the
 * kNN search in the stencil build plus one RBF-FD launch here, or both inside
 * the stencil build (this call then only takes over their status), whichever
 * hsm_plan_autotune measured fastest for the plan (the split one until tuned;
 * see hsm_plan_tuning).
 *   node_status  device u8 [N] or NULL; receives one HSM_NODE_* per node
 * A system is singular when a pivot of the scaled FP64 system (entries of
 * order one) falls below 1e-12 in magnitude or is not finite.  A singular
 * system is solved again in FP64 with the monomials of degree m-1, m-2, ..., 1
 * on the same stencil until one is not (status HSM_NODE_REDUCED_DEGREE): a
 * stencil on which the degree-m monomials are not unisolvent still gets
 * weights exact for the lower degree.  Returns
 * HSM_ESINGULAR when some node has no valid weights (its weights are then
 * zero and its status HSM_NODE_SINGULAR).  Synchronises the plan's stream
 * (the failure count is read), except after a build that solved the weights,
 * whose read-back already holds it; the retries above always synchronise.   */
hsm_status hsm_plan_compute_weights(hsm_plan plan, hsm_prec prec, uint8_t* node_status);

/* Sizes after hsm_plan_build_stencils (host outputs; any may be NULL).
 *   nnz_per_op   number of stencil entries of one operator over all nodes
 *   n_mon        nodes using MON weights
 *   n_demoted    regular-flagged nodes demoted to RBF-FD
 *   n_fallback   nodes whose requested method fell back to the FP64 solve in
 *                the last hsm_plan_compute_weights                          */
hsm_status hsm_plan_query(hsm_plan plan, int64_t* nnz_per_op, int64_t* n_mon, int64_t* n_demoted,
                          int64_t* n_fallback);

/* Exports one operator (a single hsm_op bit present in the plan's op mask) as
 * CSR into caller-allocated device arrays: row_ptr int64 [N+1], col int32
 * [nnz], val f64 [nnz] (sizes from hsm_plan_query).  Column order within a row
 * is the stencil order (centre first).                                      */
hsm_status hsm_plan_export_csr(hsm_plan plan, unsigned op, int64_t* row_ptr, int32_t* col,
                               double* val);

/* Condition number kappa_2(M) = ||M||_2 ||M^-1||_2 of every node's weight
 * system (Section 2.1, "Computational stability"): the MON matrix P^T of a
 * regular node, the augmented RBF-FD matrix [A P; P^T 0] of a scattered one,
 * both in the offsets xi = (x - x_c) / s, s = max |x_i - x_c|.  Eigenvalues
 * by the cyclic Jacobi method (at most 40 sweeps), one thread per system; a
 * diagnostic, not on the weight path.  Needs hsm_plan_build_stencils.
 *   kappa  device f64 [N]; +inf where a system is singular
 * Enqueued on the plan's stream without synchronisation.                     */
hsm_status hsm_plan_condition(hsm_plan plan, double* kappa);

/* Mean normal flux of a field over a set of nodes, the average Nusselt number
 * of Section 4.1: out[0] = scale * (1/count) * sum_i |n_i . grad T(x_i)|, the
 * gradient taken with the plan's first-derivative weights (Eq. 1).  The
 * plan's op mask must hold d/dx_k for every axis of its dimension.
 *   T        device f64 [N]
 *   nodes    device int32 [count] node ids, count >= 1; an id outside
 *            [0, N) is not followed and makes out[0] a quiet NaN
 *   normals  device f64 [dim][N] unit normals (only the listed nodes are read)
 *   scale    L / (T_H - T_C) for the Nusselt number
 *   out      device f64 [1]
 * Enqueued on the plan's stream without synchronisation.  The sum runs in a
 * fixed order, so repeated calls give the same bits.                          */
hsm_status hsm_wall_flux_mean(hsm_plan plan, const double* T, const int32_t* nodes, int64_t count,
                              const double* normals, double scale, double* out);

/* Applies the operators of op_mask (a subset of the plan's) to one field,
 * Eq. 1: out[o][c] = sum_i w_o[c][i] u[idx[c][i]], stored in FP64.
 *   in_dtype  HSM_F64: u is f64 [N], FP64 weights, FP64 sums;
 *             HSM_F32: u is f32 [N], FP32 copies of the weights, FP32 sums
 *             (error within (n+2) 2^-24 sum |w u| of the exact sum)
 *   u         device [N]
 *   out       device f64 [popcount(op_mask)][N]                             */
hsm_status hsm_apply(hsm_plan plan, unsigned op_mask, hsm_dtype in_dtype, const void* u,
                     double* out);

/* Stencil validation (no counterpart in the paper: a debugging aid).
 * hsm_plan_validate scans the plan's stencil tables on the device -- the node
 * list and the ELL index array of each group against [0, N), and the node map
 * (group 0/1, position inside its group) -- and returns HSM_EBOUNDS, naming
 * the table, when an entry is out of range.  Synchronises.
 * hsm_plan_set_checks(plan, 1) turns on check mode: every call that gathers
 * through the stencils (hsm_plan_compute_weights, hsm_apply,
 * hsm_wall_flux_mean, hsm_plan_condition, hsm_stepper_create, hsm_step)
 * validates them first and returns HSM_EBOUNDS before any gather runs.  The
 * environment variable HSM_CHECK_BOUNDS=1 turns it on for every plan at
 * creation.                                                                 */
hsm_status hsm_plan_validate(hsm_plan plan);
hsm_status hsm_plan_set_checks(hsm_plan plan, int enable);

/* Failure-path test hook: HSM_FAULT_STENCIL_INDEX writes, from the host, the
 * out-of-range index N into the last entry of the plan's first RBF-FD stencil
 * (the first MON stencil when there is none) and turns check mode on, so
 * that every gathering call returns HSM_EBOUNDS and no kernel reads through
 * the bad index.  hsm_plan_build_stencils rebuilds valid tables.  Needs
 * built stencils (HSM_ESTATE otherwise).                                    */
hsm_status hsm_plan_inject_fault(hsm_plan plan, int fault);

/* Times the kernel variants of this plan (the kNN search: 1, 2 or 4 threads
 * per query, a first window of cells sized from n and the node spacing, then
 * ring by ring; lanes per RBF-FD weight system in FP64 and FP32; the
 * arrangement of the FP64 weights and its chunk count; the apply block size)
 * on its own data and keeps the fastest of each.
 * cache_path: NULL = no cache; otherwise a text file read before and updated
 * after tuning, keyed by device name and problem shape.  Synchronises.      */
hsm_status hsm_plan_autotune(hsm_plan plan, const char* cache_path);

/* The plan's kernel variants (host outputs, any may be NULL): threads per kNN
 * query (1, 2 or 4), lanes per RBF-FD system in FP64 and in FP32 +
 * refinement, threads per block of the apply, the arrangement of the FP64
 * weights and its chunk count, and tuned = 1 after hsm_plan_autotune.
 * Arrangements:
 *   0  the stencil build computes the MON weights beside the kNN search; the
 *      weights call solves the RBF-FD group in one launch;
 *   1  the weights call computes both groups in one persistent launch with a
 *      work queue (the build computes no weights);
 *   2  the stencil build computes both groups in FP64: the MON weights beside
 *      the kNN search, and the RBF-FD group in `chunks` (1, 2 or 4) equal
 *      chunks, chunk c solved on a branch of the build graph while the kNN
 *      search runs on chunk c + 1.  The first FP64 weights call after the
 *      build without node_status then only reads the status words (the
 *      singular systems' lower-degree retry included); another precision,
 *      node_status or a second call solves again.  The plan's RBF-FD weight
 *      array then has room for N stencils.                                  */
hsm_status hsm_plan_tuning(hsm_plan plan, int* knn_qt, int* rbf_lanes, int* rbf_lanes32, int* apply_threads,
                           int* arrange, int* chunks, int* tuned);

/* Sets the plan's kernel variants instead of timing them (reproducible runs,
 * tests): knn_qt 1, 2 or 4; rbf_lanes and rbf_lanes32 4, 8, 16 or 32;
 * apply_threads 64, 128 or 256; arrange 0, 1 or 2; chunks 1, 2 or 4 (used by
 * arrangement 2).  HSM_EINVAL for other values.  Takes effect at the next
 * build / weights / apply call; arrangement 2 with systems too large for the
 * FP64 kernel's shared memory makes hsm_plan_build_stencils fail with
 * HSM_EINVAL.                                                               */
hsm_status hsm_plan_set_tuning(hsm_plan plan, int knn_qt, int rbf_lanes, int rbf_lanes32, int apply_threads,
                               int arrange, int chunks);

/* Phases timed by hsm_plan_profile. */
enum { HSM_PHASE_STENCILS = 0, HSM_PHASE_MON = 1, HSM_PHASE_RBF = 2, HSM_PHASE_APPLY = 3,
       HSM_PHASE_COUNT = 4 };

/* Device time of the last run of each phase, measured with CUDA events that
 * the library records on the plan's stream around the phase's kernels (only
 * while timing is enabled with hsm_plan_set_timing), and the number of kernels
 * the plan has launched since it was created.  With weights arrangement 2 the
 * RBF-FD phase is the span of the solve's launches inside the stencil build
 * (from the first chunk's start to the last chunk's end, overlapping the kNN
 * search): it lies inside HSM_PHASE_STENCILS.
 *   phase_ms  host float [HSM_PHASE_COUNT] or NULL (milliseconds)
 *   launches  host int64 or NULL
 * Synchronises the plan's stream.                                           */
hsm_status hsm_plan_profile(hsm_plan plan, float* phase_ms, int64_t* launches);

/* Enables (1) or disables (0) the per-phase event timing of the plan.       */
hsm_status hsm_plan_set_timing(hsm_plan plan, int enable);

/* Releases the plan and all memory it owns.  NULL is allowed.               */
hsm_status hsm_plan_destroy(hsm_plan plan);

/* ------------------------------------------------------------------------ */
/* Explicit Boussinesq stepper (Section 3, Eqs. 2-4)                         */
/* ------------------------------------------------------------------------ */

/* Boundary kind per node for hsm_phys.bc. */
enum { HSM_BC_INTERIOR = 0, HSM_BC_T_DIRICHLET = 1, HSM_BC_T_NEUMANN = 2 };

typedef struct {
  double Ra;             /* Rayleigh number                                        */
  double Pr;             /* Prandtl number                                         */
  double dt;             /* time step; Section 3 uses dt = 0.1 h^2 / 2             */
  double T_ref;          /* reference temperature of the buoyancy term             */
  const uint8_t* bc;     /* device u8 [N]: HSM_BC_*; every non-interior node is a
                            no-slip wall with a zero normal pressure derivative    */
  const double* T_bc;    /* device f64 [N]: Dirichlet temperature (read where bc=1) */
  const double* normals; /* device f64 [dim][N]: outward unit normals (bc != 0)    */
  double krylov_tol;     /* relative residual of the pressure solve (e.g. 1e-12)   */
  int krylov_max_it;     /* iteration cap of the pressure solve (e.g. 2000)        */
  int precond;           /* HSM_PRECOND_AMG (0, default) or HSM_PRECOND_JACOBI     */
  int guess_order;       /* initial guess of each pressure solve from the call's
                            previous solutions: 0 = quadratic extrapolation
                            (default), 1 = linear, -1 = the last solution      */
  int apply_f32;         /* 1: the explicit operator applications (grad and lap
                            of v in the predictor, div v*, grad p, grad T and
                            lap T) use FP32 copies of the weights and FP32
                            sums, each sum rounded to FP64 before it enters the
                            FP64 state and time update; the pressure solve
                            stays FP64.  0 (default): FP64 throughout          */
  int mg_tail_from;      /* multigrid cycle shape (the preconditioner is the same
                            operator either way): 0 = picked by timing at
                            creation (default); k >= 1: levels k.. run in the
                            thread-block-cluster kernel; -1: no such kernel    */
  int mg_fused_from;     /* 0 = picked by timing (default); k >= 1: levels k-1..
                            below the tail run their smoothing and restriction,
                            and their post-smoothing, as one kernel each;
                            -1: none                                           */
  int mg_persistent;     /* 0 = picked by timing (default); 1 = the whole cycle
                            in one cooperative kernel, its phases separated by
                            grid-wide barriers (mg_tail_from and mg_fused_from
                            then do not apply); -1: never                      */
  int mg_sweeps;         /* damped-Jacobi sweeps before and after each coarse
                            correction: 2 (default, also 0) or 1.  With 1 the
                            pre-sweep from zero is x = w f and each level runs
                            two kernels per cycle (the other cycle shapes then
                            do not apply)                                      */
  int krylov;            /* with HSM_PRECOND_AMG: HSM_KRYLOV_GMRES (0, default),
                            GMRES restarted every 30 iterations, right-
                            preconditioned by one multigrid cycle per
                            iteration; HSM_KRYLOV_BICGSTAB: BiCGSTAB, two
                            cycles per iteration.  Both stop at the same
                            relative residual.  The Jacobi preconditioner
                            always runs BiCGSTAB.                              */
} hsm_phys;

/* Right preconditioner of the pressure BiCGSTAB.  AMG: an aggregation
 * multigrid V(2,2)-cycle of the pressure operator (geometric aggregates of
 * 2^d nodes per level, Galerkin coarse operators, damped Jacobi smoothing,
 * dense solve of the coarsest bordered system), built once by
 * hsm_stepper_create.  JACOBI: the inverse diagonal.                       */
enum { HSM_PRECOND_AMG = 0, HSM_PRECOND_JACOBI = 1 };
enum { HSM_KRYLOV_GMRES = 0, HSM_KRYLOV_BICGSTAB = 1 };

/* Creates a stepper on a plan whose weights exist and whose op mask holds
 * every first derivative and the Laplacian.  Copies *phys (the device arrays
 * it points to must stay valid).  Builds the pressure operator (Laplacian rows
 * inside, normal-derivative rows on the boundary) once, from the plan's
 * weights; the steps read the plan's weights in place.  Weights recomputed
 * afterwards (or a new hsm_plan_set_spacing and rebuild) need a new stepper. */
hsm_status hsm_stepper_create(hsm_stepper* out, hsm_plan plan, const hsm_phys* phys);

/* Advances n_steps explicit steps in place (Section 3; Chorin projection):
 *   1. v* = v + dt[-(v.grad)v + Pr lap v + Ra Pr (T - T_ref) e_up], v* = 0 on
 *      walls (e_up = last axis);
 *   2. solve [Lp 1; 1^T 0][p; c] = [div(v*) / dt (0 on walls); 0] by BiCGSTAB.
 *      The first two steps of a call start from the incoming p (c = 0) and
 *      the last solution; later steps of the same call start from (p, c)
 *      extrapolated in time from the call's last two (linear, third step) or
 *      three (quadratic) solutions.  Each call starts afresh:
 *      the caller owns p, so v, T and p are the whole state to save and
 *      restore between calls;
 *   3. v = v* - dt grad p inside, 0 on walls;
 *   4. T = T + dt[-v.grad T + lap T] inside (new v advects T);
 *   5. Dirichlet T = T_bc; insulated nodes T_b = -sum_{i!=b} wn_i T_i / wn_b.
 *   v  device f64 [dim][N], T device f64 [N], p device f64 [N]
 *   krylov_iters  host int [n_steps] or NULL: pressure iterations per step
 * Synchronises once at the end to read the solver status.  Returns
 * HSM_ENOTCONV if a pressure solve hit krylov_max_it or broke down on
 * non-finite values (the steps still ran).                                  */
hsm_status hsm_step(hsm_stepper st, int n_steps, double* v, double* T, double* p,
                    int* krylov_iters);

/* Shape of the stepper's pressure solve (host outputs, any may be NULL):
 *   mg_levels        multigrid levels (0 with the Jacobi preconditioner)
 *   mg_tail_level    first level whose cycle work runs in the one
 *                    thread-block-cluster kernel (0: none)
 *   mg_tail_ctas     CTAs per cluster the device schedules (0: none)
 *   mg_fused_level   first level (below the tail) whose smoothing and
 *                    restriction, and whose two post-smoothing sweeps, run as
 *                    one kernel each (>= mg_levels: none)
 *   kernels_per_iter kernels one Krylov iteration launches
 *   tail_ms, fused_ms host f32 [16] or NULL: device time of 10 cycles with
 *                    the tail from level l (tail_ms[0]: neither form), or
 *                    with the fused kernels from level l and no tail; -1
 *                    where the choice was not timed
 *   mg_persistent    1 when the whole cycle runs as one cooperative kernel
 *                    (the level choices above then do not apply)
 *   persistent_ms    device time of 10 such cycles; -1 where not timed
 *   level_rows, level_entries  host i64 [16] or NULL: rows of each level and
 *                    the matrix entries its ELL storage holds (padding
 *                    included); 0 past the last level
 * The shape is picked by timing these cycles at hsm_stepper_create.        */
hsm_status hsm_stepper_info(hsm_stepper st, int* mg_levels, int* mg_tail_level, int* mg_tail_ctas,
                            int* mg_fused_level, int* kernels_per_iter, float* tail_ms, float* fused_ms,
                            int* mg_persistent, float* persistent_ms, int64_t* level_rows,
                            int64_t* level_entries);

hsm_status hsm_stepper_destroy(hsm_stepper st);

/* ------------------------------------------------------------------------ */
/* Learned RBF-FD weights (no counterpart in the paper: the specification's  */
/* predictor).  An MLP maps the scaled offsets (x_i - x_c)/s of a stencil,  */
/* turned into a canonical frame Q (nearest neighbour on +x, the next one in */
/* the upper half plane; 2D), to its scaled weights (Q (s w_dx, s w_dy),     */
/* s^2 w_lap, operator-major).  The output is turned back with Q^T and       */
/* projected exactly onto the monomial reproduction constraints of Eq. 1 up  */
/* to degree m; a stencil whose relative pre-projection residual exceeds 1.5 */
/* or whose post-projection residual exceeds 1e-10 is re-solved in FP64.     */
/* Dense layers run on BF16 tensor cores with FP32 accumulation.             */
/* ------------------------------------------------------------------------ */

/* Creates an MLP: Linear(n_in, hidden) GELU, (Linear(hidden, hidden) GELU)
 * x (layers-1), Linear(hidden, n_out); seeded uniform initialisation.        */
hsm_status hsm_mlp_create(hsm_mlp* out, int n_in, int hidden, int layers, int n_out, uint64_t seed,
                          void* cuda_stream);
hsm_status hsm_mlp_destroy(hsm_mlp mlp);

/* Number of parameters in the packed layout (per layer: W [out][in], b).    */
hsm_status hsm_mlp_param_count(hsm_mlp mlp, int64_t* count);
/* Host f32 copies of the parameters in the packed layout (synchronises).    */
hsm_status hsm_mlp_get_params(hsm_mlp mlp, float* host, int64_t count);
hsm_status hsm_mlp_set_params(hsm_mlp mlp, const float* host, int64_t count);

/* Loss (mean squared error over samples and outputs) and its gradient with
 * respect to the packed parameters, on count samples X device f32
 * [count][n_in], Y device f32 [count][n_out].  grads_host: host f32 [param
 * count] or NULL.  Synchronises.                                            */
hsm_status hsm_mlp_grad(hsm_mlp mlp, const float* X, const float* Y, int64_t count, float* grads_host,
                        float* loss);

/* Adam training (lr, beta1 0.9, beta2 0.999, eps 1e-8) for `steps` steps of
 * `batch` samples drawn with replacement from (X, Y) by a seeded counter
 * hash.  loss_log: host f32 [steps] or NULL.  Synchronises.                  */
hsm_status hsm_mlp_train(hsm_mlp mlp, const float* X, const float* Y, int64_t count, int steps, int batch,
                         float lr, uint64_t seed, float* loss_log);

/* Forward pass: Y device f32 [count][n_out] from X device f32 [count][n_in].
 * The fused tensor-core pass bounds every wait on its pipeline barriers; if
 * one expires, every role leaves its loop, the tensor memory is released and
 * the call returns HSM_ETIMEOUT (Y is then undefined; the handle stays
 * usable).  Synchronises the MLP's stream.                                   */
hsm_status hsm_mlp_predict(hsm_mlp mlp, const float* X, int64_t count, float* Y);

/* Failure-path test hook (no paper counterpart).  HSM_FAULT_HOLD_MLP_LOADS
 * makes the next fused forward pass issue no loads at all, so that nothing
 * is ever in flight and the waits of its tensor-core and epilogue roles run
 * out: that hsm_mlp_predict returns HSM_ETIMEOUT, and later calls work as
 * before.  The hook applies to one pass; HSM_FAULT_NONE clears it.
 * HSM_EINVAL for a NULL handle or an unknown fault.                          */
enum { HSM_FAULT_NONE = 0, HSM_FAULT_HOLD_MLP_LOADS = 1, HSM_FAULT_STENCIL_INDEX = 2 };
hsm_status hsm_mlp_inject_fault(hsm_mlp mlp, int fault);

/* Attaches the predictor used by HSM_PREC_LEARNED (n_in = d n, n_out = nops n;
 * not owned by the plan; NULL detaches).  The learned path is built for 2D
 * plans with m = 2, n = 12; other plans return HSM_EINVAL from
 * hsm_plan_compute_weights(HSM_PREC_LEARNED).                               */
hsm_status hsm_mlp_attach(hsm_plan plan, hsm_mlp mlp);

/* Batch validation of HSM_PREC_LEARNED (no paper passage; the learned path's
 * third fallback rule): `samples` stencils spread evenly over the batch are
 * solved directly (they keep those weights and status HSM_NODE_LEARNED_SOLVE);
 * when the mean over the accepted ones of max|w_learned - w_direct| /
 * max|w_direct| exceeds tol, every stencil of the batch takes the direct
 * solve.  Defaults: tol 1e-3, samples 512; samples = 0 turns it off.       */
hsm_status hsm_plan_set_learned_gate(hsm_plan plan, double tol, int64_t samples);

/* Result of the last learned batch's validation (host outputs, any may be
 * NULL): error (-1 when none was measured), failed (1 when the batch took the
 * direct solve) and accepted (validated samples that the per-stencil checks
 * had accepted, the ones the error averages).                               */
hsm_status hsm_plan_learned_gate(hsm_plan plan, double* error, int* failed, int64_t* accepted);

/* Training data of a plan: for every interior RBF-FD node in ascending node
 * order, its features (X device f32 [count][d n]) and, from the plan's current
 * weights, its labels (Y device f32 [count][nops n], may be NULL).  With X NULL
 * only count is returned.  Synchronises.                                     */
hsm_status hsm_plan_learned_data(hsm_plan plan, float* X, float* Y, int64_t* count);

/* ------------------------------------------------------------------------ */
/* Allocation-free weights for caller-supplied stencils                     */
/* ------------------------------------------------------------------------ */

/* Largest batch the allocation-free entry point accepts.                    */
#define HSM_NOALLOC_MAX_SYSTEMS (1 << 20)

/* RBF-FD weights (FP32 factorisation, FP64-residual refinement, FP64 re-solve
 * of systems whose refinement does not converge) for stencils the caller
 * already has, allocating no device memory.  The paper has no counterpart to
 * this entry point; it exists for callers that must not allocate device
 * memory while they run (for example a solver embedded in an application
 * that hands all device memory to its own pool at start-up, or a real-time
 * loop in which an allocation could stall or fail).
 *   dim, aug_m, stencil_n, op_mask  as for hsm_plan_create (stencil_n > 0);
 *               sizes for which either the FP32 kernel or the FP64 re-solve
 *               kernel has no shared-memory shape (for example 2D, m = 1,
 *               n >= 83) are rejected with HSM_EINVAL before any work
 *   coords      device f64 [dim][n_nodes]
 *   stencils    device int32 [stencil_n][count]; row 0 holds each stencil's
 *               centre, the other rows its neighbours (any order).  Every
 *               entry must lie in [0, n_nodes): a first pass checks them all
 *               and returns HSM_EBOUNDS, with weights and node_status left
 *               untouched, if one does not
 *   count       0 <= count <= HSM_NOALLOC_MAX_SYSTEMS, else HSM_EINVAL
 *   weights     device f64 [popcount(op_mask)][stencil_n][count] (output)
 *   node_status device u8 [n_nodes] or NULL: every entry is set to
 *               HSM_NODE_OK, then centres re-solved in FP64 get
 *               HSM_NODE_REFINE_FP64 and singular ones HSM_NODE_SINGULAR
 * Its scratch (a fail list of HSM_NOALLOC_MAX_SYSTEMS entries, counters and
 * small tables, 4,211,200 bytes) is one static device array in the library that
 * every GPU which loads the library holds until the process exits.  All calls
 * share it and it keeps the last call's contents; calls that overlap on the
 * GPU (other streams, other host threads) race on it, so serialise them.  The
 * first call on a device looks up the array's address for that device (with
 * it current); make that first call before any stream capture.  Synchronises
 * the stream three times.  Returns HSM_ESINGULAR when some system is
 * singular.                                                                */
hsm_status hsm_rbf_weights_fp32r_noalloc(int dim, int aug_m, int stencil_n, unsigned op_mask,
                                         const double* coords, int64_t n_nodes, const int32_t* stencils,
                                         int64_t count, double* weights, uint8_t* node_status,
                                         void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Measurement and self-check (no paper passage)                             */
/* ------------------------------------------------------------------------ */

/* FP64 fused multiply-add throughput of the current device, the bound of the
 * RBF-FD weight solves: 4 to 32 independent FMA chains per thread (with a
 * constant or a register multiplier and addend), 2 to 8 blocks of 256 threads
 * per SM, 4096 iterations; the best rate over those shapes of 3 timed launches
 * each (CUDA events on cuda_stream) after one warm-up.
 *   gflops  host f64: 2 flop per FMA / time, in GFLOP/s (required)
 *   ms      host f32 or NULL: the best launch's time
 * Synchronises the stream.                                                   */
hsm_status hsm_probe_fp64_peak(double* gflops, float* ms, void* cuda_stream);

/* Hand-written device math helpers of the weight kernels and the fused MLP
 * pass, evaluated elementwise so that tests can hold them to their error
 * bounds against IEEE results:
 *   RECIP     1/x: Newton-Raphson from the single-precision reciprocal;
 *   SQRT_NR1  sqrt x: one Newton-Raphson step from the single-precision root;
 *   SQRT_GS   sqrt x: two steps of Goldschmidt's coupled iteration;
 *   ERF_AS    erf(x) of Abramowitz and Stegun 7.1.28 in FP32 (x >= 0);
 *   GELU      z Phi(z) in FP32 through ERF_AS.
 * The FP32 helpers take x rounded to FP32 and return their FP32 result
 * widened.  x, y device f64 [n]; enqueued on cuda_stream.                    */
enum { HSM_HELPER_RECIP = 0, HSM_HELPER_SQRT_NR1 = 1, HSM_HELPER_SQRT_GS = 2, HSM_HELPER_ERF_AS = 3,
       HSM_HELPER_GELU = 4 };
hsm_status hsm_eval_helper(int fn, const double* x, double* y, int64_t n, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HSM_H */
