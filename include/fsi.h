/*
 * fsi.h -- C ABI of the GB300 (sm_103a) field-split GMG-preconditioned FGMRES
 * solver for the linearised monolithic FSI system of Calandrini, Aulisa and
 * Ke, "A field-split preconditioning technique for fluid-structure
 * interaction problems with applications in biomechanics" (arXiv:1909.13201).
 *
 * The operation: solve J2 x = f (Sec. 3.2, Eq. matrix_J2: unknowns ordered
 * d^s, d^f, p^s, u^s, u^f, p^f) by flexible GMRES, right-preconditioned by one
 * geometric-multigrid V-cycle (Sec. 3.2-3.3: damped Richardson smoothing on
 * levels l >= 1, direct solve on level 0; prolongation P2 and equation-aware
 * restriction R2 of Sec. 3.3) whose smoother preconditioner is the additive
 * field-split Schwarz method FS = blockdiag(AS1, AS2) of Sec. 3.2 (Vanka
 * blocks solved by LU, Jacobi on the lumped mass K_u^s).
 *
 * Conventions shared by every call:
 *   - all compute runs on the CUDA stream given at set-up, on the device that
 *     was current then; every call returns after its stream work completed;
 *   - vectors b, x, w, lambda are float64 arrays of the level-(L-1) dof count
 *     in J2 order (fsi_get_dof_map gives field/component/node of each entry);
 *     "device" pointers are cudaMalloc'd (or torch) memory of that device;
 *   - the caller owns every buffer it passes; the context owns (and frees in
 *     fsi_destroy) all device memory it allocates itself;
 *   - no call aborts, traps or throws: each returns an fsi_status, and
 *     fsi_last_error() gives a one-line message for the last failing call
 *     of the calling thread.
 */
#ifndef FSI_H
#define FSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsi_ctx fsi_ctx;

typedef enum {
    FSI_OK = 0,
    FSI_ERR_ARG = 1,            /* invalid argument (null, size, option range) */
    FSI_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    FSI_ERR_ALLOC = 3,          /* device or host allocation failed */
    FSI_ERR_ZERO_PIVOT = 4,     /* a Schwarz block or the coarse matrix is singular */
    FSI_ERR_NOT_CONVERGED = 5,  /* max_iters reached; x holds the last iterate */
    FSI_ERR_BREAKDOWN = 6,      /* Arnoldi breakdown without convergence */
    FSI_ERR_NONFINITE = 7,      /* NaN/Inf in a norm (input or arithmetic) */
    FSI_ERR_STATE = 8           /* call out of order (e.g. solve before smoothers) */
} fsi_status;

enum { FSI_BC_CHANNEL_2D = 0, FSI_BC_BOX_3D = 1 };
/* FSI_FP64: everything float64.  FSI_MIXED: float32 V-cycle (level operators,
 * transfers, block inverses, vectors), float64 FGMRES and outer operator.
 * FSI_MIXED_HALF: as FSI_MIXED, with the Schwarz block inverses stored in
 * float16 with one float32 scale per row (max-abs row normalisation) and
 * applied with float32 accumulation. */
enum { FSI_FP64 = 0, FSI_MIXED = 1, FSI_MIXED_HALF = 2 };

/* One linearised FSI problem on the unit square/cube (Sec. 2.2 weak form,
 * linearised at d = 0 with a frozen advection field; linear-elastic solid
 * with penalty pressure).  Host pointers, read during fsi_setup_hierarchy only. */
typedef struct {
    int dim;                    /* 2 or 3 */
    int n_fine;                 /* fine elements per direction, divisible by 2^(n_levels-1) */
    int n_levels;               /* GMG levels L >= 1 */
    const uint8_t *material;    /* n_fine^dim, lexicographic x fastest; 1 solid, 0 fluid */
    const double *advection;    /* dim x (2 n_fine + 1)^dim: w at the fine Q2 nodes, comp-major */
    double mu_s, lambda_s, rho_s, rho_f, mu_f, dt;
    int bc_preset;              /* FSI_BC_CHANNEL_2D or FSI_BC_BOX_3D */
} fsi_problem;

typedef struct {
    int restriction;            /* 0: equation-aware R2 of Sec. 3.3 (default); 1: classical P^T */
    int nonlinear;              /* 1: operator patterns hold every coupling of the Jacobian of the
                                 * nonlinear residual (Sec. 2.2: the W rows also couple to d on the
                                 * moving fluid element), as fsi_nl_setup requires; the linear
                                 * operator then carries explicit zeros there.  0: linear patterns. */
} fsi_hier_opts;

typedef struct {
    int precision;              /* FSI_FP64, FSI_MIXED or FSI_MIXED_HALF */
    int patch;                  /* Vanka group edge b >= 1: b^dim pressure vertices per block */
    double omega;               /* Richardson damping (Sec. 3.2), > 0 */
    int nu_pre, nu_post;        /* smoothing steps, >= 1 */
    int factor;                 /* block inversion ("solved by LU", Sec. 3.2):
                                 *   FSI_FACTOR_AUTO (0): float64 Gauss-Jordan for FSI_FP64,
                                 *     FSI_FACTOR_TF32 otherwise;
                                 *   FSI_FACTOR_FP64 (1): unblocked float64 Gauss-Jordan;
                                 *   FSI_FACTOR_FP32 (2): blocked float32 Gauss-Jordan, rank-32
                                 *     updates on the CUDA cores;
                                 *   FSI_FACTOR_TF32 (3): blocked float32 Gauss-Jordan, rank-32
                                 *     trailing updates on the tensor cores (tcgen05, TF32
                                 *     operands, float32 accumulation).
                                 * 2 and 3 need a mixed precision (FSI_ERR_ARG otherwise). */
    int variant;                /* level preconditioner of the Richardson smoother (Sec. 3.2):
                                 *   FSI_SMOOTHER_FS (0): the field-split FS-ASM P2 (the paper's
                                 *     method): per pressure group a solid [d^s, p^s], a fluid
                                 *     [d^f] and a fluid [u^f, p^f] block, Jacobi on K_u^s;
                                 *   FSI_SMOOTHER_AS (1): the monolithic additive Schwarz method
                                 *     the paper compares against: one block of all fields per
                                 *     pressure group.  Blocks beyond one thread-block cluster
                                 *     of the float32 factorisation (above 507 dofs: 3D) are
                                 *     inverted by a 2 x 2 split over the two field systems,
                                 *     which needs FSI_MIXED (float32 inverses); the float64
                                 *     factorisation refuses blocks its 8-CTA cluster cannot
                                 *     hold (441 dofs and more).  Both: FSI_ERR_ARG. */
    int mult_levels;            /* locally multiplicative Schwarz (Sec. 3.2, multiplicative update
                                 * formula; the paper's AS1/AS2 are multiplicative within a
                                 * process) on the mult_levels finest levels, additive below;
                                 * 0: additive everywhere; >= the number of smoothed levels: every
                                 * level.  FS only (FSI_ERR_ARG with AS or a negative value).
                                 * On such a level one smoothing step is x += omega M (b - A x)
                                 * where M sweeps each field system of P2 separately from zero:
                                 * block by block, each block correcting with the residual of
                                 * its field operator A_FF at the latest iterate (velocity field:
                                 * the K_u^s Jacobi rows first); blocks ordered by pass (solid,
                                 * fluid-d, fluid-u kind, then the colour of the block's pressure
                                 * group with period 4 / 3 / 2 per direction for b = 1 / 2 / >= 3),
                                 * so blocks of one pass share no entry of A_FF and run at once.
                                 * The transposed cycle sweeps in reverse with A_jj^{-T} and A_FF^T. */
    int cascade;                /* 1: the swapped cascade of the paper's future work (Sec. 5, the
                                 * GMG and FS boxes interchanged): FGMRES on J2 preconditioned by
                                 * the field split into the displacement system [d^s, d^f, p^s]
                                 * (rows S, A, V) and the velocity system [u^s, u^f, p^f] (rows
                                 * K, F, W), each diagonal block preconditioned by its own GMG
                                 * V-cycle with the Schwarz smoothing above.  Realised as one
                                 * V-cycle whose level operators, restrictions and coarse solve
                                 * keep only same-system entries, so it equals
                                 * blockdiag(GMG_d, GMG_u); the Krylov operator stays J2.  FS
                                 * only (FSI_ERR_ARG with AS).  0: GMG outside, FS smoothing (the
                                 * paper's method). */
} fsi_smoother_opts;

enum { FSI_SMOOTHER_FS = 0, FSI_SMOOTHER_AS = 1 };

enum { FSI_FACTOR_AUTO = 0, FSI_FACTOR_FP64 = 1, FSI_FACTOR_FP32 = 2, FSI_FACTOR_TF32 = 3 };

typedef struct {
    double rtol;                /* stop when ||f - J2 x||_2 <= rtol ||f||_2 (float64 true residual) */
    int restart;                /* FGMRES restart length m, 1..64 */
    int max_iters;              /* total inner iterations */
    int use_x0;                 /* 1: x holds the initial guess; 0: start from zero */
} fsi_solve_opts;

typedef struct {
    int iterations;             /* N of Sec. 4: total FGMRES iterations */
    int cycles;                 /* restart cycles run */
    int converged;
    int status;                 /* fsi_status of this solve */
    double r0, rN;              /* initial and final true residual norms */
    double rel_residual;        /* rN / ||f|| */
    double rho;                 /* average convergence rate (rN / r0)^(1/N), Sec. 4 */
    double solve_ms;            /* wall time of the call, host clock */
} fsi_solve_stats;

/* ---------------------------------------------------------------------------
 * fsi_setup_hierarchy -- Sec. 3.3: levels by midpoint refinement (coarse
 * element solid when any descendant is), J2 numbering per level (Eq.
 * matrix_J2), level operators by rediscretisation (Sec. 2.2 weak form),
 * transfers P2 and R2, and the coarse-level direct factorisation.
 * probs: host array of n_probs problems (n_probs > 1 only for
 * fsi_solve_batched).  cuda_stream: a cudaStream_t (NULL = legacy stream).
 * On success *out owns all device memory it allocated. */
fsi_status fsi_setup_hierarchy(const fsi_problem *probs, int n_probs, const fsi_hier_opts *opts,
                               void *cuda_stream, fsi_ctx **out);

/* fsi_setup_smoothers -- Sec. 3.2: Vanka index sets of AS1 (solid [d^s,p^s]
 * and fluid [d^f] blocks) and AS2 (fluid [u^f,p^f] blocks) on every level
 * l >= 1, gather of the dense blocks and their batched factorisation
 * (inverted, stored float64 or float32 per opts->precision).  Returns
 * FSI_ERR_ZERO_PIVOT if a block is singular.  May be called again to change
 * the options. */
fsi_status fsi_setup_smoothers(fsi_ctx *ctx, const fsi_smoother_opts *opts);

/* fsi_solve -- FGMRES(restart) on J2 x = f with one V-cycle per iteration
 * (Sec. 3.2).  b: device, f (J2 order, length fsi_get_sizes n_dofs of the
 * fine level).  x: device, in: initial guess if opts->use_x0, out: solution.
 * Problem 0 of the context.  Non-convergence returns FSI_ERR_NOT_CONVERGED
 * with x holding the last iterate and st filled. */
fsi_status fsi_solve(fsi_ctx *ctx, const double *b, double *x, const fsi_solve_opts *opts,
                     fsi_solve_stats *st);

/* fsi_solve_batched -- every problem of the context, b[i] and x[i] device
 * vectors of problem i; st: host array of n_probs stats. */
fsi_status fsi_solve_batched(fsi_ctx *ctx, const double *const *b, double *const *x,
                             const fsi_solve_opts *opts, fsi_solve_stats *st);

/* fsi_adjoint -- for J = w^T x with J2 x = f: solves J2^T lambda = w by
 * FGMRES with the transposed V-cycle (transposed smoothers, restriction P^T,
 * prolongation R^T), then dJ/df = lambda, dJ/dA_ij = -lambda_i x_j on the
 * fine operator's CSR pattern (fsi_get_matrix order) and dJ/dmu_s =
 * -lambda^T (dA/dmu_s) x at fixed lambda_s.  w, x, lambda, dA_vals: device;
 * dA_vals (nnz) and dmu_s (host scalar) may be NULL.  Problem 0. */
fsi_status fsi_adjoint(fsi_ctx *ctx, const double *w, const double *x, double *lambda,
                       double *dA_vals, double *dmu_s, const fsi_solve_opts *opts,
                       fsi_solve_stats *st);

/* fsi_autotune -- picks the Vanka group size (fsi_smoother_opts.patch) of
 * every problem (an extension; the paper fixes its blocks by hand).  Problems
 * of the same size class (dimension, fine size, level count) share one
 * choice: for the class's first problem and each of the n_cand candidate
 * sizes (1..16, n_cand <= 8) the smoothers are rebuilt and a solve of
 * A x = A 1 with opts is timed on the device (the faster of two runs; a
 * candidate that does not converge counts as infinitely slow).  Afterwards
 * every problem's smoothers use its class's fastest candidate.  chosen: host
 * int[n_probs] receives the choice; times_ms (nullable): host
 * double[n_probs * n_cand], solve time per problem and candidate.  Requires
 * fsi_setup_smoothers first (precision, omega and smoothing steps are kept). */
fsi_status fsi_autotune(fsi_ctx *ctx, const int *candidates, int n_cand, const fsi_solve_opts *opts,
                        int *chosen, double *times_ms);

/* ----------------------------- accessors --------------------------------- */

/* Sizes of level `level` (0 = coarse .. L-1 = fine) of problem `prob`:
 * out[0] n_dofs, out[1] nnz of A_l, out[2] number of Schwarz blocks,
 * out[3] largest block, out[4..10] J2 group offsets (7 entries). */
fsi_status fsi_get_sizes(const fsi_ctx *ctx, int prob, int level, int64_t *out);

/* Host copies (n_dofs each) of the J2 dof map: field (0 d, 1 u, 2 p),
 * component (pressure: 0 solid copy, 1 fluid copy) and Q2/Q1 node index. */
fsi_status fsi_get_dof_map(const fsi_ctx *ctx, int prob, int level, int32_t *field,
                           int32_t *comp, int32_t *node);

/* Host copy of the float64 CSR of A_l: row_ptr (n+1), col (nnz), val (nnz). */
fsi_status fsi_get_matrix(const fsi_ctx *ctx, int prob, int level, int64_t *row_ptr,
                          int32_t *col, double *val);

/* Host copy of the transfer between level l and l-1 (l >= 1): which = 0 P_l
 * (n_l x n_{l-1}), 1 R_l (n_{l-1} x n_l).  Call with col/val NULL to get
 * row_ptr only (row_ptr[n_rows] = nnz). */
fsi_status fsi_get_transfer(const fsi_ctx *ctx, int prob, int level, int which, int64_t *row_ptr,
                            int32_t *col, double *val);

/* Host copy of the Schwarz block index sets of level l >= 1: blk_ptr
 * (n_blocks+1), idx (blk_ptr[n_blocks]).  idx NULL: blk_ptr only. */
fsi_status fsi_get_blocks(const fsi_ctx *ctx, int prob, int level, int64_t *blk_ptr, int32_t *idx);

/* Field-split blocks of level l >= 1: pass[j] (n_blocks entries, host) is the
 * pass of block j in the locally multiplicative sweep (Sec. 3.2), kind * k^dim
 * + colour with kind 0 solid [d^s, p^s], 1 fluid [d^f], 2 fluid [u^f, p^f],
 * colour = sum_a (t_a mod k) k^a over the tile coordinates t_a of the block's
 * pressure group and k = 4 / 3 / 2 for b = 1 / 2 / >= 3 (see mult_levels).
 * Blocks are in the order fsi_get_blocks returns (sorted by pass on levels
 * with the multiplicative sweep).  FSI_ERR_STATE for monolithic (AS) blocks
 * or before the blocks exist.  Works on host-only contexts. */
fsi_status fsi_get_block_passes(const fsi_ctx *ctx, int prob, int level, int32_t *pass);

/* ------------------- single-operation entry points ------------------------
 * Device-vector calls of one piece of the path, in the level's working
 * precision converted from/to float64 at the boundary; used to check each
 * piece against the oracle.  All vectors device float64. */

/* y = A_l x (float64 operator). */
fsi_status fsi_apply_operator(fsi_ctx *ctx, int prob, int level, const double *x, double *y);


/* y = P2^{-1} r on level l >= 1 (transpose != 0: P2^{-T} r), Sec. 3.2.  On a
 * level with the locally multiplicative sweep (fsi_smoother_opts.mult_levels)
 * y = M r, the sweep of both field systems from zero (transpose: M^T r; the
 * first transposed call builds the transposed operators). */
fsi_status fsi_apply_smoother(fsi_ctx *ctx, int prob, int level, const double *r, double *y,
                              int transpose);

/* fsi_apply_smoother_noalloc -- the same y = P2^{-1} r as fsi_apply_smoother,
 * for callers that cannot allocate GPU memory at call time (for example code
 * running under a memory pool or allocator that forbids cudaMalloc/cudaFree
 * after start-up, or a real-time loop that must not block on the driver's
 * allocator).  fsi_apply_smoother allocates two working vectors per call;
 * this variant allocates nothing: its working vectors live in one file-scope
 * device array of the library holding at most FSI_NOALLOC_MAX_DOFS entries
 * per vector (2 x 2^21 float64 = 32 MiB, reserved on every GPU that loads the
 * library until the process exits).  Levels with more dofs are rejected with
 * FSI_ERR_ARG.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, with the context's device current); the first call
 * on a device may load the library's device code, so make it before any
 * stream capture.  Every call reuses the
 * same array, so calls that may overlap on the GPU (different contexts,
 * streams or threads without ordering between them) race; calls issued on
 * one stream are ordered.  On a multiplicative-sweep level the transposed
 * sweep needs the transposed operators built beforehand (by fsi_adjoint or a
 * transposed fsi_apply_smoother / fsi_apply_vcycle): FSI_ERR_STATE otherwise.
 * The paper has no counterpart to this entry point. */
#define FSI_NOALLOC_MAX_DOFS 2097152
fsi_status fsi_apply_smoother_noalloc(fsi_ctx *ctx, int prob, int level, const double *r, double *y,
                                      int transpose);

/* z = M^{-1} v: one V-cycle from zero on the fine level (transpose != 0: the
 * transposed cycle). */
fsi_status fsi_apply_vcycle(fsi_ctx *ctx, int prob, const double *v, double *z, int transpose);

/* Kernel profiling (no counterpart in the paper; measurement support).
 * mode 1: reset the counters and start recording CUDA events around the
 * fine-level smoother apply and fine-level residual SpMV launches of the
 * following solves; mode 0: stop recording; mode 2: read only; mode 3: read,
 * and measure the device's float64 FMA throughput into out[21].
 * out (host, 32 doubles): [0] smoother launches timed, [1] their total ms,
 * [2] algorithmic bytes per smoother launch (block inverses, index, weight,
 * gather and scatter traffic), [3] SpMV launches timed, [4] their total ms,
 * [5] algorithmic bytes per SpMV launch, [6] kernels launched by the library
 * since the last reset, [7] outer float64 products w = A z_j timed, [8] their
 * total ms, [9] algorithmic bytes per product, [10] nonzeros of the fine
 * operator (one float64 FMA each), [11] fine-level block inversions timed
 * (fsi_setup_smoothers while recording), [12] their total ms, [13] flops of
 * one fine-level inversion (2 n_j^3 summed over blocks), [14] fine blocks,
 * [15] fine-level restrictions timed, [16] their ms, [17] algorithmic bytes
 * per restriction, [18] fine-level prolongations timed, [19] their ms,
 * [20] algorithmic bytes per prolongation, [21] float64 GFLOP/s measured
 * by mode 3 (independent FMA chains on every SM; 0 otherwise), [22] float64
 * Gram-Schmidt passes timed (update and dots, update and norm), [23] their
 * ms, [24] their float64 FMAs in total, [25] first Gram-Schmidt passes timed,
 * [26] their ms, [27] their bytes in total, [28] bytes the float64
 * Gram-Schmidt passes of [22] must move in total (basis columns, their
 * float32 copy where read, w in and out), [29..31] reserved.  The
 * Gram-Schmidt passes are timed in host-driven solves only (solves run
 * host-driven while recording).  On a fine level with the multiplicative
 * sweep (mult_levels) a timed "smoother launch" is the whole sweep (its pass
 * residuals, applies and closing update) and [2] counts the sweep's bytes:
 * the blocks' inverse, index and vector bytes, the A_FF entries and row
 * vectors of every pass residual and the closing x += omega y.  Problem 0. */
fsi_status fsi_profile(fsi_ctx *ctx, int mode, double *out);

/* fsi_autotune_layout -- picks the lanes per row of every binned-ELL copy
 * (level operators, transfers and their transposes): for each candidate in
 * lanes[0..n_lanes) (0: the size rule -- one lane per row for large
 * operators and inside a batch, up to 16 for small ones alone; or 1, 4, 8,
 * 16 for every copy) it rebuilds the copies and times a solve of every
 * problem of the context at once (b = A 1, options opts, the second of two
 * runs, host clock); keeps the fastest.  chosen: host int, the lanes value
 * kept; times_ms: host array of n_lanes (nullable; 1e300 for a candidate
 * whose solves did not converge).  An extension: the paper's data layout is
 * PETSc's CSR.  Captured graphs are rebuilt on the next solve. */
fsi_status fsi_autotune_layout(fsi_ctx *ctx, const int *lanes, int n_lanes, const fsi_solve_opts *opts, int *chosen,
                               double *times_ms);

/* fsi_get_cost -- algorithmic bytes of one solve's parts for problem `prob`
 * (an extension for roofline accounting; the paper reports times only):
 * cost[0] one V-cycle from zero on the fine level (per level: two smoothing
 * steps as counted by fsi_profile [2], two residual products, restriction
 * and prolongation; the coarse inverse GEMV; the mixed modes' casts),
 * cost[1] one float64 outer product w = A z, cost[2] the Gram-Schmidt bytes
 * per basis vector of one Arnoldi step (the three fused passes read each
 * vector in float32 and twice in float64: 20 B per entry; FP64 mode 24 B),
 * cost[3] fine-level unknowns.  One Arnoldi step j costs cost[0] + cost[1] +
 * (j + 1) cost[2].  cost: host array of 4.  FSI_ERR_STATE before
 * fsi_setup_smoothers. */
fsi_status fsi_get_cost(fsi_ctx *ctx, int prob, double *cost);

/* Host-only inspection context: builds the levels, numbering, operator
 * sparsity patterns, transfers and (for patch >= 1) the Schwarz block index
 * sets on the host without touching a GPU, so that fsi_get_sizes,
 * fsi_get_dof_map, fsi_get_pattern, fsi_get_transfer, fsi_get_blocks and
 * fsi_get_block_passes can
 * be called on machines without CUDA devices.  Every other call on such a
 * context returns FSI_ERR_STATE.  Release with fsi_destroy. */
fsi_status fsi_setup_host_only(const fsi_problem *prob, const fsi_hier_opts *opts, int patch,
                               fsi_ctx **out);

/* Host copy of the sparsity pattern of A_l: row_ptr (n+1), col (nnz). */
fsi_status fsi_get_pattern(const fsi_ctx *ctx, int prob, int level, int64_t *row_ptr, int32_t *col);

/* ---------------------------------------------------------------------------
 * Nonlinear FSI (Sec. 2.2): the monolithic residual R(U; U_n) of the ALE
 * formulation and one implicit time step solved by exact Newton, each
 * Newton system J(U_k) dU = -R(U_k) solved by fsi_solve's FGMRES with the
 * GMG / field-split preconditioner on the level Jacobians.  2D only.
 *
 * The residual, per element of the reference mesh (3-point Gauss rule):
 *   solid (total Lagrangian): rho_s (u - u_n)/dt + div of the first
 *     Piola-Kirchhoff stress of the incompressible Mooney-Rivlin law
 *     sigma = -p I + 2 C1 (B - I) - 2 C2 (B^{-1} - I), B = F F^T
 *     (Crank-Nicolson average of the elastic stress, pressure at t_new);
 *     K rows M_L (u - (d - d_n)/dt); V rows -(J - 1, q);
 *   fluid (ALE, on the element moved by d): rho (u - u_n)/dt + the
 *     Crank-Nicolson average of rho ((u - w_m).grad) u - rho f and of the
 *     viscous stress mu (grad u + grad u^T), the pressure at t_new, the SUPG
 *     term of Eq. phi_SUPG with tau of Eq. tausupg, lambda_k of Eq. lambda_k
 *     by 50 power-method steps on the element's bubble space; mesh velocity
 *     w_m = (d - d_n)/dt; A rows: the harmonic extension k (grad d + grad
 *     d^T) (k = 1/V_el of the fine element); W rows -(J div_x u, q);
 *   fixed (Dirichlet) dofs: R_i = U_i.
 * Body force f = force sin(2 pi t / period) w(x), w the problem's advection
 * field (zero at solid-class nodes).  The Jacobian is exact (tau included),
 * assembled on every level: level L-1 at U, coarser levels at the states
 * injected at coinciding nodes.
 * ------------------------------------------------------------------------- */
typedef struct {
    double force;               /* body-force amplitude */
    double period;              /* > 0 */
    double C1, C2;              /* Mooney-Rivlin constants; C1 <= 0: C1 = mu_s / 3, C2 = C1 / 2 */
} fsi_nl_params;

#define FSI_NL_MAX_NEWTON 32

typedef struct {
    double nl_rtol;             /* stop when ||R(U_k)||_2 <= nl_rtol ||R(U_0)||_2 */
    int max_newton;             /* 1..FSI_NL_MAX_NEWTON */
    double lin_rtol;            /* relative true-residual tolerance of every Newton system */
    int restart, max_iters;     /* FGMRES restart length and iteration limit per system */
} fsi_nl_opts;

typedef struct {
    int newton_steps;           /* s_i of Sec. 4: Newton steps taken */
    int converged;              /* 1: the nonlinear tolerance was met */
    int status;                 /* fsi_status of the call */
    int lin_iterations[FSI_NL_MAX_NEWTON];   /* N_{i,s}: FGMRES iterations of Newton step s */
    double lin_rho[FSI_NL_MAX_NEWTON];       /* rho_{i,s} = (r_N / r_0)^(1/N) of that solve */
    double residual[FSI_NL_MAX_NEWTON + 1];  /* ||R(U_k)||_2, k = 0 .. newton_steps */
    double jacobian_ms;         /* Jacobian assembly on all levels, coarse inverse (host clock) */
    double setup_ms;            /* Schwarz block set-up and inversion */
    double solve_ms;            /* FGMRES solves */
    double total_ms;            /* the whole call */
} fsi_nl_stats;

/* fsi_nl_setup -- prepare the nonlinear residual on every problem of the
 * context: element tables, colour lists, injection maps.  The hierarchy must
 * have been built with fsi_hier_opts.nonlinear = 1 (FSI_ERR_STATE otherwise)
 * and be 2D (FSI_ERR_ARG otherwise).  Densities, mu_f and dt come from the
 * problem description. */
fsi_status fsi_nl_setup(fsi_ctx *ctx, const fsi_nl_params *params);

/* fsi_nl_residual -- R(U; U_n) at time t_new on level `level` (device
 * float64 vectors of that level's dof count, J2 order; R must not overlap U
 * or U_n). */
fsi_status fsi_nl_residual(fsi_ctx *ctx, int prob, int level, const double *U, const double *Un,
                           double t_new, double *R);

/* fsi_nl_inject -- the state of level `level` - 1 from the state of level
 * `level` >= 1 at the coinciding nodes (fixed dofs zero). */
fsi_status fsi_nl_inject(fsi_ctx *ctx, int prob, int level, const double *U_fine, double *U_coarse);

/* fsi_nl_jacobian -- replace every level operator of problem `prob` by the
 * exact Jacobian dR/dU (fixed rows identity, fixed columns dropped) at U, U_n
 * (level L-1; injected below) and refactor the coarse level.  Afterwards
 * fsi_get_matrix returns the Jacobians; the smoothers must be set up again
 * before a solve (FSI_ERR_STATE otherwise), and fsi_adjoint no longer offers
 * dJ/dmu_s (the stored dA/dmu_s belongs to the linear operator). */
fsi_status fsi_nl_jacobian(fsi_ctx *ctx, int prob, const double *U, const double *Un, double t_new);

/* fsi_nl_step -- one time step to t_new by exact Newton from the initial
 * guess in U (device, level L-1; on return the new state), U_n the state at
 * t_new - dt (U and U_n must not overlap).  Per Newton step: the Jacobians (fsi_nl_jacobian), the
 * smoothers with the options of the last fsi_setup_smoothers call (which
 * must have run once), FGMRES on J dU = -R from dU = 0, U += dU.  Returns
 * FSI_ERR_NOT_CONVERGED when max_newton steps do not reach nl_rtol (stats
 * filled, U the last iterate), or the status of a failing linear solve. */
fsi_status fsi_nl_step(fsi_ctx *ctx, int prob, const double *Un, double *U, double t_new, const fsi_nl_opts *opts,
                       fsi_nl_stats *stats);

/* Release everything the context owns.  NULL is a no-op. */
void fsi_destroy(fsi_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *fsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSI_H */
