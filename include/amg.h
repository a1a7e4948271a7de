/*
 * amg.h -- C ABI of the GB300 aggregation-AMG preconditioned Krylov library.
 *
 * Method: Ganesan & Shah, "SParSH-AMG: a library for hybrid CPU-GPU algebraic
 * multigrid and preconditioned iterative methods" (arXiv 2007.00056):
 *   - problem statement A u = f, A sparse N x N in CSR (Sec. 2, Sec. 2.1);
 *   - setup: pairwise heavy-edge matching (Sec. 2.1.1-2.1.2, Algorithms 2-3),
 *     piecewise-constant prolongation P, Galerkin A_c = P^T A P (Sec. 2.1.1),
 *     coarsest factorisation once (Sec. 2), all split from the solve (Sec. 3);
 *   - solve: V-cycle (Algorithm 1) or the W- and F-cycles that Sec. 2 and
 *     Sec. 3 name, AMG as a solver (Sec. 3.1), AMG-preconditioned CG
 *     (Algorithm 4) and BiCG(Stab) (Algorithm 5), stopping on ||b - A x||_2
 *     (Sec. 4).
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers on the current CUDA device
 *     (for example torch tensors' data_ptr()).  No entry point reads host
 *     arrays except where stated (amg_params, amg_solve_info are host structs;
 *     amg_batch_pcg takes host arrays of hierarchy handles and of device
 *     vector pointers).
 *   - CSR: 0-based, int32 row pointers (n+1) and column indices (nnz), columns
 *     strictly ascending within each row, square n x n, values FP64.
 *   - Work is ordered on the caller's stream; functions that return results
 *     on the host (solver info, level sizes) synchronise that stream.
 *   - The caller owns every array it passes.  amg_setup copies A; the
 *     hierarchy owns all of its device memory until amg_destroy.
 *   - No function throws, aborts or traps.  Each returns an amg_status; on an
 *     error the output arrays are unspecified.  Device-side waits are bounded
 *     and report AMG_ERR_TIMEOUT instead of hanging.
 *   - One hierarchy serves any number of right-hand sides, one call at a
 *     time: calls on the same hierarchy share its work vectors and must not
 *     overlap on the GPU.  Different hierarchies are independent.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *amg_stream_t; /* same type as cudaStream_t; NULL = legacy default stream */

typedef enum {
  AMG_OK = 0,
  AMG_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad parameter, NaN/Inf input */
  AMG_ERR_INVALID_CSR = 2,   /* row pointers / column indices violate the CSR conventions */
  AMG_ERR_ZERO_DIAG = 3,     /* a row of some level has no (or a zero) diagonal entry */
  AMG_ERR_OOM = 4,           /* device allocation failed */
  AMG_ERR_BREAKDOWN = 5,     /* Krylov breakdown: a denominator vanished or became non-finite */
  AMG_ERR_NOT_CONVERGED = 6, /* max_iter reached before the tolerance (x still holds the last iterate) */
  AMG_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  AMG_ERR_CUDA = 8,          /* a CUDA runtime call failed */
  AMG_ERR_UNSUPPORTED = 9    /* valid input outside what this library implements */
} amg_status;

typedef enum {
  AMG_FP64 = 0,          /* hierarchy values and V-cycle in FP64 */
  AMG_FP32 = 1,          /* values rounded to FP32 after the FP64 setup; V-cycle in FP32 */
  AMG_FP16_STORAGE = 2   /* D^-1/2 A D^-1/2 values stored in FP16, FP32 arithmetic */
} amg_precision;

typedef enum { AMG_COARSE_AUTO = 0, AMG_COARSE_DENSE = 1, AMG_COARSE_CG = 2 } amg_coarse_solver;

/* Multigrid cycle (Sec. 2 lists V-, W- and F-cycles; Algorithm 1 is the V).
 * The coarse correction of level k is, below the coarsest level: one cycle of
 * level k+1 (V), two (W), or an F-cycle followed by a V-cycle of level k+1
 * (F); the first from a zero guess, the second from the first one's result.
 * The coarsest level is solved once per coarse correction. */
typedef enum { AMG_CYCLE_V = 0, AMG_CYCLE_W = 1, AMG_CYCLE_F = 2 } amg_cycle_kind;

/* Order of equal edge weights in the matching.  AMG_TIE_SMALLER: total edge
 * order (w descending, min(i,j) ascending, max(i,j) ascending), i.e. a node
 * prefers the smaller of two equally heavy neighbours.  AMG_TIE_LARGER: the
 * order of Algorithm 3's lexicographically descending sort (w descending,
 * max(i,j) descending, min(i,j) descending): the larger neighbour. */
typedef enum { AMG_TIE_SMALLER = 0, AMG_TIE_LARGER = 1 } amg_tie_break;

/* Edge weight of {i,j}.  AMG_WEIGHT_ABS: max(|a_ij|, |a_ji|) (Sec. 2.1).
 * AMG_WEIGHT_SCALED, an option the paper does not have: that weight divided
 * by sqrt(|a_ii| |a_jj|), the weight of the symmetrically scaled matrix
 * D^-1/2 A D^-1/2, which keeps coarsening variable-coefficient problems
 * whose plain weights stall it. */
typedef enum { AMG_WEIGHT_ABS = 0, AMG_WEIGHT_SCALED = 1 } amg_edge_weight;

/* Setup and cycle parameters (amg_default_params fills the defaults).
 *   passes       pairwise matching passes per level (2: aggregates of <= 4; Table 2 /
 *                "pairwise, 2 passes")
 *   max_levels   levels including the finest (10; the paper's Table 2 uses 6)
 *   coarse_max   stop coarsening once a level has <= coarse_max rows; also the
 *                largest coarsest level solved by a dense factorisation (4096)
 *   stall_ratio  do not add a level whose size ratio N_{k+1}/N_k exceeds this (0.85)
 *   omega        damped-Jacobi weight of the smoother S_k (2/3)
 *   nu_pre, nu_post  pre- and post-smoothing sweeps (1, 1; Table 2 uses 6, 6)
 *   coarse_solver    AMG_COARSE_AUTO: dense if the coarsest level has <= coarse_max
 *                rows, else Jacobi-PCG to a relative residual of 1e-12 (Sec. 4.2),
 *                on one thread block cluster up to 2048 rows, else on the whole GPU.
 *                The dense solve applies the inverse formed at setup by blocked
 *                Gauss-Jordan elimination (without row interchanges when every
 *                pivot block is invertible and the inverse passes its accuracy
 *                check, else with partial pivoting): in FP64 up to
 *                2048 rows; above that in FP32 with a fixed number of FP64
 *                refinement steps per solve (x += X (f - A x)), chosen at setup
 *                so the result has FP64 accuracy (FP64 inverse if refinement
 *                cannot reach it)
 *   precision    value storage / arithmetic of the V-cycle (outer Krylov is FP64)
 *   cycle        amg_cycle_kind of every cycle the hierarchy runs (AMG_CYCLE_V).
 *                The W-cycle keeps M^{-1} symmetric for symmetric A; the
 *                F-cycle does not, so PCG with it should be flexible.
 *   tie_break    amg_tie_break of the matching (AMG_TIE_SMALLER)
 *   edge_weight  amg_edge_weight of the matching (AMG_WEIGHT_ABS)
 *   operator_form  1 (default): in the FP64 and FP32 precisions, setup also
 *                forms, for every level below the coarsest, C = I - omega A D^-1
 *                (A's pattern) and Q = P - omega D^-1 A P (the pattern of A P),
 *                and a cycle visit from the zero guess with nu_pre = nu_post = 1
 *                computes its residual as t = C f and its result as
 *                Q x_{k+1} + omega D^-1 (f + t): algebraically the same
 *                presmoothing, residual, prolongation and postsmoothing of
 *                Algorithm 1 (x = omega D^-1 f is never stored), in two
 *                matrix passes of which the second is over the smaller A P.
 *                Costs about one more copy of the level matrices in device
 *                memory.  0: only the explicit sweeps.
 *   dense_max    largest coarsest level that AMG_COARSE_AUTO solves with the
 *                dense inverse (0, the default: coarse_max).  A value above
 *                coarse_max keeps the stop size small while a hierarchy whose
 *                coarsening stalled a little above it still gets the direct
 *                coarsest solve instead of the CG.
 *   graphs       when the Krylov and stationary solvers replay one captured CUDA graph
 *                per iteration instead of launching its kernels one by one: 0 (the
 *                default) from the second solve on a hierarchy, since for a single
 *                solve the capture costs about what it saves; 1 from the first solve,
 *                for many concurrent solves whose kernel launches compete on the host;
 *                -1 never.  Results are the same either way. */
typedef struct {
  int passes;
  int max_levels;
  int coarse_max;
  double stall_ratio;
  double omega;
  int nu_pre;
  int nu_post;
  int coarse_solver;
  int precision;
  int cycle;
  int tie_break;
  int edge_weight;
  int operator_form;
  int dense_max;
  int graphs;
} amg_params;

/* Result of a Krylov solve.  iterations counts completed iterations (a
 * BiCGStab half step that meets the tolerance counts as one).
 * rel_res_recurrence is ||r||_2/||b||_2 of the recurrence residual at exit,
 * rel_res_true is ||b - A x||_2/||b||_2 recomputed from x. */
typedef struct {
  int iterations;
  double rel_res_recurrence;
  double rel_res_true;
  amg_status status;
} amg_solve_info;

typedef struct amg_hierarchy amg_hierarchy; /* opaque, device-resident */

/* Fills *p with the defaults listed above.  AMG_ERR_INVALID_ARG if p is NULL. */
amg_status amg_default_params(amg_params *p);

/* Setup phase (Sec. 3; coarsening Sec. 2.1, Algorithms 2-3; Galerkin Sec. 2.1.1).
 * Builds the hierarchy of A (n rows, nnz stored entries, device CSR arrays) on
 * the device: for each level, `passes` rounds-to-fixed-point of mutual-
 * heaviest-neighbour handshakes (edge weight max(|a_ij|,|a_ji|), equal weights
 * broken toward the smaller index; unmatched nodes stay single), aggregate ids
 * by smallest member, A_{k+1} = P^T A_k P with a fixed summation order; then
 * the coarsest solver (dense inverse, or CG).  params may be NULL (defaults).
 * The pattern of A must be structurally symmetric (AMG_ERR_UNSUPPORTED
 * otherwise).  On success *out owns a new hierarchy; on failure *out = NULL.
 * Errors: INVALID_ARG (n <= 0, nnz < 0, NULL pointers, bad params),
 * INVALID_CSR, ZERO_DIAG, OOM, CUDA, TIMEOUT, UNSUPPORTED. */
amg_status amg_setup(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                     const double *d_val, const amg_params *params, amg_stream_t stream,
                     amg_hierarchy **out);

/* One multigrid cycle from a zero initial guess (Algorithm 1 with x_0 = 0, as
 * used for z = M^{-1} r in Algorithms 4-5; the W- or F-cycle when the
 * hierarchy's params.cycle selects it): d_z = M^{-1} d_r, both length n.  The
 * two arrays must not overlap.  In FP32 / FP16-storage precision the input
 * is rounded to FP32 and the output widened back to FP64. */
amg_status amg_vcycle(const amg_hierarchy *h, const double *d_r, double *d_z, amg_stream_t stream);

/* AMG as a solver (Sec. 3.1, compared with AMG-PCG in Sec. 4.4): the
 * stationary iteration x_{j+1} = x_j + M^{-1}(b - A x_j), M^{-1} one cycle of
 * the hierarchy's kind from a zero guess.  d_x holds x_0 on entry, the last
 * iterate on exit.  After every cycle the residual b - A x_j is recomputed
 * from x_j; the solve stops when its 2-norm is <= rtol ||b||_2 or after
 * max_iter cycles (iterations counts cycles; rel_res_recurrence and
 * rel_res_true both report that residual).  b = 0 gives x = 0 and 0
 * iterations.  info may be NULL.
 * Errors: INVALID_ARG, BREAKDOWN (non-finite residual), NOT_CONVERGED,
 * TIMEOUT, CUDA. */
amg_status amg_solve(const amg_hierarchy *h, const double *d_b, double *d_x, double rtol, int max_iter,
                     amg_stream_t stream, amg_solve_info *info);

/* AMG-preconditioned CG (Sec. 3.2, Algorithm 4; residual update read as
 * r_{j+1} = r_j - alpha A p_j).  d_x holds x_0 on entry, the solution on exit.
 * Stops when ||r||_2 <= rtol ||b||_2 (recurrence residual) or after max_iter
 * iterations.  flexible != 0 uses beta = (z_{j+1}, r_{j+1} - r_j)/(z_j, r_j),
 * which stays valid when M varies slightly (mixed precision, CG coarse solve).
 * rtol = 0 runs exactly max_iter iterations unless r becomes exactly zero.
 * b = 0 gives x = 0 and 0 iterations.  info may be NULL.
 * Errors: INVALID_ARG, BREAKDOWN, NOT_CONVERGED, TIMEOUT, CUDA. */
amg_status pcg_solve(const amg_hierarchy *h, const double *d_b, double *d_x, double rtol,
                     int max_iter, int flexible, amg_stream_t stream, amg_solve_info *info);

/* AMG-preconditioned BiCGStab (Sec. 3.2, Algorithm 5), right preconditioned,
 * rbar_0 = r_0 and p_0 = r_0; p_{j+1} = r_{j+1} + beta (p_j - omega A p~_j).
 * A half step whose ||s|| meets rtol ends the solve with x += alpha p~.
 * Same argument and error conventions as pcg_solve. */
amg_status bicgstab_solve(const amg_hierarchy *h, const double *d_b, double *d_x, double rtol,
                          int max_iter, amg_stream_t stream, amg_solve_info *info);

/* Batched AMG-PCG (Algorithm 4 per system, V-cycle of Algorithm 1): solves
 * nsys independent systems in one persistent launch per team size, each
 * system on its own team -- one thread block up to 8192 rows, a thread-block
 * cluster of 2 / 4 / 8 blocks above 8192 / 24576 / 65536 rows -- running its
 * whole solve (same arguments and stopping rule as pcg_solve, applied per
 * system).  hs, d_b and d_x are host arrays of nsys entries.  hs[i] is the
 * hierarchy of system i (each
 * hierarchy at most once per call; every hierarchy must have a dense
 * coarsest level of at most 2048 rows (an FP64 inverse), the V-cycle and the
 * same precision, FP64 or FP32;
 * AMG_ERR_UNSUPPORTED otherwise); d_b[i], d_x[i] are its device right-hand
 * side and initial guess / solution.  Team reductions in a fixed order only:
 * the result of a system does not depend on the rest of the batch.  infos (host, length nsys,
 * may be NULL) receives every system's result; the return value is AMG_OK
 * when every system converged, else the first non-OK status.  Synchronises
 * the stream.  Meant for several systems at once; a lone system is faster
 * with pcg_solve, which spreads it over the whole GPU. */
amg_status amg_batch_pcg(int nsys, amg_hierarchy *const *hs, const double *const *d_b, double *const *d_x,
                         double rtol, int max_iter, int flexible, amg_stream_t stream, amg_solve_info *infos);

/* Number of levels (finest included) of h, or -1 if h is NULL. */
int amg_num_levels(const amg_hierarchy *h);

/* Size of level k (0 = finest): *n rows and *nnz stored entries (either
 * pointer may be NULL).  d_agg_out, if not NULL, receives the level's
 * fine-to-coarse aggregate map (length n, ids in [0, n_{k+1})); it must be
 * NULL for the coarsest level.  Synchronises the stream. */
amg_status amg_level_info(const amg_hierarchy *h, int level, int *n, int64_t *nnz,
                          int32_t *d_agg_out, amg_stream_t stream);

/* Copies level k's CSR (FP64 values) into caller arrays of sizes n+1, nnz, nnz. */
amg_status amg_export_level(const amg_hierarchy *h, int level, int32_t *d_row_ptr, int32_t *d_col,
                            double *d_val, amg_stream_t stream);

/* Handshake rounds run by pass p of level k during setup (the final round that
 * matched nothing included), or -1 if out of range. */
int amg_setup_rounds(const amg_hierarchy *h, int level, int pass);

/* ---- Kernel autotuning (no counterpart in the paper) ----
 * Times, on each level of h, the threads-per-row choices of the row kernels
 * (1, 2, 4, ... 32 lanes per row, and 0: one lane per row reading tiles of
 * the matrix that TMA bulk copies stage in shared memory) and the fused /
 * separate forms of the first
 * pre-smoothing sweep (with the residual) and of the prolongation (with the
 * first post-smoothing sweep), keeps the fastest for h, and remembers the
 * choice by level shape (rows, nonzeros, precision) so that every later
 * amg_setup in this process with a level of the same shape starts with it.
 * Choices change only the summation order of row sums (results stay within
 * rounding of each other).  Synchronises the stream.  Without tuning, a level
 * uses 1 lane per row up to 12 nonzeros per row and more lanes beyond. */
amg_status amg_autotune(amg_hierarchy *h, amg_stream_t stream);

/* Current kernel configuration of a level: lanes per row, fused presmoothing,
 * fused prolongation.  Returns 0, or -1 for a NULL h or a bad level. */
int amg_level_config(const amg_hierarchy *h, int level, int *tpr, int *fuse_pre, int *fuse_post);

/* Sets a level's kernel configuration by hand (tpr in {0,1,2,4,8,16,32}).
 * AMG_ERR_INVALID_ARG for a NULL h, a bad level or a bad tpr;
 * AMG_ERR_UNSUPPORTED for tpr 0 on a level without the staged form (a
 * tile of 256 rows too large for shared memory). */
amg_status amg_level_set_config(amg_hierarchy *h, int level, int tpr, int fuse_pre, int fuse_post);

/* Residual-operator form of a level (see amg_params.operator_form): returns 1
 * when zero-guess visits of the level use C and Q, 0 when they use the
 * explicit sweeps, -1 for a NULL h or a bad level. */
int amg_level_operator_form(const amg_hierarchy *h, int level);

/* Switches a level's zero-guess visits between the residual-operator form
 * (on != 0) and the explicit sweeps.  AMG_ERR_INVALID_ARG for a NULL h or a
 * bad level; AMG_ERR_UNSUPPORTED for on != 0 on a level without C and Q (the
 * coarsest level, FP16 storage, or operator_form = 0 at setup). */
amg_status amg_level_set_operator_form(amg_hierarchy *h, int level, int on);

/* ---- Instrumentation (no counterpart in the paper; used for measurement) ---- */

/* Self-test of the library's bounded device waits: `blocks` (1..64) blocks
 * wait at the grid barrier used by the coarse solver for one arrival that
 * never comes; each must give up after about 2 ms of clock cycles.  Returns
 * AMG_ERR_TIMEOUT when every block reported the timeout (the expected
 * outcome), AMG_OK if any block passed the barrier (a defect), or a CUDA
 * error.  The device stays usable afterwards.  Synchronises the stream. */
amg_status amg_selftest_wait_timeout(int blocks, amg_stream_t stream);

/* Self-test of the library's FP64 <-> FP32 conversions (the precision casts
 * of the mixed-precision V-cycle compute them on the integer pipe): for the
 * n doubles at d_in (device), writes d_f32[i] = d_in[i] rounded to FP32
 * (round to nearest even) and d_f64[i] = d_f32[i] widened back to FP64, both
 * by the library's conversion routines; the caller compares them with the
 * hardware conversions.  Device pointers, n >= 0; AMG_ERR_INVALID_ARG for a
 * null pointer with n > 0.  Asynchronous on `stream`. */
amg_status amg_selftest_convert(int64_t n, const double *d_in, float *d_f32, double *d_f64, amg_stream_t stream);

/* Coarsest CG form of h: the number of CTAs of the thread block cluster that
 * solves a small coarsest level (16 or 8, for at most 2048 rows when the
 * device schedules such a cluster), 0 when the grid-wide cooperative kernel
 * solves it, -1 when the coarsest level is solved by the dense inverse or h
 * is NULL. */
int amg_coarse_cg_cluster_size(const amg_hierarchy *h);

/* Kernel kinds reported by the per-kernel profiler.  Each kind is tracked per
 * level (0 = finest); Krylov kinds are reported at level 0. */
typedef enum {
  AMG_K_JACOBI0 = 0,        /* first presmoothing sweep from x = 0 (vector pass)      */
  AMG_K_JACOBI = 1,         /* further damped-Jacobi sweeps (matrix pass)              */
  AMG_K_RESIDUAL = 2,       /* t = f - A x (matrix pass)                               */
  AMG_K_RESTRICT = 3,       /* f_{k+1} = P^T t                                         */
  AMG_K_PROLONG_JACOBI = 4, /* x + P x_{k+1} fused with the first postsmoothing sweep  */
  AMG_K_PROLONG = 5,        /* x + P x_{k+1} alone (nu_post = 0)                       */
  AMG_K_COARSE_DENSE = 6,   /* coarsest solve, dense inverse times vector              */
  AMG_K_COARSE_CG = 7,      /* coarsest solve, persistent Jacobi-PCG                   */
  AMG_K_CAST = 8,           /* FP64 <-> FP32 conversions of the mixed-precision cycle  */
  AMG_K_KRYLOV_SPMV = 9,    /* outer Krylov SpMV with fused dot products               */
  AMG_K_KRYLOV_VEC = 10,    /* outer Krylov vector updates with fused dot products     */
  AMG_K_OP_RESIDUAL = 11,   /* residual-operator form: t = C f (matrix pass)            */
  AMG_K_OP_POST = 12        /* residual-operator form: Q x_{k+1} + omega D^-1 (f + t)   */
} amg_kernel_kind;

/* Total kernel launches this library has issued since it was loaded (a graph
 * replay counts each kernel it runs). */
unsigned long long amg_kernel_launches(void);

/* Turns per-launch CUDA-event timing of the solve phase on (on != 0) or off.
 * While on, Krylov iterations run as direct launches rather than graph
 * replays.  AMG_ERR_INVALID_ARG if h is NULL. */
amg_status amg_profile_enable(amg_hierarchy *h, int on);

/* Clears the accumulated timings of h. */
amg_status amg_profile_reset(amg_hierarchy *h);

/* Accumulated totals for one kernel kind at one level since the last reset:
 * device milliseconds (sum over launches, CUDA events on the launching
 * stream), algorithmic bytes (sum over launches: what the kernel must read and
 * write, each vector entry counted once) and launch count.  Any output pointer
 * may be NULL.  Waits for pending timed launches. */
amg_status amg_profile_read(amg_hierarchy *h, int kind, int level, double *ms, double *bytes, long long *launches);

/* ---- Allocation-free coarse solve (the paper has no counterpart) ----
 *
 * Solves A x = f by the library's Jacobi-preconditioned CG (the coarsest-level
 * solver of the V-cycle: from x = 0 until ||f - A x||_2 <= 1e-12 ||f||_2, at
 * most 1000 iterations) without allocating any device memory.  It is meant for
 * callers that cannot call cudaMalloc: plugins whose host framework owns every
 * device allocation (through its own pool or budget), and latency-critical
 * loops that cannot afford cudaMalloc's implicit device-wide synchronisation.
 *
 * All work vectors live in one fixed array inside the library (about 29 MB,
 * held on every GPU that loads the library until the process exits), so:
 *   - n must be at most 262144 (AMG_ERR_INVALID_ARG beyond that, before any
 *     device work); nnz < 2^31;
 *   - every call on a device shares that array, which keeps the previous
 *     call's contents (the entry point clears what must start at zero); calls
 *     whose GPU work overlaps -- on different streams or host threads -- race
 *     on it and must be serialised by the caller;
 *   - the first call on each device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 * Arguments: device CSR of A (same conventions as amg_setup, diagonal nonzero),
 * device vectors f (input) and x (output, length n; x must not be f).  The call
 * synchronises `stream`; *iterations (may be NULL) receives the CG iteration
 * count.  After the solve the residual is recomputed from x: AMG_OK when it is
 * at most 1e-10 ||f||_2 within the iteration limit, AMG_ERR_NOT_CONVERGED
 * otherwise (x holds the last iterate), AMG_ERR_BREAKDOWN when it is not
 * finite.  Other errors: INVALID_ARG, INVALID_CSR, ZERO_DIAG, TIMEOUT, CUDA. */
amg_status amg_coarse_cg_noalloc(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                                 const double *d_val, const double *d_f, double *d_x, amg_stream_t stream,
                                 int *iterations);

/* Where the level matrices live during the solve phase (Sec. 3.1.1, the hybrid
 * CPU/GPU-CI algorithm: a cycle works on one level at a time, so the matrices
 * of the other levels can wait in host memory and be copied to the GPU when
 * the cycle reaches them, the copy overlapping the current level's kernels).
 *   AMG_RESIDENT     everything in device memory (the state after amg_setup).
 *   AMG_HOST_MAPPED  for levels first_level..L-1, every array whose length is
 *                    the level's number of nonzeros (column indices and values
 *                    of A, of its FP32 / FP16 copies, of C and of Q) moves to
 *                    pinned host memory and the kernels read it there, over
 *                    the host-device link (NVLink-C2C on GB300).
 *   AMG_HOST_STAGED  the same arrays in pinned host memory, but each cycle
 *                    visit of such a level reads its matrix from one of two
 *                    device buffers that a second stream fills with
 *                    cudaMemcpyAsync; the copy for the visit predicted next
 *                    (V-cycle order) runs while the current visit computes,
 *                    and an unpredicted visit (W- and F-cycles) waits for its
 *                    own copy.  Level 0's A stays in device memory (the outer
 *                    Krylov method multiplies by it every iteration).  Solves
 *                    run without CUDA graphs in this mode.
 * Arrays of length n (row pointers, diagonals, aggregate maps, vectors) and
 * the coarsest level never move.  Results are bitwise the same in every mode.
 * first_level must be in [0, L) for the host modes (ignored for
 * AMG_RESIDENT).  Synchronises the hierarchy's latest stream and `stream`;
 * errors: INVALID_ARG, OOM (pinned host or device memory; the hierarchy is
 * left resident), UNSUPPORTED (no unified addressing), CUDA.  amg_autotune
 * returns UNSUPPORTED while levels are in host memory: tune first. */
typedef enum { AMG_RESIDENT = 0, AMG_HOST_MAPPED = 1, AMG_HOST_STAGED = 2 } amg_residency;
amg_status amg_set_residency(amg_hierarchy *h, int residency, int first_level, amg_stream_t stream);

/* Memory of h (any output may be NULL): device bytes it owns (staging buffers
 * included), pinned host bytes of its host-resident arrays, bytes of the two
 * staging buffers, and bytes copied host-to-device by the staging since the
 * last amg_set_residency. */
amg_status amg_memory_info(const amg_hierarchy *h, uint64_t *device_bytes, uint64_t *host_bytes,
                           uint64_t *staging_bytes, uint64_t *copied_bytes);

/* Frees every device allocation of h (NULL is a no-op).  Synchronises the
 * device work of h first. */
void amg_destroy(amg_hierarchy *h);

/* Text of the last CUDA runtime error behind an AMG_ERR_CUDA or AMG_ERR_OOM
 * returned to the calling thread, with the library source file and line of
 * the call that reported it where known ("no CUDA error" if none).  The text
 * stays valid until the thread's next call into the library. */
const char *amg_last_cuda_error(void);

/* Static English text for a status code. */
const char *amg_status_string(amg_status s);

#ifdef __cplusplus
}
#endif

#endif /* AMG_GB300_H */
