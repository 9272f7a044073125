/*
 * otgs.h -- C ABI of the GB300 (sm_103a) solver for discrete optimal
 * transport with the squared-L2 + group-lasso regulariser.
 *
 * Method: Ida et al., "Fast Regularized Discrete Optimal Transport with
 * Group-Sparse Regularizers" (AAAI 2023).  The library maximises the smooth
 * relaxed dual (Eq. 4)
 *
 *     D(alpha, beta) = alpha.a + beta.b - sum_j psi(alpha + beta_j 1_m - c_j)
 *
 * whose gradient comes from the group soft-threshold of Eq. 5,
 *
 *     grad psi(f)_[l] = ([z - mu gamma]_+ / (gamma z)) [f_[l]]_+,
 *     z = ||[f_[l]]_+||,   psi_[l] = [z - mu gamma]_+^2 / (2 gamma),
 *
 * with the safe skipping of zero blocks (Def. 1, Eq. 6, Lemma 2), the set of
 * surely-nonzero blocks (Def. 2-3, Eq. 7-8) and the outer loop of Alg. 1 around
 * an L-BFGS loop that runs entirely on the device.
 *
 * Conventions for every entry point:
 *  - Pointers documented "device" must be device memory of the current CUDA
 *    device (e.g. PyTorch tensors' data_ptr()); "host" pointers are ordinary
 *    host memory.  Nothing takes ownership of caller memory.
 *  - Every call enqueues its work on the handle's stream (a cudaStream_t
 *    passed as void*; NULL = the legacy default stream) and, unless stated
 *    otherwise, returns without synchronising.
 *  - Return value: OTGS_OK (0) or a negative ot_gs_status.  The message of
 *    the last failure on a handle is available from ot_gs_last_error().
 *  - Floating point: C is FP32; a, b, alpha, beta, gradients and D are FP64.
 *    Kernels compute in FP32 with error-free (double-float) transformations
 *    where cancellation demands it, and accumulate in FP64.
 */
#ifndef OTGS_H
#define OTGS_H

#include <stdint.h>

#if defined(__GNUC__)
#define OTGS_API __attribute__((visibility("default")))
#else
#define OTGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ot_gs ot_gs; /* opaque handle */

typedef enum {
    OTGS_OK = 0,
    OTGS_EINVAL = -1,        /* invalid argument (sizes, labels, gamma, mu, marginals, NULL) */
    OTGS_ECUDA = -2,         /* a CUDA runtime call failed (message in ot_gs_last_error) */
    OTGS_ENOMEM = -3,        /* device or host allocation failed */
    OTGS_ENOTCONV = -4,      /* ot_gs_solve stopped at maxit before ||grad D||_inf <= tol */
    OTGS_ETIMEOUT = -5,      /* ot_gs_solve stopped at its time budget */
    OTGS_ELINESEARCH = -6,   /* the line search found no acceptable step */
    OTGS_ENONFINITE = -7     /* non-finite input (C, a, b, alpha, beta) */
} ot_gs_status;

/* Solver parameters (ot_gs_set_params / ot_gs_get_params). */
typedef struct {
    double gamma;          /* gamma > 0 of Eq. 3 */
    double mu;             /* mu >= 0 of Eq. 3; the threshold is theta = mu gamma */
    int32_t r;             /* accepted iterations between snapshot refreshes (Alg. 1; paper: 10) */
    int32_t lbfgs_m;       /* L-BFGS memory (pairs), 1..32, default 10 */
    int32_t use_screening; /* 1: Alg. 1/2 screened evaluations in ot_gs_solve; 0: dense */
    int32_t use_lower_bound; /* 1: build the set N of Def. 3 every r iterations */
    double time_budget_ms; /* <= 0: none; else ot_gs_solve stops with OTGS_ETIMEOUT */
    double ftol;           /* > 0: a solve (single or batched) also stops, with OTGS_OK, after an
                              accepted iteration that raised D by at most ftol max(|D_old|, |D_new|)
                              (objective stagnation); 0 (default): off */
} ot_gs_params;

/* Counters, cumulative since create (or since ot_gs_reset_stats). */
typedef struct {
    int64_t evals;            /* dual evaluations (line-search trials included) */
    int64_t iters;            /* accepted L-BFGS iterations of the last solve */
    int64_t blocks_total;     /* (l, j) blocks visited by all evaluations = evals * L * n */
    int64_t blocks_in_N;      /* blocks computed because (l, j) in N (Alg. 2, first loop) */
    int64_t blocks_skipped;   /* blocks with zbar <= theta (Alg. 2, zero without computing) */
    int64_t blocks_checked;   /* upper bounds evaluated (blocks outside N) */
    int64_t units_total;      /* (group, 32-column tile) units visited = evals * L * ceil(n/32) */
    int64_t units_computed;   /* units whose C tile was streamed */
    int64_t snapshots;        /* snapshot refreshes (dense passes) */
    double  c_bytes;          /* bytes of C streamed by evaluation kernels */
    int64_t kernels;          /* kernels launched by ot_gs_grad / ot_gs_grad_screened calls */
    int64_t blocks_flagged;   /* blocks formed exactly (Eq. 5): those whose FP32 bound left s > 0
                                 possible, or, on a screened evaluation's block-set route, those the
                                 screen left */
} ot_gs_stats;

/*
 * Create a problem (Sec. 2.1-2.3).
 *   h       out: new handle
 *   C       device, FP32, m x n, row i at C + i*ldc (ldc >= n), c_ij >= 0, finite.
 *           Borrowed when the labels are non-decreasing, ldc % 4 == 0 and C is
 *           16-byte aligned (the layout TMA reads); the caller then keeps it alive
 *           and unchanged until ot_gs_destroy.  Otherwise the library keeps a
 *           class-sorted copy.
 *   a, b    device, FP64, m and n positive marginals with |sum a - sum b| <=
 *           1e-12 max(sum a, 1) (Sec. 2.1 uses 1/m and 1/n); copied.
 *   labels  device, int32, m class labels in [0, L) (the groups of Eq. 3); copied.
 *   gamma, mu  regularisation of Eq. 3 (gamma > 0, mu >= 0)
 *   stream  cudaStream_t (as void*) on which all later work is enqueued
 * Synchronises the stream once (validation and the group plan are built on
 * the host).  Errors: OTGS_EINVAL, OTGS_ENONFINITE, OTGS_ENOMEM, OTGS_ECUDA;
 * *h is NULL on failure.
 */
OTGS_API int ot_gs_create(ot_gs **h, const float *C, int64_t ldc, const double *a, const double *b,
                 const int32_t *labels, int64_t m, int64_t n, int32_t L, double gamma,
                 double mu, void *stream);

/*
 * A column shard of a problem (the multi-GPU split of the dual over target
 * columns, Eq. 4-5): C holds the columns J of the full cost matrix (m x |J|),
 * b the marginal b_J of those columns, a the whole a; everything else as
 * ot_gs_create, except that sum b_J need not equal sum a.  Its evaluations
 * (ot_gs_grad, ot_gs_grad_screened) give D_J = alpha.a + beta_J.b_J - sum
 * over j in J of psi, the alpha gradient a - sum_{j in J} t_.j and the beta_J
 * gradient.  Over shards J_1..J_P of all columns: D = sum_p D_Jp - (P - 1)
 * alpha.a and grad_alpha = sum_p grad_alpha_p - (P - 1) a (one sum across the
 * GPUs per evaluation); the beta gradients are the shards' own.  ot_gs_solve
 * rejects a shard handle (OTGS_EINVAL): its objective is partial.
 */
OTGS_API int ot_gs_create_shard(ot_gs **h, const float *C, int64_t ldc, const double *a, const double *b,
                 const int32_t *labels, int64_t m, int64_t n, int32_t L, double gamma,
                 double mu, void *stream);

/* Release every resource of the handle (synchronises its stream).  NULL is a no-op. */
OTGS_API int ot_gs_destroy(ot_gs *h);

/* Replace the stream used by later calls. */
OTGS_API int ot_gs_set_stream(ot_gs *h, void *stream);

OTGS_API int ot_gs_set_params(ot_gs *h, const ot_gs_params *p); /* host struct; validates */
OTGS_API int ot_gs_get_params(const ot_gs *h, ot_gs_params *p); /* host struct */

/*
 * One dense evaluation of the dual objective and its gradient (Eq. 4, Eq. 5;
 * gradient by Danskin's theorem, Sec. 2.3):
 *   alpha   device FP64 [m], caller's row order
 *   beta    device FP64 [n]
 *   out     device FP64 [1 + m + n]: out[0] = D(alpha, beta),
 *           out[1 + i] = dD/dalpha_i = a_i - sum_j t_ij,
 *           out[1 + m + j] = dD/dbeta_j = b_j - sum_i t_ij
 * Asynchronous.  Reads all of C once.  Errors: OTGS_EINVAL, OTGS_ECUDA.
 */
OTGS_API int ot_gs_grad(ot_gs *h, const double *alpha, const double *beta, double *out);

/*
 * Same evaluation, screened by the upper bound of Eq. 6 against the handle's
 * current snapshot and set N (Alg. 2): blocks with zbar <= theta are not read
 * and contribute exact zeros.  The result equals ot_gs_grad bit for bit
 * (Thm. 2; the skip test keeps a margin that covers the kernels' rounding).
 * skip_mask (device, optional, NULL to ignore) receives the per-block skip
 * decisions as L x ceil(n/32) uint32 words, bit (j % 32) of word
 * [l * ceil(n/32) + j / 32] set when block (l, j) was skipped.
 */
OTGS_API int ot_gs_grad_screened(ot_gs *h, const double *alpha, const double *beta, double *out,
                        uint32_t *skip_mask);

/*
 * Refresh the snapshot at (alpha, beta) (Alg. 1's snapshot update): one dense pass that
 * also stores z~_{l,j} (rounded up to FP32) and o~_{l,j}, and alpha~ = alpha,
 * beta~ = beta; then one pass over z~ forms each 32-column tile's largest
 * z~, with which the screened evaluation first tests whole tiles (the same
 * skip decisions as block by block, fewer bytes read).  When build_N != 0 the set N (Def. 3, Eq. 8) is first rebuilt
 * from the lower bound of Eq. 7 against the previous snapshot (Alg. 1's
 * rebuild of N).  Writes D and the gradient to out like ot_gs_grad when out != NULL.
 */
OTGS_API int ot_gs_snapshot(ot_gs *h, const double *alpha, const double *beta, int build_N, double *out);

/*
 * Copy the screening state for inspection (any pointer may be NULL); all are
 * device pointers.  zt, ot: FP32 [L * ceil(n/32)*32] (row l = group, padded
 * columns undefined); alpha_s: FP64 [m] caller order; beta_s: FP64 [n];
 * N_mask: uint32 [L * ceil(n/32)] bitmask of the set N.
 */
OTGS_API int ot_gs_get_screen_state(ot_gs *h, float *zt, float *ot, double *alpha_s, double *beta_s,
                           uint32_t *N_mask);

/*
 * Solve max D with L-BFGS (memory lbfgs_m) and a strong-Wolfe line search,
 * from the handle's current iterate (zero after create, as Alg. 1 starts; or the
 * point given to ot_gs_set_state).  With use_screening = 1 each evaluation is
 * screened (Alg. 2) and every r accepted iterations N and the snapshot are
 * rebuilt (Alg. 1).  The whole iteration -- line search, evaluation, the
 * L-BFGS update and the convergence test -- runs on the device; the host
 * waits once at the end.  Stops when ||grad D||_inf <= tol.
 * Returns OTGS_OK, OTGS_ENOTCONV (maxit), OTGS_ETIMEOUT, OTGS_ELINESEARCH,
 * OTGS_ENONFINITE (D or the gradient at the start point is not finite, e.g.
 * a NaN in the state set by ot_gs_set_state), or an error.  Synchronises the
 * stream.
 */
OTGS_API int ot_gs_solve(ot_gs *h, double tol, int32_t maxit);

/*
 * Current iterate: alpha (device FP64 [m], caller order), beta (device FP64
 * [n]); D, grad_inf (host, FP64) and iters (host) may be NULL.  Synchronises.
 */
OTGS_API int ot_gs_get_solution(ot_gs *h, double *alpha, double *beta, double *D, double *grad_inf,
                       int32_t *iters);

/*
 * Objective trace of the last ot_gs_solve: entry 0 is the start point, entry
 * k the k-th accepted iteration.  D[k] is the dual objective there, t_ms[k]
 * the device time (globaltimer) since the solve was launched, including the
 * host round trips of the line search, evals[k] the evaluations so far.  Up
 * to cap entries are written to the HOST arrays; *count (may be NULL) gets
 * the number recorded (at most 65536).  Synchronises.
 */
OTGS_API int ot_gs_get_trace(ot_gs *h, double *D, double *t_ms, int64_t *evals, int32_t cap, int32_t *count);

/* Set the iterate used by the next ot_gs_solve (warm start or resume) and
 * clear the L-BFGS memory.  alpha, beta: device FP64 [m], [n], caller order. */
OTGS_API int ot_gs_set_state(ot_gs *h, const double *alpha, const double *beta);

/*
 * Checkpoint and resume of ot_gs_solve (Alg. 1's loop state).  A saved state
 * holds everything an unfinished solve goes on with: the L-BFGS state (the
 * iterate x = (alpha, beta), the gradient, the next search direction, the
 * stored pairs (s_k, y_k) and their curvature matrices, the line search's
 * scalars, the iteration and evaluation counters) and, when the handle holds
 * a snapshot, the screening state of Alg. 1 (z~, o~, alpha~, beta~ and the
 * set N).
 *   ot_gs_state_size     *bytes (host) = size of the state of h, for a buffer
 *   ot_gs_get_state      copies the state of h into dst (device, >= that
 *                        size); needs a solver (after ot_gs_solve or
 *                        ot_gs_set_state); synchronises
 *   ot_gs_restore_state  loads a state saved from a handle of the same problem
 *                        (same m, n, classes, lbfgs_m, gamma and mu; the
 *                        caller keeps C, a, b the same) into h; the next
 *                        ot_gs_solve continues it: maxit then counts the
 *                        iterations of the whole solve, the restored ones
 *                        included, and the iterates are bit for bit those of
 *                        a solve that was never stopped (dense or screened,
 *                        with the same parameters).  Its trace starts at the
 *                        restored iterate.  Synchronises.
 * ot_gs_set_state (a warm start) drops a restored state.  Errors: OTGS_EINVAL
 * (no solver, short buffer, a state of another problem), OTGS_ECUDA.
 */
OTGS_API int ot_gs_state_size(ot_gs *h, int64_t *bytes);
OTGS_API int ot_gs_get_state(ot_gs *h, void *dst, int64_t bytes);
OTGS_API int ot_gs_restore_state(ot_gs *h, const void *src, int64_t bytes);

OTGS_API int ot_gs_get_stats(ot_gs *h, ot_gs_stats *s); /* host struct; synchronises */
OTGS_API int ot_gs_reset_stats(ot_gs *h);

/*
 * Test hooks: each changes the evaluations issued after it on this handle
 * (ot_gs_grad, ot_gs_grad_screened, ot_gs_snapshot, ot_gs_solve).
 *   OTGS_DEBUG_STALL: value in (0, 1e10] makes the evaluation kernel's
 *     consumer warps stop releasing their stages and its ring waits give up
 *     after value ns: the producer then waits (at the normal 2 s limit) for
 *     the copies it issued, the kernel records an error and returns, and D
 *     comes out NaN.  The handle's error word stays set: later evaluations
 *     of this handle give NaN too.  value <= 0 restores normal operation.
 *   OTGS_DEBUG_NAN_EVAL: value > 0 makes ot_gs_solve read the objective of
 *     its value-th evaluation and of every later one as NaN (a fake of a
 *     failing evaluation): the line search finds no acceptable step and the
 *     solve returns OTGS_ELINESEARCH (value 1, the start point: ENONFINITE).
 *     value <= 0: off.
 *   OTGS_DEBUG_SCREEN_ROUTE: the route of screened evaluations: 0 (the
 *     default) lets each evaluation choose, 1 always runs the bound pass over
 *     the needed tiles, 2 always reads the blocks the screen left from the
 *     transposed copy.  Both routes give the same bits.
 * Host only, no synchronisation.  Errors: OTGS_EINVAL (unknown switch, a
 * limit above 10 s).
 */
#define OTGS_DEBUG_STALL 2
#define OTGS_DEBUG_NAN_EVAL 3
#define OTGS_DEBUG_SCREEN_ROUTE 4
OTGS_API int ot_gs_debug(ot_gs *h, int what, int64_t value);

/*
 * Kernel timing for benchmarks: while enabled (enable != 0), every launch of
 * the evaluation kernel is bracketed by CUDA events on the handle's stream.
 * ot_gs_get_timing synchronises the stream and returns the number of timed
 * launches and their summed device time in milliseconds, then clears them.
 */
OTGS_API int ot_gs_set_timing(ot_gs *h, int enable);
OTGS_API int ot_gs_get_timing(ot_gs *h, int64_t *launches, double *total_ms);

/* Message of the last failure on h (or of the last failed ot_gs_create when
 * h is NULL).  Never NULL; valid until the next call on the handle. */
OTGS_API const char *ot_gs_last_error(const ot_gs *h);

/* Library version string, e.g. "otgs 0.1 sm_103a". */
OTGS_API const char *ot_gs_version(void);

/*
 * Host-only inspection of the group plan the library builds at create (no
 * GPU needed): for m labels in [0, L) and n columns, writes the number of
 * panels (row ranges of whole groups), of (panel, 256-column chunk) work
 * items, and of the 32-row shared-memory stages one dense evaluation streams.
 * Returns OTGS_EINVAL on bad input.  Used to test the host-side work
 * decomposition.
 */
OTGS_API int ot_gs_plan_info(const int32_t *labels_host, int64_t m, int64_t n, int32_t L,
                    int64_t *n_panels, int64_t *n_items, int64_t *n_stages);

/*
 * Downstream use of a solution (single-problem handles).
 * ot_gs_plan: the transport plan at (alpha, beta), t = grad psi (Sec. 2.3,
 * Eq. 5): t_ij = s_lj [alpha_i + beta_j - c_ij]_+ with s_lj = [z - mu gamma]_+
 * / (gamma z) of the block's positive part.  alpha: device FP64 [m] (caller
 * order), beta: device FP64 [n]; T: device FP32, m x n, row i (caller order)
 * at T + i*ldt (ldt >= n).  f is formed in FP64.
 * ot_gs_barycentric: the mapping of Sec. 2.1, out = n T^T X_S (device FP32,
 * n x d row-major): target sample j's image is n sum_i t_ij x_i; XS: device
 * FP32 m x d row-major (caller row order).  Uses m x n FP32 of scratch.
 * Both synchronise.  Errors: OTGS_EINVAL, OTGS_ENOMEM, OTGS_ECUDA.
 */
OTGS_API int ot_gs_plan(ot_gs *h, const double *alpha, const double *beta, float *T, int64_t ldt);
OTGS_API int ot_gs_barycentric(ot_gs *h, const double *alpha, const double *beta, const float *XS, int32_t d,
                               float *out);

/* ------------------------------------------------------------------------
 * Batches: many independent problems in one handle.  The paper solves one
 * problem at a time; a batch evaluates all of its problems with one launch of
 * the evaluation kernel (each problem's rows only meet its own columns) and
 * solves them with one L-BFGS state per problem, each following exactly the
 * iteration ot_gs_solve would follow alone.
 *
 * Layout of batch vectors ("concatenated"): problem k's alpha occupies
 * entries [row_off_k, row_off_k + m_k) in its caller row order, and its beta
 * entries [col_off_k, col_off_k + n_k), where row_off_k = m_0 + ... + m_{k-1}
 * and col_off_k = n_0 + ... + n_{k-1}.  A gradient vector holds the alpha
 * part (sum m_k entries) followed by the beta part (sum n_k entries).
 * ------------------------------------------------------------------------ */

/*
 * Create a batch of nprob >= 1 problems.  C, ldc, a, b, labels, m, n, L are
 * HOST arrays of nprob entries; each C[k], a[k], b[k], labels[k] is a device
 * pointer with the meaning, requirements and borrowing rule of ot_gs_create
 * for problem k.  gamma, mu are shared.  A batch handle accepts the ot_gs_batch_*
 * calls, the plan calls and the parameter, statistics and timing calls; the
 * single-problem evaluation, screening and solve calls reject it with
 * OTGS_EINVAL unless nprob == 1.  Synchronises the stream.  Errors as
 * ot_gs_create (the message names the problem).
 */
OTGS_API int ot_gs_create_batch(ot_gs **h, int32_t nprob, const float *const *C, const int64_t *ldc,
                                const double *const *a, const double *const *b, const int32_t *const *labels,
                                const int64_t *m, const int64_t *n, const int32_t *L, double gamma, double mu,
                                void *stream);

/* Number of problems and total rows / columns (any pointer may be NULL; host).
 * A handle from ot_gs_create is a batch of one. */
OTGS_API int ot_gs_batch_size(const ot_gs *h, int32_t *nprob, int64_t *m_total, int64_t *n_total);

/*
 * Dense evaluation of every problem of the batch (Eq. 4, Eq. 5), one launch
 * of the evaluation kernel for all of them:
 *   alpha, beta  device FP64, concatenated layout
 *   D            device FP64 [nprob]: D_k(alpha_k, beta_k)
 *   grad         device FP64 [sum m + sum n] (may be NULL): dD_k/dalpha_k
 *                then dD_k/dbeta_k in the concatenated layout
 * Asynchronous.  Errors: OTGS_EINVAL, OTGS_ECUDA.
 */
OTGS_API int ot_gs_batch_grad(ot_gs *h, const double *alpha, const double *beta, double *D, double *grad);

/*
 * Solve every problem of the batch: per problem the L-BFGS iteration of
 * ot_gs_solve (dense evaluations, memory lbfgs_m) from the batch iterate
 * (zero after create, or the point given to ot_gs_batch_set_state).  Problem
 * k stops when ||grad D_k||_inf <= tol, or (target_D != NULL) when D_k >=
 * target_D[k] - target_rtol |target_D[k]|, or at maxit accepted iterations,
 * or when its line search fails; stopped problems drop out of the following
 * evaluations.  The trials run in CUDA graphs of 16 trials captured once per
 * handle and relaunched until every problem has stopped; the host only reads
 * the count of running problems between graph launches.
 *   target_D  HOST FP64 [nprob] or NULL
 * Returns OTGS_OK when every problem stopped on tol or its target, else the
 * status of the first problem that did not (OTGS_ENOTCONV,
 * OTGS_ELINESEARCH), or an error.  Synchronises.
 */
OTGS_API int ot_gs_batch_solve(ot_gs *h, double tol, int32_t maxit, const double *target_D, double target_rtol);

/*
 * Best common shift of each problem's alpha: alpha_k += k_k, k_k the
 * maximiser of the concave D_k(alpha_k + k 1, beta_k) (D is unchanged by
 * alpha + k, beta - k, so this is the best point on that line through a
 * predicted start).  A bracket is doubled from [-1/16, 1/16] until it holds
 * the maximiser, then halved; each of the `iters` (1..200) steps is one
 * batch evaluation.  alpha: device FP64, concatenated layout, updated in place;
 * beta: device FP64.  Synchronises.
 */
OTGS_API int ot_gs_batch_shift(ot_gs *h, double *alpha, const double *beta, int32_t iters);

/* Set the batch iterate used by the next ot_gs_batch_solve (warm start):
 * device FP64, concatenated layout.  Clears each problem's L-BFGS memory. */
OTGS_API int ot_gs_batch_set_state(ot_gs *h, const double *alpha, const double *beta);

/*
 * Results of the last ot_gs_batch_solve.  alpha, beta: device FP64
 * (concatenated layout; both or neither).  HOST arrays of nprob entries (each
 * may be NULL): D at the final iterate, ||grad D||_inf there, accepted
 * iterations, status, evaluations (line-search trials included) and t_ms, the
 * device time from the start of the solve to the problem's stop.
 * Synchronises.
 */
OTGS_API int ot_gs_batch_result(ot_gs *h, double *alpha, double *beta, double *D, double *grad_inf,
                                int32_t *iters, int32_t *status, int64_t *evals, double *t_ms);

/*
 * Plan shape.  panel_rows: rows of whole class groups per work item (an item
 * is panel x 256 columns); split_rows: groups taller than this are cut into
 * pieces of this height, summed by different CTAs; stage_fill: 0 = C streams
 * in stages of 32 rows, k > 0 = a stage ends early, before a group of at most
 * 32 rows that would straddle its end, when it keeps at least k rows (such a
 * group's blocks are then bounded within one stage).  ot_gs_set_plan rebuilds the handle's plan (0 = the
 * default of each) and synchronises; valid ranges are [32, 4096], [64, 8192]
 * and [0, 32].  ot_gs_get_plan reports the current shape and the number of
 * work items (host pointers, each may be NULL).
 */
OTGS_API int ot_gs_set_plan(ot_gs *h, int32_t panel_rows, int32_t split_rows, int32_t stage_fill);
OTGS_API int ot_gs_get_plan(const ot_gs *h, int32_t *panel_rows, int32_t *split_rows, int32_t *stage_fill,
                            int64_t *n_items);

/*
 * Autotuner of the plan shape: times `evals` dense evaluations of all the
 * handle's problems at (alpha, beta) (device FP64, concatenated layout; the
 * cost depends on how many blocks are positive there, so pass a point like
 * those the solver visits) for each candidate (panel_rows in {32, ..., 1024},
 * split_rows in {128, ..., 1024}, stage_fill in {0, 16}), and keeps the
 * fastest.  The choice is
 * cached for the process under a key of the group-size histogram (share of
 * rows per power-of-two size class) and the size classes of the column count
 * per problem, the row count and the number of problems; a cached shape is
 * applied without measuring (*best_ms = 0).  Outputs are host pointers (each
 * may be NULL).  Synchronises.  ot_gs_autotune_clear_cache forgets all shapes.
 */
OTGS_API int ot_gs_autotune(ot_gs *h, const double *alpha, const double *beta, int32_t evals,
                            int32_t *panel_rows, int32_t *split_rows, int32_t *stage_fill, double *best_ms);
OTGS_API int ot_gs_autotune_clear_cache(void);

/* Host-only plan of a batch (no GPU needed), as ot_gs_plan_info: labels_host,
 * m, n, L are host arrays of nprob entries (labels_host[k]: host int32 [m[k]]);
 * panel_rows, split_rows, stage_fill as ot_gs_set_plan (0 = default). */
OTGS_API int ot_gs_plan_info_batch(int32_t nprob, const int32_t *const *labels_host, const int64_t *m,
                                   const int64_t *n, const int32_t *L, int32_t panel_rows, int32_t split_rows,
                                   int32_t stage_fill, int64_t *n_panels, int64_t *n_items, int64_t *n_stages);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper).  A 3-layer perceptron
 * maps per-sample features of a problem to initial duals; the zero start
 * stays the fallback and the yardstick (the solve from a warm start must
 * reach the same objective).  Network, for in_dim K and width H (multiples of 16):
 *   Z1 = q(X) q(W1)^T + b1, A1 = relu(Z1), Z2 = q(A1) q(W2)^T + b2,
 *   A2 = relu(Z2), y = q(A2) q(w3) + b3,
 * q = rounding to bfloat16 (the tensor-core operands; FP32 accumulation).
 * Parameters are FP32 master copies in one flat array:
 *   [W1 (H x K, row-major), b1 (H), W2 (H x H), b2 (H), w3 (H), b3 (1)].
 * Training minimises mean (y - t)^2 with Adam.
 * ------------------------------------------------------------------------ */
typedef struct ot_gs_mlp ot_gs_mlp;

/* New network with He-uniform weights from SplitMix64(seed) (biases 0) and
 * buffers for batches of up to max_batch samples; work goes to `stream`.
 * Synchronises once.  Errors: OTGS_EINVAL, OTGS_ENOMEM, OTGS_ECUDA. */
OTGS_API int ot_gs_mlp_create(ot_gs_mlp **h, int32_t in_dim, int32_t width, int64_t max_batch, uint64_t seed,
                              void *stream);
OTGS_API int ot_gs_mlp_destroy(ot_gs_mlp *h);
OTGS_API int ot_gs_mlp_num_params(const ot_gs_mlp *h, int64_t *n); /* host out */
/* Copy the flat FP32 parameters in (device; clears Adam's moments and step)
 * or out (device). */
OTGS_API int ot_gs_mlp_set_params(ot_gs_mlp *h, const float *p);
OTGS_API int ot_gs_mlp_get_params(ot_gs_mlp *h, float *p);
/* y[b] for the B rows of X (device FP32, B x in_dim, row-major); 0 < B <= max_batch. */
OTGS_API int ot_gs_mlp_forward(ot_gs_mlp *h, const float *X, int64_t B, float *y);
/* Loss and gradient at targets t (device FP32 [B]): loss (device FP32 scalar,
 * may be NULL) = mean (y - t)^2; grad (device FP32 flat, may be NULL) receives
 * the gradient, which is also kept for ot_gs_mlp_adam. */
OTGS_API int ot_gs_mlp_grad(ot_gs_mlp *h, const float *X, const float *t, int64_t B, float *loss, float *grad);
/* One Adam step (Kingma & Ba) with the gradient of the last ot_gs_mlp_grad. */
OTGS_API int ot_gs_mlp_adam(ot_gs_mlp *h, float lr, float beta1, float beta2, float eps);
/*
 * Input features of one problem: out (device FP32, (m + n) x in_dim) gets one
 * row per source sample, then one per target sample:
 *   source i of class l: [0, min_j c_ij, mean_j c_ij, sm_0.02, sm_0.1, g_l / m, wl_0.5, wl_1, wl_2, x_i, mu_l]
 *   target j:            [1, min_i c_ij, mean_i c_ij, sm_0.02, sm_0.1, g_k / m, wl_0.5, wl_1, wl_2, y_j, mu_k]
 * and zeros up to in_dim (>= 9 + 2 d).  mu_l = mean source feature of class l,
 * g_l its size, k the non-empty class whose mean is nearest to y_j (FP32
 * squared distance, terms in index order, ties to the lower class), sm_tau(v)
 * = -tau log mean exp(-v / tau), wl_s = the level L with sum [L - v]_+ =
 * s gamma / m over the row (s gamma / n over the column; by Newton steps).
 * C: device FP32 m x n (row stride ldc); XS: device FP32 m x d; XT: device
 * FP32 n x d; labels: device int32 [m] in [0, L); gamma > 0.
 */
OTGS_API int ot_gs_mlp_features(const float *C, int64_t ldc, int64_t m, int64_t n, const float *XS, const float *XT,
                                int32_t d, const int32_t *labels, int32_t L, float gamma, int32_t in_dim, float *out,
                                void *stream);
/* The same features for nprob problems in one launch: C, ldc, m, n, XS, XT,
 * labels, L are HOST arrays of nprob entries (pointers to device data as
 * above).  out (device FP32) gets the source rows of every problem in
 * concatenated order (sum m rows), then the target rows (sum n rows): the
 * network's output is then alpha, then beta, in the batch layout. */
OTGS_API int ot_gs_mlp_features_batch(int32_t nprob, const float *const *C, const int64_t *ldc, const int64_t *m,
                                      const int64_t *n, const float *const *XS, const float *const *XT, int32_t d,
                                      const int32_t *const *labels, const int32_t *L, float gamma, int32_t in_dim,
                                      float *out, void *stream);
/* Second-pass inputs of the warm start (from a first prediction): for
 * nprob problems (C, ldc, m, n HOST arrays as for ot_gs_mlp_features_batch)
 * and the first pass's duals alpha_hat (device FP32, sum m, batch layout) and
 * beta_hat (device FP32, sum n), writes columns [col0, col0 + 4) of every row
 * of out (device FP32, (sum m + sum n) x in_dim, the layout of
 * ot_gs_mlp_features_batch; other columns are left as they are): for source
 * row i, wl_s of the values c_ij - beta_hat_j over the problem's columns
 * (masses s gamma / m, s = 0.5, 1, 2; differences in FP32) and alpha_hat_i;
 * for target column j, wl_s of c_ij - alpha_hat_i over its rows (masses
 * s gamma / n) and beta_hat_j.  Needs 0 <= col0 <= in_dim - 4, gamma > 0. */
OTGS_API int ot_gs_mlp_refine_features(int32_t nprob, const float *const *C, const int64_t *ldc, const int64_t *m,
                                       const int64_t *n, const float *alpha_hat, const float *beta_hat, float gamma,
                                       int32_t col0, int32_t in_dim, float *out, void *stream);
/* Message of the last failure on h (NULL: of the last failed create or features call). */
OTGS_API const char *ot_gs_mlp_last_error(const ot_gs_mlp *h);

/*
 * Allocation-free dense evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code running
 * inside a custom device allocator's callbacks, frameworks whose memory pool
 * forbids allocations outside the pool, loops that cannot afford cudaMalloc's
 * implicit synchronisation.  It computes what ot_gs_grad computes without a
 * handle and calls no cudaMalloc, cudaFree or other allocating routine: all
 * scratch (plan, partial sums, reduction state) lives in one static device
 * array of OTGS_STATIC_SCRATCH_BYTES bytes that every GPU loading this part of
 * the library keeps until the process exits.
 *   C            device FP32, m x n, row stride ldc; rows class-sorted
 *                (labels_host non-decreasing); ldc % 4 == 0 and C 16-byte
 *                aligned (no sorted copy can be made without allocating)
 *   a, b         device FP64 marginals [m], [n]
 *   labels_host  HOST int32 [m], non-decreasing, values in [0, L)
 *   alpha, beta  device FP64 [m], [n];  out: device FP64 [1 + m + n] as ot_gs_grad
 *   stream       cudaStream_t as void*
 * Inputs are not otherwise validated.  The scratch a problem needs is 52
 * bytes per row, 16 per column (rounded up to a multiple of 256 columns), 64
 * per work item (a panel of whole classes, up to 512 rows, x 256 columns), 32
 * per (non-empty class, 32-column tile), and 2 KB per 256-row piece x 256
 * columns of every class taller than 256 rows; the Zipf-class workload at m
 * = n = 2 x 10^4 needs about 30 MB.  Larger problems are rejected with
 * OTGS_EINVAL before any GPU work; the message says how many
 * bytes were needed.  The first call made on a device looks up the array's
 * device address there (once per device).  Each call uploads its plan with
 * cudaMemcpyAsync from pageable host memory, which the runtime stages
 * synchronously: the call returns once its inputs are staged, the host waits
 * for work already queued on the stream before the copy, and the call must
 * not be made while the stream is being captured into a CUDA graph.  Every
 * call shares the array and leaves the last call's contents in it (the values
 * that must start at zero are cleared by each call); calls that overlap on
 * the GPU race with each other.
 * Asynchronous with respect to the host.  Errors: OTGS_EINVAL, OTGS_ECUDA;
 * message from ot_gs_noalloc_last_error().
 */
#define OTGS_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
OTGS_API int ot_gs_grad_noalloc(const float *C, int64_t ldc, const double *a, const double *b,
                                const int32_t *labels_host, int64_t m, int64_t n, int32_t L, double gamma,
                                double mu, const double *alpha, const double *beta, double *out, void *stream);
OTGS_API const char *ot_gs_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OTGS_H */
