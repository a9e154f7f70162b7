/*
 * gabp.h -- C ABI of the GB300 (sm_103a) Gaussian belief propagation solver.
 *
 * The solver computes x = A^{-1} b for a sparse symmetric A by synchronous
 * Gaussian belief propagation (GaBP), the message-passing method of
 * D. Bickson, "Gaussian Belief Propagation: Theory and Application":
 *   - the linear system is read as a Gaussian Markov random field whose
 *     marginal means are A^{-1} b (Sec. "From Linear Algebra to Probabilistic
 *     Inference", Proposition on linear systems and inference);
 *   - every directed edge i->j carries a precision message P_ij and a mean
 *     message mu_ij (eq_prec_message, eq_mean_message; Algorithm 1);
 *   - each message is node i's aggregate minus the reverse message j->i, the
 *     broadcast form (Algorithm 2, Sec. "GaBP Broadcast Variant");
 *   - by default all messages of a round are computed from the previous
 *     round's messages (parallel / synchronous schedule); the serial schedule
 *     (one store updated in place, nodes firing colour by colour) is an
 *     option (Sec. "The Gaussian BP Algorithm", scheduling paragraph);
 *   - options add Aitken's method or Steffensen's iterations on the marginal
 *     means (Sec. "Convergence Acceleration") and the convergence fix for
 *     non-walk-summable A, as a double loop or a damped single loop (Chapter
 *     "Fixing convergence of GaBP");
 *   - rectangular systems: regularised least squares through the symmetric
 *     augmented system (Sec. "Extension to General Linear Systems");
 *   - the answer is the marginal mean vector and, optionally, the marginal
 *     precisions (Algorithm 1, steps 4-5);
 *   - the messages are the solver's state: they can be exported and loaded
 *     (checkpoint / resume, warm starts), a solve can start from a caller's
 *     iterate, and FP64 runs can record their residual per round.
 *
 * Conventions for every function below
 *   - Return value: a gabp_status.  Negative values are errors; on an error
 *     no output is written unless stated.
 *   - Device pointers are CUDA device (or managed) addresses on the device
 *     that was current when the handle was created.  Host pointers are plain
 *     host memory.  The caller owns every array it passes; the library copies
 *     what it keeps.
 *   - Work is enqueued on the handle's stream (gabp_create / gabp_set_stream).
 *     Solves synchronise on that stream before they return, because the
 *     convergence decision is read back to the host.
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - int32 indices: n < 2^31 and nnz < 2^31.
 */
#ifndef GABP_H_
#define GABP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gabp_handle_s *gabp_handle;

typedef enum {
  GABP_OK = 0,             /* converged: relative residual <= tol */
  GABP_NOT_CONVERGED = 1,  /* max_iter rounds ran; x holds the last iterate */
  GABP_DIVERGED = 2,       /* a non-finite value appeared; x holds the last finite-checked iterate */
  GABP_BREAKDOWN = 3,      /* a cavity precision P_{i\j} (or a marginal precision) was exactly 0 */
  GABP_TIMEOUT = 4,        /* a bounded device-side wait gave up (multi-system persistent kernel) */
  GABP_ERR_INVALID = -1,   /* bad argument or matrix (see gabp_create) */
  GABP_ERR_CUDA = -2,      /* a CUDA runtime call failed; gabp_last_error() has the text */
  GABP_ERR_NOMEM = -3      /* device allocation failed */
} gabp_status;

/* Message arithmetic of a solve. */
typedef enum {
  GABP_PREC_FP64 = 0,        /* plain FP64 GaBP: precision and mean messages in FP64 */
  GABP_PREC_FP32_REFINE = 1  /* FP32 precision and mean messages; FP64 residual r = b - A x and
                                update x += d (iterative refinement) are the only FP64 steps */
} gabp_precision;

/* How an FP64 round is organised on the GPU; both compute Algorithm 2 and give
 * the same iterates.  (The FP32 path always uses its own recompute form.) */
typedef enum {
  GABP_VARIANT_NODE = 0,  /* one fused kernel per round: a sub-warp per row gathers each sender's
                             aggregate and the reverse message, writes the row's in-messages, and
                             forms the row's aggregate, x and residual in the same pass */
  GABP_VARIANT_EDGE = 1   /* two kernels per round: one thread per directed edge computes its
                             message (aggregate minus reverse message), then a row kernel sums them */
} gabp_variant;

typedef struct {
  int variant;          /* gabp_variant, default GABP_VARIANT_NODE */
  int precision;        /* gabp_precision, default GABP_PREC_FP64 */
  int check_every;      /* rounds per convergence read-back (CUDA-graph replay length), default 16.
                           Plain FP64 solves (node variant, no acceleration) of graphs of at most
                           131,072 rows run every round in one launch that decides on the device
                           (up to 2,048 rows, or 4,096 in slices of at most 8 slots a row: one
                           thread-block cluster; above: a cooperative grid),
                           and do not use it; nor do FP64 serial-schedule solves of graphs of at
                           most 4,096 rows (2,048 with a mean degree of 8 or more, 1,024 with 24 or
                           more): one cluster runs every sweep (with Steffensen's step, where its
                           state fits in the cluster's shared memory) */
  int freeze_precisions;/* plain FP64 solves (node variant or serial schedule, no acceleration): 1 =
                           freeze the precision messages once they have stopped moving (on the serial
                           schedule "round" below reads "sweep").  Screen: after two consecutive
                           rounds in which no node's P~_i moved by more than 16 units in the last
                           place (~2^-48 relative), one round checks every precision message against its previous
                           round's the same way while it stores each edge's coefficient
                           -A_ki / P_k\i and each node's 1/P~; if none moved, later rounds update
                           the mean messages only (the precisions do not depend on b), else the
                           screen resumes.  Every round up to the stored one is bitwise the plain
                           solve's; after it x differs from the plain iterate by rounding only.
                           Pays on solves that need many more rounds than the precisions do
                           (FP64-bound rounds); the screen costs a few percent per round.  0 =
                           every round updates both (Algorithm 2 as printed).  The edge variant
                           and the accelerated solves ignore it (the FP32 path always freezes).
                           Default 0 */
  double inner_tol;     /* loosest target of an FP32 inner solve (relative change of its iterate); each
                           inner solve aims at min(inner_tol, max(1e-6, 0.1 tol ||b|| / ||r||)),
                           the reduction still needed.  Default 1e-4 */
  int inner_max_iter;   /* rounds per inner solve, default 400 */
  int max_refine;       /* refinement steps, default 30 */
  int gamma_mode;       /* convergence fix: 0 off, 1 Gamma = gamma * diag(A),
                           2 Gamma_ii = max(0, sum_j |A_ij| - A_ii) + gamma * A_ii; default 0 */
  double gamma;         /* loading parameter for gamma_mode, default 0.25 */
  int lanes;            /* lanes per row of the FP32 R = 1 round kernels (1..32, power of two; they
                           use at most 16); 0 = autotune.  The FP64 parallel rounds always run one
                           row per lane on a sliced layout (rows sorted by degree in windows of 4096,
                           slices of 32 rows) and ignore it */
  int profile;          /* 1: time every phase with CUDA events (read with gabp_profile_read), default 0 */
  int reuse_precisions; /* FP32 path: 1 keeps the converged precision messages of A for later
                           solves (they do not depend on b); 0 re-runs the precision phase in every
                           solve.  Default 1 */
  int multi_split;      /* gabp_solve_systems: systems with rows + off-diagonal entries >= this go to a
                           thread-block cluster, smaller ones to one block; 0 = autotune.  Default 0 */
  int prec_stop_log2;   /* FP32 precision phase stops at a max relative change <= 2^-prec_stop_log2 in
                           two consecutive rounds (10..23).  Default 16 */
  int multi_mode;       /* gabp_solve_systems kernel: 0 autotune, 1 grid-persistent (every round sweeps
                           all running systems; its shape autotuned over the row-CSR and the sliced
                           layouts), 2 cluster / single-block teams, 3 grid-persistent on the sliced
                           layout only (each system's rows sorted by degree and cut into 32-row
                           slices, one lane per row; built once per offsets array).  Default 0 */
  int overlap_precision; /* FP32_REFINE, one right-hand side: 1 = while the precisions converge, the
                           rounds update precision AND mean messages (Algorithm 2's full round), so
                           the first inner solve starts with the precision phase; 0 = precision-only
                           rounds first.  Default 1 */
  int device_loop;      /* FP32_REFINE, one right-hand side, no loading, profile 0: 1 = the whole
                           refinement loop (rounds, stop decisions, residuals, updates) runs as ONE
                           CUDA graph with conditional while/if nodes, no host round trip until the
                           result; 0 = host-driven batches of check_every rounds.  Default 1 */
  int schedule;         /* message schedule (Sec. "The Gaussian BP Algorithm", parallel vs serial):
                           0 parallel (synchronous, two stores); 1 serial (one store updated in place,
                           nodes firing colour by colour in a greedy index-order colouring; rounds then
                           count sweeps).  gabp_solve, FP64 and FP32_REFINE without loading.  Default 0 */
  int fix_single_loop;  /* convergence fix (gamma_mode != 0): 0 the double loop (inner GaBP solves on
                           A + Gamma, FP32 messages, FP64 outer steps); 1 the single loop of the same
                           chapter: one FP64 GaBP round on A + Gamma per outer step, the node potentials
                           moved by h <- (1 - s) h + s (b + Gamma x).  Default 0 */
  int accel;            /* Acceleration of plain FP64 GaBP (Sec. "Convergence Acceleration"),
                           node variant.  1 = Aitken's method on the marginal means, parallel
                           schedule only -- every node extrapolates its last three iterates,
                           y = x0 - (x1 - x0)^2 / (x2 - 2 x1 + x0); the stop rule and the answer
                           use y; the GaBP iteration is unchanged.  Pays on smooth problems (the
                           paper's Poisson example: 25 rounds instead of 134), not on rough
                           right-hand sides.  2 = Steffensen's iterations, parallel or serial
                           schedule: rounds (sweeps) pair into cycles; after a cycle's second
                           round the marginal-mean vector is extrapolated with one scalar step,
                           y = x2 - lam (x2 - x1), lam = <x2 - x1, D> / <D, D>,
                           D = x2 - 2 x1 + x0, and y replaces the iterate: the mean messages
                           move by the same step (h <- h2 - lam (h2 - h1); precisions kept),
                           which gives marginal means y once the precisions are stationary, and
                           GaBP runs on from there.  The iterate of a cycle's second round is the
                           extrapolated one.  Pays mostly on the serial schedule (32 x 32 grid:
                           37 sweeps instead of 59).  accel = 1 with schedule = 1 is
                           GABP_ERR_INVALID.  Default 0 */
  int unroll;           /* FP32 R = 1 round kernels with lanes pinned: slots per lane whose loads are
                           issued together (1, 2, 4 or 8); 0 = 4 (1 at 16 lanes).  The pinned
                           (lanes, unroll) pair must be one the library is built with: (1|2|4|8, 4),
                           (1|2|4, 8), (2|4|8, 2), (16, 1), (16, 2); others give GABP_ERR_INVALID.
                           Ignored when lanes = 0 (autotuned).  Default 0 */
  int history;          /* FP64 parallel rounds: record the relative residual of the first `history`
                           iterates of each solve (read with gabp_residual_history), the curve the
                           paper plots against the iteration count; 0 = off.  Default 0 */
  double fix_step;      /* the single loop's step s in (0, 1], default 0.5 */
  int warm_start;       /* plain FP64 parallel rounds: 1 = round 0 takes the messages of the handle's
                           last FP64 solve (or those loaded by gabp_set_messages) instead of zero
                           messages, with the new b; the iteration has the same fixed point from any
                           start, so a nearby b converges in fewer rounds.  Ignored until the handle
                           has such messages, and by the other paths.  Default 0 */
  int initial_guess;    /* gabp_solve / gabp_solve_host (every single right-hand-side path): 1 = x holds
                           an initial iterate x0 on entry; the path solves the correction system
                           A d = b - A x0 (FP64 residual) to the tolerance that makes
                           ||b - A (x0 + d)|| <= tol ||b||, and returns x = x0 + d (x0 itself when it
                           already meets tol; x = 0 for b = 0).  Rounds, stats and messages are those of
                           the correction solve.  Default 0 */
  int graphs;           /* 1 = rounds replayed from captured CUDA graphs (and the FP32 refinement loop run
                           as one graph, device_loop); 0 = every kernel launched on its own, for
                           per-kernel profilers (kernels in graphs that can set conditional handles
                           cannot be profiled one by one).  Same kernels and results.  Default 1 */
  int reserved;
} gabp_options;

/* Fill *o with the defaults listed above. */
gabp_status gabp_options_default(gabp_options *o);

/*
 * gabp_create -- validate A, upload it and build the device graph.
 *
 * A is given as FULL symmetric CSR: rowptr[n+1], col[nnz], val[nnz], the
 * diagonal included, column indices strictly increasing within each row.
 * mem_space 0: the three arrays are host memory; 1: device memory.
 * The graph of A: nodes are variables, edges are the nonzero off-diagonal
 * entries (Sec. "From Linear Algebra to Probabilistic Inference").
 *
 * Returns GABP_ERR_INVALID (and no handle) when: n < 1, nnz out of range,
 * rowptr not monotone, a column index out of range or not strictly increasing,
 * a row without a diagonal entry or with A_ii = 0, a stored zero off the
 * diagonal, an asymmetric pattern or value (A_ij != A_ji bit for bit), or a
 * non-finite value.  The handle owns all device memory it allocates; free it
 * with gabp_destroy.  stream is a cudaStream_t; NULL (the legacy default
 * stream) makes the handle create and own a non-blocking stream, which every
 * call first orders after the work already queued on the legacy default stream
 * (round graphs cannot be captured on the legacy stream).  opt may be NULL
 * (defaults).
 */
gabp_status gabp_create(gabp_handle *out, int32_t n, int64_t nnz, const int32_t *rowptr,
                        const int32_t *col, const double *val, int mem_space, void *stream,
                        const gabp_options *opt);

/* New values for the same sparsity pattern (the full symmetric CSR values in
 * the order of the rowptr/col given to gabp_create, host (mem_space 0) or
 * device (1)), e.g. the matrix of a learning step.  The reverse-edge index,
 * the layout and the autotuner's choices are kept; the precision state is
 * recomputed by the next solve (eq_prec depends on A only, Sec. "The Gaussian BP Algorithm").
 * Checked like gabp_create's values (finite, nonzero diagonal and
 * off-diagonals, A_ij == A_ji bit for bit); on GABP_ERR_INVALID the handle
 * holds no valid matrix and every solve fails until a valid call. */
gabp_status gabp_set_values(gabp_handle h, const double *val, int mem_space);

/* Replace the handle's options (validated) / stream.  gabp_set_stream waits
 * for the work on the old stream; NULL switches to the handle's own stream
 * (as gabp_create with NULL). */
gabp_status gabp_set_options(gabp_handle h, const gabp_options *opt);
gabp_status gabp_set_stream(gabp_handle h, void *stream);

/*
 * gabp_solve -- solve A x = b (b, x: device arrays of n doubles).
 *
 * Messages start at zero (Algorithm 1, step 1).  After round t the tentative
 * means x_t are formed (Algorithm 1, step 4) and the run stops at the first t
 * with ||b - A x_t||_2 <= tol ||b||_2, or at t = max_iter.  With the FP32
 * refinement precision, tol is the target of the outer FP64 loop.  With
 * gamma_mode != 0 the convergence fix runs: x <- x + (A + Gamma)^{-1} (b - A x)
 * (Chapter "Fixing convergence of GaBP", double loop), GaBP being run on
 * A + Gamma.
 * iters_out (nullable): rounds of the returned iterate (FP64) or total inner
 * rounds (FP32 refinement / convergence fix).  relres_out (nullable): final
 * ||b - A x|| / ||b||.  On GABP_NOT_CONVERGED / GABP_DIVERGED x holds the last
 * iterate.  b = 0 gives x = 0 and 0 rounds.
 */
gabp_status gabp_solve(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                       int32_t *iters_out, double *relres_out);

/* As gabp_solve with b and x in host memory; the copies run on the handle's stream. */
gabp_status gabp_solve_host(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                            int32_t *iters_out, double *relres_out);

/*
 * gabp_solve_batched -- nrhs right-hand sides in one launch sequence, FP32
 * messages + FP64 refinement (the precision messages depend on A only, eq_prec
 * and eq_prec_message, so they are converged once and shared).
 * B, X: device, column r at B + r*ld (ld >= n).  iters_out: total inner rounds.
 * relres_out (nullable): HOST array of nrhs doubles receiving each column's
 * final relative residual.
 * Returns the worst status over the columns.
 */
gabp_status gabp_solve_batched(gabp_handle h, int32_t nrhs, const double *B, double *X, int64_t ld,
                               double tol, int32_t max_iter, int32_t *iters_out, double *relres_out);

/*
 * gabp_solve_systems -- solve nsys independent systems in ONE persistent launch.
 * The handle's A must be block diagonal: system s owns rows and columns
 * [offsets[s], offsets[s+1]) (host array of nsys+1 ints, offsets[0] = 0,
 * offsets[nsys] = n, strictly increasing); an entry coupling two systems gives
 * GABP_ERR_INVALID.  b, x: device arrays of n doubles.  Every system runs its own
 * FP32 precision phase, FP32 mean rounds and FP64 refinement to
 * ||b_s - A_s x_s|| <= tol ||b_s|| (the batching direction of the paper's method:
 * systems share nothing).  Large systems are solved by a thread-block cluster,
 * small ones by a single thread block (a host scheduler balances the work; the
 * size threshold between the two is autotuned on the handle's first call).
 * status_out / iters_out / relres_out: nullable HOST arrays of nsys receiving each
 * system's status, rounds (precision + inner) and final relative residual.
 * Returns the worst status.
 */
gabp_status gabp_solve_systems(gabp_handle h, int32_t nsys, const int32_t *offsets, const double *b, double *x,
                               double tol, int32_t max_iter, int32_t *status_out, int32_t *iters_out,
                               double *relres_out);

/* The colouring of the serial schedule (options.schedule = 1): nodes in index
 * order, each taking the smallest colour not used by a lower-indexed
 * neighbour; a sweep fires colour 0, then colour 1, ...  colour: device array
 * of n int32 (nullable); *ncolours (nullable) the number of colours.  Computed
 * once per handle (on the device) and kept. */
gabp_status gabp_serial_colours(gabp_handle h, int32_t *colour, int32_t *ncolours);

/*
 * gabp_create_dense -- a handle for a dense symmetric matrix A (n x n, row-major, leading
 * dimension lda >= n, FP64), e.g. the kernel matrices of Chapter "Support Vector Regression"
 * (Sec. "Our novel construction": the kernel matrix with its main diagonal weighted until it
 * is diagonally dominant, solved by GaBP with the n node aggregates broadcast every round).
 * The broadcast form (Algorithm 2) needs no sparsity: the entry keeps A's nonzero entries
 * (and the diagonal), builds their row-CSR on the device and creates an ordinary handle on
 * it, so every solve path and option applies.  A in host (mem_space 0) or device (1) memory;
 * a host A is copied to the device first.  *nnz_out (nullable) receives the entries kept.
 * GABP_ERR_INVALID for bad arguments, more than 2^31 - 1 kept entries, or an A that
 * gabp_create rejects (not symmetric, non-finite, zero diagonal); otherwise as gabp_create.
 */
gabp_status gabp_create_dense(gabp_handle *out, int32_t n, const double *A, int64_t lda, int mem_space,
                              void *stream, const gabp_options *options, int64_t *nnz_out);

/*
 * gabp_create_lsq -- a handle for regularised least squares / MMSE estimation with a
 * rectangular J (m x k): x = (J^T J + gamma I)^{-1} J^T y (Sec. "Extension to General
 * Linear Systems", the -gamma I block that makes the augmented matrix invertible; Chapter
 * "Extending GaBP to support non-square matrices", its MMSE detector with Psi = gamma I).
 * The handle's matrix is the sparse symmetric augmented system
 *     [[I_k, J^T], [J, -gamma I_m]]  (n = k + m rows: x first, the auxiliary z after),
 * so no J^T J is formed and every solver path and option applies to it; GaBP on it gives
 * x in its first k marginal means.  The model is walk-summable for gamma > sigma_max(|J|)^2
 * (the section's condition); below that plain FP64 GaBP often still converges, while the
 * FP32-messages path may report GABP_DIVERGED.
 * J: CSR rowptr[m+1], col[nnz], val[nnz] (columns strictly increasing within a row, in
 * [0, k); finite nonzero values), host (mem_space 0) or device (1) memory; device arrays
 * are read after synchronising `stream` (when not NULL).  gamma > 0 and finite.  The
 * augmented CSR is assembled once in host memory (an O(nnz) transpose of J) and handed to
 * gabp_create.  Returns GABP_ERR_INVALID for bad arguments or a bad J, or when
 * k + m + 2 nnz does not fit int32; otherwise as gabp_create.  gabp_destroy frees it.
 */
gabp_status gabp_create_lsq(gabp_handle *out, int32_t m, int32_t k, int64_t nnz, const int32_t *rowptr,
                            const int32_t *col, const double *val, double gamma, int mem_space, void *stream,
                            const gabp_options *opt);

/* Solve on a gabp_create_lsq handle: y (device, m) -> x (device, k) and, when z is not
 * NULL, the auxiliary z = (J x - y) / gamma (device, m).  The augmented right-hand side is
 * [0_k; y]; the run is the handle's gabp_solve path (options as set), its stop rule the
 * augmented system's relative residual ||[0; y] - A_aug [x; z]|| <= tol ||y||.
 * iters_out / relres_out as gabp_solve.  GABP_ERR_INVALID on a handle not created by
 * gabp_create_lsq, on host arrays, or with options.initial_guess = 1. */
gabp_status gabp_solve_lsq(gabp_handle h, const double *y, double *x, double *z, double tol, int32_t max_iter,
                           int32_t *iters_out, double *relres_out);

/* Marginal precisions P_i = A_ii + sum_k P_ki of the last solve (Algorithm 1,
 * step 4), device array of n doubles.  Exact (= 1/(A^{-1})_ii) on trees; an
 * approximation on loopy graphs.  GABP_ERR_INVALID before the first solve. */
gabp_status gabp_marginal_precisions(gabp_handle h, double *Pi);

/* Messages of the last FP64 solve at its returned round (or sweep), in the receiver
 * layout of the input CSR: for slot p of row i with col[p] = k != i,
 * P[p] = P_ki and hm[p] = P_ki * mu_ki (the information-form mean message);
 * diagonal slots get 0.  After a solve with options.freeze_precisions the precision
 * messages are those of the stored round or the round before it (later rounds do not
 * rewrite them; the two agree to 16 units in the last place).  Device arrays of nnz
 * doubles. */
gabp_status gabp_get_messages(gabp_handle h, double *P, double *hm);

/* Gradient of a scalar loss through x = A^{-1} b, given lambda = A^{-1} dL/dx
 * (obtain it with a second gabp_solve on dL/dx: A is symmetric) and x:
 * grad_val[p] for every CSR slot p = (i, j) of the input:
 *   off-diagonal: -(lambda_i x_j + lambda_j x_i) / 2   (symmetrised),
 *   diagonal:     -lambda_i x_i.
 * dL/db is lambda itself.  Device arrays. */
gabp_status gabp_grad_values(gabp_handle h, const double *lambda, const double *x, double *grad_val);

/* Statistics of the last solve (all outputs nullable): rounds executed
 * (precision-phase plus inner mean rounds; for gabp_solve_systems the largest
 * over the systems), the directed-edge count E (off-diagonal nnz), the number
 * of edge-updates performed (one directed edge's messages recomputed in one
 * round, summed over rounds, right-hand sides and systems), and refinement steps. */
gabp_status gabp_last_stats(gabp_handle h, int64_t *rounds, int64_t *num_edges, int64_t *edge_updates,
                            int32_t *refine_steps);

/* The precision freeze of the last FP64 solve (options.freeze_precisions), outputs
 * nullable: *round receives the round whose coefficients -A_ki / P_k\i and 1/P~
 * were stored (that round and every earlier one are the plain solve's; later rounds
 * update the mean messages only), or 0 if the freeze was off or never verified;
 * *checks the number of verification rounds run (failed ones included).
 * GABP_ERR_INVALID for a null handle. */
gabp_status gabp_last_freeze(gabp_handle h, int32_t *round, int32_t *checks);

/* Per-phase device time of the solves since the last reset (options.profile = 1):
 * phase 0 FP64 GaBP rounds, 1 FP32 precision rounds (joint precision + mean
 * rounds with overlap_precision), 2 FP32 mean rounds, 3 FP64 refinement steps
 * (residual + update), 4 the persistent multi-system kernel (always timed),
 * 5 the coefficient freeze (with overlap_precision: the first mean round,
 * which also computes the frozen coefficients).  ms: summed CUDA-event time around the phase's
 * launches on the handle's stream (it includes the few rounds launched after a
 * decision, which return at once); rounds: round kernels that did work (phase
 * 4: the largest per-system round count); launches: every kernel the library
 * launched. */
typedef struct {
  double ms[6];
  int64_t rounds[6];
  int64_t launches;
} gabp_profile;
gabp_status gabp_profile_read(gabp_handle h, gabp_profile *out, int reset);

/*
 * gabp_solve_noalloc -- plain FP64 solve of a small system without any device
 * allocation.  The paper has no counterpart: this is a deployment variant of
 * gabp_solve for callers that cannot call cudaMalloc at solve time (latency-
 * critical loops that cannot absorb its device synchronisation, processes
 * whose device memory another allocator has already reserved, code under
 * no-allocation-after-start-up rules).
 *
 * A is FULL symmetric CSR as for gabp_create; rowptr, col, val, b, x are DEVICE
 * arrays owned by the caller (host pointers return GABP_ERR_INVALID before
 * anything is launched); stream is a cudaStream_t.  Same iteration, stop rule
 * and statuses as gabp_solve with GABP_PREC_FP64; iters_out / relres_out are
 * nullable host pointers.  A matrix the kernel rejects (CSR structure,
 * diagonal, symmetry) returns GABP_ERR_INVALID with "matrix rejected" in
 * gabp_last_error().
 *
 * Every call synchronises `stream` before it returns (the status is read back
 * to the host), so it cannot be called while that stream is being captured
 * into a CUDA graph.
 *
 * Working memory is one fixed array (about 5.6 MB) inside the library's device
 * memory, held by every GPU that loads the library until the process exits.
 * Limits: 1 <= n <= 16384 and n <= nnz <= 131072; larger sizes return
 * GABP_ERR_INVALID without launching anything.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it for
 * the process; calls after a cudaDeviceReset of that device are not supported.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or other allocating call
 * is made.
 */
gabp_status gabp_solve_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                               const double *val, const double *b, double *x, double tol,
                               int32_t max_iter, void *stream, int32_t *iters_out, double *relres_out);

/* Loads messages as the handle's FP64 state (the checkpoint counterpart of
 * gabp_get_messages, same layout: device arrays of nnz doubles, P[p] = P_ki and
 * hm[p] = P_ki mu_ki for slot p of row i with col[p] = k != i, diagonal slots
 * ignored).  The next gabp_solve with options.warm_start = 1 (FP64 parallel
 * rounds) starts from them; any finite messages are a valid start, a poor one
 * costs rounds (or, outside the convergent cases, convergence).  The handle
 * keeps its own copy.  GABP_ERR_INVALID for null pointers or host arrays. */
gabp_status gabp_set_messages(gabp_handle h, const double *P, const double *hm);

/* Residual history of the last solve (options.history > 0, plain FP64 parallel
 * rounds, node or edge variant): relres[t] = ||b - A x^(t)|| / ||b|| for the
 * iterates t = 0, 1, ... the rounds checked (x^(0) = b_i / A_ii; with Aitken's
 * method the accelerated iterate), at most cap entries copied into the HOST
 * array relres; *count (nullable) = entries recorded (at most options.history).
 * Other paths record none (*count = 0).  GABP_ERR_INVALID for cap < 0 or a
 * null relres with cap > 0. */
gabp_status gabp_residual_history(gabp_handle h, double *relres, int32_t cap, int32_t *count);

/* The autotuner's choices for this handle (0 where not tuned yet; all outputs
 * nullable): the FP64 round's lanes per row (1 once its sliced layout is built:
 * one row per lane); the FP32 precision-phase round's
 * shape (the joint precision + mean round when options.overlap_precision = 1,
 * else the precision-only round) and the mean round's shape, packed as
 * lanes | unroll << 8; the multi-system size split;
 * the multi-system kernel (1 grid-persistent, 2 teams) | the grid-persistent
 * kernel's shape << 8 (shape: lanes | unroll << 8, plus 1 << 16 on the sliced
 * layout).  The FP64 and FP32 choices are remembered for the
 * process per (device, n, directed-edge count): a later handle of a matrix of
 * that size starts with them instead of tuning again. */
gabp_status gabp_tuned_shapes(gabp_handle h, int32_t *fp64_lanes, int32_t *prec32_shape, int32_t *mean32_shape,
                              int64_t *multi_split, int32_t *multi_mode);

/* Free everything the handle owns.  NULL is accepted. */
gabp_status gabp_destroy(gabp_handle h);

/* Static text for a status; thread-local text of the last CUDA error. */
const char *gabp_status_string(gabp_status s);
const char *gabp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GABP_H_ */
