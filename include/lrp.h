/*
 * lrp.h -- C ABI of the GB300 low-rank Poisson solver (Cross-DEIM on the
 * sine-transformed 5-point Poisson equation).
 *
 * Problem (paper Sec. 3, Eq. matrix_poisson): on the n x n interior grid of
 * the unit square with zero Dirichlet data, h = 1/(n+1), solve
 *
 *     T W + W T = h^2 F,      T = tridiag(-1, 2, -1)  (n x n),
 *
 * for a right-hand side given by factors F = U_f diag(s_f) V_f^T (Sec. 3.2).
 * The solver transforms the factors with the orthonormal DST-I Z (Sec. 3),
 * runs Cross-DEIM (Algorithm "Cross-DEIM", Sec. 2.2.3) on the transformed
 * solution What(i,j) = h^2 Fhat(i,j) / (lambda_i + lambda_j) (Eq. g_for_p)
 * and transforms the result back: W = (Z Uhat) diag(S) (Z Vhat)^T.
 * The n x n grid is never formed.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major FP64 with a leading dimension ld >= n.
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device; the
 *     caller allocates and owns them.  h_* pointers are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Every call returns an lrp_status; no call aborts, throws or exits.  On an
 *     error the thread-local message lrp_last_error() says what failed.
 *   - Results: W ~= U diag(S) V^T, U and V with orthonormal columns, S >= 0
 *     descending, the sign of each singular pair unspecified.
 */
#ifndef LRP_H_
#define LRP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lrp_status {
  LRP_OK = 0,
  LRP_EINVAL = 1,          /* bad argument (size, pointer, leading dimension, option) */
  LRP_ENOMEM = 2,          /* device or host allocation failed */
  LRP_ECUDA = 3,           /* a CUDA runtime call failed (see lrp_last_error) */
  LRP_ETIMEDOUT = 4,       /* a bounded wait gave up (server drain, device flag) */
  LRP_NOT_CONVERGED = 5,   /* the stop test was not met (max_iter reached, or a mixed-precision
                              correction solve stalled first); a valid result was still written */
  LRP_RANK_CAPPED = 6,     /* tolerance needs rank > max_rank; result truncated */
  LRP_EAGAIN = 7,          /* lrp_poll: not finished yet; lrp_submit: server full, retry */
  LRP_ECAPACITY = 8        /* server admission: request larger than the memory cap */
} lrp_status;

typedef enum lrp_precision {
  LRP_FP64 = 0,   /* every step in FP64 */
  LRP_MIXED = 1   /* FP32 transforms/contractions, FP64 Gram/Cholesky/core, one
                     FP64-residual refinement step (not in the paper) */
} lrp_precision;

typedef enum lrp_selector {
  LRP_SEL_LEVERAGE = 0,  /* leverage scores, deterministic top-c: the c = columns rows of largest
                            score (Sec. 2.2.2 with the sampling replaced by a selection) */
  LRP_SEL_QDEIM = 1,     /* Algorithm (Q)DEIM: pivoted QR of U^T (Sec. 2.2.1) */
  LRP_SEL_BERNOULLI = 2  /* the default: Algorithm LeverageScores as printed (Sec. 2.2.2): row i
                            sampled with probability min(1, c pi_i), c = sample_factor x columns;
                            draws from Philox4x32-10 keyed by seed, counter (row, iteration, side, 0) */
} lrp_selector;

/* The matrix Cross-DEIM approximates.  LRP_MAT_POISSON: the transformed solution
   of the Poisson problem (Sec. 3.2), right-hand side F = U_f diag(s_f) V_f^T.
   The test matrices of Sec. 4.1 (n x n, FP64 plans only): lrp_problem.d_U_f and
   d_V_f are then the initial guesses U_0, V_0 (n x r_f; orthonormalised by the
   solver), d_s_f is unused and may be NULL, and U, S, V approximate the matrix
   itself. */
typedef enum lrp_matrix {
  LRP_MAT_POISSON = 0,
  LRP_MAT_HILBERT = 1,   /* H(i, j) = 1 / (1 + i + j), i, j from 0 */
  LRP_MAT_K = 2          /* K(i, j) = (|x_i + y_j| / 2)^5, x_i = -1 + 2i/(n-1), y_j likewise */
} lrp_matrix;

/* Solver options.  lrp_default_opts fills the defaults noted here. */
typedef struct lrp_opts {
  int32_t precision;     /* lrp_precision, default LRP_FP64 */
  int32_t selector;      /* lrp_selector, default LRP_SEL_BERNOULLI */
  int32_t max_iter;      /* Cross-DEIM iterations, default 30 */
  int32_t refine_steps;  /* LRP_MIXED only: residual-correction steps: 0 (the FP32 result), 1, or 2
                            (default): a second step for the problems whose first step looks
                            unreliable (LRP_FLAG_REFINED_TWICE; the others are unchanged) */
  int32_t max_rhs_rank;  /* capacity for r_f, default 64 (<= 256) */
  int32_t batch;         /* max problems per lrp_solve_batch call, default 1 */
  int32_t m_cap;         /* index-set capacity, default min(2*max_rank + max_rhs_rank, 256) */
  int32_t check_every;   /* host reads the active-solve count every this many
                            iterations, default 1 */
  uint64_t seed;         /* key of the growth-index generator (SplitMix64) and of the
                            Bernoulli draws (Philox4x32-10), default 0 */
  double sample_factor;  /* LRP_SEL_BERNOULLI: c / columns, the expected sample size over the
                            basis width (> 0), default 1 */
  int32_t matrix;        /* lrp_matrix, default LRP_MAT_POISSON */
  int32_t loop_on_device; /* 0 (default): the host reads the count of still-iterating problems after
                            every Cross-DEIM iteration and launches the next one over the active ones;
                            1: the whole solve is one captured CUDA graph whose iteration loops are
                            conditional while-nodes, continued by the device while any problem is
                            active (bounded by max_iter), so a solve is one graph launch and the call
                            returns without waiting for it (the mixed path's second refinement step
                            is a conditional if-node of the same graph).  The graph is captured on a
                            batch size's first solve; a plan keeps up to eight (one per batch size,
                            least recently used replaced). */
  /* Launch shapes (no counterpart in the paper).  Both are result-neutral: every
     output is computed by the same operations in the same order whatever the
     value, so they change only the speed (lrp_group and the autotuner in
     tune.py pick them by timing). */
  int32_t gemm_rows_per_thread; /* rows per thread of the narrow tall products (thread per
                            row, at most 32 input columns): 1 or 2; 0 (default): 2 for FP32
                            data, 1 for FP64 */
  int32_t dst_cta_threads; /* threads per CTA of the shared-memory DST-I (n+1 <= 8192, or
                            16384 in FP32), which then transforms threads / ((n+1)/16)
                            columns at once: 256, 512 or 1024; 0 (default): 256.  FP64 and
                            double-float transforms use at most 512 */
} lrp_opts;

/* Per-problem report, written by the device into caller memory. */
/* lrp_info.flags */
#define LRP_FLAG_CONVERGED 1   /* the stop test passed (mixed: the FP32 trial passed it or stalled at its
                                  noise floor, and every correction solve passed it) */
#define LRP_FLAG_RANK_CAPPED 2 /* r* > max_rank */
#define LRP_FLAG_CAPACITY 4    /* an index set reached m_cap */
#define LRP_FLAG_BAD_INPUT 8   /* non-finite data met */
#define LRP_FLAG_STALLED 16    /* an FP32 solve stopped at its noise floor: the change stopped halving */
#define LRP_FLAG_ROLLED_BACK 32 /* a stalled FP32 solve returned its previous iterate (the last step grew the change) */
#define LRP_FLAG_REFINED_TWICE 64 /* the first correction looked unreliable: a second refinement step ran */

typedef struct lrp_info {
  int32_t rank;          /* r = max(min(r*, max_rank), 1) columns written to U, V, S */
  int32_t iterations;    /* Cross-DEIM iterations taken (last solve of a refinement) */
  int32_t status;        /* LRP_OK, LRP_NOT_CONVERGED or LRP_RANK_CAPPED */
  int32_t r_star;        /* tail-rule rank before the max_rank cap */
  int32_t size_I;        /* |I| at exit */
  int32_t size_J;        /* |J| at exit */
  int32_t total_iterations; /* summed over the initial solve and refinement solves */
  int32_t flags;         /* LRP_FLAG_* bits */
  double rho;            /* last relative change ||A_k - A_{k-1}||_F / ||A_k||_F */
  double eta_smin;       /* last min(eta1(1+eta2), eta2(1+eta1)) * S_min / ||S||_F */
  double sigma_max;      /* largest singular value of the result */
  double reserved1;
} lrp_info;

/*
 * Warm-start record of one problem: the index sets I, J and the transformed
 * iterate (Uh, Vh) that a solve ended with (device memory owned by the record,
 * sized by the plan it was created for).  Algorithm Cross-DEIM starts from
 * initial bases and empty index sets; a record that holds a result instead seeds
 * the next solve of a related problem with them (the abstract presents
 * Cross-DEIM as a warm-startable iteration).  The first iteration's change rho
 * is measured from zero as in a cold start, so a warm solve runs at least two
 * iterations.  A record serves one problem at a time: lrp_solve_batch rejects a
 * batch that names one record twice (LRP_EINVAL), and two batches in flight on
 * unordered streams must not share a record.
 */
typedef struct lrp_warm_s* lrp_warm_t;

/* One problem of a batch (all problems of a plan share n). */
typedef struct lrp_problem {
  int32_t r_f;           /* right-hand-side rank, 1 <= r_f <= max_rhs_rank */
  int32_t reserved;
  const double* d_U_f;   /* n x r_f, ld ldu_f */
  int64_t ldu_f;
  const double* d_s_f;   /* r_f weights of F = U_f diag(s_f) V_f^T */
  const double* d_V_f;   /* n x r_f, ld ldv_f */
  int64_t ldv_f;
  double* d_U;           /* out: n x max_rank, ld ldu (first rank columns written) */
  int64_t ldu;
  double* d_S;           /* out: max_rank singular values (first rank written) */
  double* d_V;           /* out: n x max_rank, ld ldv */
  int64_t ldv;
  lrp_info* d_info;      /* out: device memory for one lrp_info (may be NULL) */
  lrp_warm_t warm;       /* NULL, or a record of this plan: when it holds a result the
                            solve starts from its I, J and iterate; on return it holds
                            this solve's (mixed precision: its first FP32 solve's) */
} lrp_problem;

typedef struct lrp_plan_s* lrp_plan_t;

/* Fill *opts with the defaults.  Returns LRP_EINVAL for NULL. */
lrp_status lrp_default_opts(lrp_opts* opts);

/*
 * Create a plan for grids with n interior points per dimension, relative
 * tolerance tol (Algorithm Cross-DEIM's epsilon: stop test and final
 * truncation sum_{l>r} S_l^2 < tol^2 ||S||^2) and output rank cap max_rank
 * (the paper's r_max).  opts may be NULL (defaults).  The plan allocates and
 * owns all device workspace on the current device; its size grows with
 * batch * n * m_cap.  Supported: 1 <= n <= 8191 with n+1 a power of two is
 * the shared-memory DST path; other n (n+1 a power of two up to 2^20) use the
 * multi-pass DST.  Errors: LRP_EINVAL (n+1 not a power of two, tol <= 0,
 * max_rank < 1, options out of range), LRP_ENOMEM, LRP_ECUDA.
 */
lrp_status lrp_plan(lrp_plan_t* out, int64_t n, double tol, int32_t max_rank,
                    const lrp_opts* opts);

/*
 * Pack the results of the plan's most recent solve (lrp_solve / lrp_solve_batch)
 * compactly: for each problem i of that batch, in order, the block
 * [U (n x r_i) | S (r_i) | V (n x r_i)] (column-major, ld n; r_i the problem's
 * rank) into d_packed, starting d_offsets[i] doubles in; d_offsets[count]
 * receives the total.  d_offsets (device, count + 1 int64) and d_packed
 * (device, capacity doubles) are the caller's.  Asynchronous on `stream`, which
 * must be ordered after the solve; a block that would end beyond capacity is not
 * written (detect it from d_offsets[count] > capacity).  Errors: LRP_EINVAL (NULL
 * plan or offsets, no solve yet), LRP_ECUDA.
 */
lrp_status lrp_plan_pack(lrp_plan_t plan, double* d_packed, int64_t capacity, int64_t* d_offsets, void* stream);

/*
 * Device bytes that lrp_plan(n, tol, max_rank, opts) would allocate in its
 * workspace arena (the figure lrp_plan_workspace_bytes reports for the plan),
 * computed on the host without touching a device.  Same argument checks and
 * errors as lrp_plan (LRP_EINVAL), plus LRP_EINVAL for NULL bytes.
 */
lrp_status lrp_plan_estimate_bytes(int64_t n, double tol, int32_t max_rank, const lrp_opts* opts, size_t* bytes);

/*
 * Create an empty warm-start record for problems of `plan` (device memory of
 * about 2 n m_cap doubles).  Errors: LRP_EINVAL, LRP_ENOMEM.
 */
lrp_status lrp_warm_create(lrp_plan_t plan, lrp_warm_t* out);

/* Mark a record empty again (the next solve starts cold and refills it). */
lrp_status lrp_warm_reset(lrp_warm_t warm);

/* Release a record (synchronises the device first). */
lrp_status lrp_warm_destroy(lrp_warm_t warm);

/* Release a plan and its workspace (synchronises the device first). */
lrp_status lrp_plan_destroy(lrp_plan_t plan);

/* Bytes of device workspace the plan holds. */
lrp_status lrp_plan_workspace_bytes(lrp_plan_t plan, size_t* bytes);

/*
 * Solve one problem (Sec. 3.2: DST of the factors, Cross-DEIM on Eq. g_for_p,
 * back DST).  Inputs and outputs are device pointers as in lrp_problem.  Work
 * is enqueued on `stream`; the call returns once the iteration loop has ended
 * (it reads a device counter of active solves between iterations) with the
 * output writes enqueued on `stream`.  Errors: LRP_EINVAL, LRP_ECUDA.  The
 * per-problem outcome (LRP_NOT_CONVERGED, LRP_RANK_CAPPED) is in d_info.
 */
lrp_status lrp_solve(lrp_plan_t plan, int32_t r_f,
                     const double* d_U_f, int64_t ldu_f, const double* d_s_f,
                     const double* d_V_f, int64_t ldv_f,
                     double* d_U, int64_t ldu, double* d_S, double* d_V, int64_t ldv,
                     lrp_info* d_info, void* stream);

/*
 * Solve `count` independent problems of the plan's n in one set of launches
 * (every kernel covers all problems).  h_problems is a HOST array of count
 * descriptors; count <= opts.batch.  Same completion rule as lrp_solve.
 */
lrp_status lrp_solve_batch(lrp_plan_t plan, int32_t count, const lrp_problem* h_problems,
                           void* stream);

/*
 * Orthonormal DST-I of ncols columns (Sec. 3: Y = Z X, Z_{ik} =
 * sqrt(2/(n+1)) sin(i k pi/(n+1))), FP64, n+1 a power of two up to 2^20.
 * X and Y are device, column-major, may not overlap.  Enqueued on stream.
 */
lrp_status lrp_dst1(int64_t n, int32_t ncols, const double* d_X, int64_t ldx,
                    double* d_Y, int64_t ldy, void* stream);

/*
 * lrp_dst1 without any device allocation.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory when they call in (a host
 * callback or plugin running while another framework owns the memory pool, a
 * fixed memory budget handed out up front, or code that must avoid the implicit
 * synchronisation of cudaMalloc/cudaFree).  Its scratch (one twiddle table and
 * the job descriptor, 128 KiB + 256 B) is a fixed array inside the library that
 * every device which loads the library holds until the process exits.
 * Arguments and result are those of lrp_dst1, restricted to n+1 <= 8192;
 * larger n returns LRP_EINVAL.  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (for example on two
 * unordered streams) race on it.
 */
lrp_status lrp_dst1_noalloc(int64_t n, int32_t ncols, const double* d_X, int64_t ldx,
                            double* d_Y, int64_t ldy, void* stream);

/*
 * Measurement hooks (not part of the paper's method).  Kernel classes of the
 * solve, for per-class launch counts and CUDA-event timings.
 */
typedef enum lrp_kernel_class {
  LRP_K_DST = 0,       /* forward and back DST-I */
  LRP_K_CROSS = 1,     /* sampled columns/rows of the transformed solution */
  LRP_K_GRAM = 2,      /* per-block partial Gram / cross-Gram products, FP64 accumulation */
  LRP_K_REDUCE = 3,    /* reduction of the Gram partials */
  LRP_K_GEMM = 4,      /* tall-skinny n x m times m x m' products on FP64 data */
  LRP_K_LEVERAGE = 5,  /* leverage scores and block top-c */
  LRP_K_CHOL = 6,      /* small Cholesky / triangular inverse per problem */
  LRP_K_CORE = 7,      /* small pseudoinverse / SVD core per problem */
  LRP_K_SELECT = 8,    /* index-set enrichment per problem */
  LRP_K_STOP = 9,      /* convergence test per problem */
  LRP_K_OTHER = 10,    /* setup, finalize, counters */
  LRP_K_REFINE = 11,   /* mixed precision: residual/sum assembly and recompression cores */
  LRP_K_GRAM_F32 = 12, /* partial Gram products with FP32 accumulation (FP32 iterations) */
  LRP_K_GEMM_F32 = 13, /* tall-skinny products on FP32 data (FP32 iterations) */
  LRP_K_GRAM_DF = 14,  /* Gram partials in double-float arithmetic on the FP32 pipe (mixed precision) */
  LRP_K_GEMM_DF = 15,  /* tall-skinny products in double-float arithmetic on the FP32 pipe (mixed precision) */
  LRP_K_DST_DF = 16,   /* DST-I of FP64 data in double-float arithmetic (mixed precision) */
  LRP_K_COUNT = 17
} lrp_kernel_class;

/*
 * enable != 0: every kernel launch of later solves on this plan is bracketed
 * by a CUDA event pair recorded on the solve's stream (no host synchronisation
 * is added); enable == 0 stops recording.  Launch counting is always on.
 */
lrp_status lrp_plan_set_timing(lrp_plan_t plan, int32_t enable);

/*
 * Per-iteration trace of Algorithm Cross-DEIM (Sec. 3.1): with enable != 0 every
 * later solve records, for each problem slot and each iteration (the mixed
 * path's FP32 solves in order, the correction solve after the first), the
 * quantities of the stop test.  The first call allocates
 * batch * LRP_TRACE_LEN * LRP_TRACE_WIDTH doubles of device memory (freed with
 * the plan).  Toggling re-captures the iteration graphs on the next solve.
 * Errors: LRP_EINVAL (NULL plan), LRP_ENOMEM.
 */
#define LRP_TRACE_LEN 96
#define LRP_TRACE_WIDTH 8
lrp_status lrp_plan_set_trace(lrp_plan_t plan, int32_t enable);

/*
 * Copy the trace of batch slot `slot` of the last solve to host memory `out`
 * (row-major, LRP_TRACE_WIDTH doubles per iteration: iteration index within its
 * solve, rho, min(eta1(1+eta2), eta2(1+eta1)) S_min, |I_k|, |J_k| before
 * redundancy removal, in-loop rank r_k, ||S_k||_F, |I_k| after removal), at
 * most max_entries rows; *n_entries receives the rows written.  Synchronises
 * the device.  Errors: LRP_EINVAL (NULL pointer, slot out of range, tracing
 * never enabled), LRP_ECUDA.
 */
lrp_status lrp_plan_trace(lrp_plan_t plan, int32_t slot, double* out, int32_t max_entries, int32_t* n_entries);

/*
 * Launches and summed event-timed milliseconds of kernel class kclass
 * (0 <= kclass < LRP_K_COUNT, or -1 for all classes) since the last reset.
 * Synchronises the device first.  *total_ms is 0 when timing was off.
 */
lrp_status lrp_plan_kernel_stats(lrp_plan_t plan, int32_t kclass, int64_t* launches, double* total_ms);

/*
 * Algorithmic work of kernel class kclass (or -1 for all) since the last reset,
 * summed over problems: the minimal flops and HBM bytes of the method's steps
 * at the sizes each iteration actually had (|I|, |J|, ranks), independent of
 * the kernels' tiling.  Synchronises the device first.
 */
lrp_status lrp_plan_kernel_work(lrp_plan_t plan, int32_t kclass, double* flops, double* bytes);

/* Clear the launch counts, timings and work totals of a plan. */
lrp_status lrp_plan_reset_stats(lrp_plan_t plan);

/* ------------------------------------------------------------------ groups
 *
 * A group solves one batch as `lanes` concurrent sub-batches: one plan, one CUDA
 * stream and one host worker thread per lane, so that the lanes' iterations
 * (each driven from the host) interleave on the GPU and per-problem cores of one
 * lane overlap tall products of another.  Problems are split into contiguous,
 * nearly equal shares in order.
 */
typedef struct lrp_group_s* lrp_group_t;

/*
 * Create a group of `lanes` (1..16) plans for n, tol, max_rank; opts->batch is
 * the group's total capacity, each lane holding ceil(batch / lanes).  Errors as
 * lrp_plan, plus LRP_EINVAL for lanes out of range or batch < lanes.
 */
lrp_status lrp_group_create(lrp_group_t* out, int64_t n, double tol, int32_t max_rank, const lrp_opts* opts,
                            int32_t lanes);

/*
 * Solve `count` problems (as lrp_solve_batch; warm-start records are not
 * accepted).  The lanes start after the work `stream` holds at the call; on
 * return every lane's work has been enqueued and `stream` waits for it.  Returns
 * the first lane error, if any.
 */
lrp_status lrp_group_solve(lrp_group_t group, int32_t count, const lrp_problem* problems, void* stream);

/* The plan of lane `lane` (for statistics and traces; owned by the group). */
lrp_status lrp_group_plan(lrp_group_t group, int32_t lane, lrp_plan_t* out);

/* As lrp_plan_pack over the group's last solve: all problems, in order, back to back. */
lrp_status lrp_group_pack(lrp_group_t group, double* d_packed, int64_t capacity, int64_t* d_offsets, void* stream);

/* Stop the workers and free the lanes' plans. */
lrp_status lrp_group_destroy(lrp_group_t group);

/* ------------------------------------------------------------------ mixed sizes, one launch
 *
 * A multi-size set: one plan per grid size (each with loop_on_device), solved
 * together as ONE CUDA graph launch.  lrp_multi_solve sorts a call's problems
 * into their size's plan and runs every size's whole solve (forward DST,
 * Cross-DEIM, refinement, back DST) as one concurrent branch of the graph; each
 * branch continues its iteration loops on the device while any of its problems
 * is active, so the host neither waits nor launches between iterations.  The
 * graph is captured on first use for each vector of per-size problem counts
 * (and warm-record / trace use) and replayed afterwards.  Results are those of
 * each size's plan alone (the branches share no workspace).
 */
typedef struct lrp_multi_s* lrp_multi_t;

/*
 * Create a set for nsizes distinct grid sizes ns[i] (n+1 powers of two), with
 * room for batches[i] problems of size ns[i] per call; tol, max_rank and opts
 * (NULL = defaults; opts->batch and opts->loop_on_device are ignored) are shared.
 * Errors: as lrp_plan, plus LRP_EINVAL for a repeated size or nsizes outside 1..64.
 */
lrp_status lrp_multi_create(lrp_multi_t* out, int32_t nsizes, const int64_t* ns, const int32_t* batches,
                            double tol, int32_t max_rank, const lrp_opts* opts);

/*
 * Solve `count` problems in one graph launch on `stream`: problem i has grid
 * size ns[i] (HOST array) and descriptor problems[i] (HOST array, device
 * factors as in lrp_solve_batch); at most batches[b] problems per size.  The
 * call returns once the launch is enqueued; results are complete when `stream`
 * reaches it.  Errors: LRP_EINVAL (a size not in the set, too many problems of
 * one size, a bad descriptor), LRP_ECUDA.
 */
lrp_status lrp_multi_solve(lrp_multi_t m, int32_t count, const int64_t* ns, const lrp_problem* problems,
                           void* stream);

/* The plan of size index b (statistics, traces, packing; owned by the set). */
lrp_status lrp_multi_plan(lrp_multi_t m, int32_t size_index, lrp_plan_t* out);

/* Free the set and its plans (synchronises the device first). */
lrp_status lrp_multi_destroy(lrp_multi_t m);

/* ------------------------------------------------------------------ serving
 *
 * A request server over the batched solver for streams of independent
 * problems of varying n, precision and tolerance (one GPU, one process).
 * Admission: each request's working set is estimated as
 * 8 n (2 r_f + 4 m_cap + 2 max_rank) bytes, with r_f' = r_f rounded up to a
 * multiple of 16 and m_cap the index-set capacity of its bucket's plan:
 * min(2 max_rank + r_f', 256) in FP64; in mixed precision 64 while r_f' + 16 <=
 * 64 (else r_f' + 16), which keeps the refinement in double-float arithmetic; a
 * request is refused with LRP_ECAPACITY when it alone exceeds the memory cap,
 * and with LRP_EAGAIN when the queued and running requests' estimates plus its
 * own would exceed the cap or the queue is full (retry later).  Scheduling:
 * worker lanes (one host thread and one CUDA stream each) take the oldest
 * waiting request that can start and solve it with up to a plan's batch of
 * waiting requests of its bucket (n, precision, tol, max_rank, r_f'), in
 * arrival order, as one graph launch (the plans run their iteration loops on
 * the device).  A bucket holds up to one plan per lane, so a request that
 * arrives while a batch of its bucket runs starts on another lane (continuous
 * batching: later arrivals join the next batch).  Plans are created on first
 * use with as many batch slots as fit a quarter of the cap, and idle plans are
 * destroyed least recently used when a new plan or warm-start record would not
 * fit.  Warm start: requests that name the same nonzero warm_key share a
 * warm-start record of a plan of their bucket (created by the first, reused by
 * later ones that run on that plan; at most warm_capacity records per plan,
 * least recently used dropped); a batch holds at most one request per key.
 */
typedef struct lrp_server_s* lrp_server_t;

typedef struct lrp_server_opts {
  int64_t memory_cap_bytes;  /* device bytes for plans and warm records, and the admission cap (40 GiB) */
  int32_t lanes;             /* concurrent batches, 1..16 (2) */
  int32_t max_batch;         /* upper bound of a plan's batch slots (64) */
  int32_t max_queue;         /* waiting requests before LRP_EAGAIN (65536) */
  int32_t warm_capacity;     /* warm-start records per plan (64) */
} lrp_server_opts;

typedef struct lrp_request {
  int64_t n;            /* interior points per dimension, n+1 a power of two */
  int32_t r_f;          /* right-hand-side rank */
  int32_t max_rank;     /* output rank cap (r_max) */
  double tol;           /* relative tolerance of Algorithm Cross-DEIM */
  int32_t precision;    /* lrp_precision */
  int32_t reserved;
  uint64_t warm_key;    /* 0, or the key of a warm-start record (see above) */
  const double* U_f;    /* host, n x r_f column-major (ld n); copied by lrp_submit */
  const double* s_f;    /* host, r_f; copied */
  const double* V_f;    /* host, n x r_f; copied */
  double* U;            /* host out, n x max_rank (ld n): first rank columns written */
  double* S;            /* host out, max_rank singular values */
  double* V;            /* host out, n x max_rank */
} lrp_request;

typedef struct lrp_result {
  int32_t status;       /* the solve's lrp_status (OK, NOT_CONVERGED, RANK_CAPPED) or the error */
  int32_t rank;         /* columns written to U, V */
  int32_t iterations;   /* Cross-DEIM iterations, all solves of the request */
  int32_t warm_used;    /* 1 if the solve started from a filled warm-start record */
  double latency_us;    /* lrp_submit to completion */
  double queue_us;      /* lrp_submit to the start of its batch */
} lrp_result;

typedef struct lrp_server_stats {
  int64_t submitted, completed, rejected;  /* since creation or the last reset */
  int64_t queued, running, plans;
  int64_t device_bytes;                    /* plans + warm records held */
  int64_t admitted_bytes;                  /* estimates of queued + running requests */
  double p50_us, p99_us, mean_us, max_us;  /* latency of completed requests (nearest rank) */
} lrp_server_stats;

/* Fill *opts with the defaults.  Returns LRP_EINVAL for NULL. */
lrp_status lrp_server_default_opts(lrp_server_opts* opts);

/* The admission estimate above in bytes for an FP64 request (an upper bound for mixed
   precision); 0 for out-of-range arguments. */
size_t lrp_request_footprint(int64_t n, int32_t r_f, int32_t max_rank);

/*
 * Start a server on the current device (opts may be NULL).  Errors:
 * LRP_EINVAL (options out of range), LRP_ECUDA (no device), LRP_ENOMEM.
 */
lrp_status lrp_server_create(lrp_server_t* out, const lrp_server_opts* opts);

/*
 * Admit one request without blocking on the GPU: the inputs are copied, the
 * output buffers must stay valid until the request's result has been taken.
 * *ticket identifies it.  Errors: LRP_EINVAL (bad request), LRP_ECAPACITY,
 * LRP_EAGAIN (see above), LRP_ENOMEM.
 */
lrp_status lrp_submit(lrp_server_t server, const lrp_request* req, uint64_t* ticket);

/*
 * LRP_EAGAIN while the request runs or waits; once it has finished, LRP_OK with
 * *out filled, after which the ticket is released (a second poll is LRP_EINVAL).
 */
lrp_status lrp_poll(lrp_server_t server, uint64_t ticket, lrp_result* out);

/* As lrp_poll, but waits up to timeout_us; LRP_ETIMEDOUT if still unfinished. */
lrp_status lrp_wait(lrp_server_t server, uint64_t ticket, lrp_result* out, int64_t timeout_us);

/* Counters and latency percentiles (microseconds). */
lrp_status lrp_server_get_stats(lrp_server_t server, lrp_server_stats* out);

/* Copy the message of the most recent failed batch (empty if none) into buf (len bytes, NUL-terminated). */
lrp_status lrp_server_last_error(lrp_server_t server, char* buf, size_t len);

/* Clear the counters and the latency record. */
lrp_status lrp_server_reset_stats(lrp_server_t server);

/*
 * Finish every admitted request, stop the lanes and free all device memory.
 * Results not yet taken are discarded.
 */
lrp_status lrp_server_destroy(lrp_server_t server);

/* Thread-local text of the last error (empty string if none). */
const char* lrp_last_error(void);

/* Static name of a status code. */
const char* lrp_status_string(lrp_status s);

#ifdef __cplusplus
}
#endif

#endif /* LRP_H_ */
