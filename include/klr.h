/*
 * klr.h -- C ABI of the GB300 rational-program library.
 *
 * The library implements the data-parallel hot path of the rational-program
 * method for choosing CUDA launch parameters (KLARAPTOR, arXiv 1911.02373):
 *
 *   1. fitting each low-level performance metric as a rational function
 *      p(N, b) / q(N, b) of the data size N and the block shape b, posed as the
 *      linearised least-squares problem [M_p | -y M_q] c = 0 over monomial
 *      design matrices (Section V-E; Section IV, step 2);
 *   2. evaluating the resulting rational program -- fitted metrics, integer
 *      occupancy (Fig. 1, Eq. 1), the MWP-CWP cycle model (Example 2) -- over
 *      every candidate block shape, and choosing the constrained argmin
 *      (Section IV, steps 4 and 5), returned as the six launch integers of the
 *      paper's IO function (Section V-C).
 *
 * Conventions for every entry point:
 *   - Pointers documented as "device" must point to memory of the context's
 *     device (cudaMalloc'd or a PyTorch CUDA tensor); "host" pointers to host
 *     memory.  The inputs klr_fit and klr_argmin only read (a batch's
 *     offsets, x and y; a query set's q_offsets and q_N) may also be
 *     page-locked host memory (cudaHostAlloc / cudaMallocHost) on a device
 *     with unified addressing: the kernels then read them in place over the
 *     interconnect.  The caller owns every array; the library never frees
 *     them.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising, except where noted.
 *   - Argument errors are detected on the host before anything is enqueued
 *     and return KLR_EINVAL; nothing is written then.  Per-item problems (a
 *     degenerate fit, a query without a usable configuration) do not fail the
 *     call: they are reported in the per-item status arrays.
 *   - A context's scratch memory is allocated by klr_ctx_reserve() or, when the
 *     stream is not capturing a CUDA graph, grown on demand by the first call
 *     that needs more.  During graph capture a call that would need to grow it
 *     returns KLR_ENOMEM instead, so reserve before capturing.
 *   - A context is used by one host thread at a time; calls sharing a context
 *     on different streams must not overlap (they share its scratch memory).
 */
#ifndef KLR_H
#define KLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KLR_VERSION_MAJOR 0
#define KLR_VERSION_MINOR 1

/* ---- status codes ------------------------------------------------------ */
typedef int32_t klr_status;
#define KLR_OK        0
#define KLR_EINVAL    1   /* bad argument (NULL pointer, bad size, bad enum)   */
#define KLR_ECUDA     2   /* a CUDA runtime call failed; see klr_last_error()   */
#define KLR_ENOMEM    3   /* scratch memory could not be provided               */
#define KLR_ENOTSUP   4   /* valid but unsupported combination of options       */

/* ---- element types ----------------------------------------------------- */
#define KLR_F32 0
#define KLR_F64 1
/* Sample coordinates as 8-bit base-2 logarithms (klr_fit_batch.sample_dtype):
 * x holds uint8 e, the coordinate is 2^e exactly (e > 127 is not finite), and
 * y is FP32.  7 bytes per sample at n_vars = 3 instead of 16 for FP32: the
 * paper's data sizes and block dimensions are powers of two. */
#define KLR_EXP8 2
/* Sample coordinates packed in one 16-bit code per sample
 * (klr_fit_batch.sample_dtype, n_vars = 3): x holds, for sample s, the uint16
 * e_N | e_b0 << 6 | e_b1 << 11 (x_stride unused), the coordinates being
 * (2^e_N, 2^e_b0, 2^e_b1) exactly (N up to 2^63, block dimensions up to
 * 2^31), and y is FP32: 6 bytes per sample.  Accepted where KLR_EXP8 is; a fit
 * of KLR_EXP16 samples equals the fit of the same samples in FP32 bit for
 * bit. */
#define KLR_EXP16 3

/* ---- fit precision modes (how the Gram matrix is accumulated) ------------
 * The Gram matrix G = A^T A of the design matrix A = [Phi | -y Phi] is built
 * from the moment sums  sum_s y_s^k x_s^mu  (k = 0, 1, 2; mu over monomials of
 * degree <= 2d), which determine every entry of G.  The small null-vector
 * solve and the optional refinement passes are FP64 in every mode.
 *   KLR_FIT_FP64: moments accumulated in FP64.
 *   KLR_FIT_DF32: moments accumulated in double-FP32 (error-free transforms on
 *                 FP32 pipes, ~2^-44 relative); needs KLR_F32 samples.  Exact
 *                 products need sample coordinates that are powers of two; a
 *                 fit with other coordinates is flagged KLR_FIT_INEXACT.
 *   KLR_FIT_FP32: moments accumulated in plain FP32 (fast, inaccurate).
 *   KLR_FIT_TF32, KLR_FIT_BF16: Gram products on tensor cores with operands
 *                 rounded to TF32 / BF16, FP32 accumulation.               */
#define KLR_FIT_FP64 0
#define KLR_FIT_DF32 1
#define KLR_FIT_FP32 2
#define KLR_FIT_TF32 3
#define KLR_FIT_BF16 4

/* ---- per-fit status bits ------------------------------------------------- */
#define KLR_FIT_OK              0
#define KLR_FIT_EMPTY           1  /* no samples: coefficients are zero        */
#define KLR_FIT_NONFINITE       2  /* NaN/Inf in the samples: coefficients zero */
#define KLR_FIT_RANK_DEFICIENT  4  /* null space of dimension > 1 (estimated)  */
#define KLR_FIT_INEXACT         8  /* DF32 with non-power-of-two coordinates    */
#define KLR_FIT_SOLVE_FAILED   16  /* the FP64 factorisation broke down         */

/* ---- per-query status bits ----------------------------------------------- */
#define KLR_Q_OK             0
#define KLR_Q_BAD_METRIC     1  /* some meaningful config had q(x) = 0 or a
                                   non-finite metric; it was skipped           */
#define KLR_Q_NONE_FEASIBLE  2  /* no meaningful configuration: best = -1      */
#define KLR_Q_TIE_RESOLVED   4  /* FP32 near-tie re-decided in FP64            */
#define KLR_Q_HISTORY        8  /* answered from the runtime history            */
#define KLR_Q_REFINED       16  /* secondary metric chose another configuration */

typedef struct klr_ctx klr_ctx;

/* Create a context on CUDA device `device` (made current for the call).
 * *out receives the context.  Returns KLR_EINVAL for a bad device index. */
klr_status klr_ctx_create(klr_ctx** out, int device);

/* Destroy a context and free its scratch memory (synchronises the device). */
klr_status klr_ctx_destroy(klr_ctx* ctx);

/* Pre-allocate scratch memory for up to `max_fits` fits and `max_queries`
 * queries, so that later calls of that size allocate nothing (required before
 * capturing calls into a CUDA graph).  Synchronous. */
klr_status klr_ctx_reserve(klr_ctx* ctx, int64_t max_fits, int64_t max_queries);

/* Message of the last error on this thread (static storage, never NULL). */
const char* klr_last_error(void);

/* Library version as major * 100 + minor. */
int klr_version(void);

/* ---- E1: the configuration set F -----------------------------------------
 * Section IV (step 4 and its footnote) and Section V: the candidate block
 * shapes are tuples of powers of two (b0[, b1[, b2]]) whose thread count T is
 * a multiple of 32 with min_threads <= T <= max_threads, ordered by T, then by
 * decreasing b0, then decreasing b1.  dims in 1..3.
 * cfg_out: host, capacity `capacity` rows of 3 int32 (unused dims = 1), may
 * be NULL to query the count; *count receives |F|.  Returns KLR_EINVAL when
 * capacity < |F| and cfg_out is not NULL. */
klr_status klr_enumerate_configs(int dims, int min_threads, int max_threads,
                                 int32_t* cfg_out, int capacity, int* count);

/* ---- F1-F4: batched rational fits ----------------------------------------
 * Section V-E and Section IV step 2.  Fit f owns samples
 * s in [offsets[f], offsets[f+1]).  Sample s has raw coordinates
 * x[v * x_stride + s] (v = 0: N, v = 1..n_vars-1: b0, b1[, b2]) and value y[s].
 * The monomial basis is every monomial of total degree <= degree in the scaled
 * variables (N 2^-n_scale_log2, b 2^-b_scale_log2, ...), ordered by degree,
 * then by decreasing exponent tuple; m = C(n_vars + degree, degree) monomials.
 * The fitted coefficients c = (alpha_1..alpha_m, beta_1..beta_m) of
 * p = sum alpha Phi and q = sum beta Phi are the least-squares null vector of
 * the column-equilibrated design matrix A D, A = [Phi | -y Phi]: D scales
 * column j by 2^-floor(e_j / 2), e_j the binary exponent (frexp) of the
 * column's squared 2-norm; c = D v, normalised to unit 2-norm, with the
 * denominator's constant coefficient positive (if it is below 1e-12 in
 * magnitude, the largest-magnitude denominator coefficient is positive). */
typedef struct klr_fit_batch {
    int32_t n_fits;        /* >= 0                                           */
    int32_t n_vars;        /* 3 (N, b0, b1) or 4 (N, b0, b1, b2)             */
    int32_t degree;        /* total degree, 1..3                             */
    int32_t n_scale_log2;  /* N is scaled by 2^-n_scale_log2                  */
    int32_t b_scale_log2;  /* block dimensions are scaled by 2^-b_scale_log2  */
    int32_t sample_dtype;  /* KLR_F32 or KLR_F64: element type of x and y;
                            * KLR_EXP8: x uint8 log2, y FP32; KLR_EXP16: x
                            * one packed uint16 per sample, y FP32 (both with
                            * KLR_FIT_DF32, the degree-2 basis in (N, b0, b1)
                            * and no refinement; else KLR_ENOTSUP)          */
    const int64_t* offsets;/* device, n_fits + 1, non-decreasing, >= 0        */
    const void* x;         /* device, n_vars rows, row stride x_stride        */
    int64_t x_stride;      /* elements between rows of x, >= offsets[n_fits]  */
    const void* y;         /* device, y[s]                                    */
    int32_t precision;     /* KLR_FIT_*                                        */
    int32_t refine_iters;  /* FP64 refinement passes over the samples, 0..8   */
    int32_t var_degree[4]; /* all 0: the total-degree basis of `degree`; else
                            * var_degree[0] >= 1: the basis of every monomial
                            * with exponent <= var_degree[v] in variable v
                            * (0..3 each, at most 35 monomials; Section V-E's
                            * per-variable degree bounds); `degree` is then
                            * ignored.  Ordered by total degree, then by
                            * decreasing exponent tuple.                       */
} klr_fit_batch;

/* coef_out: device, n_fits x 2m elements of coef_dtype (row-major).
 * fit_status: device, n_fits int32 (KLR_FIT_* bits).
 * fit_diag: device, n_fits x 4 doubles or NULL: (lambda_min / lambda_max of
 *   the equilibrated Gram matrix, an estimate of its next-smallest eigenvalue
 *   over lambda_max, rms of A c over the samples, refinement passes run). */
klr_status klr_fit(klr_ctx* ctx, const klr_fit_batch* batch, void* coef_out,
                   int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                   void* stream);

/* klr_fit in its two stages, for callers that time or schedule them apart.
 * klr_fit_gram: F1-F2, the per-fit moment sums (or, in the TF32/BF16 modes,
 * the tensor-core Gram matrices) into the context's scratch memory.
 * klr_fit_solve: F3-F4 from that scratch, with klr_fit's outputs.  The pair
 * gives bitwise the same outputs as klr_fit when klr_fit_solve follows
 * klr_fit_gram for the same batch, on the same context and stream, with no
 * other call of the context in between (otherwise the solve reads whatever
 * the scratch holds: wrong results, not a fault).  Errors as klr_fit. */
klr_status klr_fit_gram(klr_ctx* ctx, const klr_fit_batch* batch, void* stream);
klr_status klr_fit_solve(klr_ctx* ctx, const klr_fit_batch* batch, void* coef_out,
                         int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                         void* stream);

/* Held-out error of fitted coefficients (for choosing among bases, Section
 * V-E): per fit, sqrt(mean over its samples s of (((p/q)(x_s) - y_s) / y_s)^2)
 * in FP64, with the batch's basis (degree or var_degree), scaling and CSR
 * samples (precision and refine_iters are ignored).  coef: device, n_fits x 2m
 * of coef_dtype.  err_out: device, n_fits doubles (0 for a fit without
 * samples; NaN where q vanishes or a sample is not finite). */
klr_status klr_fit_heldout(klr_ctx* ctx, const klr_fit_batch* batch, const void* coef,
                           int32_t coef_dtype, double* err_out, void* stream);

/* Choice of a basis per fit from held-out errors (Section V-E bounds each
 * variable's degree separately and leaves the bounds to be chosen).  This
 * library's rule: among the candidates whose error is finite and at most
 * (1 + tol) times the fit's least error plus floor, the one with the fewest
 * monomials; ties go to the lower column.  The threshold is computed in FP64
 * as (least * (1 + tol)) + floor, rounded after each operation.
 * errors: device, n_fits x n_cand doubles, row-major (e.g. one klr_fit_heldout
 *   output per column).
 * sizes: HOST, n_cand int32, the monomials of each candidate basis (> 0).
 * choice_out: device, n_fits int32: the chosen column, -1 when no error of the
 *   fit is finite.
 * 1 <= n_cand <= KLR_CHOOSE_BASIS_MAX_CAND, tol >= 0 and floor >= 0 (finite),
 * else KLR_EINVAL before anything is enqueued. */
#define KLR_CHOOSE_BASIS_MAX_CAND 64
klr_status klr_choose_basis(klr_ctx* ctx, const double* errors, const int32_t* sizes,
                            int64_t n_fits, int32_t n_cand, double tol, double floor,
                            int32_t* choice_out, void* stream);

/* ---- E2-E5: the rational program ----------------------------------------- */

/* Hardware parameters H.  Integer limits per SM feed the occupancy program of
 * Fig. 1 / Eq. 1; the rest feed MWP-CWP (Example 2). */
typedef struct klr_hw {
    int32_t n_sm;                  /* number of SMs                            */
    int32_t max_warps_per_sm;      /* W_max                                    */
    int32_t regs_per_sm;           /* R_max (per SM)                           */
    int32_t smem_per_sm;           /* Z_max, bytes per SM                      */
    int32_t max_blocks_per_sm;     /* B_max                                    */
    int32_t max_threads_per_block; /* T_max                                    */
    double mem_latency;            /* cycles (Mem_LD)                          */
    double mem_bandwidth;          /* bytes / second                           */
    double clock_hz;               /* SM clock                                 */
    double departure_delay_coal;   /* cycles between coalesced transactions    */
    double departure_delay_uncoal; /* cycles between uncoalesced transactions  */
} klr_hw;

/* A rational program per kernel: eight fitted metrics, in the order
 * comp_insts, coal_mem_insts, uncoal_mem_insts, synch_insts, coal_per_mw,
 * uncoal_per_mw, load_bytes_per_warp, issue_cycles.  Metric i of a kernel is
 * L_i = metric_lo[i] + metric_scale[i] * |p_i(x) / q_i(x)|, x the scaled
 * (N, b...) point, p_i and q_i in the basis documented for klr_fit.
 * coef_lo + metric_scale must make coal + uncoal >= 1. */
typedef struct klr_program {
    int32_t n_kernels;
    int32_t n_vars;        /* 3 (2D blocks) or 4 (3D blocks)                 */
    int32_t degree;        /* 1..3                                           */
    int32_t n_scale_log2;
    int32_t b_scale_log2;
    int32_t coef_dtype;    /* KLR_F32 or KLR_F64                              */
    const void* coef;      /* device, n_kernels x 8 x 2m                      */
    const int32_t* regs;   /* device, n_kernels: registers per thread R       */
    const int32_t* smem;   /* device, n_kernels: shared memory bytes/block Z  */
    double metric_lo[8];
    double metric_scale[8];
    int32_t var_degree[4]; /* the basis of the fits, as in klr_fit_batch      */
} klr_program;

/* Queries, grouped by kernel: kernel k asks for data sizes
 * q_N[q_offsets[k] .. q_offsets[k+1]) (device arrays; q_offsets has
 * n_kernels + 1 entries, non-decreasing, q_offsets[0] = 0). */
typedef struct klr_queries {
    const int64_t* q_offsets;
    const int64_t* q_N;    /* data sizes, >= 1                               */
    int64_t n_queries;     /* = q_offsets[n_kernels]                         */
} klr_queries;

/* Table mode: cycles of every (query, configuration) pair.
 * cfg: device, n_cfg x 3 int32 block shapes (unused dims 1), n_cfg <= 256,
 *   e.g. from klr_enumerate_configs.  A configuration is meaningful for a
 *   query when B_active > 0, T <= T_max and every block dimension <= N
 *   (footnote to Section IV step 4).
 * cycles_out: device, n_queries x n_cfg of out_dtype; +inf where the
 *   configuration is not meaningful or a metric is invalid.
 * out_dtype selects the arithmetic: KLR_F32 evaluates in FP32, KLR_F64 in FP64.
 */
klr_status klr_eval(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                    const int32_t* cfg, int n_cfg, const klr_queries* q,
                    void* cycles_out, int32_t out_dtype, void* stream);

/* Argmin mode (Section IV step 5): per query the meaningful configuration of
 * least cycles (ties: lowest index; none: -1).
 * best_idx: device int32[n_queries]; best_cycles: device [n_queries] of
 * out_dtype (+inf when none); margin: device float[n_queries] or NULL,
 * (runner-up - best) / best (+inf with one candidate, 0 with none);
 * q_status: device int32[n_queries] or NULL (KLR_Q_* bits);
 * launch_out: device int32[n_queries x 6] or NULL: (gx, gy, gz, bx, by, bz)
 * with g_i = ceil(N / b_i) for the used dimensions (Section V-A, V-C).
 * With out_dtype KLR_F32 the sweep runs in FP32 and every query whose FP32
 * runner-up lies within the FP32 error bound of its best is re-decided by
 * FP64 evaluation of the tied configurations (KLR_Q_TIE_RESOLVED). */
klr_status klr_argmin(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                      const int32_t* cfg, int n_cfg, const klr_queries* q,
                      int32_t* best_idx, void* best_cycles, int32_t out_dtype,
                      float* margin, int32_t* q_status, int32_t* launch_out,
                      void* stream);

/* Section IV, step 5: several configurations may optimise the estimate up to
 * some margin, and a secondary performance metric may refine the choice.
 * The paper fixes neither; this call takes occupancy, a metric the paper
 * names: per query, among the configurations whose cycles in cycles_table
 * (klr_eval's FP32 output for the same queries, n_queries x n_cfg, +inf where
 * not meaningful) are <= (1 + eps) times the least (compared in FP64), the one
 * with the most active warps per SM (Eq. 1); ties by fewer cycles, then the
 * lower index.  best_idx, best_cycles (its cycles), q_status (device, or NULL:
 * KLR_Q_REFINED when the choice differs from the first least-cycles
 * configuration, KLR_Q_NONE_FEASIBLE when nothing is finite).  eps >= 0;
 * eps = 0 gives the plain argmin except among exact ties. */
klr_status klr_argmin_refined(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                              const int32_t* cfg, int n_cfg, const klr_queries* q,
                              const float* cycles_table, double eps, int32_t* best_idx,
                              float* best_cycles, int32_t* q_status, void* stream);

/* ---- runtime history ---------------------------------------------------------
 * Section III-B: the tool keeps a runtime history of its decisions so that
 * later launches get theirs at once.  A history is a device hash table from
 * (kernel index, N) to the outputs of klr_argmin (FP32 mode): best index,
 * best cycles, margin and status.  It belongs to one program, hardware
 * description and configuration set; clear it when any of them changes.
 *   klr_history_create: 2^capacity_log2 slots (10..30; 24 bytes each) on the
 *     context's device; KLR_ENOMEM if the allocation fails.  Synchronous.
 *   klr_history_clear: forget every entry (asynchronous on `stream`).
 *   klr_history_destroy: synchronises the device and frees the table.
 *   klr_argmin_history: klr_argmin with out_dtype KLR_F32 and the same
 *     arguments, where every query whose (kernel, N) is in the history takes
 *     its outputs from there (q_status adds KLR_Q_HISTORY) and is not
 *     evaluated (a kernel whose queries all hit is skipped); the evaluated
 *     queries are recorded afterwards (linear probing over at most 64 slots;
 *     a query that finds no free slot, or has N >= 2^40, is not recorded).
 *     The outputs equal klr_argmin's for the same program.  The context's
 *     scratch holds one byte per query more than klr_argmin's (sized by
 *     klr_ctx_reserve). */
typedef struct klr_history klr_history;
klr_status klr_history_create(klr_ctx* ctx, int32_t capacity_log2, klr_history** out);
klr_status klr_history_clear(klr_history* hist, void* stream);
klr_status klr_history_destroy(klr_history* hist);
klr_status klr_argmin_history(klr_ctx* ctx, klr_history* hist, const klr_program* prog,
                              const klr_hw* hw, const int32_t* cfg, int n_cfg,
                              const klr_queries* q, int32_t* best_idx, float* best_cycles,
                              float* margin, int32_t* q_status, int32_t* launch_out,
                              void* stream);

/* ---- autotuning of the library's launch shapes ----------------------------
 * The paper tunes the launch parameters of the user's kernels; these two calls
 * tune the library's own.  Each runs the operation once per candidate launch
 * shape (one untimed run, then three timed between CUDA events on `stream`),
 * keeps the fastest in the context under the call's problem class (basis,
 * precision, mode and log2 buckets of the batch sizes) and runs it once more,
 * so the outputs are exactly those of klr_fit / klr_argmin with that shape.
 * Later calls of the same class on this context, including calls captured
 * into a CUDA graph, launch with the tuned shape; other classes keep the
 * built-in default.
 *   klr_autotune_fit: moments kernel warps per block (1, 2, 4), then lanes per
 *     fit of the double-word solver (2, 4, 8) where that solver runs.
 *   klr_autotune_argmin: evaluator threads per block (32, 64, 128, 256).
 * Arguments are those of klr_fit / klr_argmin (same layouts, ownership and
 * per-item status), plus choice_out (int32, host, may be NULL: the chosen
 * shape code) and ms_out (float, host, may be NULL: its mean time per call in
 * milliseconds).  Synchronises `stream`.  Returns KLR_EINVAL while `stream` is
 * capturing a graph (tune before capturing) and the operation's own errors. */
klr_status klr_autotune_fit(klr_ctx* ctx, const klr_fit_batch* batch, void* coef_out,
                            int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                            int32_t* choice_out, float* ms_out, void* stream);
klr_status klr_autotune_argmin(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                               const int32_t* cfg, int n_cfg, const klr_queries* q,
                               int32_t* best_idx, void* best_cycles, int32_t out_dtype,
                               float* margin, int32_t* q_status, int32_t* launch_out,
                               int32_t* choice_out, float* ms_out, void* stream);

/* The context's tuned launch shapes as (problem-class key, shape code) pairs,
 * to keep them across runs.  klr_tune_export writes up to `cap` pairs into the
 * host arrays keys/choices (NULL allowed when cap is 0) and sets *n_out to
 * the number the context holds.  klr_tune_import stores n pairs (replacing
 * an existing key's choice); a code outside 0..255 is KLR_EINVAL and stores
 * nothing.  A code is only meaningful for the operation and library version
 * that produced it; out-of-range shape fields fall back to the nearest valid
 * shape.  Host only, no device work. */
klr_status klr_tune_export(klr_ctx* ctx, uint64_t* keys, int32_t* choices, int cap, int* n_out);
klr_status klr_tune_import(klr_ctx* ctx, const uint64_t* keys, const int32_t* choices, int n);

/* ---- learned proposer ------------------------------------------------------
 * The paper has no learned component; these calls add a surrogate of the
 * rational program that proposes candidate block shapes, which the exact
 * program then re-ranks (klr_argmin_candidates), so the rational program is
 * both the fallback and the arbiter of the surrogate.
 *
 * Network (FP32 master parameters, BF16 operands, FP32 accumulation; every
 * dense layer y = x W^T + b with W stored out x in, row-major):
 *   emb  = coef E^T,  E: 64 x n_coef        coef: a kernel's 8 x 2m fitted
 *                                           coefficients (n_coef = 16 m)
 *   x0   = [features(16) | emb(64)]         features: log2 N / 23, log2 b0 / 10,
 *          log2 b1 / 10, log2 b2 / 10 (0 for 2D shapes), the 7 hardware
 *          features hw_feat[7], then zeros
 *   a1 = gelu(x0 W1^T + b1)  W1: 256 x 80;  a2 = gelu(a1 W2^T + b2)  W2: 256 x 256
 *   a3 = gelu(a2 W3^T + b3)  W3: 256 x 256; pred = a3 W4^T + b4      W4: k x 256
 *   gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
 * Two output forms (n_out in klr_mlp):
 *   n_out = 0, per row: k = 1; a row is (kernel, N, block shape); loss = mean
 *     squared error of pred against target[n].
 *   n_out = |F| > 0, per query: k = n_out; a row is (kernel, N), its shape
 *     features are 0 and output c predicts shape c; target is n x n_out and
 *     non-finite entries (shapes that are not meaningful) are masked: loss =
 *     sum of squared errors over the finite targets / their count.  51
 *     outputs per row cost about 1/40 of 51 per-row evaluations.
 * The parameter vector holds E, W1, b1, W2, b2, W3, b3, W4, b4 in that order;
 * klr_mlp_param_count(n_coef, n_out) floats.  pred is trained against a
 * target the caller chooses (normalised log2 cycles). */
typedef struct klr_mlp {
    int32_t n_coef;        /* coefficients per kernel, a multiple of 8        */
    int32_t n_out;         /* 0: per-row output; 1..256: per-query outputs    */
    float* params;         /* device, param_count floats (FP32 master copy)   */
    float* adam_m;         /* device, param_count floats (training only)      */
    float* adam_v;         /* device, param_count floats (training only)      */
    int64_t step;          /* AdamW steps taken; klr_mlp_train_step adds one  */
    float hw_feat[7];      /* hardware features fed to every row              */
} klr_mlp;

/* Rows for the network: row r is (kernel[r], N[r], block shape cfg[cfg_idx[r]]);
 * for a per-query network cfg_idx is ignored (may be NULL) and target holds
 * n x n_out values. */
typedef struct klr_mlp_rows {
    int64_t n;
    const int32_t* kernel;   /* device [n], indexes coef rows                 */
    const int64_t* N;        /* device [n], >= 1                              */
    const int32_t* cfg_idx;  /* device [n], rows of the cfg table             */
    const float* target;     /* device [n] (training only)                    */
} klr_mlp_rows;

/* Number of parameters for n_coef coefficients per kernel and n_out outputs
 * (0: per-row form); 0 for arguments out of range. */
int64_t klr_mlp_param_count(int32_t n_coef, int32_t n_out);

/* One training step on a batch (n <= 262144): forward, mean-squared-error
 * loss, backward, and (if apply_update) one AdamW step with bias correction,
 * betas (0.9, 0.999), eps 1e-8, decoupled weight decay on every parameter.
 * coef: device, n_kernels x n_coef FP32.  cfg: device n_cfg x 3 int32.
 * loss_out: device float or NULL.  grads_out: device, param_count floats or
 * NULL (the batch gradient, before the update). */
klr_status klr_mlp_train_step(klr_ctx* ctx, klr_mlp* net, const float* coef,
                              const int32_t* cfg, int n_cfg, const klr_mlp_rows* rows,
                              float lr, float weight_decay, int apply_update,
                              float* loss_out, float* grads_out, void* stream);

/* Forward pass for a batch of rows (n <= 262144): pred_out device FP32, [n]
 * per row or [n x n_out] per query. */
klr_status klr_mlp_predict(klr_ctx* ctx, const klr_mlp* net, const float* coef,
                           const int32_t* cfg, int n_cfg, const klr_mlp_rows* rows,
                           float* pred_out, void* stream);

/* Training targets from an FP32 cycles table (klr_eval output, n_rows x
 * n_cfg): out[r][c] = log2 cycles[r][c] minus the mean of log2 cycles over
 * row r's finite positive entries (a per-query offset does not change which
 * shape is best), NaN where the entry is not finite or not positive.  Device
 * arrays; asynchronous on `stream`. */
klr_status klr_mlp_query_targets(const float* cycles, int64_t n_rows, int32_t n_cfg, float* out,
                                 void* stream);

/* Proposal: for every query of q (CSR by kernel) predict all n_cfg shapes and
 * keep the k (1..16) of least predicted value among the meaningful ones
 * (B_active > 0, T <= T_max, every b_i <= N; integer occupancy as in
 * klr_argmin).  cand_out: device int32 [n_queries x k], -1 past the number of
 * meaningful shapes.  regs, smem: device int32 [n_kernels].  A per-query
 * network needs n_out == n_cfg (else KLR_EINVAL) and runs once per query; a
 * per-row network runs once per (query, shape). */
klr_status klr_propose(klr_ctx* ctx, const klr_mlp* net, const float* coef,
                       const int32_t* regs, const int32_t* smem, int32_t n_kernels,
                       const klr_hw* hw, const int32_t* cfg, int n_cfg,
                       const klr_queries* q, int k, int32_t* cand_out, void* stream);

/* Exact re-ranking (Section IV, step 5, restricted to candidates): per query,
 * the meaningful candidate of least cycles by the FP32 rational program as
 * klr_argmin's sweep evaluates it (per kernel, only the proposed shapes are
 * specialised); ties go to the lowest shape index; no meaningful candidate:
 * -1 and KLR_Q_NONE_FEASIBLE.  As in klr_argmin, a query whose FP32 least has
 * another candidate shape within the FP32 error window is re-decided by FP64
 * evaluation of the tied candidates (KLR_Q_TIE_RESOLVED; best_cycles then
 * holds the FP64 value rounded to FP32).  cand: device int32 [n_queries x k]
 * shape indices (entries outside 0..n_cfg-1 are skipped; a repeated shape
 * counts once).  best_cycles: device float [n_queries]; q_status: device int32
 * [n_queries] or NULL.  Uses the context's scratch memory (tie records). */
klr_status klr_argmin_candidates(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                                 const int32_t* cfg, int n_cfg, const klr_queries* q,
                                 const int32_t* cand, int k, int32_t* best_idx,
                                 float* best_cycles, int32_t* q_status, void* stream);

/* Argmin without allocation.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate device memory -- a launch hook that
 * picks block shapes right before each kernel launch (a cudaMalloc there would
 * synchronise the application), code that runs while a stream captures a CUDA
 * graph, or a process whose device memory is owned by another allocator.
 *
 * Same computation and outputs as klr_argmin with out_dtype KLR_F32 (best_cycles
 * is float[n_queries]), on the current CUDA device, without a context.  Its
 * scratch (a tie counter and KLR_ARGMIN_NOALLOC_TIE_RECORDS tie records, about
 * 512 KiB) is a static device array of the library, held by every GPU that loads
 * the library until the process exits.  The call allocates nothing: it makes no
 * cudaMalloc, cudaFree or allocating library call.
 *
 * Limits and caveats:
 *   - n_queries must not exceed KLR_ARGMIN_NOALLOC_MAX_QUERIES; larger calls
 *     return KLR_EINVAL and enqueue nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (the call zeroes the counter it needs).  Calls that overlap
 *     on the GPU -- on different streams, or from several host threads --
 *     race on it; serialise them. */
#define KLR_ARGMIN_NOALLOC_MAX_QUERIES 65536
#define KLR_ARGMIN_NOALLOC_TIE_RECORDS 16384
klr_status klr_argmin_noalloc(const klr_program* prog, const klr_hw* hw,
                              const int32_t* cfg, int n_cfg, const klr_queries* q,
                              int32_t* best_idx, float* best_cycles, float* margin,
                              int32_t* q_status, int32_t* launch_out, void* stream);

/* ---- measured peaks ----------------------------------------------------------
 * The denominators of the rooflines of the ALU-bound kernels, measured on the
 * context's device: each probe runs independent dependency chains of one
 * instruction (8 per thread, 64 warps per SM) and takes the best of five
 * timed launches (CUDA events).  Units: 10^12 flop/s (an FMA is 2 flop) or
 * 10^12 operations/s.
 *   fp32_fma_tflops       FFMA (fma.rn.f32)
 *   fp32x2_fma_tflops     packed FFMA2 (fma.rn.f32x2, 4 flop per instruction)
 *   fp64_fma_tflops       DFMA (fma.rn.f64)
 *   mufu_rcp_tops         reciprocal approximations (rcp.approx.ftz.f32)
 *   tf32_mma_sync_tflops  mma.sync.m16n8k8 TF32 with FP32 accumulation (the
 *                         warp-level tensor path; the precision modes' Gram
 *                         and the surrogate's inference issue tcgen05)
 * Synchronous: waits for `stream` (not capturable: KLR_EINVAL while it
 * captures a graph); allocates and frees a few KB of device memory. */
typedef struct klr_peaks {
    double fp32_fma_tflops;
    double fp32x2_fma_tflops;
    double fp64_fma_tflops;
    double mufu_rcp_tops;
    double tf32_mma_sync_tflops;
} klr_peaks;
klr_status klr_probe_peaks(klr_ctx* ctx, klr_peaks* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KLR_H */
