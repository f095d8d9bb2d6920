/*
 * sme.h -- C ABI of the GB300 (sm_103a) library for stochastic matrix-free
 * equilibration (Diamond & Boyd, "Stochastic Matrix-Free Equilibration").
 *
 * The library finds diagonal scalings D = diag(e^u), E = diag(e^v) that
 * approximately equilibrate A in the l2 norm (Section 1: rows of DAE with norm
 * alpha, columns with norm beta, m alpha^2 = n beta^2), by projected stochastic
 * gradient on the regularised, box-constrained problem (eq. (3), Section 2.3)
 * with the randomised row-norm estimator of Section 3.1 (Algorithm 1), and then
 * uses D and E as a diagonal preconditioner for LSQR (Section 5.1).
 *
 * Conventions shared by every entry point
 *   - All pointers to vectors are DEVICE pointers unless the argument says
 *     "host".  Vectors are dense, contiguous, in the op's state type: double
 *     for an SME_F64 op, float otherwise.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it in order; an entry point that returns host results
 *     synchronises that stream before returning and says so.
 *   - Errors are returned as sme_status; nothing throws across the ABI.
 *     sme_last_error() gives a one-line description of the last failure on
 *     the calling thread.  After SME_ERR_CUDA the op should be destroyed.
 *   - The op owns its device copies of A and all scratch it allocates; the
 *     caller owns every vector it passes in.
 *   - Indices are 0-based.  m, n >= 1; nnz < 2^31.
 */
#ifndef SME_H
#define SME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sme_op_s *sme_op;

typedef enum {
    SME_OK = 0,
    SME_ERR_ARG = -1,           /* a null pointer, a size out of range or an inconsistent parameter */
    SME_ERR_INVALID_CSR = -2,   /* row_ptr not monotone / not starting at 0 / not ending at nnz, a column
                                   index outside [0, n), or columns not strictly increasing in a row */
    SME_ERR_OOM = -3,           /* a device allocation failed */
    SME_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    SME_ERR_NONFINITE = -5,     /* a NaN or Inf in the input values or in an iterate */
    SME_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    SME_ERR_NOT_CONVERGED = -7, /* LSQR stopped at max_iters above its tolerance (results still written) */
    SME_ERR_UNSUPPORTED = -8    /* a valid request the library does not implement (e.g. an unsupported k) */
} sme_status;

typedef enum {
    SME_F64 = 0,   /* double values, double state vectors */
    SME_F32 = 1,   /* float values, float state vectors */
    SME_BF16 = 2,  /* dense only: bfloat16 values, float state vectors */
    SME_FP8E4M3 = 3 /* dense only: e4m3 values with one float scale per row, float state vectors */
} sme_dtype;

const char *sme_status_string(sme_status s);
const char *sme_last_error(void);

/*
 * sme_release_cached_memory -- return the library's idle device memory to the system.
 *
 * The device buffers of destroyed operators (and the staging of host input during
 * operator creation) are kept, by exact size, for later operators: creating and
 * destroying an operator per solve then allocates nothing after the first time.
 * Stream-ordered scratch of the device builds comes from a library memory pool that
 * keeps its memory between calls.  This call frees every idle block and trims the
 * pool; an allocation that fails does the same before trying again.  Operators that
 * are alive are not affected.  Synchronises the device.  Always SME_OK.
 */
sme_status sme_release_cached_memory(void);

/* ------------------------------------------------------------------ operators */

/*
 * sme_op_create_csr -- build the operator for a sparse A (m x n) given in CSR.
 *
 * The method touches A only through products with A and A^T (Section 3,
 * "matrix-free").  The op keeps, on the device:
 *   - a sliced-ELL copy of A (32-row slices, rows ordered by length), for A.x;
 *   - a transposed copy built ON THE DEVICE from the CSR by a stable radix
 *     sort on column index (no atomics in the products), for A^T.y.
 * row_ptr: int32[m+1], row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz.
 * col_idx: int32[nnz], strictly increasing within each row, in [0, n).
 * vals:    nnz values of `dtype` (SME_F64 or SME_F32).
 * on_device = 0: the three arrays are host memory (validated on the host);
 * on_device = 1: they are device memory (validated by a device check).
 * Empty rows and columns are allowed (problem (3) stays bounded, Section 2.3).
 * Synchronises `stream`.  Returns SME_ERR_INVALID_CSR / SME_ERR_NONFINITE on bad input.
 */
sme_status sme_op_create_csr(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                             const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device,
                             void *stream);

/*
 * sme_op_create_dense -- build the operator for a dense row-major A (m x n).
 * dtype SME_BF16: A is bfloat16, lda >= n elements.
 * dtype SME_FP8E4M3: A is e4m3 (one byte per entry), row_scales[m] floats with
 *   A_ij = row_scales[i] * e4m3(A_ij); pass NULL for unit scales.
 * Products with the +-1 probe blocks run on the tcgen05 tensor cores with FP32
 * accumulation (Section 3.1 estimator, dense A).  m and n must be multiples of 128,
 * and m*n below 2^37 (SME_ERR_UNSUPPORTED otherwise).  The op holds A and A^T (2 bytes
 * per entry each) in a K-blocked order.  on_device as for the CSR form.  Synchronises
 * `stream`.
 */
sme_status sme_op_create_dense(sme_op *out, int64_t m, int64_t n, const void *A, int64_t lda, sme_dtype dtype,
                               const float *row_scales, int on_device, void *stream);

/*
 * sme_op_destroy -- release an operator (NULL is allowed).  Synchronises the device; the
 * op's device blocks are then kept for reuse by later operators of the same sizes (see
 * sme_release_cached_memory).  Always SME_OK.
 */
sme_status sme_op_destroy(sme_op op);

typedef struct {
    int64_t m, n, nnz;          /* nnz = m*n for a dense op */
    int32_t dtype;              /* sme_dtype of the values */
    int32_t state_is_double;    /* 1 when state vectors are double */
    int64_t device_bytes;       /* device memory the op holds */
    int64_t padded_entries_fwd; /* sliced-ELL entries incl. padding, A and A^T copies */
    int64_t padded_entries_bwd;
    double last_loop_ms;        /* with SME_EQ_TIMED: device time of the last call's iteration loop */
    int64_t last_loop_iters;    /* iterations in that loop */
} sme_op_info;

sme_status sme_op_get_info(sme_op op, sme_op_info *info);

/* ------------------------------------------------------------------ probes */

/*
 * sme_draw_probes -- the IID uniform {-1,+1} probe draw of Algorithm 1, as bits.
 *
 * Philox4x32-10 (Salmon et al., SC'11) with
 *   key = (seed mod 2^32, seed >> 32), counter = (index, t, stream_id, p >> 7),
 *   word = out[(p >> 5) & 3], sign of probe p at `index` = bit (p & 31) set ? -1 : +1.
 * Writes words[w * len + index] for w < ceil(k/32), index < len (device uint32).
 * Stream ids: 2*b for s (columns) and 2*b+1 for w (rows) of matrix b of a batch.
 */
sme_status sme_draw_probes(uint64_t seed, int32_t t, int32_t stream_id, int64_t len, int32_t k,
                           uint32_t *words, void *stream);

/* ------------------------------------------------------------------ equilibration */

typedef struct {
    double alpha, beta;   /* target row / column norms; <= 0 selects (n/m)^(1/4), (m/n)^(1/4) (Section 4) */
    double gamma;         /* regularisation of eq. (3); <= 0 selects 0.1 (Section 4) */
    double M;             /* box |u|,|v| <= M of eq. (3); <= 0 selects log(1e4) (Section 4) */
    int32_t T;            /* iterations performed by this call, >= 0 */
    int32_t k;            /* probes per iteration (estimates averaged over the k probes); 1,2,4,...,64 */
    int32_t t_begin;      /* index t of the first iteration (>= 1); > 1 resumes a run */
    int32_t t0;           /* step offset: eta_t = 2 / (gamma (t + t0 + 1)); 0 is Algorithm 1 */
    uint64_t seed;        /* Philox key for the probes */
    int32_t stream_base;  /* Philox stream pair: stream_base for s, stream_base + 1 for w */
    int32_t flags;        /* SME_EQ_* bits */
} sme_equil_params;

#define SME_EQ_ASYNC 1    /* do not synchronise or read the status word; see sme_op_check */
#define SME_EQ_NO_GRAPH 2 /* launch the iterations directly instead of through a cached CUDA graph */
#define SME_EQ_TIMED 4    /* time the iteration loop with CUDA events on `stream` (read by sme_op_get_info) */
/* Test of the failure path of the tensor-core (dense) operators: the TMA producer's and the MMA issuer's
 * waits get a bound of zero polls, so every launch gives up before its first MMA, writes no iterate, and the
 * call returns SME_ERR_TIMEOUT; the drain waits (the accumulator, MMAs in flight before TMEM is freed, copies
 * landing) keep their full bound.  The iterates are left as passed in.  Sparse operators ignore it. */
#define SME_EQ_EXPIRE_PIPELINE_WAITS 8

/*
 * sme_equilibrate -- iterations t_begin .. t_begin+T-1 of Algorithm 1 (Section 3.2):
 *   D = diag(e^{u^{t-1}}), E = diag(e^{v^{t-1}});
 *   z_u = (1/k) sum_p |D A E s_p|^2,  z_v = (1/k) sum_p |E A^T D w_p|^2   (both from the previous iterate);
 *   u^t = Pi_[-M,M](u^{t-1} - 2 (z_u - alpha^2 + gamma u^{t-1}) / (gamma (t + t0 + 1))), v^t likewise;
 *   ubar <- 2 u^t / (t + 2) + t ubar / (t + 2), vbar likewise.
 * u[m], v[n]: in: u^{t_begin-1}, v^{t_begin-1} (zeros for the paper's start); out: the last iterate.
 * u_bar[m], v_bar[n]: in: the averages after t_begin-1 iterations (zeros at the start); out: updated.
 * The outputs D = diag(e^{u_bar}), E = diag(e^{v_bar}) are the method's result.
 * Unless SME_EQ_ASYNC, synchronises `stream` and returns SME_ERR_NONFINITE if an iterate was not finite.
 */
sme_status sme_equilibrate(sme_op op, const sme_equil_params *p, void *u, void *v, void *u_bar, void *v_bar,
                           void *stream);

/*
 * sme_op_autotune -- choose the launch shape of the iteration kernel for probe count k on this sparse
 * operator: 32-row slices per CTA (4, 8 or 16; FP32 with k = 16 or 32, otherwise 8) and whether the
 * A^T CTAs are dispatched before the A CTAs.  Every candidate is timed (CUDA events, estimate mode) and
 * the fastest is kept for later calls with this k.  Outputs are optional host pointers.  The rows'
 * ordering (the length sort of the sliced ELL) is fixed at creation.  sme_batch_equilibrate calls this
 * on its first use of a k.  Synchronises `stream`.
 */
sme_status sme_op_autotune(sme_op op, int32_t k, int32_t *slices_per_cta, int32_t *cols_first,
                           float *ms_per_iteration, void *stream);

/*
 * sme_equilibrate_targets -- Algorithm 1 for varying row and column norms (Section 6): the rows of DAE
 * should have squared norms row_targets_sq[i] and the columns col_targets_sq[j] (device vectors in the
 * state type, original order; the problem is consistent when their sums agree).  The gradient estimate
 * becomes |DAE s|^2 - r + gamma u (and likewise for v); alpha and beta in p are ignored.  Sparse,
 * single (non-batch) operators.  Otherwise as sme_equilibrate.
 */
sme_status sme_equilibrate_targets(sme_op op, const sme_equil_params *p, const void *row_targets_sq,
                                   const void *col_targets_sq, void *u, void *v, void *u_bar, void *v_bar,
                                   void *stream);

/*
 * sme_equilibrate_symmetric -- Algorithm 2 (symmetric equilibration, Section 6): D = E = diag(e^u) for a
 * square symmetric A, one probe block s per iteration (Philox stream stream_base), estimate
 * z = (1/k) sum_p |D A D s_p|^2 and the projected step of Algorithm 1 on u alone.  u[n], u_bar[n] in/out
 * as in sme_equilibrate; alpha <= 0 selects 1.  A's symmetry is the caller's promise (not checked).
 */
sme_status sme_equilibrate_symmetric(sme_op op, const sme_equil_params *p, void *u, void *u_bar, void *stream);

/*
 * sme_equilibrate_block -- block equilibration (Section 6): rows in p_blocks contiguous blocks
 * [row_block_ptr[b], row_block_ptr[b+1]) share the scaling e^{u_b}, columns in q_blocks blocks share
 * e^{v_c} (HOST offset arrays of p_blocks+1 and q_blocks+1 entries, starting at 0 and ending at m / n).
 * The block gradient is sum_{i in b} (|DAE|^2 1)_i - alpha^2 m_b + gamma u_b, estimated by summing the
 * rows' estimates of the block.  u, u_bar hold p_blocks entries, v, v_bar q_blocks (device, state type).
 */
sme_status sme_equilibrate_block(sme_op op, const sme_equil_params *p, int64_t p_blocks,
                                 const int64_t *row_block_ptr, int64_t q_blocks, const int64_t *col_block_ptr,
                                 void *u, void *v, void *u_bar, void *v_bar, void *stream);

/* sme_op_check -- synchronise `stream`, return and clear the op's device status word. */
sme_status sme_op_check(sme_op op, void *stream);

/*
 * sme_estimate -- the estimator alone (Section 3.1) for iteration t's probes:
 *   z_u[i] = (1/k) sum_p ((D A E s_p)_i)^2,  z_v[j] = (1/k) sum_p ((E A^T D w_p)_j)^2
 * with D = diag(e^u), E = diag(e^v), probes from (seed, t, stream_base[+1]).  z_u[m], z_v[n] device
 * outputs in the state type; either may be NULL to skip it.
 */
sme_status sme_estimate(sme_op op, const void *u, const void *v, int32_t t, int32_t k, uint64_t seed,
                        int32_t stream_base, void *z_u, void *z_v, void *stream);

/* ------------------------------------------------------------------ evaluation */

typedef struct {
    double row_spread;   /* max/min l2 norm over nonempty rows of DAE */
    double col_spread;   /* max/min l2 norm over nonempty columns of DAE */
    double rms;          /* RMS equilibration error (Section 4) */
    double objective;    /* f(u, v) of eq. (3) */
    int64_t empty_rows, empty_cols;
} sme_eval_result;

/*
 * sme_evaluate -- exact squared row and column norms of DAE (the optimality
 * conditions of Section 2.1) with FP64 accumulation, and the metrics above.
 * r2[m], c2[n]: optional device outputs (double), may be NULL.  `res` is a host
 * struct.  alpha, beta, gamma <= 0 select the Section 4 defaults.  Synchronises `stream`.
 */
sme_status sme_evaluate(sme_op op, const void *u, const void *v, double alpha, double beta, double gamma,
                        double *r2, double *c2, sme_eval_result *res, void *stream);

/* ------------------------------------------------------------------ LSQR */

typedef struct {
    double tol;          /* stop when the selected residual <= tol (e.g. 1e-6) */
    int64_t max_iters;   /* iteration cap */
    int32_t check_every; /* true residual (FP64) checked every this many iterations (>= 1) */
    int32_t stop_rule;   /* 0: ||A x - b|| / ||b||;  1: ||A^T r|| / (||A||_F ||r||) (least squares) */
    double *history;     /* HOST, may be NULL: the selected residual at every check, in order (sme_lsqr only) */
    int64_t history_cap; /* entries history can hold */
    int32_t predict_check; /* sme_lsqr, stop_rule 0, tol > 0: bring a check forward to the iteration at which
                              the geometric trend of the last two checked residuals (the first being 1 at
                              x = 0) reaches tol; checks stay at most check_every apart, and stopping still
                              rests only on the checked FP64 residual */
} sme_lsqr_params;

typedef struct {
    int64_t iters;            /* LSQR iterations performed */
    double rel_residual;      /* ||A x - b|| / ||b|| of the ORIGINAL system, FP64 */
    double normal_residual;   /* ||A^T (A x - b)|| / (||A||_F ||A x - b||), FP64 */
    int32_t converged;
    int64_t kernel_launches;  /* device kernels this call launched */
    int64_t history_count;    /* entries written to p->history */
} sme_lsqr_result;

/*
 * sme_lsqr -- LSQR (Paige & Saunders 1982) on the equilibrated operator (Section 5.1):
 * solves (D A E) xbar = D b from xbar = 0 and returns x = E xbar.  D = diag(e^{u_bar}),
 * E = diag(e^{v_bar}); u_bar == NULL means D = I (column scaling only, which keeps the
 * least-squares minimiser of an inconsistent system), and both NULL is plain LSQR.
 * Vectors are in the state type; the scalar recurrences (rho, phibar, norms) and the
 * residual checks run in FP64 on the device, so there is no host round trip per iteration.
 * b[m] device input, x[n] device output.  Synchronises `stream`; `res` is a host struct.
 * Returns SME_ERR_NOT_CONVERGED (x still written) when max_iters is reached above tol.
 */
sme_status sme_lsqr(sme_op op, const void *u_bar, const void *v_bar, const void *b, void *x,
                    const sme_lsqr_params *p, sme_lsqr_result *res, void *stream);

/* ------------------------------------------------------------------ batches */

/*
 * A batch of sparse matrices equilibrated together (Algorithm 1 run on each matrix, all matrices
 * advanced by the same launches).  The batch is one block-diagonal operator diag(A_0, ..., A_{B-1})
 * laid out matrix by matrix (each matrix's rows and columns sorted by length), so one launch serves
 * matrices of very different sizes.  Matrix b draws its probes from Philox streams stream_base + 2b (s)
 * and stream_base + 2b + 1 (w) with counters indexed inside matrix b, so its result equals a separate
 * sme_equilibrate of A_b with stream_base + 2b (bit for bit when both share slices among the same number
 * of warps, which is always the case for rows and columns under 48 nonzeros on average).
 * SME_BATCH_GROUP_BYTES (environment) > 0 lays out groups of consecutive matrices whose gather tables fit
 * that many bytes instead of single matrices.
 */
typedef struct sme_batch_s *sme_batch;

/*
 * sme_batch_create -- count matrices in CSR, HOST arrays: m[b], n[b], row_ptr[b] (int32[m[b]+1]),
 * col_idx[b], vals[b] (dtype SME_F32 or SME_F64), each validated as in sme_op_create_csr.  The totals of
 * rows, columns and nonzeros must stay below 2^31.  Synchronises `stream`.
 */
sme_status sme_batch_create(sme_batch *out, int32_t count, const int64_t *m, const int64_t *n,
                            const int32_t *const *row_ptr, const int32_t *const *col_idx, const void *const *vals,
                            sme_dtype dtype, void *stream);
sme_status sme_batch_destroy(sme_batch b);

/* Number of matrices and the offsets of matrix b's rows [row_off[b], row_off[b+1]) and columns in the
 * concatenated vectors (host arrays of count + 1 entries, either may be NULL). */
sme_status sme_batch_get_info(sme_batch b, int32_t *count, int64_t *row_off, int64_t *col_off);

/*
 * sme_batch_equilibrate -- sme_equilibrate for every matrix of the batch at once.  u, u_bar are the
 * concatenated row vectors (sum of m[b] entries, matrix order), v, v_bar the concatenated column
 * vectors.  alpha, beta <= 0 select each matrix's own (n_b/m_b)^(1/4), (m_b/n_b)^(1/4); gamma, M, T, k,
 * t_begin, t0, seed, flags apply to all.  Unless SME_EQ_ASYNC, synchronises and checks the status word.
 */
sme_status sme_batch_equilibrate(sme_batch b, const sme_equil_params *p, void *u, void *v, void *u_bar,
                                 void *v_bar, void *stream);

/* sme_estimate for every matrix of the batch (concatenated vectors; probes as in sme_batch_equilibrate). */
sme_status sme_batch_estimate(sme_batch b, const void *u, const void *v, int32_t t, int32_t k, uint64_t seed,
                              int32_t stream_base, void *z_u, void *z_v, void *stream);

/*
 * sme_batch_lsqr -- sme_lsqr for every matrix of the batch, each with its own LSQR (own FP64 scalar
 * recurrence, own residual checks and convergence; a converged matrix stops changing while the others
 * continue).  u_bar, v_bar (nullable), b and x are the concatenated vectors; results is a HOST array of
 * one sme_lsqr_result per matrix (kernel_launches is reported in results[0]).  Returns
 * SME_ERR_NOT_CONVERGED when any matrix stopped above tol (all results still written).  Synchronises.
 */
sme_status sme_batch_lsqr(sme_batch b, const void *u_bar, const void *v_bar, const void *bvec, void *x,
                          const sme_lsqr_params *p, sme_lsqr_result *results, void *stream);

/* The block-diagonal operator of the batch (owned by the batch; do not destroy it), for sme_evaluate
 * of all matrices at once (row / column norms come back concatenated). */
sme_status sme_batch_op(sme_batch b, sme_op *op);

/*
 * sme_batch_evaluate -- sme_evaluate for every matrix of the batch: res is a HOST array of one
 * sme_eval_result per matrix (spread over that matrix's nonempty rows / columns, RMS against its own
 * targets, its own f(u, v) of eq. (3)).  alpha, beta <= 0 select each matrix's Section 4 defaults
 * (n_b/m_b)^(1/4), (m_b/n_b)^(1/4); gamma <= 0 selects 0.1.  u, v: concatenated state vectors.
 * Synchronises `stream`.
 */
sme_status sme_batch_evaluate(sme_batch b, const void *u, const void *v, double alpha, double beta, double gamma,
                              sme_eval_result *res, void *stream);

/* ------------------------------------------------------------------ Chambolle-Cremers-Pock (Section 5.2) */

/*
 * sme_op_norm2 -- ||D A E||_2 by `iters` steps of power iteration on K^T K (K = D A E), started at the unit
 * vector 1/sqrt(n); returns sqrt(||K^T K p||) for the last unit iterate p in *norm (host).  u_bar, v_bar
 * (state type, device) may be NULL for D = I or E = I.  Single sparse operators only.  Synchronises.
 */
sme_status sme_op_norm2(sme_op op, const void *u_bar, const void *v_bar, int32_t iters, double *norm, void *stream);

typedef struct {
    double lambda;       /* > 0: the Lasso weight; the paper uses 1e-3 ||A^T b||_inf */
    double tau, sigma;   /* primal / dual steps; <= 0 selects 0.9 / ||D A E||_2 (Section 5.2) */
    double theta;        /* extrapolation; <= 0 selects 1 */
    int64_t max_iters;
    int32_t check_every; /* the objective is evaluated (FP64, original system) every check_every iterations */
    int32_t norm_iters;  /* power iterations for ||D A E||_2 when a step is selected; <= 0 selects 100 */
    double p_star;       /* known optimal value (> 0), for the stopping rule; <= 0: run max_iters */
    double tol;          /* stop at the first check with (f(x) - p_star) / f(0) <= tol */
} sme_ccp_params;

typedef struct {
    int64_t iters;        /* iterations done */
    double objective;     /* f(x) at the returned x */
    double objective0;    /* f(0) = ||b||^2 / sqrt(lambda) */
    double rel_gap;       /* (f(x) - p_star) / f(0), NaN without p_star */
    double op_norm;       /* ||D A E||_2 used for the steps (0 when both steps were given) */
    double tau, sigma;    /* the steps used */
    int32_t converged;    /* 1 when rel_gap <= tol */
    int64_t kernel_launches;
    int64_t history_count; /* entries written to history */
} sme_ccp_result;

/*
 * sme_ccp_lasso -- the Lasso problem of Section 5.2,
 *     minimize ||A x - b||^2 / sqrt(lambda) + sqrt(lambda) ||x||_1,
 * by the Chambolle-Cremers-Pock primal-dual method on the equilibrated operator D A E (x = E xs), all
 * iterates starting at 0.  u_bar, v_bar: the log-scalings (device, state type; NULL for no scaling on that
 * side).  b[m] (device) and x[n] (device, output, original variables).  history (host, may be NULL): f(x)
 * at every check, up to history_cap entries.  Single sparse operators only.  Synchronises.
 */
sme_status sme_ccp_lasso(sme_op op, const void *u_bar, const void *v_bar, const void *b, void *x,
                         const sme_ccp_params *p, sme_ccp_result *res, double *history, int64_t history_cap,
                         void *stream);

/* ------------------------------------------------------------------ learned warm start */

/*
 * A small MLP that predicts initial log-scalings u^0, v^0 from per-row / per-column features, so that
 * Algorithm 1 can start near its optimum.  The paper has no such component; it uses the paper's method
 * unchanged.  Because the paper's first step eta_1 = 1/gamma discards u^0 (u^1 depends on u^0 only
 * through the estimate), a warm start is used with a step offset t0 > 0 in sme_equil_params.
 *
 * Network: 8 normalised features -> 128 (ReLU) -> 128 (ReLU) -> 1, BF16 weights for the forward pass,
 * FP32 master weights and FP32 accumulation, trained on the device by sme_mlp_train_step (mean squared
 * error, Adam).  The 128 x 128 layer and its gradients run on the tensor cores (BF16 operands, the
 * activations split into several BF16 terms so that the results keep FP32 accuracy).  Their completion
 * waits are bounded: one that runs out leaves NaN in that call's outputs and sets a status word that the
 * next sme_mlp_gradient / sme_mlp_train_step with a loss read reports as SME_ERR_TIMEOUT.  Features of row i (column j), see sme_op_features:
 *   [ 1/2 log of the k = 8 sketch of the squared norm (sme_estimate at u = v = 0, t = 1),
 *     log(1 + nonzeros), log(mean |A_ij|), side (0 rows, 1 columns),
 *     mean sketch log-norm of the rows, of the columns, log m, log n ].
 */
typedef struct sme_mlp_s *sme_mlp;

sme_status sme_mlp_create(sme_mlp *out, uint64_t seed);  /* He initialisation from `seed` */
sme_status sme_mlp_destroy(sme_mlp mlp);
int64_t sme_mlp_param_count(void);
/* Host copies of the FP32 parameters (sme_mlp_param_count floats) and of the input normalisation
 * (8 means then 8 scales); either pointer may be NULL.  set_params synchronises the device. */
sme_status sme_mlp_get_params(sme_mlp mlp, float *params, float *norm);
sme_status sme_mlp_set_params(sme_mlp mlp, const float *params, const float *norm);
/* y[i] = MLP(X[i, :]) for X a device float array N x 8 (row-major). */
sme_status sme_mlp_forward(sme_mlp mlp, const float *X, int64_t N, float *y, void *stream);
/* Gradient of (1/N) sum_i (MLP(X_i) - target_i)^2 with respect to the parameters (device grad, may be
 * NULL) and the loss (host, may be NULL; synchronises when given).  Deterministic. */
sme_status sme_mlp_gradient(sme_mlp mlp, const float *X, const float *target, int64_t N, float *grad,
                            float *loss, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999) on the same loss with learning rate lr. */
sme_status sme_mlp_train_step(sme_mlp mlp, const float *X, const float *target, int64_t N, float lr, float *loss,
                              void *stream);
/* Input normalisation fitted to training features X (N x 8 device floats, 16-byte aligned, N >= 2): the
 * per-feature mean and standard deviation (N - 1 in the denominator; a deviation <= 1e-6 is replaced by 1),
 * each summed in FP64 in a fixed order; then set as by sme_mlp_set_params.  Synchronises `stream`. */
sme_status sme_mlp_fit_normalisation(sme_mlp mlp, const float *X, int64_t N, void *stream);
/* A minibatch for sme_mlp_train_step: X_batch (batch x 8), target_batch (batch) filled with rows of (X, target)
 * (N rows, N < 2^32) drawn uniformly with replacement.  Draw b of step `step` takes row floor(r N / 2^32), r the
 * first output word of Philox4x32-10 at counter (b mod 2^32, b >> 32, step, 0x6D6C7000) with key
 * (seed mod 2^32, seed >> 32).  X and X_batch 16-byte aligned. */
sme_status sme_mlp_draw_batch(const float *X, const float *target, int64_t N, int64_t batch, uint64_t seed,
                              int64_t step, float *X_batch, float *target_batch, void *stream);
/* Features of every row (m x 8) and column (n x 8) of a sparse operator, device float arrays.  For the
 * operator of a batch, the mean sketch norms and the sizes are those of each row's / column's own matrix. */
sme_status sme_op_features(sme_op op, uint64_t seed, float *row_features, float *col_features, void *stream);
/* u0[m], v0[n] (state type) = the MLP's prediction for every row and column of `op`. */
sme_status sme_warm_start(sme_op op, sme_mlp mlp, uint64_t seed, void *u0, void *v0, void *stream);
/* The same two for all matrices of a batch (concatenated rows, concatenated columns). */
sme_status sme_batch_features(sme_batch b, uint64_t seed, float *row_features, float *col_features, void *stream);
sme_status sme_batch_warm_start(sme_batch b, sme_mlp mlp, uint64_t seed, void *u0, void *v0, void *stream);

/* ------------------------------------------------------------------ one matrix split over several devices */

/*
 * Algorithm 1 on one matrix split over P devices (one process per device).  Rows and columns are cut
 * into P contiguous blocks, block q = [len q / P, len (q + 1) / P).  Part p holds row block p of A (its
 * forward products, Section 3.1: z_u of its rows) and column block p of A^T (z_v of its columns), and
 * nothing else of the matrix.  Every iteration of Algorithm 1 needs both estimates at the previous iterate
 * (u^{t-1}, v^{t-1}): a part's rows read e^{v_j} and the probe signs s_j of EVERY column, its columns read
 * e^{u_i} and w_i of every row.  These live in two gather tables that each part writes for its own rows
 * and columns and that the caller all-gathers between iterations (the one exchange of the method: m + n
 * entries per iteration; probe signs are counter-based, so none are exchanged).
 *
 * Tables: the row table has P * row_chunk entries, the column table P * col_chunk, of entry_bytes each
 * (sme_shard_get_info); part q writes entries [q * chunk, (q + 1) * chunk) (its block's rows in the
 * library's internal order, the rest of the chunk unused), so an in-place all-gather of equal chunks
 * assembles them.  The caller owns the tables (device memory) and keeps two of each, for the current and
 * the next iteration.  A run:
 *     sme_shard_begin (writes this part's chunks of the tables of iteration t_begin)
 *     all-gather both tables
 *     for t = t_begin .. t_begin + T - 1:
 *         sme_shard_step(t, current tables -> this part's chunks of the next tables); all-gather the next tables
 *     sme_shard_end
 * Each part draws exactly the probes an unsplit run draws (probe counters use the whole matrix's index), so
 * the parts' results together equal the unsplit sme_equilibrate's (bit for bit where no row is long enough
 * for the kernel to share it among warps; otherwise up to the order of the sums).
 */
typedef struct {
    int32_t parts, part;
    int64_t m, n;                    /* the whole matrix */
    int64_t row_begin, row_end;      /* this part's rows [row_begin, row_end) */
    int64_t col_begin, col_end;      /* this part's columns */
    int64_t row_chunk, col_chunk;    /* table entries per part */
    int32_t entry_bytes;             /* bytes per table entry for the k given to sme_shard_get_info */
} sme_shard_info;

/* Part `part` of `parts` of the CSR matrix (the whole matrix is passed; host or device as in
 * sme_op_create_csr, SME_F64 or SME_F32).  1 <= parts <= min(m, n).  The op refuses the whole-matrix calls
 * (sme_equilibrate, sme_estimate, sme_lsqr, ...: SME_ERR_UNSUPPORTED) and runs only sme_shard_*. */
sme_status sme_op_create_csr_shard(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                   const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device,
                                   int32_t parts, int32_t part, void *stream);
sme_status sme_shard_get_info(sme_op op, int32_t k, sme_shard_info *info);
/* u[row_end - row_begin], u_bar (this part's rows, in row order), v[col_end - col_begin], v_bar: the start
 * state (state type); p as for sme_equilibrate (alpha, beta default from the whole matrix's m, n). */
sme_status sme_shard_begin(sme_op op, const sme_equil_params *p, const void *u, const void *v, const void *u_bar,
                           const void *v_bar, void *row_table, void *col_table, void *stream);
/* Iteration t: reads the whole current tables, writes this part's chunks of the next ones (other buffers).
 * SME_ERR_ARG, with nothing launched, before a successful sme_shard_begin on this op or when p->k needs table
 * entries of another size than the k given to sme_shard_begin (the tables are sized for one entry size). */
sme_status sme_shard_step(sme_op op, const sme_equil_params *p, int32_t t, const void *row_table_in,
                          const void *col_table_in, void *row_table_out, void *col_table_out, void *stream);
/* This part's u, v, u_bar, v_bar after the last step (SME_ERR_ARG before a successful sme_shard_begin). */
sme_status sme_shard_end(sme_op op, void *u, void *v, void *u_bar, void *v_bar, void *stream);

/* ------------------------------------------------------------------ allocation-free estimator */

/*
 * sme_estimate_rows_static -- the row-side estimate of sme_estimate (z_u only, FP32),
 * for callers that must not allocate device memory on this path: code whose device
 * memory is already owned by a caching allocator (a framework pool that reserved the
 * free memory), a latency-critical loop that cannot take the device-wide
 * synchronisation an allocation or a free may cause, or a plug-in handed fixed device
 * buffers by a host application that keeps the memory budget to itself.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 *
 * Works directly on the caller's device CSR (row_ptr int32[m+1], col_idx int32[nnz],
 * vals float[nnz]) and device vectors u[m], v[n]; writes z_u[m].  Probes as in
 * sme_estimate (iteration t, Philox stream stream_base for s).  k in {1,2,4,...,32}.
 *
 * Calls no cudaMalloc/cudaFree.  Its only scratch, a gather table of n entries,
 * is a fixed array of SME_STATIC_MAX_COLS entries (8 bytes each, 8 MiB) inside the
 * library; every GPU that loads the library holds it until the process exits.
 * n > SME_STATIC_MAX_COLS returns SME_ERR_ARG.  All calls on a device share the
 * array and it keeps the last call's contents (each call rewrites the n entries it
 * reads, so nothing needs clearing): calls whose GPU work overlaps (unordered
 * streams) race on it.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it, so make that first call before
 * beginning any stream capture; a device reset (cudaDeviceReset) invalidates the
 * kept address, so do not call this entry point again in a process after one.
 *
 * The CSR is not validated on the host (row_ptr must be nondecreasing from 0, with
 * row_ptr[m] entries in col_idx and vals).  A column index outside [0, n) is never
 * used to address the table: its row is written as NaN, the other rows are exact.
 */
#define SME_STATIC_MAX_COLS (1 << 20)

sme_status sme_estimate_rows_static(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                    const float *vals, const float *u, const float *v, int32_t t, int32_t k,
                                    uint64_t seed, int32_t stream_base, float *z_u, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SME_H */
