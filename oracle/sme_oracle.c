/*
 * Plain FP64 CPU oracle for stochastic matrix-free equilibration
 * (Diamond & Boyd, "Stochastic Matrix-Free Equilibration").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by the test
 * suite, by the smoke check and by the bench's CPU-baseline leg.  The product
 * path never links or calls it, and it shares no code, header or constant
 * table with the CUDA library.
 *
 * Everything here is written for a reader to check against the paper by eye:
 * loops follow the definitions, in FP64, with no blocking, fusion or
 * reordering beyond what the definition states.
 *
 *   - Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
 *     as easy as 1, 2, 3", SC'11 (round function and constants from that
 *     paper).  The equilibration paper only asks for IID uniform {-1,+1}
 *     probes (Algorithm 1); the counter layout that makes both sides draw the
 *     same signs is the probe contract below.
 *   - Row-norm estimator z = |B s|^2 (Section 3.1, "Estimating row norms
 *     squared"), averaged over k probes.
 *   - One step of Algorithm 1 (Section 3.2): both estimates use the previous
 *     iterate (u^{t-1}, v^{t-1}); step 2/(gamma (t + t0 + 1)); projection on
 *     [-M, M]; running weighted averages.  t0 = 0 is the paper's method.
 *   - Exact squared row/column norms of DAE (Section 2.1 optimality
 *     conditions), used for the spread and RMS metrics (Section 4).
 *
 * Probe contract (the paper draws s, w IID and says nothing about how):
 *   key     = (seed mod 2^32, seed >> 32)
 *   counter = (index, t, stream, p >> 7)       stream 0: s over columns,
 *                                              stream 1: w over rows
 *   word    = out[(p >> 5) & 3]
 *   sign    = bit (p & 31) of word set ? -1 : +1
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Threads.  The checker build is single-threaded; a second build of this same file with OpenMP times the
 * oracle on all host cores.  The parallel loops only split independent outputs between threads (rows,
 * columns, probe-table entries): every sum is still taken in the order written, so both builds give the
 * same bits.
 */
#ifdef _OPENMP
#include <omp.h>
#define OR_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
static int or_thread_count(void) { return omp_get_num_threads(); }
static int or_thread_id(void) { return omp_get_thread_num(); }
#define OR_PARALLEL _Pragma("omp parallel")
int or_max_threads(void) { return omp_get_max_threads(); }
#else
#define OR_PARALLEL_FOR
#define OR_PARALLEL
static int or_thread_count(void) { return 1; }
static int or_thread_id(void) { return 0; }
int or_max_threads(void) { return 1; }
#endif

/* ---------------------------------------------------------------- Philox */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u; /* key schedule increments */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

double or_probe_sign(uint64_t seed, uint32_t index, uint32_t t, uint32_t stream, uint32_t p)
{
    uint32_t ctr[4] = {index, t, stream, p >> 7};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    uint32_t word = out[(p >> 5) & 3u];
    return ((word >> (p & 31u)) & 1u) ? -1.0 : 1.0;
}

/* sgn[idx * k + p] for idx in [0, len), p in [0, k). */
void or_draw_probes(uint64_t seed, int32_t t, int32_t stream, int64_t len, int32_t k, double *sgn)
{
    OR_PARALLEL_FOR
    for (int64_t idx = 0; idx < len; ++idx)
        for (int32_t p = 0; p < k; ++p)
            sgn[idx * k + p] = or_probe_sign(seed, (uint32_t)idx, (uint32_t)t, (uint32_t)stream, (uint32_t)p);
}

/* ------------------------------------------------------------ estimators */

/* z[i] = (1/k) sum_p ((D A E s_p)_i)^2, D = diag(e^u), E = diag(e^v); s is n x k. */
void or_row_estimate(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                     const double *u, const double *v, const double *s, int32_t k, double *z)
{
    (void)n;
    OR_PARALLEL_FOR
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p) {
            double y = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int64_t j = col[e];
                double b = exp(u[i]) * val[e] * exp(v[j]);
                y += b * s[j * k + p];
            }
            acc += y * y;
        }
        z[i] = acc / (double)k;
    }
}

/* z[j] = (1/k) sum_p ((E A^T D w_p)_j)^2; w is m x k.  Accumulated by scattering over the CSR, rows in
 * order.  With several threads, each owns a contiguous range of columns and scatters only into those. */
void or_col_estimate(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                     const double *u, const double *v, const double *w, int32_t k, double *z)
{
    double *y = (double *)calloc((size_t)(n * k), sizeof(double));
    OR_PARALLEL
    {
        const int64_t nt = or_thread_count(), id = or_thread_id();
        const int64_t j0 = n * id / nt, j1 = n * (id + 1) / nt;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int64_t j = col[e];
                if (j < j0 || j >= j1)
                    continue;
                double b = exp(v[j]) * val[e] * exp(u[i]);
                for (int32_t p = 0; p < k; ++p)
                    y[j * k + p] += b * w[i * k + p];
            }
    }
    OR_PARALLEL_FOR
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p)
            acc += y[j * k + p] * y[j * k + p];
        z[j] = acc / (double)k;
    }
    free(y);
}

/* ----------------------------------------------------------- Algorithm 1 */

static double clip(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

/* One iteration t of Algorithm 1 with explicit probe signs s (n x k) and w (m x k), and optional
 * per-row / per-column squared target norms rt (m), ct (n) in place of alpha^2, beta^2 (the varying-norm
 * variant of Section 6: gradient |DAE|^2 1 - r + gamma u).
 * u, v hold u^{t-1}, v^{t-1} on entry and u^t, v^t on exit; ubar, vbar are the running averages. */
void or_psgd_step_targets(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          const double *rt, const double *ct, double alpha, double beta, double gamma, double M,
                          int32_t t, int32_t t0, const double *s, const double *w, int32_t k,
                          double *u, double *v, double *ubar, double *vbar)
{
    double *zu = (double *)malloc((size_t)m * sizeof(double));
    double *zv = (double *)malloc((size_t)n * sizeof(double));
    or_row_estimate(m, n, row_ptr, col, val, u, v, s, k, zu);
    or_col_estimate(m, n, row_ptr, col, val, u, v, w, k, zv);
    double eta = 2.0 / (gamma * ((double)t + (double)t0 + 1.0));
    OR_PARALLEL_FOR
    for (int64_t i = 0; i < m; ++i) {
        double target = rt ? rt[i] : alpha * alpha;
        double un = clip(u[i] - eta * (zu[i] - target + gamma * u[i]), -M, M);
        u[i] = un;
        ubar[i] = 2.0 * un / ((double)t + 2.0) + (double)t * ubar[i] / ((double)t + 2.0);
    }
    OR_PARALLEL_FOR
    for (int64_t j = 0; j < n; ++j) {
        double target = ct ? ct[j] : beta * beta;
        double vn = clip(v[j] - eta * (zv[j] - target + gamma * v[j]), -M, M);
        v[j] = vn;
        vbar[j] = 2.0 * vn / ((double)t + 2.0) + (double)t * vbar[j] / ((double)t + 2.0);
    }
    free(zu);
    free(zv);
}

void or_psgd_step(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                  double alpha, double beta, double gamma, double M, int32_t t, int32_t t0,
                  const double *s, const double *w, int32_t k,
                  double *u, double *v, double *ubar, double *vbar)
{
    or_psgd_step_targets(m, n, row_ptr, col, val, NULL, NULL, alpha, beta, gamma, M, t, t0, s, w, k, u, v, ubar,
                         vbar);
}

/* One iteration t of Algorithm 2 (symmetric equilibration, Section 6): D = E = diag(e^u),
 * z_i = (1/k) sum_p ((D A D s_p)_i)^2 with signs s (n x k), then the projected step and the average. */
void or_psgd_step_symmetric(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                            double alpha, double gamma, double M, int32_t t, int32_t t0, const double *s, int32_t k,
                            double *u, double *ubar)
{
    double *z = (double *)malloc((size_t)n * sizeof(double));
    or_row_estimate(n, n, row_ptr, col, val, u, u, s, k, z);
    double eta = 2.0 / (gamma * ((double)t + (double)t0 + 1.0));
    for (int64_t i = 0; i < n; ++i) {
        double un = clip(u[i] - eta * (z[i] - alpha * alpha + gamma * u[i]), -M, M);
        u[i] = un;
        ubar[i] = 2.0 * un / ((double)t + 2.0) + (double)t * ubar[i] / ((double)t + 2.0);
    }
    free(z);
}

/* One iteration t of block equilibration (Section 6): rows split into p contiguous blocks
 * [rb[b], rb[b+1]) sharing the scaling e^{ub[b]}, columns into q blocks [cb[c], cb[c+1]) sharing e^{vb[c]}.
 * The block gradient is sum_{i in b} (|DAE|^2 1)_i - alpha^2 m_b + gamma u_b; its estimate sums the row
 * estimates of the block.  ub, vb (block iterates) and ubb, vbb (block averages) are updated. */
void or_block_step(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                   int64_t p, const int64_t *rb, int64_t q, const int64_t *cb, double alpha, double beta,
                   double gamma, double M, int32_t t, int32_t t0, const double *s, const double *w, int32_t k,
                   double *ub, double *vb, double *ubb, double *vbb)
{
    double *u = (double *)malloc((size_t)m * sizeof(double));
    double *v = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t b = 0; b < p; ++b)
        for (int64_t i = rb[b]; i < rb[b + 1]; ++i)
            u[i] = ub[b];
    for (int64_t c = 0; c < q; ++c)
        for (int64_t j = cb[c]; j < cb[c + 1]; ++j)
            v[j] = vb[c];
    double *zu = (double *)malloc((size_t)m * sizeof(double));
    double *zv = (double *)malloc((size_t)n * sizeof(double));
    or_row_estimate(m, n, row_ptr, col, val, u, v, s, k, zu);
    or_col_estimate(m, n, row_ptr, col, val, u, v, w, k, zv);
    double eta = 2.0 / (gamma * ((double)t + (double)t0 + 1.0));
    for (int64_t b = 0; b < p; ++b) {
        double zb = 0.0;
        for (int64_t i = rb[b]; i < rb[b + 1]; ++i)
            zb += zu[i];
        double mb = (double)(rb[b + 1] - rb[b]);
        double un = clip(ub[b] - eta * (zb - alpha * alpha * mb + gamma * ub[b]), -M, M);
        ub[b] = un;
        ubb[b] = 2.0 * un / ((double)t + 2.0) + (double)t * ubb[b] / ((double)t + 2.0);
    }
    for (int64_t c = 0; c < q; ++c) {
        double zc = 0.0;
        for (int64_t j = cb[c]; j < cb[c + 1]; ++j)
            zc += zv[j];
        double nc = (double)(cb[c + 1] - cb[c]);
        double vn = clip(vb[c] - eta * (zc - beta * beta * nc + gamma * vb[c]), -M, M);
        vb[c] = vn;
        vbb[c] = 2.0 * vn / ((double)t + 2.0) + (double)t * vbb[c] / ((double)t + 2.0);
    }
    free(u);
    free(v);
    free(zu);
    free(zv);
}

/* Iterations t_begin .. t_begin + T - 1 of Algorithm 1 with Philox probes.
 * stream_base selects the Philox stream pair (stream_base for s, stream_base + 1 for w). */
void or_equilibrate(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                    double alpha, double beta, double gamma, double M, int32_t t_begin, int32_t T,
                    int32_t t0, int32_t k, uint64_t seed, int32_t stream_base,
                    double *u, double *v, double *ubar, double *vbar)
{
    double *s = (double *)malloc((size_t)(n * k) * sizeof(double));
    double *w = (double *)malloc((size_t)(m * k) * sizeof(double));
    for (int32_t t = t_begin; t < t_begin + T; ++t) {
        or_draw_probes(seed, t, stream_base, n, k, s);
        or_draw_probes(seed, t, stream_base + 1, m, k, w);
        or_psgd_step(m, n, row_ptr, col, val, alpha, beta, gamma, M, t, t0, s, w, k, u, v, ubar, vbar);
    }
    free(s);
    free(w);
}

/* One iteration t evaluated only at the listed rows and columns, for spot checks on large inputs.
 * Reads the full u^{t-1}, v^{t-1}; writes u^t, ubar at rows[] into u_out, ubar_out (indexed like rows[]),
 * and likewise for columns. */
void or_psgd_step_sampled(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          double alpha, double beta, double gamma, double M, int32_t t, int32_t t0, int32_t k,
                          uint64_t seed, int32_t stream_base,
                          const double *u, const double *v, const double *ubar, const double *vbar,
                          int64_t n_rows, const int64_t *rows, int64_t n_cols, const int64_t *cols,
                          double *u_out, double *ubar_out, double *v_out, double *vbar_out)
{
    double eta = 2.0 / (gamma * ((double)t + (double)t0 + 1.0));
    for (int64_t q = 0; q < n_rows; ++q) {
        int64_t i = rows[q];
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p) {
            double y = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int64_t j = col[e];
                double sj = or_probe_sign(seed, (uint32_t)j, (uint32_t)t, (uint32_t)stream_base, (uint32_t)p);
                y += exp(u[i]) * val[e] * exp(v[j]) * sj;
            }
            acc += y * y;
        }
        double z = acc / (double)k;
        double un = clip(u[i] - eta * (z - alpha * alpha + gamma * u[i]), -M, M);
        u_out[q] = un;
        ubar_out[q] = 2.0 * un / ((double)t + 2.0) + (double)t * ubar[i] / ((double)t + 2.0);
    }
    if (n_cols == 0)
        return;
    /* Column sums need every row that touches a sampled column: one pass over the CSR. */
    int64_t *slot = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j)
        slot[j] = -1;
    for (int64_t q = 0; q < n_cols; ++q)
        slot[cols[q]] = q;
    double *y = (double *)calloc((size_t)(n_cols * k), sizeof(double));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t q = slot[col[e]];
            if (q < 0)
                continue;
            int64_t j = col[e];
            double b = exp(v[j]) * val[e] * exp(u[i]);
            for (int32_t p = 0; p < k; ++p)
                y[q * k + p] += b * or_probe_sign(seed, (uint32_t)i, (uint32_t)t, (uint32_t)(stream_base + 1), (uint32_t)p);
        }
    for (int64_t q = 0; q < n_cols; ++q) {
        int64_t j = cols[q];
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p)
            acc += y[q * k + p] * y[q * k + p];
        double z = acc / (double)k;
        double vn = clip(v[j] - eta * (z - beta * beta + gamma * v[j]), -M, M);
        v_out[q] = vn;
        vbar_out[q] = 2.0 * vn / ((double)t + 2.0) + (double)t * vbar[j] / ((double)t + 2.0);
    }
    free(y);
    free(slot);
}

/* ------------------------------------------------------------ evaluation */

/* r2[i] = sum_j (e^{u_i} A_ij e^{v_j})^2 and c2[j] = sum_i (e^{u_i} A_ij e^{v_j})^2. */
void or_exact_norms_sq(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       const double *u, const double *v, double *r2, double *c2)
{
    for (int64_t j = 0; j < n; ++j)
        c2[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t j = col[e];
            double b = exp(u[i]) * val[e] * exp(v[j]);
            acc += b * b;
            c2[j] += b * b;
        }
        r2[i] = acc;
    }
}

/* y = A x (FP64), for the LSQR residual checks of the oracle. */
void or_csr_matvec(int64_t m, const int64_t *row_ptr, const int32_t *col, const double *val,
                   const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            acc += val[e] * x[col[e]];
        y[i] = acc;
    }
}

/* Dense A (m x n, row-major, float values widened to FP64): the estimates of iteration t at the listed
 * rows and columns, with sign tables s (n x k) and w (m x k) drawn once from Philox.
 *   zu[q] = (1/k) sum_p (sum_j e^{u_i} A_ij e^{v_j} s_jp)^2   for i = rows[q]
 *   zv[q] = (1/k) sum_p (sum_i e^{v_j} A_ij e^{u_i} w_ip)^2   for j = cols[q]
 * row_scale (nullable) multiplies row i of A. */
void or_dense_estimate_sampled(int64_t m, int64_t n, const float *A, const double *row_scale, const double *u,
                               const double *v, int32_t t, int32_t k, uint64_t seed, int32_t stream_base,
                               int64_t n_rows, const int64_t *rows, int64_t n_cols, const int64_t *cols,
                               double *zu, double *zv)
{
    double *s = (double *)malloc((size_t)(n * k) * sizeof(double));
    double *w = (double *)malloc((size_t)(m * k) * sizeof(double));
    or_draw_probes(seed, t, stream_base, n, k, s);
    or_draw_probes(seed, t, stream_base + 1, m, k, w);
    OR_PARALLEL_FOR
    for (int64_t q = 0; q < n_rows; ++q) {
        double *y = (double *)malloc((size_t)k * sizeof(double));
        int64_t i = rows[q];
        double ci = row_scale ? row_scale[i] : 1.0;
        for (int32_t p = 0; p < k; ++p)
            y[p] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double b = exp(u[i]) * ci * (double)A[i * n + j] * exp(v[j]);
            for (int32_t p = 0; p < k; ++p)
                y[p] += b * s[j * k + p];
        }
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p)
            acc += y[p] * y[p];
        zu[q] = acc / (double)k;
        free(y);
    }
    OR_PARALLEL_FOR
    for (int64_t q = 0; q < n_cols; ++q) {
        double *y = (double *)malloc((size_t)k * sizeof(double));
        int64_t j = cols[q];
        for (int32_t p = 0; p < k; ++p)
            y[p] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double ci = row_scale ? row_scale[i] : 1.0;
            double b = exp(v[j]) * ci * (double)A[i * n + j] * exp(u[i]);
            for (int32_t p = 0; p < k; ++p)
                y[p] += b * w[i * k + p];
        }
        double acc = 0.0;
        for (int32_t p = 0; p < k; ++p)
            acc += y[p] * y[p];
        zv[q] = acc / (double)k;
        free(y);
    }
    free(s);
    free(w);
}
