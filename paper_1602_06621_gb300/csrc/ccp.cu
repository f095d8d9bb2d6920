// The Chambolle-Cremers-Pock application of Section 5.2: the Lasso problem
//     minimize  f(x) = ||A x - b||^2 / sqrt(lam) + sqrt(lam) ||x||_1
// solved by the primal-dual method on the equilibrated operator K = D A E (x = E xs), with step sizes
// tau = sigma = 0.9 / ||K||_2 and theta = 1, all iterates starting at 0.  One iteration is one product with
// K and one with K^T, as for LSQR:
//   rows:    y_i  <- a_i (w_i - sigma d_i b_i) / (a_i + sigma),   w = y + sigma K xbar,  a_i = 2 / (d_i^2 sqrt(lam))
//            (the closed-form prox of sigma F*, F(y) = ||D^{-1} y - b||^2 / sqrt(lam))
//   columns: xs'_j <- soft(xs_j - tau (K^T y)_j, tau sqrt(lam) e_j),  xbar_j <- xs'_j + theta (xs'_j - xs_j)
//            (the prox of tau G, G(xs) = sqrt(lam) ||E xs||_1)
// Vectors live in the operators' sorted orders.  Each product gathers a pre-scaled vector (e xbar for K,
// d y for K^T), so every nonzero costs one gather, as in the iteration kernel.  ||K||_2 comes from power
// iteration on K^T K started at the unit vector 1/sqrt(n).  Every check_every iterations the objective is
// evaluated in FP64 on the original problem (x = E xs), with deterministic reductions; with a known optimal
// value the run stops at a relative gap (f - p*) / f(0) <= tol.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sell_ops.cuh"
#include "sme_internal.cuh"

namespace sme {

struct CcpScalars {
    double tau, sigma, theta, sqrt_lam;
    double inv_lam_pw;       // 1 / ||K^T K p|| of the last power step (normalises the next one)
    double pw_norm;          // ||K^T K p|| of the last power step
    double f0, f, xnorm1, p_star, tol, rel_gap;
    long long iters;
    int done;                // 0 running, 1 converged
    int pad;
};

struct CcpState {
    void *d = nullptr, *e = nullptr, *bs = nullptr, *y = nullptr, *yd = nullptr, *xs = nullptr, *xe = nullptr,
         *xt = nullptr;
    double *partials = nullptr;
    unsigned *counter = nullptr;
    CcpScalars *sc = nullptr, *host = nullptr;
};

template <typename real>
__global__ void ccp_scales(int64_t n, const int32_t *perm, const real *logscale, real *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = logscale ? (real)exp((double)logscale[perm[i]]) : real(1);
}

// Power iteration, start: xe = e / sqrt(n) (the unit vector in K's column space, pre-scaled by E).
template <typename real>
__global__ void ccp_power_init(int64_t n, const real *e, real *xe, CcpScalars *sc)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) sc->inv_lam_pw = 1.0;
    if (c < n) xe[c] = e[c] * (real)(1.0 / sqrt((double)n));
}

// Power iteration, rows: yd = D (K p) with K p = D A (E p); p is xe * inv_lam_pw.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) ccp_power_rows(Sell S, const real *d, const real *xe, real *yd,
                                                              const CcpScalars *sc)
{
    const SplitSlice<SPLIT> w;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, w, xe);
    const int64_t r = w.slice * 32 + w.lane;
    if (!w.lead() || w.slice >= S.nslices || r >= S.rows) return;
    const real dr = d[r];
    yd[r] = dr * dr * acc * (real)sc->inv_lam_pw;
}

// Power iteration, columns: q = K^T (K p) = E A^T (D K p); xe = E q; ||q|| reduced in FP64.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) ccp_power_cols(Sell S, const real *e, const real *yd, real *xe,
                                                              double *partials, unsigned *counter, CcpScalars *sc)
{
    const SplitSlice<SPLIT> w;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, w, yd);
    const int64_t c = w.slice * 32 + w.lane;
    double part = 0.0;
    if (w.lead() && w.slice < S.nslices && c < S.rows) {
        const real ec = e[c];
        const real q = ec * acc;
        xe[c] = ec * q;
        part = (double)q * (double)q;
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x == 0) {
        sc->pw_norm = sqrt(tot);
        sc->inv_lam_pw = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    }
}

// Start of the solve: b in sorted row order, y = 0, and f(0) = ||b||^2 / sqrt(lam).
template <typename real>
__global__ void ccp_init_rows(int64_t m, const int32_t *perm, const real *b, real *bs, real *y, real *yd,
                              double *partials, unsigned *counter, CcpScalars *sc)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (r < m) {
        const real bi = b[perm[r]];
        bs[r] = bi;
        y[r] = real(0);
        yd[r] = real(0);
        part = (double)bi * (double)bi;
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x == 0) {
        sc->f0 = tot / sc->sqrt_lam;
        sc->f = sc->f0;
        sc->iters = 0;
        sc->done = 0;
        sc->rel_gap = sc->p_star > 0.0 ? (sc->f0 - sc->p_star) / sc->f0 : NAN;
    }
}

template <typename real>
__global__ void ccp_init_cols(int64_t n, real *xs, real *xe)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        xs[c] = real(0);
        xe[c] = real(0);
    }
}

// Dual step (rows): w = y + sigma d (A xe), y <- a (w - sigma d b) / (a + sigma), yd = d y.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) ccp_rows(Sell S, const real *d, const real *bs, const real *xe,
                                                        real *y, real *yd, const CcpScalars *sc)
{
    if (((volatile const CcpScalars *)sc)->done) return;  // the same for every thread of the block
    const real sigma = (real)sc->sigma;
    const double sqrt_lam = sc->sqrt_lam;
    const SplitSlice<SPLIT> w;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, w, xe);
    const int64_t r = w.slice * 32 + w.lane;
    if (!w.lead() || w.slice >= S.nslices || r >= S.rows) return;
    const real dr = d[r];
    const real wv = y[r] + sigma * dr * acc;
    const real a = (real)(2.0 / ((double)dr * (double)dr * sqrt_lam));
    const real yn = a * (wv - sigma * dr * bs[r]) / (a + sigma);
    y[r] = yn;
    yd[r] = dr * yn;
}

// Primal step (columns): xs' = soft(xs - tau e (A^T yd), tau sqrt(lam) e), xbar = xs' + theta (xs' - xs),
// xe = e xbar.  The last block counts the iteration.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) ccp_cols(Sell S, const real *e, const real *yd, real *xs, real *xe,
                                                        unsigned *counter, CcpScalars *sc)
{
    if (((volatile const CcpScalars *)sc)->done) return;  // the same for every thread of the block
    const real tau = (real)sc->tau, theta = (real)sc->theta;
    const real thr0 = (real)(sc->tau * sc->sqrt_lam);
    const SplitSlice<SPLIT> w;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, w, yd);
    const int64_t c = w.slice * 32 + w.lane;
    if (w.lead() && w.slice < S.nslices && c < S.rows) {
        const real ec = e[c];
        const real xo = xs[c];
        const real z = xo - tau * ec * acc;
        const real thr = thr0 * ec;
        const real az = z < real(0) ? -z : z;
        const real xn = az > thr ? (z < real(0) ? -(az - thr) : az - thr) : real(0);
        xs[c] = xn;
        xe[c] = ec * (xn + theta * (xn - xo));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(counter, 1u) == gridDim.x - 1) {
            *counter = 0u;
            sc->iters += 1;
        }
    }
}

// x = E xs (sorted column order) and ||x||_1 in FP64; with perm, also x_out in original order.
template <typename real>
__global__ void ccp_current_x(int64_t n, const real *e, const real *xs, real *xt, const int32_t *perm, real *x_out,
                              double *partials, unsigned *counter, CcpScalars *sc, int final_pass)
{
    if (!final_pass && ((volatile const CcpScalars *)sc)->done) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (c < n) {
        const real v = e[c] * xs[c];
        xt[c] = v;
        if (perm) x_out[perm[c]] = v;
        part = fabs((double)v);
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x == 0) sc->xnorm1 = tot;
}

// f(x) = ||A x - b||^2 / sqrt(lam) + sqrt(lam) ||x||_1 in FP64 on the original system; the stopping rule.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) ccp_objective(Sell S, const real *xt, const real *bs, double *partials,
                                                             unsigned *counter, CcpScalars *sc, int final_pass)
{
    if (!final_pass && ((volatile const CcpScalars *)sc)->done) return;  // uniform over the block
    const SplitSlice<SPLIT> w;
    const double acc = sell_row_dot_split<real, double, real, SPLIT>(S, w, xt);
    const int64_t i = w.slice * 32 + w.lane;
    double part = 0.0;
    if (w.lead() && w.slice < S.nslices && i < S.rows) {
        const double ri = acc - (double)bs[i];
        part = ri * ri;
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x != 0) return;
    sc->f = tot / sc->sqrt_lam + sc->sqrt_lam * sc->xnorm1;
    if (sc->p_star > 0.0) {
        sc->rel_gap = (sc->f - sc->p_star) / sc->f0;
        if (!final_pass && sc->tol > 0.0 && sc->rel_gap <= sc->tol) sc->done = 1;
    }
}


static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static void ccp_release(CcpState *C)
{
    for (void *p : {C->d, C->e, C->bs, C->y, C->yd, C->xs, C->xe, C->xt, (void *)C->partials, (void *)C->counter,
                    (void *)C->sc})
        if (p) cudaFree(p);
    delete C->host;
    delete C;
}

static sme_status ccp_alloc(sme_op op, CcpState *C, size_t sz)
{
    const int64_t m = op->m, n = op->n;
    // One partial per block of any pass: at most one block per slice (8 warps on one slice).
    const int64_t maxb = std::max<int64_t>(std::max<int64_t>(op->fwd.nslices, op->bwd.nslices),
                                           (std::max(m, n) + 255) / 256);
    void **mv[5] = {&C->d, &C->bs, &C->y, &C->yd, nullptr};
    void **nv[5] = {&C->e, &C->xs, &C->xe, &C->xt, nullptr};
    bool ok = true;
    for (int i = 0; mv[i]; ++i) ok = ok && cudaMalloc(mv[i], (size_t)m * sz) == cudaSuccess;
    for (int i = 0; nv[i]; ++i) ok = ok && cudaMalloc(nv[i], (size_t)n * sz) == cudaSuccess;
    if (!ok ||cudaMalloc(&C->partials, (size_t)maxb * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&C->counter, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&C->sc, sizeof(CcpScalars)) != cudaSuccess) {
        cudaGetLastError();
        return SME_ERR_OOM;
    }
    C->host = new CcpScalars();
    return SME_OK;
}

// Power iteration on K^T K: `iters` steps from the unit vector; returns ||K||_2 (host).
template <typename real>
static sme_status power_norm_t(sme_op op, CcpState *C, int iters, double *norm, int64_t *launches, cudaStream_t s)
{
    const Sell &F = op->fwd, &B = op->bwd;
    const Pass pf = pass_for(F), pb = pass_for(B);
    ccp_power_init<real><<<nblk(op->n), 256, 0, s>>>(op->n, (const real *)C->e, (real *)C->xe, C->sc);
    for (int i = 0; i < iters; ++i) {
        SPLIT_LAUNCH(ccp_power_rows, real, pf, s, F, (const real *)C->d, (const real *)C->xe, (real *)C->yd, C->sc);
        SPLIT_LAUNCH(ccp_power_cols, real, pb, s, B, (const real *)C->e, (const real *)C->yd, (real *)C->xe,
                   C->partials, C->counter, C->sc);
    }
    *launches += 1 + 2 * (int64_t)iters;
    SME_CUDA(cudaGetLastError());
    SME_CUDA(cudaMemcpyAsync(C->host, C->sc, sizeof(CcpScalars), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    *norm = std::sqrt(C->host->pw_norm);
    return SME_OK;
}

template <typename real>
static sme_status prepare(sme_op op, CcpState *C, const real *ubar, const real *vbar, cudaStream_t s)
{
    SME_TRY(ccp_alloc(op, C, sizeof(real)));
    SME_CUDA(cudaMemsetAsync(C->counter, 0, sizeof(unsigned), s));
    SME_CUDA(cudaMemsetAsync(C->sc, 0, sizeof(CcpScalars), s));
    ccp_scales<real><<<nblk(op->m), 256, 0, s>>>(op->m, op->fwd.perm, ubar, (real *)C->d);
    ccp_scales<real><<<nblk(op->n), 256, 0, s>>>(op->n, op->bwd.perm, vbar, (real *)C->e);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

template <typename real>
static sme_status ccp_t(sme_op op, const real *ubar, const real *vbar, const real *b, real *x_out,
                        const sme_ccp_params *p, sme_ccp_result *res, double *history, int64_t history_cap,
                        cudaStream_t s)
{
    CcpState *C = new CcpState();
    auto done = [&](sme_status st) {
        ccp_release(C);
        return st;
    };
    sme_status st = prepare<real>(op, C, ubar, vbar, s);
    if (st != SME_OK) return done(st);
    int64_t launches = 2;
    double nrm = 0.0;
    double tau = p->tau, sigma = p->sigma;
    if (tau <= 0.0 || sigma <= 0.0) {
        st = power_norm_t<real>(op, C, p->norm_iters > 0 ? p->norm_iters : 100, &nrm, &launches, s);
        if (st != SME_OK) return done(st);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) {
            set_error("sme_ccp_lasso: ||D A E||_2 is zero or not finite");
            return done(SME_ERR_NONFINITE);
        }
        if (tau <= 0.0) tau = 0.9 / nrm;
        if (sigma <= 0.0) sigma = 0.9 / nrm;
    }
    CcpScalars h{};
    h.tau = tau;
    h.sigma = sigma;
    h.theta = p->theta > 0.0 ? p->theta : 1.0;
    h.sqrt_lam = std::sqrt(p->lambda);
    h.p_star = p->p_star;
    h.tol = p->tol;
    *C->host = h;
    if (cudaMemcpyAsync(C->sc, C->host, sizeof(CcpScalars), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return done(SME_ERR_CUDA);
    const Sell &F = op->fwd, &B = op->bwd;
    const int64_t m = op->m, n = op->n;
    const Pass pf = pass_for(F), pb = pass_for(B);
    real *d = (real *)C->d, *e = (real *)C->e, *bs = (real *)C->bs, *y = (real *)C->y, *yd = (real *)C->yd,
         *xs = (real *)C->xs, *xe = (real *)C->xe, *xt = (real *)C->xt;
    ccp_init_rows<real><<<nblk(m), 256, 0, s>>>(m, F.perm, b, bs, y, yd, C->partials, C->counter, C->sc);
    ccp_init_cols<real><<<nblk(n), 256, 0, s>>>(n, xs, xe);
    launches += 2;
    const int every = std::max(1, p->check_every);
    // A chunk of `every` iterations and its objective check, all on fixed buffers.
    auto enqueue_chunk = [&](int64_t chunk, cudaStream_t q) {
        for (int64_t j = 0; j < chunk; ++j) {
            SPLIT_LAUNCH(ccp_rows, real, pf, q, F, d, bs, xe, y, yd, C->sc);
            SPLIT_LAUNCH(ccp_cols, real, pb, q, B, e, yd, xs, xe, C->counter, C->sc);
        }
        ccp_current_x<real><<<nblk(n), 256, 0, q>>>(n, e, xs, xt, nullptr, nullptr, C->partials, C->counter, C->sc,
                                                   0);
        SPLIT_LAUNCH(ccp_objective, real, pf, q, F, xt, bs, C->partials, C->counter, C->sc, 0);
    };
    // Full chunks are captured once as a CUDA graph and replayed (on a private stream: the caller's may be
    // the legacy default stream, which cannot be captured); without a graph they are launched directly.
    GraphOnce chunk_graph;
    if (p->max_iters >= 2 * (int64_t)every) chunk_graph.capture([&](cudaStream_t q) { enqueue_chunk(every, q); });
    int64_t it = 0, hcount = 0;
    bool stop = false;
    while (it < p->max_iters && !stop) {
        const int64_t chunk = std::min<int64_t>(every, p->max_iters - it);
        if (chunk == every && chunk_graph.exec) {
            if (cudaGraphLaunch(chunk_graph.exec, s) != cudaSuccess) {
                cuda_fail(cudaGetLastError(), "sme_ccp_lasso", __LINE__);
                return done(SME_ERR_CUDA);
            }
        } else {
            enqueue_chunk(chunk, s);
        }
        it += chunk;
        launches += 2 * chunk + 2;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(C->host, C->sc, sizeof(CcpScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cuda_fail(cudaGetLastError(), "sme_ccp_lasso", __LINE__);
            return done(SME_ERR_CUDA);
        }
        if (history && hcount < history_cap) history[hcount] = C->host->f;
        ++hcount;
        if (!std::isfinite(C->host->f)) {
            set_error("sme_ccp_lasso: the objective became non-finite");
            return done(SME_ERR_NONFINITE);
        }
        stop = C->host->done != 0;
    }
    ccp_current_x<real><<<nblk(n), 256, 0, s>>>(n, e, xs, xt, B.perm, x_out, C->partials, C->counter, C->sc, 1);
    SPLIT_LAUNCH(ccp_objective, real, pf, s, F, xt, bs, C->partials, C->counter, C->sc, 1);
    launches += 2;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(C->host, C->sc, sizeof(CcpScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cuda_fail(cudaGetLastError(), "sme_ccp_lasso", __LINE__);
        return done(SME_ERR_CUDA);
    }
    const CcpScalars &r = *C->host;
    res->iters = r.iters;
    res->objective = r.f;
    res->objective0 = r.f0;
    res->rel_gap = r.rel_gap;
    res->op_norm = nrm;
    res->tau = tau;
    res->sigma = sigma;
    res->converged = r.p_star > 0.0 && r.tol > 0.0 && r.rel_gap <= r.tol ? 1 : 0;
    res->kernel_launches = launches;
    res->history_count = std::min(hcount, history_cap);
    return done(SME_OK);
}

}  // namespace sme

using namespace sme;

static bool ccp_op_ok(sme_op op, const char *who)
{
    if (!op || op->dense || op->batch) {
        set_error("%s: a single sparse operator is required", who);
        return false;
    }
    return true;
}

extern "C" sme_status sme_op_norm2(sme_op op, const void *u_bar, const void *v_bar, int32_t iters, double *norm,
                                   void *stream)
{
    SME_TRY(no_shard(op, "sme_op_norm2"));
    if (!ccp_op_ok(op, "sme_op_norm2") || !norm || iters < 1) {
        if (op && norm && iters < 1) set_error("sme_op_norm2: iters must be >= 1");
        return SME_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CcpState *C = new CcpState();
    int64_t launches = 0;
    sme_status st;
    if (op->dbl) {
        st = prepare<double>(op, C, (const double *)u_bar, (const double *)v_bar, s);
        if (st == SME_OK) st = power_norm_t<double>(op, C, iters, norm, &launches, s);
    } else {
        st = prepare<float>(op, C, (const float *)u_bar, (const float *)v_bar, s);
        if (st == SME_OK) st = power_norm_t<float>(op, C, iters, norm, &launches, s);
    }
    ccp_release(C);
    return st;
}

extern "C" sme_status sme_ccp_lasso(sme_op op, const void *u_bar, const void *v_bar, const void *b, void *x,
                                    const sme_ccp_params *p, sme_ccp_result *res, double *history,
                                    int64_t history_cap, void *stream)
{
    NvtxRange range("sme ccp lasso");
    SME_TRY(no_shard(op, "sme_ccp_lasso"));
    if (!ccp_op_ok(op, "sme_ccp_lasso")) return SME_ERR_ARG;
    if (!b || !x || !p || !res || !(p->lambda > 0.0) || p->max_iters < 0 || history_cap < 0 ||
        (history_cap > 0 && !history)) {
        set_error("sme_ccp_lasso: bad arguments");
        return SME_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (op->dbl)
        return ccp_t<double>(op, (const double *)u_bar, (const double *)v_bar, (const double *)b, (double *)x, p, res,
                             history, history_cap, s);
    return ccp_t<float>(op, (const float *)u_bar, (const float *)v_bar, (const float *)b, (float *)x, p, res, history,
                        history_cap, s);
}
