// LSQR for every matrix of a batch at once (Section 5.1 applied matrix by matrix).
//
// The products run over the batch's block-diagonal operator, as for a single matrix, but every matrix
// keeps its own LSQR: its own FP64 scalars (alpha, beta, rho, phibar, ...), its own residual checks and its
// own convergence flag.  Norms are segmented reductions: each kernel scatters its rows' squares into the
// batch's original (matrix-contiguous) order, then one CTA per matrix sums its range in a fixed order and
// runs that matrix's scalar recurrence.  A converged matrix stops changing; the others go on.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "sell_ops.cuh"
#include "sme_internal.cuh"

namespace sme {

struct BScal {
    double alpha, beta, rhobar, phibar, phi, rho, theta, bnorm, rel_res, rnorm, normal_res, afro;
    long long iters;
    int done;   // 0 running, 1 converged (checked), 2 exact breakdown
    int first;
};

struct BLsqr {
    int count = 0;
    void *ud = nullptr, *ve = nullptr, *w = nullptr, *x = nullptr, *d = nullptr, *e = nullptr, *bs = nullptr,
         *xt = nullptr;
    double *sq_r = nullptr, *sq_c = nullptr, *sq_r2 = nullptr, *r = nullptr;
    int64_t *roff = nullptr, *coff = nullptr;  // device copies of the batch offsets
    BScal *sc = nullptr, *host = nullptr;
    int32_t *list_r = nullptr, *list_c = nullptr;  // slices of unfinished matrices (matrix-major layout)
};

// ------------------------------------------------------------------ kernels

// The slice a warp takes: its own index, or an entry of a list of the slices still at work (slices of
// matrices that have not converged); past the end of the list, no slice.
__device__ __forceinline__ int64_t listed_slice(const int32_t *list, int64_t nlist, int64_t idx)
{
    return list ? (idx < nlist ? (int64_t)list[idx] : INT64_MAX) : idx;
}

template <typename real>
__global__ void bl_init_rows(int64_t M, const int32_t *perm, const real *bvec, const real *d, real *bs, real *ud,
                             double *sq_db, double *sq_b)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int32_t i = perm[r];
    const real bi = bvec[i], dr = d[r], db = dr * bi;
    bs[r] = bi;
    ud[r] = dr * db;
    sq_db[i] = (double)db * (double)db;
    sq_b[i] = (double)bi * (double)bi;
}

template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) bl_rows(Sell S, const int32_t *mid, const real *d, const real *ve,
                                                       real *ud, double *sq, const BScal *sc, const int32_t *list,
                                                       int64_t nlist)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = listed_slice(list, nlist, (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp);
    if (slice >= S.nslices) return;
    const int64_t r = slice * 32 + lane;
    // Rows of finished matrices (and padding rows) do no work.
    const bool live = r < S.rows && !sc[mid[r]].done;
    const real acc = sell_row_dot<real, real, real>(S, slice, lane, ve, live);
    if (!live) return;
    const BScal &c = sc[mid[r]];
    const real inv_alpha = (real)(c.alpha > 0.0 ? 1.0 / c.alpha : 0.0);
    const real inv_beta = (real)(c.beta > 0.0 ? 1.0 / c.beta : 0.0);
    const real dr = d[r];
    const real uhat = dr * acc * inv_alpha - (real)c.alpha * (ud[r] / dr) * inv_beta;
    ud[r] = dr * uhat;
    sq[S.perm[r]] = (double)uhat * (double)uhat;
}

template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) bl_cols(Sell S, const int32_t *mid, const real *e, const real *ud,
                                                       real *ve, real *w, real *x, double *sq, const BScal *sc,
                                                       int init, const int32_t *list, int64_t nlist)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = listed_slice(list, nlist, (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp);
    if (slice >= S.nslices) return;
    const int64_t c = slice * 32 + lane;
    const bool live = c < S.rows && !sc[mid[c]].done;
    const real acc = sell_row_dot<real, real, real>(S, slice, lane, ud, live);
    if (!live) return;
    const BScal &p = sc[mid[c]];
    const real inv_alpha = (real)(p.alpha > 0.0 ? 1.0 / p.alpha : 0.0);
    const real inv_beta = (real)(p.beta > 0.0 ? 1.0 / p.beta : 0.0);
    const real ec = e[c];
    real vhat;
    if (init) {
        vhat = ec * acc * inv_beta;
        w[c] = real(0);
        x[c] = real(0);
    } else {
        const real v = ve[c] / ec * inv_alpha;
        if (p.first) {
            w[c] = v;
            x[c] = real(0);
        } else {
            const real wo = w[c];
            x[c] = x[c] + (real)(p.phi / p.rho) * wo;
            w[c] = v - (real)(p.theta / p.rho) * wo;
        }
        vhat = ec * acc * inv_beta - (real)p.beta * v;
    }
    ve[c] = ec * vhat;
    sq[S.perm[c]] = (double)vhat * (double)vhat;
}

// One CTA per matrix: sum of sq over the matrix's range [off[b], off[b+1]), then the action.
enum { RED_INIT_BETA, RED_INIT_ALPHA, RED_BETA, RED_ALPHA, RED_RESID, RED_NORMAL, RED_FRO };

__global__ void __launch_bounds__(LQ_THREADS) bl_reduce(const double *sq, const double *sq2, const int64_t *off,
                                                         BScal *sc, int action, double tol, int stop_rule,
                                                         int final_check)
{
    const int b = blockIdx.x;
    BScal &c = sc[b];
    const bool frozen = (action == RED_BETA || action == RED_ALPHA) && c.done;
    if (frozen) return;
    if ((action == RED_RESID || action == RED_NORMAL) && !final_check && c.done == 1) return;
    const int64_t lo = off[b], hi = off[b + 1];
    double v = 0.0, v2 = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        v += sq[i];
        if (sq2) v2 += sq2[i];
    }
    const double s = block_sum(v);
    const double s2 = sq2 ? block_sum(v2) : 0.0;
    if (threadIdx.x != 0) return;
    switch (action) {
        case RED_INIT_BETA:
            c.beta = sqrt(s);
            c.phibar = c.beta;
            c.bnorm = sqrt(s2);
            c.phi = 0.0;
            c.rho = 1.0;
            c.theta = 0.0;
            c.iters = 0;
            c.first = 1;
            c.done = c.beta > 0.0 ? 0 : 2;
            c.rel_res = c.bnorm > 0.0 ? 1.0 : 0.0;
            break;
        case RED_INIT_ALPHA:
            if (c.done) break;
            c.alpha = sqrt(s);
            c.rhobar = c.alpha;
            if (c.alpha == 0.0) c.done = 2;
            break;
        case RED_BETA:
            c.beta = sqrt(s);
            break;
        case RED_ALPHA: {
            const double alpha_n = sqrt(s), beta = c.beta;
            const double rho = hypot(c.rhobar, beta);
            const double cs = c.rhobar / rho, sn = beta / rho;
            c.theta = sn * alpha_n;
            c.rhobar = -cs * alpha_n;
            c.phi = cs * c.phibar;
            c.phibar = sn * c.phibar;
            c.rho = rho;
            c.alpha = alpha_n;
            c.first = 0;
            c.iters += 1;
            if (beta == 0.0 || alpha_n == 0.0) c.done = 2;
            break;
        }
        case RED_RESID:
            c.rnorm = sqrt(s);
            c.rel_res = c.bnorm > 0.0 ? c.rnorm / c.bnorm : c.rnorm;
            if (!final_check && stop_rule == 0 && c.rel_res <= tol && c.done == 0) c.done = 1;
            break;
        case RED_NORMAL:
            c.normal_res = (c.rnorm > 0.0 && c.afro > 0.0) ? sqrt(s) / (c.afro * c.rnorm) : 0.0;
            if (!final_check && stop_rule == 1 && c.normal_res <= tol && c.done == 0) c.done = 1;
            break;
        case RED_FRO:
            c.afro = sqrt(s);
            break;
    }
}

template <typename real>
__global__ void bl_current_x(int64_t N, const int32_t *mid, const int32_t *perm, const real *e, const real *x,
                             const real *w, const BScal *sc, real *xt, real *x_out, int skip_done)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const BScal &p = sc[mid[c]];
    if (skip_done && p.done == 1) return;
    const real v = e[c] * (x[c] + (real)(p.phi / p.rho) * w[c]);
    xt[c] = v;
    if (x_out) x_out[perm[c]] = v;
}

// Residual r = A x - b in FP64.  Between checks (skip_done) the rows of matrices that already converged are
// skipped: their partial sums are not read again before the final pass, which computes every row.
template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) bl_residual(Sell S, const int32_t *mid, const BScal *sc, int skip_done,
                                                           const real *xt, const real *bs, double *r, double *sq,
                                                           const int32_t *list, int64_t nlist)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = listed_slice(list, nlist, (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp);
    if (slice >= S.nslices) return;
    const int64_t i = slice * 32 + lane;
    const bool live = i < S.rows && !(skip_done && sc[mid[i]].done == 1);
    const double acc = sell_row_dot<real, double, real>(S, slice, lane, xt, live);
    if (!live) return;
    const double ri = acc - (double)bs[i];
    r[i] = ri;
    sq[S.perm[i]] = ri * ri;
}

template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) bl_normal(Sell S, const double *r, double *sq)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp;
    if (slice >= S.nslices) return;
    const double acc = sell_row_dot<real, double, double>(S, slice, lane, r);
    const int64_t c = slice * 32 + lane;
    if (c < S.rows) sq[S.perm[c]] = acc * acc;
}

template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) bl_row_sq(Sell S, double *sq)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp;
    if (slice >= S.nslices) return;
    const int np = S.slice_w[slice] / 2;
    const int64_t pbase = S.slice_off[slice] / 2 + lane;
    double a2 = 0.0;
    for (int q = 0; q < np; ++q) {
        int c0, c1;
        real a0, a1;
        pair_load<real>(S, pbase + (int64_t)q * 32, c0, a0, c1, a1);
        a2 += (double)a0 * (double)a0 + (double)a1 * (double)a1;
    }
    const int64_t i = slice * 32 + lane;
    if (i < S.rows) sq[S.perm[i]] = a2;
}

template <typename real>
__global__ void bl_scales(int64_t n, const int32_t *perm, const real *logscale, real *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = logscale ? (real)exp((double)logscale[perm[i]]) : real(1);
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static void bl_release(BLsqr *L)
{
    if (!L) return;
    for (void *p : {L->ud, L->ve, L->w, L->x, L->d, L->e, L->bs, L->xt, (void *)L->sq_r, (void *)L->sq_c,
                    (void *)L->sq_r2, (void *)L->r, (void *)L->roff, (void *)L->coff, (void *)L->sc,
                    (void *)L->list_r, (void *)L->list_c})
        if (p) cudaFree(p);
    delete[] L->host;
    delete L;
}

template <typename real>
static sme_status batch_lsqr_t(sme_op op, const real *ubar, const real *vbar, const real *bvec, real *x_out,
                               const sme_lsqr_params *p, sme_lsqr_result *res, cudaStream_t s)
{
    BatchInfo *B = op->batch;
    const int count = B->count;
    const int64_t M = op->m, N = op->n;
    // Released on every return path (the early returns of SME_CUDA included).
    std::unique_ptr<BLsqr, void (*)(BLsqr *)> owner(new BLsqr(), bl_release);
    BLsqr *L = owner.get();
    L->count = count;
    auto fail = [](sme_status e) { return e; };
    const size_t sz = sizeof(real);
    void **bufs[8] = {&L->ud, &L->bs, &L->d, &L->ve, &L->w, &L->x, &L->e, &L->xt};
    const int64_t lens[8] = {M, M, M, N, N, N, N, N};
    for (int i = 0; i < 8; ++i)
        if (cudaMalloc(bufs[i], lens[i] * sz) != cudaSuccess) return fail(SME_ERR_OOM);
    if (cudaMalloc(&L->sq_r, M * 8) != cudaSuccess || cudaMalloc(&L->sq_r2, M * 8) != cudaSuccess ||
        cudaMalloc(&L->r, M * 8) != cudaSuccess || cudaMalloc(&L->sq_c, N * 8) != cudaSuccess ||
        cudaMalloc(&L->roff, (count + 1) * 8) != cudaSuccess || cudaMalloc(&L->coff, (count + 1) * 8) != cudaSuccess ||
        cudaMalloc(&L->sc, count * sizeof(BScal)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SME_ERR_OOM);
    }
    L->host = new BScal[count]();
    const Sell &F = op->fwd, &Bk = op->bwd;
    const int32_t *mid_r = B->mid[0], *mid_c = B->mid[1];
    real *ud = (real *)L->ud, *ve = (real *)L->ve, *w = (real *)L->w, *x = (real *)L->x, *d = (real *)L->d,
         *e = (real *)L->e, *bs = (real *)L->bs, *xt = (real *)L->xt;
    const unsigned fb = (unsigned)std::max<int64_t>((F.nslices + 7) / 8, 1);
    const unsigned bb = (unsigned)std::max<int64_t>((Bk.nslices + 7) / 8, 1);
    int64_t launches = 0;
    SME_CUDA(cudaMemcpyAsync(L->roff, B->row_off, (count + 1) * 8, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemcpyAsync(L->coff, B->col_off, (count + 1) * 8, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemsetAsync(L->sc, 0, count * sizeof(BScal), s));
    SME_CUDA(cudaMemsetAsync(x, 0, N * sz, s));
    SME_CUDA(cudaMemsetAsync(w, 0, N * sz, s));
    bl_row_sq<real><<<fb, LQ_THREADS, 0, s>>>(F, L->sq_r);
    bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_r, nullptr, L->roff, L->sc, RED_FRO, p->tol, p->stop_rule, 0);
    bl_scales<real><<<nblk(M), 256, 0, s>>>(M, F.perm, ubar, d);
    bl_scales<real><<<nblk(N), 256, 0, s>>>(N, Bk.perm, vbar, e);
    bl_init_rows<real><<<nblk(M), 256, 0, s>>>(M, F.perm, bvec, d, bs, ud, L->sq_r, L->sq_r2);
    bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_r, L->sq_r2, L->roff, L->sc, RED_INIT_BETA, p->tol, p->stop_rule, 0);
    bl_cols<real><<<bb, LQ_THREADS, 0, s>>>(Bk, mid_c, e, ud, ve, w, x, L->sq_c, L->sc, 1, nullptr, 0);
    bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_c, nullptr, L->coff, L->sc, RED_INIT_ALPHA, p->tol, p->stop_rule, 0);
    launches += 8;
    SME_CUDA(cudaGetLastError());
    const int every = std::max(1, p->check_every);
    // With one group per matrix, matrix b's rows are sorted positions row_off[b] .. row_off[b+1]-1 (columns
    // likewise), so once some matrices have converged the products run over the slices of the others only.
    const bool compact = B->matrix_major;
    std::vector<int32_t> lr, lc;
    std::vector<char> active_prev(count, 1);
    int64_t nlr = 0, nlc = 0;
    unsigned gr = fb, gc = bb;
    if (compact) {
        if (cudaMalloc(&L->list_r, F.nslices * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&L->list_c, Bk.nslices * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(SME_ERR_OOM);
        }
    }
    auto slices_of_active = [&](const int64_t *off, std::vector<int32_t> &out) {
        out.clear();
        int64_t last = -1;
        for (int b = 0; b < count; ++b) {
            if (L->host[b].done) continue;
            const int64_t s0 = std::max<int64_t>(off[b] / 32, last + 1), s1 = (off[b + 1] + 31) / 32;
            for (int64_t q = s0; q < s1; ++q) out.push_back((int32_t)q);
            last = std::max<int64_t>(last, s1 - 1);
        }
    };
    const int32_t *use_lr = nullptr, *use_lc = nullptr;
    int64_t it = 0;
    bool all_done = false;
    while (it < p->max_iters && !all_done) {
        const int64_t chunk = std::min<int64_t>(every, p->max_iters - it);
        for (int64_t j = 0; j < chunk; ++j) {
            bl_rows<real><<<gr, LQ_THREADS, 0, s>>>(F, mid_r, d, ve, ud, L->sq_r, L->sc, use_lr, nlr);
            bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_r, nullptr, L->roff, L->sc, RED_BETA, p->tol, p->stop_rule, 0);
            bl_cols<real><<<gc, LQ_THREADS, 0, s>>>(Bk, mid_c, e, ud, ve, w, x, L->sq_c, L->sc, 0, use_lc, nlc);
            bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_c, nullptr, L->coff, L->sc, RED_ALPHA, p->tol, p->stop_rule, 0);
        }
        it += chunk;
        bl_current_x<real><<<nblk(N), 256, 0, s>>>(N, mid_c, Bk.perm, e, x, w, L->sc, xt, nullptr, 1);
        bl_residual<real><<<gr, LQ_THREADS, 0, s>>>(F, mid_r, L->sc, 1, xt, bs, L->r, L->sq_r, use_lr, nlr);
        bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_r, nullptr, L->roff, L->sc, RED_RESID, p->tol, p->stop_rule, 0);
        launches += 4 * chunk + 3;
        if (p->stop_rule == 1) {
            bl_normal<real><<<bb, LQ_THREADS, 0, s>>>(Bk, L->r, L->sq_c);
            bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_c, nullptr, L->coff, L->sc, RED_NORMAL, p->tol, 1, 0);
            launches += 2;
        }
        SME_CUDA(cudaGetLastError());
        SME_CUDA(cudaMemcpyAsync(L->host, L->sc, count * sizeof(BScal), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaStreamSynchronize(s));
        all_done = true;
        bool changed = false;
        for (int b = 0; b < count; ++b) {
            const char act = L->host[b].done == 0;
            all_done = all_done && !act;
            changed = changed || act != active_prev[b];
            active_prev[b] = act;
        }
        if (compact && changed && !all_done) {
            slices_of_active(B->row_off, lr);
            slices_of_active(B->col_off, lc);
            nlr = (int64_t)lr.size();
            nlc = (int64_t)lc.size();
            SME_CUDA(cudaMemcpyAsync(L->list_r, lr.data(), nlr * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SME_CUDA(cudaMemcpyAsync(L->list_c, lc.data(), nlc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SME_CUDA(cudaStreamSynchronize(s));  // the host vectors may change before the copies complete
            use_lr = L->list_r;
            use_lc = L->list_c;
            gr = (unsigned)std::max<int64_t>((nlr + 7) / 8, 1);
            gc = (unsigned)std::max<int64_t>((nlc + 7) / 8, 1);
        }
    }
    bl_current_x<real><<<nblk(N), 256, 0, s>>>(N, mid_c, Bk.perm, e, x, w, L->sc, xt, x_out, 0);
    bl_residual<real><<<fb, LQ_THREADS, 0, s>>>(F, mid_r, L->sc, 0, xt, bs, L->r, L->sq_r, nullptr, 0);
    bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_r, nullptr, L->roff, L->sc, RED_RESID, p->tol, p->stop_rule, 1);
    bl_normal<real><<<bb, LQ_THREADS, 0, s>>>(Bk, L->r, L->sq_c);
    bl_reduce<<<count, LQ_THREADS, 0, s>>>(L->sq_c, nullptr, L->coff, L->sc, RED_NORMAL, p->tol, p->stop_rule, 1);
    launches += 5;
    SME_CUDA(cudaGetLastError());
    SME_CUDA(cudaMemcpyAsync(L->host, L->sc, count * sizeof(BScal), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    bool all_conv = true, finite = true;
    for (int b = 0; b < count; ++b) {
        const BScal &h = L->host[b];
        const double metric = p->stop_rule == 1 ? h.normal_res : h.rel_res;
        res[b].iters = h.iters;
        res[b].rel_residual = h.rel_res;
        res[b].normal_residual = h.normal_res;
        res[b].converged = metric <= p->tol ? 1 : 0;
        res[b].kernel_launches = b == 0 ? launches : 0;
        res[b].history_count = 0;
        all_conv = all_conv && res[b].converged;
        finite = finite && std::isfinite(h.rel_res);
    }
    if (!finite) {
        set_error("sme_batch_lsqr: a residual became non-finite");
        return SME_ERR_NONFINITE;
    }
    if (!all_conv) {
        set_error("sme_batch_lsqr: some matrices stopped above tol");
        return SME_ERR_NOT_CONVERGED;
    }
    return SME_OK;
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_batch_lsqr(sme_batch b, const void *u_bar, const void *v_bar, const void *bvec, void *x,
                                     const sme_lsqr_params *p, sme_lsqr_result *results, void *stream)
{
    NvtxRange range("sme batch lsqr");
    if (!b || !bvec || !x || !p || !results || p->max_iters < 0 || p->tol < 0 ||
        (p->stop_rule != 0 && p->stop_rule != 1)) {
        set_error("sme_batch_lsqr: bad arguments");
        return SME_ERR_ARG;
    }
    sme_op op = b->op;
    if (op->dbl)
        return batch_lsqr_t<double>(op, (const double *)u_bar, (const double *)v_bar, (const double *)bvec, (double *)x,
                                    p, results, (cudaStream_t)stream);
    return batch_lsqr_t<float>(op, (const float *)u_bar, (const float *)v_bar, (const float *)bvec, (float *)x, p,
                               results, (cudaStream_t)stream);
}
