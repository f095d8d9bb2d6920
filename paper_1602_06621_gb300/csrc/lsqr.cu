// Evaluation of a scaling (exact norms of DAE) and LSQR on the equilibrated operator.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sme_internal.cuh"
#include "sell_ops.cuh"

namespace sme {

constexpr int EV_THREADS = 256;

__device__ __forceinline__ void load_pair_any(const void *ent, const double *val64, bool dbl, int64_t pi, int &c0,
                                              double &a0, int &c1, double &a1)
{
    if (!dbl) {
        const int4 e = __ldcs((const int4 *)ent + pi);
        c0 = e.x;
        c1 = e.z;
        a0 = (double)__int_as_float(e.y);
        a1 = (double)__int_as_float(e.w);
    } else {
        const int2 c = __ldcs((const int2 *)ent + pi);
        const double2 v = __ldcs((const double2 *)val64 + pi);
        c0 = c.x;
        c1 = c.y;
        a0 = v.x;
        a1 = v.y;
    }
}

// sq[r] = e^{2 x[perm[r]]} for the gather side, in sorted order (FP64).
template <typename real>
__global__ void exp2_sorted(int64_t rows, const int32_t *perm, const real *x, double *sq)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const double e = exp((double)x[perm[r]]);
    sq[r] = e * e;
}

// out[perm[r]] = e^{2 x_own} * sum_l a_l^2 * sq[c_l]  (exact squared norms, FP64 accumulation).
template <typename real>
__global__ void exact_norms_kernel(Sell S, bool dbl, const double *sq, const real *x_own, double *out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slice = r >> 5;
    if (slice >= S.nslices) return;
    const int lane = (int)(r & 31);
    const int w = S.slice_w[slice];
    const int64_t pbase = S.slice_off[slice] / 2 + lane;
    double acc = 0.0;
    for (int q = 0; q < w / 2; ++q) {
        int c0, c1;
        double a0, a1;
        load_pair_any(S.ent, S.val64, dbl, pbase + (int64_t)q * 32, c0, a0, c1, a1);
        acc += a0 * a0 * sq[c0];
        acc += a1 * a1 * sq[c1];
    }
    if (r >= S.rows) return;
    const int32_t i = S.perm[r];
    const double e = exp((double)x_own[i]);
    out[i] = e * e * acc;
}

struct EvalPart {
    double sum_sq_dev;  // sum (sqrt(r2) - target)^2
    double sum_r2;      // sum r2
    double sum_x, sum_x2;
    double maxn, minn;  // over nonempty
    double empty;
};

template <typename real>
__global__ void eval_partials(int64_t n, const double *r2, const real *x, double target, EvalPart *parts)
{
    __shared__ EvalPart sh[EV_THREADS];
    EvalPart p{0, 0, 0, 0, 0, INFINITY, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = r2[i];
        const double nv = sqrt(v);
        p.sum_sq_dev += (nv - target) * (nv - target);
        p.sum_r2 += v;
        const double xi = (double)x[i];
        p.sum_x += xi;
        p.sum_x2 += xi * xi;
        if (v > 0) {
            p.maxn = fmax(p.maxn, nv);
            p.minn = fmin(p.minn, nv);
        } else {
            p.empty += 1.0;
        }
    }
    sh[threadIdx.x] = p;
    __syncthreads();
    for (int o = EV_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            EvalPart &a = sh[threadIdx.x];
            const EvalPart &b = sh[threadIdx.x + o];
            a.sum_sq_dev += b.sum_sq_dev;
            a.sum_r2 += b.sum_r2;
            a.sum_x += b.sum_x;
            a.sum_x2 += b.sum_x2;
            a.maxn = fmax(a.maxn, b.maxn);
            a.minn = fmin(a.minn, b.minn);
            a.empty += b.empty;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Metrics from exact squared norms r2[m], c2[n] (original order) and the state u, v.
template <typename real>
static sme_status evaluate_from_norms(int64_t m, int64_t n, const double *r2, const double *c2, const real *u,
                                      const real *v, double alpha, double beta, double gamma, sme_eval_result *res,
                                      EvalPart *parts, cudaStream_t s)
{
    const int NB = 152;
    eval_partials<real><<<NB, EV_THREADS, 0, s>>>(m, r2, u, alpha, parts);
    eval_partials<real><<<NB, EV_THREADS, 0, s>>>(n, c2, v, beta, parts + NB);
    SME_CUDA(cudaGetLastError());
    std::vector<EvalPart> h(2 * NB);
    SME_CUDA(cudaMemcpyAsync(h.data(), parts, 2 * NB * sizeof(EvalPart), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    EvalPart R{0, 0, 0, 0, 0, INFINITY, 0}, C{0, 0, 0, 0, 0, INFINITY, 0};
    for (int b = 0; b < NB; ++b) {
        for (int side = 0; side < 2; ++side) {
            EvalPart &a = side ? C : R;
            const EvalPart &p = h[side * NB + b];
            a.sum_sq_dev += p.sum_sq_dev;
            a.sum_r2 += p.sum_r2;
            a.sum_x += p.sum_x;
            a.sum_x2 += p.sum_x2;
            a.maxn = std::max(a.maxn, p.maxn);
            a.minn = std::min(a.minn, p.minn);
            a.empty += p.empty;
        }
    }
    res->row_spread = R.minn > 0 && std::isfinite(R.minn) ? R.maxn / R.minn : INFINITY;
    res->col_spread = C.minn > 0 && std::isfinite(C.minn) ? C.maxn / C.minn : INFINITY;
    res->rms = std::sqrt(R.sum_sq_dev + C.sum_sq_dev) / std::sqrt((double)(m + n));
    // f(u,v) of eq. (3): (1/2) sum_ij A_ij^2 e^{2u_i+2v_j} = (1/2) sum_i r2_i.
    res->objective = 0.5 * R.sum_r2 - alpha * alpha * R.sum_x - beta * beta * C.sum_x +
                     0.5 * gamma * (R.sum_x2 + C.sum_x2);
    res->empty_rows = (int64_t)R.empty;
    res->empty_cols = (int64_t)C.empty;
    return SME_OK;
}

template <typename real>
static sme_status evaluate_t(sme_op op, const real *u, const real *v, double alpha, double beta, double gamma,
                             double *r2_out, double *c2_out, sme_eval_result *res, cudaStream_t s)
{
    const int64_t m = op->m, n = op->n;
    const int NB = 152;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc((size_t)(2 * (m + n)) * sizeof(double) + 2 * NB * sizeof(EvalPart)));
    double *buf = scratch.as<double>();
    double *sq_u = buf, *sq_v = buf + m, *r2 = buf + m + n, *c2 = buf + 2 * m + n;
    EvalPart *parts = (EvalPart *)(buf + 2 * (m + n));
    if (r2_out) r2 = r2_out;
    if (c2_out) c2 = c2_out;
    if (op->dense) {
        SME_TRY(dense_exact_norms(op, (const float *)u, (const float *)v, sq_u, sq_v, r2, c2, s));
    } else {
        exp2_sorted<real><<<nblk(m), 256, 0, s>>>(m, op->fwd.perm, u, sq_u);
        exp2_sorted<real><<<nblk(n), 256, 0, s>>>(n, op->bwd.perm, v, sq_v);
        exact_norms_kernel<real><<<nblk(op->fwd.nslices * 32), 256, 0, s>>>(op->fwd, op->dbl, sq_v, u, r2);
        exact_norms_kernel<real><<<nblk(op->bwd.nslices * 32), 256, 0, s>>>(op->bwd, op->dbl, sq_u, v, c2);
    }
    return evaluate_from_norms<real>(m, n, r2, c2, u, v, alpha, beta, gamma, res, parts, s);
}

// Per-matrix partials of a batch: block (b, side) reduces matrix b's rows (side 0) or columns (side 1), whose
// entries are off[b] .. off[b+1]-1 in the batch's original order; targets[side][b] is the matrix's norm target.
template <typename real>
__global__ void __launch_bounds__(EV_THREADS) segment_eval(int count, const int64_t *off_r, const int64_t *off_c,
                                                           const double *r2, const double *c2, const real *u,
                                                           const real *v, const double *targets, EvalPart *parts)
{
    __shared__ EvalPart sh[EV_THREADS];
    const int b = blockIdx.x, side = blockIdx.y;
    const int64_t *off = side ? off_c : off_r;
    const double *q = side ? c2 : r2;
    const real *x = side ? v : u;
    const double target = targets[side * count + b];
    EvalPart p{0, 0, 0, 0, 0, INFINITY, 0};
    for (int64_t i = off[b] + threadIdx.x; i < off[b + 1]; i += blockDim.x) {
        const double w = q[i];
        const double nv = sqrt(w);
        p.sum_sq_dev += (nv - target) * (nv - target);
        p.sum_r2 += w;
        const double xi = (double)x[i];
        p.sum_x += xi;
        p.sum_x2 += xi * xi;
        if (w > 0) {
            p.maxn = fmax(p.maxn, nv);
            p.minn = fmin(p.minn, nv);
        } else {
            p.empty += 1.0;
        }
    }
    sh[threadIdx.x] = p;
    __syncthreads();
    for (int o = EV_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            EvalPart &a = sh[threadIdx.x];
            const EvalPart &c = sh[threadIdx.x + o];
            a.sum_sq_dev += c.sum_sq_dev;
            a.sum_r2 += c.sum_r2;
            a.sum_x += c.sum_x;
            a.sum_x2 += c.sum_x2;
            a.maxn = fmax(a.maxn, c.maxn);
            a.minn = fmin(a.minn, c.minn);
            a.empty += c.empty;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[side * count + b] = sh[0];
}

template <typename real>
static sme_status batch_evaluate_t(sme_op op, const real *u, const real *v, double alpha, double beta, double gamma,
                                   sme_eval_result *res, cudaStream_t s)
{
    const BatchInfo *B = op->batch;
    const int count = B->count;
    const int64_t m = op->m, n = op->n;
    std::vector<int64_t> offs(2 * (count + 1));
    std::memcpy(offs.data(), B->row_off, (count + 1) * sizeof(int64_t));
    std::memcpy(offs.data() + count + 1, B->col_off, (count + 1) * sizeof(int64_t));
    std::vector<double> al(count), be(count), targets(2 * count);
    for (int b = 0; b < count; ++b) {
        const double mb = (double)(B->row_off[b + 1] - B->row_off[b]), nb = (double)(B->col_off[b + 1] - B->col_off[b]);
        al[b] = alpha > 0 ? alpha : std::pow(nb / mb, 0.25);
        be[b] = beta > 0 ? beta : std::pow(mb / nb, 0.25);
        targets[b] = al[b];
        targets[count + b] = be[b];
    }
    const size_t bytes = (size_t)(2 * (m + n)) * 8 + offs.size() * 8 + targets.size() * 8 + 2 * count * sizeof(EvalPart);
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc(bytes));
    char *buf = scratch.as<char>();
    double *sq_u = (double *)buf, *sq_v = sq_u + m, *r2 = sq_v + n, *c2 = r2 + m;
    int64_t *d_off = (int64_t *)(c2 + n);
    double *d_tg = (double *)(d_off + offs.size());
    EvalPart *parts = (EvalPart *)(d_tg + targets.size());
    SME_CUDA(cudaMemcpyAsync(d_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemcpyAsync(d_tg, targets.data(), targets.size() * 8, cudaMemcpyHostToDevice, s));
    exp2_sorted<real><<<nblk(m), 256, 0, s>>>(m, op->fwd.perm, u, sq_u);
    exp2_sorted<real><<<nblk(n), 256, 0, s>>>(n, op->bwd.perm, v, sq_v);
    exact_norms_kernel<real><<<nblk(op->fwd.nslices * 32), 256, 0, s>>>(op->fwd, op->dbl, sq_v, u, r2);
    exact_norms_kernel<real><<<nblk(op->bwd.nslices * 32), 256, 0, s>>>(op->bwd, op->dbl, sq_u, v, c2);
    segment_eval<real><<<dim3(count, 2), EV_THREADS, 0, s>>>(count, d_off, d_off + count + 1, r2, c2, u, v, d_tg,
                                                             parts);
    SME_CUDA(cudaGetLastError());
    std::vector<EvalPart> h(2 * count);
    SME_CUDA(cudaMemcpyAsync(h.data(), parts, h.size() * sizeof(EvalPart), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < count; ++b) {
        const EvalPart &R = h[b], &C = h[count + b];
        sme_eval_result &o = res[b];
        o.row_spread = R.minn > 0 && std::isfinite(R.minn) ? R.maxn / R.minn : INFINITY;
        o.col_spread = C.minn > 0 && std::isfinite(C.minn) ? C.maxn / C.minn : INFINITY;
        const double len = (double)(offs[b + 1] - offs[b] + offs[count + 2 + b] - offs[count + 1 + b]);
        o.rms = std::sqrt(R.sum_sq_dev + C.sum_sq_dev) / std::sqrt(len);
        o.objective = 0.5 * R.sum_r2 - al[b] * al[b] * R.sum_x - be[b] * be[b] * C.sum_x +
                      0.5 * gamma * (R.sum_x2 + C.sum_x2);
        o.empty_rows = (int64_t)R.empty;
        o.empty_cols = (int64_t)C.empty;
    }
    return SME_OK;
}

// ------------------------------------------------------------------ LSQR
//
// Paige & Saunders (1982) LSQR on K = D A E, used as in Section 5.1: solve K xbar = D b from
// xbar = 0 and return x = E xbar; accuracy is measured on the original system.
//
// Vectors live in sorted order.  The products gather pre-scaled vectors so each nonzero costs a
// single gather: ud = D uhat (uhat = beta u, unnormalised) for the products with A^T, and
// ve = E vhat (vhat = alpha v) for the products with A.  The norms beta and alpha are FP64
// reductions (block partials summed in a fixed order by the last block), and the scalar
// recurrence runs in FP64 in the last block of each A^T-kernel, so the host only looks at the
// state every check_every iterations.  The update x <- x + (phi/rho) w, w <- v - (theta/rho) w of
// iteration i needs alpha_{i+1}, so it is applied by the A^T-kernel of iteration i+1 (and by the
// final kernel), which reads v_{i+1} there anyway.

struct LsqrScalars {
    double alpha, beta;      // alpha_i (normalises ve), beta (normalises ud)
    double rhobar, phibar;
    double phi, rho, theta;  // phi_i, rho_i, theta_{i+1} of the last completed iteration i
    double bnorm, tol;
    double rel_res, normal_res, afro;
    long long iters;         // completed iterations
    int done;                // 0 running, 1 converged (checked), 2 exact breakdown (beta or alpha = 0)
    int first;               // next A^T-kernel starts the w/x sequence (w_1 = v_1, x_0 = 0)
    int stop_rule;
    int pad;
};

struct LsqrState {
    void *ud, *ve, *w, *x, *d, *e, *bs, *xt;
    double *r;
    double *partials;  // 2 * max blocks
    unsigned *counter;
    LsqrScalars *sc;
    LsqrScalars *host;  // host mirror
    int64_t bytes;
    int64_t fwd_blocks, bwd_blocks;
    double afro;  // cached ||A||_F (< 0: not computed)
    // The graph of one chunk of check_every iterations and its check, kept for later calls on this op (it
    // reads only the op's own buffers); rebuilt when check_every or the stop rule changes.
    cudaGraphExec_t chunk = nullptr;
    int chunk_every = 0, chunk_rule = -1;
};



// b in sorted row order, u_1 = D b / beta_1 stored as ud = D (D b); beta_1 and ||b|| reduced.
template <typename real>
__global__ void lsqr_init_rows(int64_t m, const int32_t *perm, const real *b, const real *d, real *bs, real *ud,
                               double *partials, unsigned *counter, LsqrScalars *sc)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double pb = 0.0, pdb = 0.0;
    if (r < m) {
        const real bi = b[perm[r]];
        const real dr = d[r];
        bs[r] = bi;
        const real db = dr * bi;
        ud[r] = dr * db;
        pb = (double)bi * (double)bi;
        pdb = (double)db * (double)db;
    }
    // Two sums through the same partial array: [0, grid) for ||D b||^2, [grid, 2 grid) for ||b||^2.
    const double s1 = block_sum(pdb);
    const double s2 = block_sum(pb);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s1;
        partials[gridDim.x + blockIdx.x] = s2;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v1 = 0.0, v2 = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        v1 += __ldcg(partials + i);
        v2 += __ldcg(partials + gridDim.x + i);
    }
    const double t1 = block_sum(v1);
    const double t2 = block_sum(v2);
    if (threadIdx.x == 0) {
        *counter = 0u;
        sc->beta = sqrt(t1);
        sc->phibar = sc->beta;
        sc->bnorm = sqrt(t2);
        sc->phi = 0.0;
        sc->rho = 1.0;
        sc->theta = 0.0;
        sc->iters = 0;
        sc->first = 1;
        sc->done = sc->beta > 0.0 ? 0 : 2;
        sc->rel_res = sc->bnorm > 0.0 ? 1.0 : 0.0;
    }
}

// Products with A (rows): uhat = K v_i - alpha_i u_i; beta_{i+1} = ||uhat||.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS, 8) lsqr_rows(Sell S, const real *d, const real *ve, real *ud,
                                                         double *partials, unsigned *counter, LsqrScalars *sc)
{
    if (((volatile LsqrScalars *)sc)->done) return;  // the same for every thread of the block
    const double alpha = sc->alpha, beta = sc->beta;
    const real inv_alpha = (real)(alpha > 0.0 ? 1.0 / alpha : 0.0);
    const real alpha_r = (real)alpha;
    const real inv_beta = (real)(beta > 0.0 ? 1.0 / beta : 0.0);
    const SplitSlice<SPLIT> sw;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, sw, ve);
    double part = 0.0;
    if (sw.lead() && sw.slice < S.nslices) {
        const int64_t r = sw.slice * 32 + sw.lane;
        if (r < S.rows) {
            const real dr = d[r];
            const real uhat = dr * acc * inv_alpha - alpha_r * (ud[r] / dr) * inv_beta;
            ud[r] = dr * uhat;
            part = (double)uhat * (double)uhat;
        }
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x == 0) sc->beta = sqrt(tot);
}

// Products with A^T (columns): the lagged x/w update of the previous iteration, then
// vhat = K^T u_{i+1} - beta_{i+1} v_i, alpha_{i+1} = ||vhat||, and the scalar recurrence of iteration i.
// init = 1 computes vhat = K^T u_1 only (alpha_1, rhobar_1).
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS, 8) lsqr_cols(Sell S, const real *e, const real *ud, real *ve, real *w,
                                                         real *x, double *partials, unsigned *counter,
                                                         LsqrScalars *sc, int init)
{
    if (((volatile LsqrScalars *)sc)->done) return;  // the same for every thread of the block
    const double alpha = sc->alpha, beta = sc->beta;
    const int first = sc->first;
    const real inv_alpha = (real)(alpha > 0.0 ? 1.0 / alpha : 0.0);
    const real inv_beta = (real)(beta > 0.0 ? 1.0 / beta : 0.0);
    const real beta_r = (real)beta;
    const real x_step = (real)(sc->phi / sc->rho);
    const real w_step = (real)(sc->theta / sc->rho);
    const SplitSlice<SPLIT> sw;
    const real acc = sell_row_dot_split<real, real, real, SPLIT>(S, sw, ud);
    double part = 0.0;
    if (sw.lead() && sw.slice < S.nslices) {
        const int64_t c = sw.slice * 32 + sw.lane;
        if (c < S.rows) {
            const real ec = e[c];
            real vhat;
            if (init) {
                vhat = ec * acc * inv_beta;
                w[c] = real(0);
                x[c] = real(0);
            } else {
                const real v = ve[c] / ec * inv_alpha;
                if (first) {
                    w[c] = v;
                    x[c] = real(0);
                } else {
                    const real wo = w[c];
                    x[c] = x[c] + x_step * wo;
                    w[c] = v - w_step * wo;
                }
                vhat = ec * acc * inv_beta - beta_r * v;
            }
            ve[c] = ec * vhat;
            part = (double)vhat * (double)vhat;
        }
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x != 0) return;
    const double alpha_n = sqrt(tot);
    if (init) {
        sc->alpha = alpha_n;
        sc->rhobar = alpha_n;
        if (alpha_n == 0.0) sc->done = 2;
        return;
    }
    const double rho = hypot(sc->rhobar, beta);
    const double cs = sc->rhobar / rho, sn = beta / rho;
    sc->theta = sn * alpha_n;
    sc->rhobar = -cs * alpha_n;
    sc->phi = cs * sc->phibar;
    sc->phibar = sn * sc->phibar;
    sc->rho = rho;
    sc->alpha = alpha_n;
    sc->first = 0;
    sc->iters += 1;
    if (beta == 0.0 || alpha_n == 0.0) sc->done = 2;
}

// xt = E (x + (phi/rho) w): the current iterate x_i = E xbar_i; with perm != NULL also written to
// x_out in original column order (the final result).
template <typename real>
__global__ void lsqr_current_x(int64_t n, const real *e, const real *x, const real *w, const LsqrScalars *sc,
                               real *xt, const int32_t *perm, real *x_out)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (sc->done == 1 && !perm) return;
    const real step = (real)(sc->phi / sc->rho);
    const real v = e[c] * (x[c] + step * w[c]);
    if (xt) xt[c] = v;
    if (perm) x_out[perm[c]] = v;
}

// r = A xt - b in FP64 (rows); ||r|| / ||b|| against tol (stop_rule 0).
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) lsqr_residual(Sell S, const real *xt, const real *bs, double *r,
                                                             double *partials, unsigned *counter, LsqrScalars *sc,
                                                             int final_check)
{
    if (!final_check && ((volatile LsqrScalars *)sc)->done == 1) return;  // uniform over the block
    const SplitSlice<SPLIT> sw;
    const double acc = sell_row_dot_split<real, double, real, SPLIT>(S, sw, xt);
    double part = 0.0;
    if (sw.lead() && sw.slice < S.nslices) {
        const int64_t i = sw.slice * 32 + sw.lane;
        if (i < S.rows) {
            const double ri = acc - (double)bs[i];
            r[i] = ri;
            part = ri * ri;
        }
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x != 0) return;
    sc->rel_res = sc->bnorm > 0.0 ? sqrt(tot) / sc->bnorm : sqrt(tot);
    sc->normal_res = sqrt(tot);  // ||r||, turned into the normal residual by lsqr_normal
    if (!final_check && sc->stop_rule == 0 && sc->rel_res <= sc->tol && sc->done == 0) sc->done = 1;
}

// ||A^T r|| / (||A||_F ||r||) (columns), FP64.
template <typename real, int SPLIT>
__global__ void __launch_bounds__(LQ_THREADS) lsqr_normal(Sell S, const double *r, double *partials,
                                                           unsigned *counter, LsqrScalars *sc, int final_check)
{
    if (!final_check && ((volatile LsqrScalars *)sc)->done == 1) return;  // uniform over the block
    const SplitSlice<SPLIT> sw;
    const double acc = sell_row_dot_split<real, double, double, SPLIT>(S, sw, r);
    double part = 0.0;
    if (sw.lead() && sw.slice < S.nslices && sw.slice * 32 + sw.lane < S.rows) part = acc * acc;
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x != 0) return;
    const double rn = sc->normal_res;
    sc->normal_res = (rn > 0.0 && sc->afro > 0.0) ? sqrt(tot) / (sc->afro * rn) : 0.0;
    if (!final_check && sc->stop_rule == 1 && sc->normal_res <= sc->tol && sc->done == 0) sc->done = 1;
}

template <typename real>
__global__ void scales_sorted(int64_t n, const int32_t *perm, const real *logscale, real *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = logscale ? (real)exp((double)logscale[perm[i]]) : real(1);
}

template <typename real>
__global__ void __launch_bounds__(LQ_THREADS) frobenius_sq(Sell S, double *partials, unsigned *counter, double *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slice = (int64_t)blockIdx.x * (LQ_THREADS / 32) + warp;
    double part = 0.0;
    if (slice < S.nslices) {
        const int np = S.slice_w[slice] / 2;
        const int64_t pbase = S.slice_off[slice] / 2 + lane;
        for (int q = 0; q < np; ++q) {
            int c0, c1;
            real a0, a1;
            pair_load<real>(S, pbase + (int64_t)q * 32, c0, a0, c1, a1);
            part += (double)a0 * (double)a0 + (double)a1 * (double)a1;
        }
    }
    if (!arrive_last(part, partials, counter)) return;
    const double tot = sum_partials(partials, counter);
    if (threadIdx.x == 0) *out = tot;
}

static LsqrState *lsqr_state(sme_op op) { return (LsqrState *)op->ws.lsqr; }

void release_lsqr(sme_op op)
{
    LsqrState *L = lsqr_state(op);
    if (!L) return;
    for (void *p : {L->ud, L->ve, L->w, L->x, L->d, L->e, L->bs, L->xt, (void *)L->r, (void *)L->partials,
                    (void *)L->counter, (void *)L->sc})
        dev_release(p);
    if (L->chunk) cudaGraphExecDestroy(L->chunk);
    delete L->host;
    delete L;
    op->ws.lsqr = nullptr;
}

static sme_status alloc_lsqr(sme_op op, cudaStream_t s);

// The op's LSQR state, allocated on first use; a failed allocation leaves no partial state behind.
static sme_status ensure_lsqr(sme_op op, cudaStream_t s)
{
    if (lsqr_state(op)) return SME_OK;
    const sme_status st = alloc_lsqr(op, s);
    if (st != SME_OK) release_lsqr(op);
    return st;
}

static sme_status alloc_lsqr(sme_op op, cudaStream_t s)
{
    LsqrState *L = new LsqrState();
    op->ws.lsqr = L;
    const size_t sz = op->dbl ? 8 : 4;
    const int64_t m = op->m, n = op->n;
    L->fwd_blocks = (op->fwd.nslices + 7) / 8;
    L->bwd_blocks = (op->bwd.nslices + 7) / 8;
    // One partial per block of any pass: at most one block per slice (8 warps on one slice).
    const int64_t maxb = std::max<int64_t>(std::max(op->fwd.nslices, op->bwd.nslices), (std::max(m, n) + 255) / 256);
    SME_TRY(dev_alloc(op, &L->ud, m * sz));
    SME_TRY(dev_alloc(op, &L->bs, m * sz));
    SME_TRY(dev_alloc(op, &L->d, m * sz));
    SME_TRY(dev_alloc(op, (void **)&L->r, m * sizeof(double)));
    SME_TRY(dev_alloc(op, &L->ve, n * sz));
    SME_TRY(dev_alloc(op, &L->w, n * sz));
    SME_TRY(dev_alloc(op, &L->x, n * sz));
    SME_TRY(dev_alloc(op, &L->e, n * sz));
    SME_TRY(dev_alloc(op, &L->xt, n * sz));
    SME_TRY(dev_alloc(op, (void **)&L->partials, 2 * maxb * sizeof(double)));
    SME_TRY(dev_alloc(op, (void **)&L->counter, sizeof(unsigned)));
    SME_TRY(dev_alloc(op, (void **)&L->sc, sizeof(LsqrScalars)));
    L->host = new LsqrScalars();  // a one-struct mirror: pageable memory is as fast as pinned here
    SME_CUDA(cudaMemsetAsync(L->counter, 0, sizeof(unsigned), s));
    L->afro = -1.0;
    return SME_OK;
}

template <typename real>
static sme_status lsqr_t(sme_op op, const real *ubar, const real *vbar, const real *b, real *x_out,
                         const sme_lsqr_params *p, sme_lsqr_result *res, cudaStream_t s)
{
    SME_TRY(ensure_lsqr(op, s));
    LsqrState *L = lsqr_state(op);
    const int64_t m = op->m, n = op->n;
    const Sell &F = op->fwd, &B = op->bwd;
    real *ud = (real *)L->ud, *ve = (real *)L->ve, *w = (real *)L->w, *x = (real *)L->x;
    real *d = (real *)L->d, *e = (real *)L->e, *bs = (real *)L->bs, *xt = (real *)L->xt;
    const unsigned fb = (unsigned)std::max<int64_t>(L->fwd_blocks, 1);
    const Pass pf = pass_for(F), pb = pass_for(B);
    int64_t launches = 0;
    LsqrScalars init{};
    init.tol = p->tol;
    init.stop_rule = p->stop_rule;
    init.afro = L->afro;
    SME_CUDA(cudaMemcpyAsync(L->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemsetAsync(x, 0, n * sizeof(real), s));
    SME_CUDA(cudaMemsetAsync(w, 0, n * sizeof(real), s));
    if (L->afro < 0) {
        double *fro = &L->sc->afro;
        frobenius_sq<real><<<fb, LQ_THREADS, 0, s>>>(F, L->partials, L->counter, fro);
        double h = 0.0;
        SME_CUDA(cudaMemcpyAsync(&h, fro, sizeof(double), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaStreamSynchronize(s));
        L->afro = std::sqrt(h);
        SME_CUDA(cudaMemcpyAsync(fro, &L->afro, sizeof(double), cudaMemcpyHostToDevice, s));
        ++launches;
    }
    scales_sorted<real><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, F.perm, ubar, d);
    scales_sorted<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, B.perm, vbar, e);
    lsqr_init_rows<real><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, F.perm, b, d, bs, ud, L->partials,
                                                                       L->counter, L->sc);
    SPLIT_LAUNCH(lsqr_cols, real, pb, s, B, e, ud, ve, w, x, L->partials, L->counter, L->sc, 1);
    launches += 4;
    SME_CUDA(cudaGetLastError());
    const int every = std::max(1, p->check_every);
    // A chunk of `every` iterations and its residual check, on fixed buffers: captured once as a CUDA graph
    // (on a private stream) and replayed; partial chunks and graph-less runs launch directly.
    auto enqueue_chunk = [&](int64_t chunk, cudaStream_t q) {
        for (int64_t j = 0; j < chunk; ++j) {
            SPLIT_LAUNCH(lsqr_rows, real, pf, q, F, d, ve, ud, L->partials, L->counter, L->sc);
            SPLIT_LAUNCH(lsqr_cols, real, pb, q, B, e, ud, ve, w, x, L->partials, L->counter, L->sc, 0);
        }
        lsqr_current_x<real><<<(unsigned)((n + 255) / 256), 256, 0, q>>>(n, e, x, w, L->sc, xt, nullptr, nullptr);
        SPLIT_LAUNCH(lsqr_residual, real, pf, q, F, xt, bs, L->r, L->partials, L->counter, L->sc, 0);
        if (p->stop_rule == 1) SPLIT_LAUNCH(lsqr_normal, real, pb, q, B, L->r, L->partials, L->counter, L->sc, 0);
    };
    if (L->chunk && (L->chunk_every != every || L->chunk_rule != p->stop_rule)) {
        cudaGraphExecDestroy(L->chunk);
        L->chunk = nullptr;
    }
    if (!L->chunk && p->max_iters >= 2 * (int64_t)every) {
        GraphOnce g;
        g.capture([&](cudaStream_t q) { enqueue_chunk(every, q); });
        L->chunk = g.exec;
        g.exec = nullptr;
        L->chunk_every = every;
        L->chunk_rule = p->stop_rule;
    }
    int64_t it = 0, hcount = 0;
    // Predicted checks: the last two checked residuals (the first is 1 at x = 0) give a geometric trend.
    const bool predict = p->predict_check && p->stop_rule == 0 && p->tol > 0.0;
    double res_prev = 1.0, res_last = 1.0;
    int64_t it_prev = 0, it_last = 0;
    while (it < p->max_iters) {
        int64_t chunk = std::min<int64_t>(every, p->max_iters - it);
        if (predict && it_last > it_prev && res_last > p->tol && res_last < res_prev) {
            const double per_iter = std::log(res_last / res_prev) / (double)(it_last - it_prev);  // < 0
            const double need = std::ceil(std::log(p->tol / res_last) / per_iter);
            if (need < (double)chunk) chunk = std::max<int64_t>(1, (int64_t)need);
        }
        if (chunk == every && L->chunk)
            SME_CUDA(cudaGraphLaunch(L->chunk, s));
        else
            enqueue_chunk(chunk, s);
        it += chunk;
        launches += 2 * chunk + 2 + (p->stop_rule == 1 ? 1 : 0);
        SME_CUDA(cudaGetLastError());
        SME_CUDA(cudaMemcpyAsync(L->host, L->sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaStreamSynchronize(s));
        if (p->history && hcount < p->history_cap)
            p->history[hcount] = p->stop_rule == 1 ? L->host->normal_res : L->host->rel_res;
        ++hcount;
        if (L->host->done) break;
        if (std::isfinite(L->host->rel_res)) {
            res_prev = res_last;
            it_prev = it_last;
            res_last = L->host->rel_res;
            it_last = it;
        }
    }
    // Final x in original order, and both residuals of exactly that x.
    lsqr_current_x<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, e, x, w, L->sc, xt, B.perm, x_out);
    SPLIT_LAUNCH(lsqr_residual, real, pf, s, F, xt, bs, L->r, L->partials, L->counter, L->sc, 1);
    SPLIT_LAUNCH(lsqr_normal, real, pb, s, B, L->r, L->partials, L->counter, L->sc, 1);
    launches += 3;
    SME_CUDA(cudaGetLastError());
    SME_CUDA(cudaMemcpyAsync(L->host, L->sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    const LsqrScalars &h = *L->host;
    res->iters = h.iters;
    res->rel_residual = h.rel_res;
    res->normal_residual = h.normal_res;
    const double final_metric = p->stop_rule == 1 ? h.normal_res : h.rel_res;
    res->converged = (h.done != 0 && final_metric <= p->tol) || final_metric <= p->tol ? 1 : 0;
    res->kernel_launches = launches;
    res->history_count = p->history ? std::min(hcount, p->history_cap) : 0;
    if (!std::isfinite(h.rel_res)) {
        set_error("sme_lsqr: residual became non-finite");
        return SME_ERR_NONFINITE;
    }
    if (!res->converged) {
        set_error("sme_lsqr: %lld iterations, residual %.3e above tol %.1e", (long long)h.iters, final_metric,
                  p->tol);
        return SME_ERR_NOT_CONVERGED;
    }
    return SME_OK;
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_evaluate(sme_op op, const void *u, const void *v, double alpha, double beta, double gamma,
                                   double *r2, double *c2, sme_eval_result *res, void *stream)
{
    NvtxRange range("sme evaluate");
    SME_TRY(no_shard(op, "sme_evaluate"));
    if (!op || !u || !v || !res) {
        set_error("sme_evaluate: bad arguments");
        return SME_ERR_ARG;
    }
    if (alpha <= 0) alpha = std::pow((double)op->n / (double)op->m, 0.25);
    if (beta <= 0) beta = std::pow((double)op->m / (double)op->n, 0.25);
    if (gamma <= 0) gamma = 0.1;
    if (op->dbl)
        return evaluate_t<double>(op, (const double *)u, (const double *)v, alpha, beta, gamma, r2, c2, res,
                                  (cudaStream_t)stream);
    return evaluate_t<float>(op, (const float *)u, (const float *)v, alpha, beta, gamma, r2, c2, res,
                             (cudaStream_t)stream);
}

extern "C" sme_status sme_batch_evaluate(sme_batch bt, const void *u, const void *v, double alpha, double beta,
                                         double gamma, sme_eval_result *res, void *stream)
{
    if (!bt || !u || !v || !res) {
        set_error("sme_batch_evaluate: bad arguments");
        return SME_ERR_ARG;
    }
    if (gamma <= 0) gamma = 0.1;
    sme_op op = bt->op;
    if (op->dbl)
        return batch_evaluate_t<double>(op, (const double *)u, (const double *)v, alpha, beta, gamma, res,
                                        (cudaStream_t)stream);
    return batch_evaluate_t<float>(op, (const float *)u, (const float *)v, alpha, beta, gamma, res,
                                   (cudaStream_t)stream);
}

extern "C" sme_status sme_lsqr(sme_op op, const void *u_bar, const void *v_bar, const void *b, void *x,
                               const sme_lsqr_params *p, sme_lsqr_result *res, void *stream)
{
    NvtxRange range("sme lsqr");
    SME_TRY(no_shard(op, "sme_lsqr"));
    if (!op || !b || !x || !p || !res || p->max_iters < 0 || p->tol < 0 || (p->stop_rule != 0 && p->stop_rule != 1) ||
        p->history_cap < 0 || (p->history_cap > 0 && !p->history)) {
        set_error("sme_lsqr: bad arguments");
        return SME_ERR_ARG;
    }
    if (op->dense) {
        set_error("sme_lsqr: dense operators are not supported");
        return SME_ERR_UNSUPPORTED;
    }
    *res = sme_lsqr_result{};
    if (op->dbl)
        return lsqr_t<double>(op, (const double *)u_bar, (const double *)v_bar, (const double *)b, (double *)x, p, res,
                              (cudaStream_t)stream);
    return lsqr_t<float>(op, (const float *)u_bar, (const float *)v_bar, (const float *)b, (float *)x, p, res,
                         (cudaStream_t)stream);
}
