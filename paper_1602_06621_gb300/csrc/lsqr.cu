// Evaluation of a scaling (exact norms of DAE) and LSQR on the equilibrated operator.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sme_internal.cuh"

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

template <typename real>
static sme_status evaluate_t(sme_op op, const real *u, const real *v, double alpha, double beta, double gamma,
                             double *r2_out, double *c2_out, sme_eval_result *res, cudaStream_t s)
{
    const int64_t m = op->m, n = op->n;
    double *buf = nullptr;
    const int NB = 152;
    SME_CUDA(cudaMallocAsync((void **)&buf, (size_t)(2 * (m + n)) * sizeof(double) + 2 * NB * sizeof(EvalPart), s));
    double *sq_u = buf, *sq_v = buf + m, *r2 = buf + m + n, *c2 = buf + 2 * m + n;
    EvalPart *parts = (EvalPart *)(buf + 2 * (m + n));
    if (r2_out) r2 = r2_out;
    if (c2_out) c2 = c2_out;
    exp2_sorted<real><<<nblk(m), 256, 0, s>>>(m, op->fwd.perm, u, sq_u);
    exp2_sorted<real><<<nblk(n), 256, 0, s>>>(n, op->bwd.perm, v, sq_v);
    exact_norms_kernel<real><<<nblk(op->fwd.nslices * 32), 256, 0, s>>>(op->fwd, op->dbl, sq_v, u, r2);
    exact_norms_kernel<real><<<nblk(op->bwd.nslices * 32), 256, 0, s>>>(op->bwd, op->dbl, sq_u, v, c2);
    eval_partials<real><<<NB, EV_THREADS, 0, s>>>(m, r2, u, alpha, parts);
    eval_partials<real><<<NB, EV_THREADS, 0, s>>>(n, c2, v, beta, parts + NB);
    SME_CUDA(cudaGetLastError());
    std::vector<EvalPart> h(2 * NB);
    SME_CUDA(cudaMemcpyAsync(h.data(), parts, 2 * NB * sizeof(EvalPart), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    SME_CUDA(cudaFreeAsync(buf, s));
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

void release_lsqr(sme_op op) { (void)op; }

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_evaluate(sme_op op, const void *u, const void *v, double alpha, double beta, double gamma,
                                   double *r2, double *c2, sme_eval_result *res, void *stream)
{
    if (!op || !u || !v || !res) {
        set_error("sme_evaluate: bad arguments");
        return SME_ERR_ARG;
    }
    if (op->dense) {
        set_error("sme_evaluate: dense operators are evaluated through sme_estimate");
        return SME_ERR_UNSUPPORTED;
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

extern "C" sme_status sme_lsqr(sme_op op, const void *u_bar, const void *v_bar, const void *b, void *x,
                               const sme_lsqr_params *p, sme_lsqr_result *res, void *stream)
{
    (void)op;
    (void)u_bar;
    (void)v_bar;
    (void)b;
    (void)x;
    (void)p;
    (void)res;
    (void)stream;
    set_error("sme_lsqr: not built yet");
    return SME_ERR_UNSUPPORTED;
}
