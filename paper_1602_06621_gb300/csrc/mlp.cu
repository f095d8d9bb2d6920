// Learned warm start for Algorithm 1: a small MLP that maps per-row / per-column features of A to
// initial log-scalings u^0, v^0.  (Algorithm 1 itself is unchanged; a warm start needs a step offset
// t0 > 0, since the first step of the paper's schedule, eta_1 = 1/gamma, discards u^0.)
//
// Network: 8 inputs (normalised) -> 128 (ReLU) -> 128 (ReLU) -> 1.  Weights are stored in BF16 for the
// forward pass with FP32 master copies for training; all accumulation is FP32.
//
// Kernels work on tiles of 32 samples: a CTA of 128 threads (thread j = hidden unit j) keeps the layer-2
// weights (FP32, rows padded to 129 words so that the unit-per-thread access pattern is free of bank
// conflicts) and the tile's activations in shared memory.  Training fuses forward and backward per tile;
// each CTA accumulates its gradient partials in shared memory, writes them once, and a second kernel sums
// the partials in CTA order (deterministic) before an Adam step updates the masters and BF16 copies.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "sme_internal.cuh"

namespace sme {

constexpr int MLP_IN = 8, MLP_H = 128, MLP_TS = 32;
constexpr int W2P = MLP_H + 1;  // padded row length of W2 / dW2 in shared memory
// Parameter layout (FP32): W1[H][IN], b1[H], W2[H][H], b2[H], W3[H], b3.
constexpr int P_W1 = 0, P_B1 = P_W1 + MLP_H * MLP_IN, P_W2 = P_B1 + MLP_H, P_B2 = P_W2 + MLP_H * MLP_H,
              P_W3 = P_B2 + MLP_H, P_B3 = P_W3 + MLP_H, P_COUNT = P_B3 + 1;

struct Mlp {
    float *master = nullptr;  // P_COUNT FP32 parameters
    __nv_bfloat16 *wbf = nullptr;  // BF16 copies (same layout; biases copied too)
    float *m1 = nullptr, *m2 = nullptr;  // Adam moments
    float *partials = nullptr;  // per-CTA gradient partials
    float *grad = nullptr;      // reduced gradient
    float *loss_part = nullptr; // per-CTA loss partials
    float *loss_dev = nullptr;  // reduced loss
    int max_ctas = 0;
    float norm_mean[MLP_IN], norm_std[MLP_IN];
    float *d_norm = nullptr;  // device copy: mean[8], 1/std[8]
    long long adam_t = 0;
};

}  // namespace sme

struct sme_mlp_s {
    sme::Mlp m;
};

namespace sme {

struct MlpSmem {
    float W2[MLP_H * W2P];
    float X[MLP_TS][MLP_IN];
    float H1[MLP_TS][MLP_H];
    float H2[MLP_TS][MLP_H];
    float D2[MLP_TS][MLP_H];  // dL/dz2 (training)
    float Y[MLP_TS], DY[MLP_TS];
};

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// Forward of one tile; thread j computes unit j for all samples of the tile.  Returns nothing; results in sm.
__device__ __forceinline__ void tile_forward(MlpSmem &sm, const __nv_bfloat16 *w, int ns)
{
    const int j = threadIdx.x;
    // Layer 1.
    float w1[MLP_IN];
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) w1[f] = bf(w, P_W1 + j * MLP_IN + f);
    const float b1 = __bfloat162float(w[P_B1 + j]);
    for (int s = 0; s < MLP_TS; ++s) {
        float z = b1;
#pragma unroll
        for (int f = 0; f < MLP_IN; ++f) z += w1[f] * sm.X[s][f];
        sm.H1[s][j] = s < ns ? fmaxf(z, 0.f) : 0.f;
    }
    __syncthreads();
    // Layer 2: 32 accumulators per thread.
    float acc[MLP_TS];
    const float b2 = __bfloat162float(w[P_B2 + j]);
#pragma unroll
    for (int s = 0; s < MLP_TS; ++s) acc[s] = b2;
    for (int i = 0; i < MLP_H; ++i) {
        const float wji = sm.W2[j * W2P + i];
#pragma unroll
        for (int s = 0; s < MLP_TS; ++s) acc[s] += wji * sm.H1[s][i];
    }
#pragma unroll
    for (int s = 0; s < MLP_TS; ++s) sm.H2[s][j] = fmaxf(acc[s], 0.f);
    __syncthreads();
    // Layer 3: warp w sums samples w, w+4, ... over the 128 units.
    const int warp = j >> 5, lane = j & 31;
    const float b3 = __bfloat162float(w[P_B3]);
    for (int s = warp; s < MLP_TS; s += MLP_H / 32) {
        float p = 0.f;
        for (int u = lane; u < MLP_H; u += 32) p += bf(w, P_W3 + u) * sm.H2[s][u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0) sm.Y[s] = p + b3;
    }
    __syncthreads();
}

__device__ __forceinline__ void load_tile(MlpSmem &sm, const float *X, int64_t N, int64_t base, const float *norm,
                                          int &ns)
{
    const int64_t rem = N - base;
    ns = (int)(rem < MLP_TS ? rem : (int64_t)MLP_TS);
    for (int e = threadIdx.x; e < MLP_TS * MLP_IN; e += blockDim.x) {
        const int s = e / MLP_IN, f = e % MLP_IN;
        sm.X[s][f] = s < ns ? (X[(base + s) * MLP_IN + f] - norm[f]) * norm[MLP_IN + f] : 0.f;
    }
    __syncthreads();
}

__device__ __forceinline__ void load_w2(MlpSmem &sm, const __nv_bfloat16 *w)
{
    for (int e = threadIdx.x; e < MLP_H * MLP_H; e += blockDim.x)
        sm.W2[(e / MLP_H) * W2P + (e % MLP_H)] = bf(w, P_W2 + e);
    __syncthreads();
}

__global__ void __launch_bounds__(MLP_H) mlp_infer(const __nv_bfloat16 *w, const float *norm, const float *X,
                                                   int64_t N, float *y)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(raw);
    load_w2(sm, w);
    for (int64_t base = (int64_t)blockIdx.x * MLP_TS; base < N; base += (int64_t)gridDim.x * MLP_TS) {
        int ns;
        load_tile(sm, X, N, base, norm, ns);
        tile_forward(sm, w, ns);
        if (threadIdx.x < ns) y[base + threadIdx.x] = sm.Y[threadIdx.x];
        __syncthreads();
    }
}

// Fused forward + backward of the mean squared error (1/N) sum (y - target)^2 over all tiles of this CTA.
// Writes this CTA's gradient partial (P_COUNT floats) and loss partial.
__global__ void __launch_bounds__(MLP_H) mlp_grad(const __nv_bfloat16 *w, const float *norm, const float *X,
                                                  const float *target, int64_t N, float *partials, float *loss_part)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(raw);
    float *dW2 = reinterpret_cast<float *>(raw + sizeof(MlpSmem));  // [H][W2P]
    const int j = threadIdx.x, warp = j >> 5, lane = j & 31;
    load_w2(sm, w);
    for (int e = j; e < MLP_H * W2P; e += blockDim.x) dW2[e] = 0.f;
    float gW1[MLP_IN] = {0.f}, gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, loss = 0.f;
    const float w3j = bf(w, P_W3 + j);
    const float invN = 1.f / (float)N;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * MLP_TS; base < N; base += (int64_t)gridDim.x * MLP_TS) {
        int ns;
        load_tile(sm, X, N, base, norm, ns);
        tile_forward(sm, w, ns);
        if (j < MLP_TS) {
            const float r = j < ns ? sm.Y[j] - target[base + j] : 0.f;
            sm.DY[j] = 2.f * r * invN;
            loss += r * r;
        }
        __syncthreads();
        // Layer 3 and the ReLU of layer 2: dz2[s][j] = dy[s] * W3[j] * (h2 > 0).
        for (int s = 0; s < MLP_TS; ++s) {
            const float dy = sm.DY[s], h2 = sm.H2[s][j];
            gW3 += dy * h2;
            const float d2 = h2 > 0.f ? dy * w3j : 0.f;
            sm.D2[s][j] = d2;
            gb2 += d2;
            if (j == 0) gb3 += dy;
        }
        __syncthreads();
        // dW2[j][i] += sum_s dz2[s][j] h1[s][i]  (thread j owns row j).
        for (int i = 0; i < MLP_H; ++i) {
            float g = 0.f;
#pragma unroll 8
            for (int s = 0; s < MLP_TS; ++s) g += sm.D2[s][j] * sm.H1[s][i];
            dW2[j * W2P + i] += g;
        }
        // dz1[s][j] = (sum_u W2[u][j] dz2[s][u]) * (h1 > 0), thread j = unit j of layer 1.
        for (int s = 0; s < MLP_TS; ++s) {
            float d1 = 0.f;
            for (int u = 0; u < MLP_H; ++u) d1 += sm.W2[u * W2P + j] * sm.D2[s][u];
            d1 = sm.H1[s][j] > 0.f ? d1 : 0.f;
            gb1 += d1;
#pragma unroll
            for (int f = 0; f < MLP_IN; ++f) gW1[f] += d1 * sm.X[s][f];
        }
        __syncthreads();
    }
    float *P = partials + (int64_t)blockIdx.x * P_COUNT;
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) P[P_W1 + j * MLP_IN + f] = gW1[f];
    P[P_B1 + j] = gb1;
    for (int i = 0; i < MLP_H; ++i) P[P_W2 + j * MLP_H + i] = dW2[j * W2P + i];
    P[P_B2 + j] = gb2;
    P[P_W3 + j] = gW3;
    // Loss and db3: block sums in a fixed order.
    __shared__ float red[2][MLP_H / 32];
    float l = loss, b = gb3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        red[0][warp] = l;
        red[1][warp] = b;
    }
    __syncthreads();
    if (j == 0) {
        float lt = 0.f, bt = 0.f;
        for (int q = 0; q < MLP_H / 32; ++q) {
            lt += red[0][q];
            bt += red[1][q];
        }
        P[P_B3] = bt;
        loss_part[blockIdx.x] = lt;
    }
}

// grad[e] = sum over CTAs (in order) of partials; loss = sum of loss partials / N.
__global__ void mlp_reduce(const float *partials, int nparts, float *grad, const float *loss_part, float *loss_out,
                           int64_t N)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < P_COUNT) {
        float g = 0.f;
        for (int c = 0; c < nparts; ++c) g += partials[(int64_t)c * P_COUNT + e];
        grad[e] = g;
    }
    if (e == 0 && loss_out) {
        float l = 0.f;
        for (int c = 0; c < nparts; ++c) l += loss_part[c];
        *loss_out = l / (float)N;
    }
}

__global__ void mlp_adam(float *master, __nv_bfloat16 *wbf, float *m1, float *m2, const float *grad, float lr,
                         float b1, float b2, float eps, float c1, float c2)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P_COUNT) return;
    const float g = grad[e];
    const float a = b1 * m1[e] + (1.f - b1) * g;
    const float v = b2 * m2[e] + (1.f - b2) * g * g;
    m1[e] = a;
    m2[e] = v;
    const float p = master[e] - lr * (a * c1) / (sqrtf(v * c2) + eps);
    master[e] = p;
    wbf[e] = __float2bfloat16_rn(p);
}

__global__ void mlp_to_bf16(const float *master, __nv_bfloat16 *wbf)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < P_COUNT) wbf[e] = __float2bfloat16_rn(master[e]);
}

// Row features of a sliced-ELL operator side: nnz count and mean |value|, written in original order.
template <typename real>
__global__ void side_stats(Sell S, float *cnt, float *meanabs)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S.rows) return;
    const int64_t slice = r >> 5;
    const int lane = (int)(r & 31);
    const int w = S.slice_w[slice];
    const int64_t pbase = S.slice_off[slice] / 2 + lane;
    double sabs = 0.0;
    int c = 0;
    for (int q = 0; q < w / 2; ++q) {
        double a0, a1;
        if (sizeof(real) == 4) {
            const int4 e = ((const int4 *)S.ent)[pbase + (int64_t)q * 32];
            a0 = __int_as_float(e.y);
            a1 = __int_as_float(e.w);
        } else {
            const double2 v = ((const double2 *)S.val64)[pbase + (int64_t)q * 32];
            a0 = v.x;
            a1 = v.y;
        }
        if (a0 != 0.0) {
            sabs += fabs(a0);
            ++c;
        }
        if (a1 != 0.0) {
            sabs += fabs(a1);
            ++c;
        }
    }
    const int32_t i = S.perm[r];
    cnt[i] = (float)c;
    meanabs[i] = c ? (float)(sabs / c) : 0.f;
}

// Matrix of entry i when the entries of matrix b are off[b] .. off[b+1]-1 (count matrices).
__device__ __forceinline__ int segment_of(const int64_t *off, int count, int64_t i)
{
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Feature rows: [log sketch norm, log(1 + nnz), log mean|a|, side, mean sketch of the matrix's rows, of its
// columns, log m, log n], each matrix of a batch with its own means and sizes.
template <typename real>
__global__ void assemble_features(int64_t len, const real *z, const float *cnt, const float *meanabs, float side,
                                  int count, const int64_t *off_own, const int64_t *off_r, const int64_t *off_c,
                                  const float *mu_r, const float *mu_c, float *F)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int b = segment_of(off_own, count, i);
    float *f = F + i * MLP_IN;
    f[0] = 0.5f * logf(fmaxf((float)z[i], 1e-30f));
    f[1] = log1pf(cnt[i]);
    f[2] = logf(fmaxf(meanabs[i], 1e-30f));
    f[3] = side;
    f[4] = mu_r[b];
    f[5] = mu_c[b];
    f[6] = logf((float)(off_r[b + 1] - off_r[b]));
    f[7] = logf((float)(off_c[b + 1] - off_c[b]));
}

// Mean of 1/2 log(sketch) over each matrix's entries (FP64 sums): one CTA per matrix.
template <typename real>
__global__ void __launch_bounds__(1024) segment_mean_log_sketch(const int64_t *off, const real *z, float *out)
{
    __shared__ double sh[1024];
    const int b = blockIdx.x;
    const int64_t lo = off[b], hi = off[b + 1];
    double v = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v += 0.5 * log(fmax((double)z[i], 1e-30));
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = (float)(sh[0] / (double)(hi - lo));
}

template <typename real>
__global__ void cast_out(int64_t n, const float *y, real *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (real)y[i];
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static size_t infer_smem() { return sizeof(MlpSmem); }
static size_t grad_smem() { return sizeof(MlpSmem) + (size_t)MLP_H * W2P * sizeof(float); }

// ------------------------------------------------------------------ training data on the device

constexpr int NORM_THREADS = 256;
constexpr int NORM_BLOCKS = 152 * 2;

// Per-block FP64 sums over rows of X (N x 8) of x_f - shift_f (pass 1: shift = 0) or of (x_f - shift_f)^2
// (pass 2: shift = the mean); rows split evenly over the blocks, each block sums its rows in order.
__global__ void __launch_bounds__(NORM_THREADS) feature_sums(const float *X, int64_t N, const double *shift,
                                                              int squared, double *partials)
{
    __shared__ double sh[NORM_THREADS][MLP_IN + 1];
    double acc[MLP_IN];
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) acc[f] = 0.0;
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(N, lo + per);
    for (int64_t i = lo + threadIdx.x; i < hi; i += NORM_THREADS)
#pragma unroll
        for (int f = 0; f < MLP_IN; ++f) {
            const double d = (double)X[i * MLP_IN + f] - (shift ? shift[f] : 0.0);
            acc[f] += squared ? d * d : d;
        }
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) sh[threadIdx.x][f] = acc[f];
    __syncthreads();
    if (threadIdx.x < MLP_IN) {
        double t = 0.0;
        for (int j = 0; j < NORM_THREADS; ++j) t += sh[j][threadIdx.x];
        partials[(int64_t)blockIdx.x * MLP_IN + threadIdx.x] = t;
    }
}

// out_f = (sum of the blocks' partials in block order) / div.
__global__ void feature_finish(const double *partials, int nblocks, double div, double *out)
{
    const int f = threadIdx.x;
    if (f >= MLP_IN) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[(int64_t)b * MLP_IN + f];
    out[f] = t / div;
}

// Minibatch of `batch` rows of (X, y) drawn uniformly with replacement: row of draw b at step `step` is
// floor(r N / 2^32), r the first word of Philox4x32-10 at counter (b mod 2^32, b >> 32, step, 0x6D6C7000),
// key (seed mod 2^32, seed >> 32).
__global__ void draw_batch_rows(const float *X, const float *y, int64_t N, int64_t batch, uint32_t k0, uint32_t k1,
                                uint32_t step, float *Xb, float *yb)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const U4 o = philox10(U4{(uint32_t)b, (uint32_t)(b >> 32), step, 0x6D6C7000u}, k0, k1);
    const int64_t i = (int64_t)(((uint64_t)o.x * (uint64_t)N) >> 32);
    const float4 *src = reinterpret_cast<const float4 *>(X + i * MLP_IN);
    float4 *dst = reinterpret_cast<float4 *>(Xb + b * MLP_IN);
    dst[0] = src[0];
    dst[1] = src[1];
    yb[b] = y[i];
}

template <typename real>
static sme_status features_t(sme_op op, uint64_t seed, float *rowF, float *colF, cudaStream_t s)
{
    const int64_t m = op->m, n = op->n;
    // Matrix boundaries: one matrix for a single operator, the batch's offsets otherwise.
    const int count = op->batch ? op->batch->count : 1;
    std::vector<int64_t> offs(2 * (count + 1));
    if (op->batch) {
        std::memcpy(offs.data(), op->batch->row_off, (count + 1) * sizeof(int64_t));
        std::memcpy(offs.data() + count + 1, op->batch->col_off, (count + 1) * sizeof(int64_t));
    } else {
        offs = {0, m, 0, n};
    }
    const size_t bytes = (size_t)(m + n) * (sizeof(real) * 2 + 8) + offs.size() * 8 + 2 * (size_t)count * 4 + 64;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc(bytes));
    char *buf = scratch.as<char>();
    real *u0 = (real *)buf, *v0 = u0 + m, *zu = v0 + n, *zv = zu + m;
    float *cnt = (float *)(zv + n), *mab = cnt + (m + n);
    int64_t *d_off = (int64_t *)(((uintptr_t)(mab + (m + n)) + 15) & ~(uintptr_t)15);
    float *mu = (float *)(d_off + offs.size());
    SME_CUDA(cudaMemcpyAsync(d_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemsetAsync(u0, 0, (size_t)(m + n) * sizeof(real), s));
    SME_TRY(estimate_sparse(op, u0, v0, 1, 8, seed, 0, zu, zv, s));
    side_stats<real><<<nblk(m), 256, 0, s>>>(op->fwd, cnt, mab);
    side_stats<real><<<nblk(n), 256, 0, s>>>(op->bwd, cnt + m, mab + m);
    const int64_t *off_r = d_off, *off_c = d_off + count + 1;
    segment_mean_log_sketch<real><<<count, 1024, 0, s>>>(off_r, zu, mu);
    segment_mean_log_sketch<real><<<count, 1024, 0, s>>>(off_c, zv, mu + count);
    if (rowF)
        assemble_features<real><<<nblk(m), 256, 0, s>>>(m, zu, cnt, mab, 0.f, count, off_r, off_r, off_c, mu,
                                                        mu + count, rowF);
    if (colF)
        assemble_features<real><<<nblk(n), 256, 0, s>>>(n, zv, cnt + m, mab + m, 1.f, count, off_c, off_r, off_c, mu,
                                                        mu + count, colF);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_mlp_create(sme_mlp *out, uint64_t seed)
{
    if (!out) return SME_ERR_ARG;
    *out = nullptr;
    sme_mlp M = new sme_mlp_s();
    Mlp &m = M->m;
    // He initialisation from a seeded host generator (splitmix64 + Box-Muller), biases zero.
    std::vector<float> p(P_COUNT, 0.f);
    uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() { return std::sqrt(-2.0 * std::log(1.0 - next())) * std::cos(6.283185307179586 * next()); };
    for (int e = 0; e < MLP_H * MLP_IN; ++e) p[P_W1 + e] = (float)(normal() * std::sqrt(2.0 / MLP_IN));
    for (int e = 0; e < MLP_H * MLP_H; ++e) p[P_W2 + e] = (float)(normal() * std::sqrt(2.0 / MLP_H));
    for (int e = 0; e < MLP_H; ++e) p[P_W3 + e] = (float)(normal() * std::sqrt(1.0 / MLP_H));
    for (int f = 0; f < MLP_IN; ++f) {
        m.norm_mean[f] = 0.f;
        m.norm_std[f] = 1.f;
    }
    m.max_ctas = 152;
    auto fail = [&]() {
        sme_mlp_destroy(M);
        return SME_ERR_OOM;
    };
    if (cudaMalloc(&m.master, P_COUNT * 4) != cudaSuccess || cudaMalloc(&m.wbf, P_COUNT * 2) != cudaSuccess ||
        cudaMalloc(&m.m1, P_COUNT * 4) != cudaSuccess || cudaMalloc(&m.m2, P_COUNT * 4) != cudaSuccess ||
        cudaMalloc(&m.grad, P_COUNT * 4) != cudaSuccess ||
        cudaMalloc(&m.partials, (size_t)m.max_ctas * P_COUNT * 4) != cudaSuccess ||
        cudaMalloc(&m.loss_part, m.max_ctas * 4) != cudaSuccess || cudaMalloc(&m.d_norm, 2 * MLP_IN * 4) != cudaSuccess ||
        cudaMalloc(&m.loss_dev, 4) != cudaSuccess) {
        cudaGetLastError();
        return fail();
    }
    cudaMemcpy(m.master, p.data(), P_COUNT * 4, cudaMemcpyHostToDevice);
    cudaMemset(m.m1, 0, P_COUNT * 4);
    cudaMemset(m.m2, 0, P_COUNT * 4);
    mlp_to_bf16<<<nblk(P_COUNT), 256>>>(m.master, m.wbf);
    float nh[2 * MLP_IN];
    for (int f = 0; f < MLP_IN; ++f) {
        nh[f] = 0.f;
        nh[MLP_IN + f] = 1.f;
    }
    cudaMemcpy(m.d_norm, nh, sizeof(nh), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail();
    cudaFuncSetAttribute(mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)infer_smem());
    cudaFuncSetAttribute(mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    *out = M;
    return SME_OK;
}

extern "C" sme_status sme_mlp_destroy(sme_mlp M)
{
    if (!M) return SME_OK;
    Mlp &m = M->m;
    for (void *p : {(void *)m.master, (void *)m.wbf, (void *)m.m1, (void *)m.m2, (void *)m.grad, (void *)m.partials,
                    (void *)m.loss_part, (void *)m.d_norm, (void *)m.loss_dev})
        if (p) cudaFree(p);
    delete M;
    return SME_OK;
}

extern "C" int64_t sme_mlp_param_count(void) { return P_COUNT; }

extern "C" sme_status sme_mlp_get_params(sme_mlp M, float *host, float *norm_host)
{
    if (!M) return SME_ERR_ARG;
    if (host) SME_CUDA(cudaMemcpy(host, M->m.master, P_COUNT * 4, cudaMemcpyDeviceToHost));
    if (norm_host)
        for (int f = 0; f < MLP_IN; ++f) {
            norm_host[f] = M->m.norm_mean[f];
            norm_host[MLP_IN + f] = M->m.norm_std[f];
        }
    return SME_OK;
}

extern "C" sme_status sme_mlp_set_params(sme_mlp M, const float *host, const float *norm_host)
{
    if (!M) return SME_ERR_ARG;
    Mlp &m = M->m;
    if (host) {
        SME_CUDA(cudaMemcpy(m.master, host, P_COUNT * 4, cudaMemcpyHostToDevice));
        mlp_to_bf16<<<nblk(P_COUNT), 256>>>(m.master, m.wbf);
        SME_CUDA(cudaGetLastError());
    }
    if (norm_host) {
        float nh[2 * MLP_IN];
        for (int f = 0; f < MLP_IN; ++f) {
            if (!(norm_host[MLP_IN + f] > 0.f)) {
                set_error("sme_mlp_set_params: feature scales must be positive");
                return SME_ERR_ARG;
            }
            m.norm_mean[f] = norm_host[f];
            m.norm_std[f] = norm_host[MLP_IN + f];
            nh[f] = norm_host[f];
            nh[MLP_IN + f] = 1.f / norm_host[MLP_IN + f];
        }
        SME_CUDA(cudaMemcpy(m.d_norm, nh, sizeof(nh), cudaMemcpyHostToDevice));
    }
    SME_CUDA(cudaDeviceSynchronize());
    return SME_OK;
}

extern "C" sme_status sme_mlp_forward(sme_mlp M, const float *X, int64_t N, float *y, void *stream)
{
    if (!M || !X || !y || N < 0) return SME_ERR_ARG;
    if (N == 0) return SME_OK;
    const unsigned grid = (unsigned)std::min<int64_t>((N + MLP_TS - 1) / MLP_TS, 152 * 4);
    mlp_infer<<<grid, MLP_H, infer_smem(), (cudaStream_t)stream>>>(M->m.wbf, M->m.d_norm, X, N, y);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_mlp_gradient(sme_mlp M, const float *X, const float *target, int64_t N, float *grad_out,
                                       float *loss_host, void *stream)
{
    if (!M || !X || !target || N < 1) return SME_ERR_ARG;
    Mlp &m = M->m;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (int)std::min<int64_t>((N + MLP_TS - 1) / MLP_TS, m.max_ctas);
    mlp_grad<<<grid, MLP_H, grad_smem(), s>>>(m.wbf, m.d_norm, X, target, N, m.partials, m.loss_part);
    mlp_reduce<<<nblk(P_COUNT), 256, 0, s>>>(m.partials, grid, m.grad, m.loss_part, m.loss_dev, N);
    SME_CUDA(cudaGetLastError());
    if (grad_out) SME_CUDA(cudaMemcpyAsync(grad_out, m.grad, P_COUNT * 4, cudaMemcpyDeviceToDevice, s));
    if (loss_host) {
        SME_CUDA(cudaMemcpyAsync(loss_host, m.loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaStreamSynchronize(s));
    }
    return SME_OK;
}

extern "C" sme_status sme_mlp_train_step(sme_mlp M, const float *X, const float *target, int64_t N, float lr,
                                         float *loss_host, void *stream)
{
    NvtxRange range("sme mlp train step");
    SME_TRY(sme_mlp_gradient(M, X, target, N, nullptr, loss_host, stream));
    Mlp &m = M->m;
    m.adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)m.adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)m.adam_t));
    mlp_adam<<<nblk(P_COUNT), 256, 0, (cudaStream_t)stream>>>(m.master, m.wbf, m.m1, m.m2, m.grad, lr, b1, b2, 1e-8f,
                                                              c1, c2);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_mlp_fit_normalisation(sme_mlp M, const float *X, int64_t N, void *stream)
{
    if (!M || !X || N < 2) {
        set_error("sme_mlp_fit_normalisation: a network and at least two feature rows are required");
        return SME_ERR_ARG;
    }
    if ((uintptr_t)X % 16) {
        set_error("sme_mlp_fit_normalisation: X must be 16-byte aligned");
        return SME_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc((size_t)(NORM_BLOCKS + 2) * MLP_IN * sizeof(double)));
    double *partials = scratch.as<double>(), *mean = partials + NORM_BLOCKS * MLP_IN, *var = mean + MLP_IN;
    feature_sums<<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(X, N, nullptr, 0, partials);
    feature_finish<<<1, 32, 0, s>>>(partials, NORM_BLOCKS, (double)N, mean);
    feature_sums<<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(X, N, mean, 1, partials);
    feature_finish<<<1, 32, 0, s>>>(partials, NORM_BLOCKS, (double)(N - 1), var);
    SME_CUDA(cudaGetLastError());
    double h[2 * MLP_IN];
    SME_CUDA(cudaMemcpyAsync(h, mean, sizeof(h), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    float norm[2 * MLP_IN];
    for (int f = 0; f < MLP_IN; ++f) {
        const double sd = std::sqrt(h[MLP_IN + f]);
        norm[f] = (float)h[f];
        norm[MLP_IN + f] = sd > 1e-6 ? (float)sd : 1.f;  // constant features are left unscaled
    }
    return sme_mlp_set_params(M, nullptr, norm);
}

extern "C" sme_status sme_mlp_draw_batch(const float *X, const float *target, int64_t N, int64_t batch, uint64_t seed,
                                         int64_t step, float *X_batch, float *target_batch, void *stream)
{
    if (!X || !target || !X_batch || !target_batch || N < 1 || N > 0xffffffffLL || batch < 0 || step < 0) {
        set_error("sme_mlp_draw_batch: bad arguments");
        return SME_ERR_ARG;
    }
    if ((uintptr_t)X % 16 || (uintptr_t)X_batch % 16) {
        set_error("sme_mlp_draw_batch: feature arrays must be 16-byte aligned");
        return SME_ERR_ARG;
    }
    if (batch == 0) return SME_OK;
    draw_batch_rows<<<nblk(batch), 256, 0, (cudaStream_t)stream>>>(X, target, N, batch, (uint32_t)seed,
                                                                   (uint32_t)(seed >> 32), (uint32_t)step, X_batch,
                                                                   target_batch);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_op_features(sme_op op, uint64_t seed, float *row_features, float *col_features,
                                      void *stream)
{
    SME_TRY(no_shard(op, "sme_op_features"));
    if (!op || op->dense) {
        set_error("sme_op_features: sparse operators only");
        return SME_ERR_ARG;
    }
    if (op->dbl) return features_t<double>(op, seed, row_features, col_features, (cudaStream_t)stream);
    return features_t<float>(op, seed, row_features, col_features, (cudaStream_t)stream);
}

extern "C" sme_status sme_warm_start(sme_op op, sme_mlp M, uint64_t seed, void *u0, void *v0, void *stream)
{
    NvtxRange range("sme warm start");
    SME_TRY(no_shard(op, "sme_warm_start"));
    if (!op || !M || !u0 || !v0 || op->dense) {
        set_error("sme_warm_start: bad arguments");
        return SME_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = op->m, n = op->n;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc((size_t)(m + n) * (MLP_IN + 1) * sizeof(float)));
    float *buf = scratch.as<float>();
    float *F = buf, *y = buf + (m + n) * MLP_IN;
    SME_TRY(sme_op_features(op, seed, F, F + m * MLP_IN, stream));
    SME_TRY(sme_mlp_forward(M, F, m + n, y, stream));
    if (op->dbl) {
        cast_out<double><<<nblk(m), 256, 0, s>>>(m, y, (double *)u0);
        cast_out<double><<<nblk(n), 256, 0, s>>>(n, y + m, (double *)v0);
    } else {
        cast_out<float><<<nblk(m), 256, 0, s>>>(m, y, (float *)u0);
        cast_out<float><<<nblk(n), 256, 0, s>>>(n, y + m, (float *)v0);
    }
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_batch_features(sme_batch b, uint64_t seed, float *row_features, float *col_features,
                                         void *stream)
{
    if (!b) return SME_ERR_ARG;
    return sme_op_features(b->op, seed, row_features, col_features, stream);
}

extern "C" sme_status sme_batch_warm_start(sme_batch b, sme_mlp M, uint64_t seed, void *u0, void *v0, void *stream)
{
    if (!b) return SME_ERR_ARG;
    return sme_warm_start(b->op, M, seed, u0, v0, stream);
}
