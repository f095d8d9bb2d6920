// Learned warm start for Algorithm 1: a small MLP that maps per-row / per-column features of A to
// initial log-scalings u^0, v^0.  (Algorithm 1 itself is unchanged; a warm start needs a step offset
// t0 > 0, since the first step of the paper's schedule, eta_1 = 1/gamma, discards u^0.)
//
// Network: 8 inputs (normalised) -> 128 (ReLU) -> 128 (ReLU) -> 1.  Weights are stored in BF16 for the
// forward pass with FP32 master copies for training; all accumulation is FP32.
//
// Kernels work on tiles of 128 samples, one sample per thread, with the 128 x 128 contractions of layer 2
// and of its gradients on the tensor cores (tcgen05.mma, accumulators in TMEM; details with the kernels).
// Training fuses forward and backward per tile; each CTA accumulates its gradient in TMEM across its tiles,
// writes it once as a partial, and a second kernel sums the partials in CTA order (deterministic) before an
// Adam step updates the masters and BF16 copies.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "sme_internal.cuh"
#include "tc_common.cuh"

namespace sme {

constexpr int MLP_IN = 8, MLP_H = 128;
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
    int *d_status = nullptr;  // device status word of the tensor-core kernels (ST_TIMEOUT)
    long long adam_t = 0;
};

}  // namespace sme

struct sme_mlp_s {
    sme::Mlp m;
};

namespace sme {

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// ------------------------------------------------------------------ tensor-core tiles
//
// A CTA of 128 threads works on tiles of 128 samples; thread s owns sample s of the tile, which is also row s
// of every product whose M runs over samples (TMEM lane s).  The 128 x 128 contractions run on tcgen05.mma
// (kind::f16, BF16 operands in shared memory with the 128-byte swizzle, FP32 accumulators in TMEM), issued
// by one thread:
//   forward   Z   = H1 W2^T             M = samples, N = units j, K = units i
//   backward  dH1 = D2 W2               M = samples, N = units i, K = units j  (W2^T kept as a second copy)
//             dW2 (+)= D2^T H1, db2     M = units j, N = units i + a ones row, K = samples (64 per step)
//             dW1 (+)= dZ1^T X, db1     M = units i, N = 8 features + a ones row (16), K = samples
// The weights are BF16 already.  The forward operand H1 is split into three BF16 terms (hi = bf16(x),
// mid = bf16(x - hi), lo = bf16(x - hi - mid), |x - hi - mid - lo| <= 2^-27 |x|), so the forward product is
// FP32-accurate.  The gradient operands are pairs hi + lo (|x - hi - lo| <= 2^-18 |x|); a product of two
// pairs keeps hi*hi + hi*lo + lo*hi.  All accumulation is FP32.
// Layer 1 (K = 8) and layer 3 (N = 1) stay on the FP32 pipe in the thread that owns the sample.

constexpr int TT = 128;              // samples per tile: the M of every product
constexpr int HT_ROWS = MLP_H + 16;  // H1^T rows, the ones row (db2) and zero rows: N of dW2 (a multiple of 16)
constexpr int XT_ROWS = 16;          // 8 feature rows, the ones row (db1) and zero rows: N of dW1
constexpr int CH = 64;               // samples per step of the gradient products (one 128-byte K-atom)

// Shared-memory offsets (bytes) of the operands; every base is 1024-aligned.
struct TcPlan {
    int w2, w2t, ha_h, ha_l, ha_m, ht_h, ht_l, dt_h, dt_l, xt_h, xt_l, total;
};
constexpr int OPB = TT * MLP_H * 2;  // one 128 x 128 BF16 operand: 32 KB
// The middle term of the forward operand (H1 as three BF16 terms) lives where H1^T and D2^T go later: the
// forward product completes before those are written.
constexpr TcPlan TRAIN_PLAN = {0,
                               OPB,
                               2 * OPB,
                               3 * OPB,
                               4 * OPB,
                               4 * OPB,
                               4 * OPB + HT_ROWS * CH * 2,
                               4 * OPB + 2 * HT_ROWS * CH * 2,
                               4 * OPB + 2 * HT_ROWS * CH * 2 + MLP_H * CH * 2,
                               4 * OPB + 2 * HT_ROWS * CH * 2 + 2 * MLP_H * CH * 2,
                               4 * OPB + 2 * HT_ROWS * CH * 2 + 2 * MLP_H * CH * 2 + XT_ROWS * CH * 2,
                               4 * OPB + 2 * HT_ROWS * CH * 2 + 2 * MLP_H * CH * 2 + 2 * XT_ROWS * CH * 2};
constexpr TcPlan INFER_PLAN = {0, 0, OPB, 2 * OPB, 3 * OPB, 0, 0, 0, 0, 0, 0, 4 * OPB};  // forward operands only
static_assert(TRAIN_PLAN.ht_l % 1024 == 0 && TRAIN_PLAN.dt_h % 1024 == 0 && TRAIN_PLAN.dt_l % 1024 == 0 &&
                  TRAIN_PLAN.xt_h % 1024 == 0 && TRAIN_PLAN.xt_l % 1024 == 0,
              "operand bases must be 1024-aligned");
static_assert(TRAIN_PLAN.total + 1024 + 8 * 1024 <= 227 * 1024, "shared memory of the training kernel");

// Byte offset of element (r, k) of a K-major BF16 operand of `rows` rows: K-atoms of 64 elements, each a block
// of rows x 128 bytes; the 16-byte chunk c of row r sits at chunk c ^ (r mod 8) (128-byte swizzle).
__device__ __forceinline__ uint32_t sw_off(int rows, int r, int k)
{
    const int atom = k >> 6, kin = k & 63;
    return (uint32_t)(atom * rows * 128 + r * 128 + ((((kin >> 3) ^ (r & 7))) << 4) + (kin & 7) * 2);
}

__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ void sts16(uint32_t a, uint16_t v)
{
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t a)
{
    uint4 r;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(a) : "memory");
    return r;
}

// x = hi + lo + r, hi and lo BF16 (bit patterns); x - hi and (x - hi) - lo are exact in FP32.
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
}

// Eight values k0 .. k0 + 7 of row r into the hi and lo operands (one 16-byte chunk each).
__device__ __forceinline__ void put_row8(uint32_t hbase, uint32_t lbase, int rows, int r, int k0, const float (&v)[8])
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint16_t h0, l0, h1, l1;
        split_bf16(v[2 * q], h0, l0);
        split_bf16(v[2 * q + 1], h1, l1);
        h[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        l[q] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
    const uint32_t o = sw_off(rows, r, k0);
    sts128(hbase + o, h[0], h[1], h[2], h[3]);
    sts128(lbase + o, l[0], l[1], l[2], l[3]);
}

// Eight values k0 .. k0 + 7 of row r as three BF16 terms (hi + mid + lo, |x - hi - mid - lo| <= 2^-27 |x|).
__device__ __forceinline__ void put_row8_3(uint32_t hbase, uint32_t mbase, uint32_t lbase, int rows, int r, int k0,
                                           const float (&v)[8])
{
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint16_t t[2][3];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float x = v[2 * q + e];
            const __nv_bfloat16 bh = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(bh);
            const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
            t[e][0] = __bfloat16_as_ushort(bh);
            t[e][1] = __bfloat16_as_ushort(bm);
            t[e][2] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(bm)));
        }
        h[q] = (uint32_t)t[0][0] | ((uint32_t)t[1][0] << 16);
        m[q] = (uint32_t)t[0][1] | ((uint32_t)t[1][1] << 16);
        l[q] = (uint32_t)t[0][2] | ((uint32_t)t[1][2] << 16);
    }
    const uint32_t o = sw_off(rows, r, k0);
    sts128(hbase + o, h[0], h[1], h[2], h[3]);
    sts128(mbase + o, m[0], m[1], m[2], m[3]);
    sts128(lbase + o, l[0], l[1], l[2], l[3]);
}

// One value at (r, k) into the hi and lo operands.
__device__ __forceinline__ void put_one(uint32_t hbase, uint32_t lbase, int rows, int r, int k, float v)
{
    uint16_t h, l;
    split_bf16(v, h, l);
    const uint32_t o = sw_off(rows, r, k);
    sts16(hbase + o, h);
    sts16(lbase + o, l);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Instruction descriptor: kind::f16, BF16 A and B (both K-major), FP32 D, shape M x N.
__host__ __device__ constexpr uint32_t mlp_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_cta1(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit_cta1(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// D (+)= A B^T over K elements (K a multiple of 16): A = [128][K], B = [n_rows][K], K-major, 128-byte swizzle.
__device__ __forceinline__ void mma_kmajor(uint32_t d, uint32_t a, uint32_t b, int n_rows, int K, uint32_t idesc,
                                           bool accumulate)
{
    for (int k = 0; k < K; k += 16) {
        const int atom = k >> 6, kin = k & 63;
        const uint64_t ad = smem_desc_sw128_u32(a + (uint32_t)(atom * TT * 128 + kin * 2));
        const uint64_t bd = smem_desc_sw128_u32(b + (uint32_t)(atom * n_rows * 128 + kin * 2));
        mma_cta1(d, ad, bd, idesc, (accumulate || k > 0) ? 1u : 0u);
    }
}

// Every thread waits for the next phase of `bar`; true in every thread if any thread's bounded wait ran out.
__device__ __forceinline__ bool wait_all(uint64_t *bar, uint32_t &phase)
{
    const bool ok = mbar_wait(bar, phase & 1u);
    ++phase;
    return __syncthreads_or(ok ? 0 : 1) != 0;
}

// v[q] given in every lane; returns in lane l the sum over the warp's lanes of v[l] (a fixed tree per index).
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// Layer 1 of one unit in FP32 (zero for samples past the end of the data).
__device__ __forceinline__ float layer1(const float *W1s, const float *b1s, const float (&x)[MLP_IN], int i, bool valid)
{
    float z = b1s[i];
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) z += W1s[i * MLP_IN + f] * x[f];
    return valid ? fmaxf(z, 0.f) : 0.f;
}

// Forward (TRAIN = false: y for every sample) or fused forward and backward of the mean squared error
// (1/N) sum (y - target)^2 (TRAIN = true: this CTA's gradient partial, P_COUNT floats, and loss partial) over
// tiles blockIdx.x, blockIdx.x + gridDim.x, ...  A bounded wait that runs out sets ST_TIMEOUT in *status and
// leaves NaN in this CTA's outputs.
template <bool TRAIN>
__global__ void __launch_bounds__(TT, 1)
    mlp_tc(const __nv_bfloat16 *w, const float *norm, const float *X, const float *target, int64_t N, float *y_out,
           float *partials, float *loss_part, int *status)
{
    constexpr TcPlan P = TRAIN ? TRAIN_PLAN : INFER_PLAN;
    constexpr uint32_t NCOL = TRAIN ? 512u : 128u;  // Z / dH1 (128 columns), dW2 (144), dW1 (16)
    constexpr uint32_t ID_Z = mlp_idesc(TT, MLP_H), ID_W2 = mlp_idesc(TT, HT_ROWS), ID_W1 = mlp_idesc(TT, XT_ROWS);
    extern __shared__ __align__(1024) uint8_t raw[];
    __shared__ float W1s[MLP_H * MLP_IN], b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    __shared__ float red[TT / 32][MLP_H];
    __shared__ float lred[2][TT / 32];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_sh;
    const uint32_t sb = (smem_u32(raw) + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < MLP_H * MLP_IN; e += TT) W1s[e] = bf(w, P_W1 + e);
    b1s[tid] = bf(w, P_B1 + tid);
    b2s[tid] = bf(w, P_B2 + tid);
    w3s[tid] = bf(w, P_W3 + tid);
    const float b3 = bf(w, P_B3);
    {  // W2 as the B operand of the forward product: row j = tid as stored, 16-byte chunks
        const uint4 *src = reinterpret_cast<const uint4 *>(w + P_W2 + tid * MLP_H);
#pragma unroll 4
        for (int c = 0; c < MLP_H / 8; ++c) {
            const uint4 q = src[c];
            sts128(sb + P.w2 + sw_off(MLP_H, tid, c * 8), q.x, q.y, q.z, q.w);
        }
    }
    if (TRAIN) {
        // W2^T (row i = tid) as the B operand of dH1, and the zero rows of X^T.
        const uint16_t *w16 = reinterpret_cast<const uint16_t *>(w + P_W2);
        for (int c = 0; c < MLP_H / 8; ++c) {
            uint32_t q[4];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                q[h] = (uint32_t)w16[(c * 8 + 2 * h) * MLP_H + tid] |
                       ((uint32_t)w16[(c * 8 + 2 * h + 1) * MLP_H + tid] << 16);
            sts128(sb + P.w2t + sw_off(MLP_H, tid, c * 8), q[0], q[1], q[2], q[3]);
        }
        for (int e = tid; e < (XT_ROWS - MLP_IN - 1) * CH; e += TT) {
            const int r = MLP_IN + 1 + e / CH, k = e % CH;
            sts16(sb + P.xt_h + sw_off(XT_ROWS, r, k), 0);
            sts16(sb + P.xt_l + sw_off(XT_ROWS, r, k), 0);
        }
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_sh;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes

    uint32_t phase = 0;
    bool bad = false, first2 = true, first1 = true;
    float loss = 0.f, gw3 = 0.f, gb3 = 0.f;
    const float invN = 1.f / (float)N;
    int64_t base = (int64_t)blockIdx.x * TT;
    for (; base < N; base += (int64_t)gridDim.x * TT) {
        const bool valid = tid < N - base;
        float x[MLP_IN];
#pragma unroll
        for (int f = 0; f < MLP_IN; ++f)
            x[f] = valid ? (X[(base + tid) * MLP_IN + f] - norm[f]) * norm[MLP_IN + f] : 0.f;
        // Layer 1 into the A operand of the forward product; its ReLU mask kept for dZ1.
        uint32_t mask1[MLP_H / 32];
#pragma unroll 1
        for (int c = 0; c < MLP_H / 32; ++c) {
            uint32_t m = 0;
#pragma unroll
            for (int k0 = 0; k0 < 32; k0 += 8) {
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    v[q] = layer1(W1s, b1s, x, c * 32 + k0 + q, valid);
                    if (v[q] > 0.f) m |= 1u << (k0 + q);
                }
                put_row8_3(sb + P.ha_h, sb + P.ha_m, sb + P.ha_l, TT, tid, c * 32 + k0, v);
            }
            mask1[c] = m;
        }
        fence_async_smem();
        tc_before();
        __syncthreads();
        if (tid == 0) {
            tc_after();
            mma_kmajor(tmem, sb + P.ha_h, sb + P.w2, MLP_H, MLP_H, ID_Z, false);
            mma_kmajor(tmem, sb + P.ha_m, sb + P.w2, MLP_H, MLP_H, ID_Z, true);
            mma_kmajor(tmem, sb + P.ha_l, sb + P.w2, MLP_H, MLP_H, ID_Z, true);
            commit_cta1(&bar);
        }
        if ((bad = wait_all(&bar, phase))) break;
        tc_after();
        // Layer 2's ReLU and layer 3 (FP32) from row tid of Z.
        float yv = 0.f;
        uint32_t mask2[MLP_H / 32];
#pragma unroll 1
        for (int c = 0; c < MLP_H / 32; ++c) {
            float z[32];
            tmem_ld32(t_lane + c * 32, z);
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float h2 = fmaxf(z[q] + b2s[c * 32 + q], 0.f);
                yv += w3s[c * 32 + q] * h2;
                if (h2 > 0.f) m |= 1u << q;
            }
            mask2[c] = m;
        }
        yv += b3;
        if (!TRAIN) {
            if (valid) y_out[base + tid] = yv;
            tc_before();  // these TMEM loads precede the next tile's product
            continue;
        }
        const float r = valid ? yv - target[base + tid] : 0.f;
        loss += r * r;
        const float dy = 2.f * r * invN;
        gb3 += dy;
        // dW3 partials and D2 = dy w3 (h2 > 0), written over the forward operand (its product is complete) as
        // the A operand of dH1.
#pragma unroll 1
        for (int c = 0; c < MLP_H / 32; ++c) {
            float z[32];
            tmem_ld32(t_lane + c * 32, z);
            float v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = dy * fmaxf(z[q] + b2s[c * 32 + q], 0.f);
#pragma unroll
            for (int k0 = 0; k0 < 32; k0 += 8) {
                float d[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) d[q] = ((mask2[c] >> (k0 + q)) & 1u) ? dy * w3s[c * 32 + k0 + q] : 0.f;
                put_row8(sb + P.ha_h, sb + P.ha_l, TT, tid, c * 32 + k0, d);
            }
            red[warp][c * 32 + lane] = warp_transpose_sum(v, lane);
        }
        fence_async_smem();
        tc_before();
        __syncthreads();
        gw3 += red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
        if (tid == 0) {
            tc_after();
            mma_kmajor(tmem, sb + P.ha_h, sb + P.w2t, MLP_H, MLP_H, ID_Z, false);
            mma_kmajor(tmem, sb + P.ha_l, sb + P.w2t, MLP_H, MLP_H, ID_Z, true);
            commit_cta1(&bar);
        }
        if ((bad = wait_all(&bar, phase))) break;
        tc_after();
        // dW2 and db2, 64 samples per step: D2^T (this thread's own D2 words, scattered into column sl) and
        // H1^T (layer 1 recomputed with the same arithmetic) with its ones row and zero rows.
#pragma unroll 1
        for (int c = 0; c < TT / CH; ++c) {
            if (tid / CH == c) {
                const int sl = tid - c * CH;
#pragma unroll 1
                for (int k0 = 0; k0 < MLP_H; k0 += 8) {
                    const uint32_t o = sw_off(TT, tid, k0);
                    const uint4 hv = lds128(sb + P.ha_h + o), lv = lds128(sb + P.ha_l + o);
                    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t od = sw_off(MLP_H, k0 + q, sl);
                        sts16(sb + P.dt_h + od, (uint16_t)(hw[q >> 1] >> (16 * (q & 1))));
                        sts16(sb + P.dt_l + od, (uint16_t)(lw[q >> 1] >> (16 * (q & 1))));
                    }
                }
#pragma unroll 4
                for (int i = 0; i < MLP_H; ++i)
                    put_one(sb + P.ht_h, sb + P.ht_l, HT_ROWS, i, sl, layer1(W1s, b1s, x, i, valid));
                put_one(sb + P.ht_h, sb + P.ht_l, HT_ROWS, MLP_H, sl, valid ? 1.f : 0.f);
                for (int i = MLP_H + 1; i < HT_ROWS; ++i)  // zero rows (the forward's middle term overlaps them)
                    put_one(sb + P.ht_h, sb + P.ht_l, HT_ROWS, i, sl, 0.f);
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_after();
                const uint32_t d = tmem + MLP_H;
                mma_kmajor(d, sb + P.dt_h, sb + P.ht_h, HT_ROWS, CH, ID_W2, !first2);
                mma_kmajor(d, sb + P.dt_h, sb + P.ht_l, HT_ROWS, CH, ID_W2, true);
                mma_kmajor(d, sb + P.dt_l, sb + P.ht_h, HT_ROWS, CH, ID_W2, true);
                commit_cta1(&bar);
            }
            first2 = false;
            if ((bad = wait_all(&bar, phase))) break;
        }
        if (bad) break;
        // dW1 and db1, 64 samples per step: dZ1^T = (dH1 masked by layer 1's ReLU)^T and X^T with its ones row.
#pragma unroll 1
        for (int c = 0; c < TT / CH; ++c) {
            if (tid / CH == c) {  // whole warps
                const int sl = tid - c * CH;
#pragma unroll 1
                for (int cc = 0; cc < MLP_H / 32; ++cc) {
                    float g[32];
                    tmem_ld32(t_lane + cc * 32, g);
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        put_one(sb + P.dt_h, sb + P.dt_l, MLP_H, cc * 32 + q, sl, ((mask1[cc] >> q) & 1u) ? g[q] : 0.f);
                }
#pragma unroll
                for (int f = 0; f < MLP_IN; ++f) put_one(sb + P.xt_h, sb + P.xt_l, XT_ROWS, f, sl, x[f]);
                put_one(sb + P.xt_h, sb + P.xt_l, XT_ROWS, MLP_IN, sl, valid ? 1.f : 0.f);
            }
            fence_async_smem();
            tc_before();
            __syncthreads();
            if (tid == 0) {
                tc_after();
                const uint32_t d = tmem + MLP_H + HT_ROWS;
                mma_kmajor(d, sb + P.dt_h, sb + P.xt_h, XT_ROWS, CH, ID_W1, !first1);
                mma_kmajor(d, sb + P.dt_h, sb + P.xt_l, XT_ROWS, CH, ID_W1, true);
                mma_kmajor(d, sb + P.dt_l, sb + P.xt_h, XT_ROWS, CH, ID_W1, true);
                commit_cta1(&bar);
            }
            first1 = false;
            if ((bad = wait_all(&bar, phase))) break;
        }
        if (bad) break;
        tc_before();  // this tile's TMEM loads precede the next tile's forward product
    }
    const float qnan = __int_as_float(0x7fc00000);
    if (bad) {
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            mbar_wait(&bar, (phase - 1u) & 1u);  // once more, bounded: the product still in flight
        }
        if (!TRAIN)
            for (; base < N; base += (int64_t)gridDim.x * TT)
                if (tid < N - base) y_out[base + tid] = qnan;
    }
    if (TRAIN) {
        tc_before();
        __syncthreads();
        tc_after();
        // Thread tid = TMEM lane tid = unit j of dW2 and unit i of dW1.
        float *Pp = partials + (int64_t)blockIdx.x * P_COUNT;
        if (!bad && !first2) {
#pragma unroll 1
            for (int c = 0; c < MLP_H / 32; ++c) {
                float g[32];
                tmem_ld32(t_lane + MLP_H + c * 32, g);
#pragma unroll
                for (int q = 0; q < 32; ++q) Pp[P_W2 + tid * MLP_H + c * 32 + q] = g[q];
            }
            float g[32];
            tmem_ld32(t_lane + 2 * MLP_H, g);  // columns 256..287: db2, dW2's zero rows, then dW1 and db1
            Pp[P_B2 + tid] = g[0];
#pragma unroll
            for (int f = 0; f < MLP_IN; ++f) Pp[P_W1 + tid * MLP_IN + f] = g[HT_ROWS - MLP_H + f];
            Pp[P_B1 + tid] = g[HT_ROWS - MLP_H + MLP_IN];
        } else {
            const float fill = bad ? qnan : 0.f;
            for (int i = 0; i < MLP_H; ++i) Pp[P_W2 + tid * MLP_H + i] = fill;
            Pp[P_B2 + tid] = fill;
            for (int f = 0; f < MLP_IN; ++f) Pp[P_W1 + tid * MLP_IN + f] = fill;
            Pp[P_B1 + tid] = fill;
        }
        Pp[P_W3 + tid] = bad ? qnan : gw3;
        float l = loss, b = gb3;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            lred[0][warp] = l;
            lred[1][warp] = b;
        }
        __syncthreads();
        if (tid == 0) {
            float lt = 0.f, bt = 0.f;
            for (int q = 0; q < TT / 32; ++q) {
                lt += lred[0][q];
                bt += lred[1][q];
            }
            Pp[P_B3] = bad ? qnan : bt;
            loss_part[blockIdx.x] = bad ? qnan : lt;
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
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

static size_t infer_smem() { return (size_t)INFER_PLAN.total + 1024; }
static size_t grad_smem() { return (size_t)TRAIN_PLAN.total + 1024; }

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
        cudaMalloc(&m.loss_dev, 4) != cudaSuccess || cudaMalloc(&m.d_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail();
    }
    cudaMemcpy(m.master, p.data(), P_COUNT * 4, cudaMemcpyHostToDevice);
    cudaMemset(m.m1, 0, P_COUNT * 4);
    cudaMemset(m.m2, 0, P_COUNT * 4);
    cudaMemset(m.d_status, 0, sizeof(int));
    mlp_to_bf16<<<nblk(P_COUNT), 256>>>(m.master, m.wbf);
    float nh[2 * MLP_IN];
    for (int f = 0; f < MLP_IN; ++f) {
        nh[f] = 0.f;
        nh[MLP_IN + f] = 1.f;
    }
    cudaMemcpy(m.d_norm, nh, sizeof(nh), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail();
    if (cudaFuncSetAttribute(mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)infer_smem()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()) !=
            cudaSuccess) {
        cudaGetLastError();
        set_error("sme_mlp_create: the tensor-core kernels cannot get their shared memory");
        sme_mlp_destroy(M);
        return SME_ERR_CUDA;
    }
    *out = M;
    return SME_OK;
}

extern "C" sme_status sme_mlp_destroy(sme_mlp M)
{
    if (!M) return SME_OK;
    Mlp &m = M->m;
    for (void *p : {(void *)m.master, (void *)m.wbf, (void *)m.m1, (void *)m.m2, (void *)m.grad, (void *)m.partials,
                    (void *)m.loss_part, (void *)m.d_norm, (void *)m.loss_dev, (void *)m.d_status})
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
    const unsigned grid = (unsigned)std::min<int64_t>((N + TT - 1) / TT, 152);
    mlp_tc<false><<<grid, TT, infer_smem(), (cudaStream_t)stream>>>(M->m.wbf, M->m.d_norm, X, nullptr, N, y, nullptr,
                                                                   nullptr, M->m.d_status);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_mlp_gradient(sme_mlp M, const float *X, const float *target, int64_t N, float *grad_out,
                                       float *loss_host, void *stream)
{
    if (!M || !X || !target || N < 1) return SME_ERR_ARG;
    Mlp &m = M->m;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (int)std::min<int64_t>((N + TT - 1) / TT, m.max_ctas);
    mlp_tc<true><<<grid, TT, grad_smem(), s>>>(m.wbf, m.d_norm, X, target, N, nullptr, m.partials, m.loss_part,
                                               m.d_status);
    mlp_reduce<<<nblk(P_COUNT), 256, 0, s>>>(m.partials, grid, m.grad, m.loss_part, m.loss_dev, N);
    SME_CUDA(cudaGetLastError());
    if (grad_out) SME_CUDA(cudaMemcpyAsync(grad_out, m.grad, P_COUNT * 4, cudaMemcpyDeviceToDevice, s));
    if (loss_host) {
        // The loss is read back anyway; the status word with it (a bounded wait that ran out in a kernel).
        int st = 0;
        SME_CUDA(cudaMemcpyAsync(loss_host, m.loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaMemcpyAsync(&st, m.d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        SME_CUDA(cudaStreamSynchronize(s));
        if (st) {
            SME_CUDA(cudaMemsetAsync(m.d_status, 0, sizeof(int), s));
            set_error("sme_mlp_gradient: a tensor-core wait ran out (results are NaN)");
            return SME_ERR_TIMEOUT;
        }
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
