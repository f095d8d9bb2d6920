// Dense operator on E4M3 (FP8) data: the probe products of Algorithm 1 with tcgen05.mma kind::f8f6f4.
//
// The matrix stays E4M3 in HBM (one byte per entry, with one FP32 scale c_i per row: A_ij = c_i q_ij),
// as A and a transposed copy A^T, both K-blocked in 128 x 128-byte blocks so that every TMA tile load is
// one contiguous 16 KB run.  The B operand of each product is a single E4M3 term (the single-term reading of the
// Section 3.1 estimator on dense A: the +-1 probes are exact, the scaling e^{x_j} is rounded to the 4
// significant bits of E4M3, a relative error of at most 2^-4 per scaling):
//     B[p][j] = e4m3( 2^S e^{x_j} c_j ) * s_jp          (c_j = 1 on the forward side)
// S is a power-of-two exponent per operand and iteration, chosen so that the largest magnitude lands
// at <= 256 (the largest E4M3 value is 448), which leaves 2^-17 of dynamic range below it.  The
// accumulators are divided by 2^S exactly in the epilogue.
//
// Choosing S needs the largest e^{x_j} c_j of the NEXT iterate while the epilogue is still producing it,
// so it is bounded instead of measured.  One step of Algorithm 1 cannot raise a coordinate by more than
// its target term: z >= 0 gives x^t <= (1 - eta gamma) x^{t-1} + eta target, and eta gamma <= 1, so with
// Q = max_j (x_j^{t-1} + log|c_j|) of the previous iterate,
//     max_j (x_j^t + log|c_j|) <= (1 - eta gamma) Q + eta gamma max log|c| + eta target   (and <= M + max log|c|).
// Every iteration records its own Q with one atomic max per warp into a ring of three slots (read the
// previous one, fill the current one, clear the next one), and the scale exponents of the operands are
// kept by iteration parity.  The first operand of a call is scaled from the exact maximum.
//
// Launch structure, rings, bounded waits and the drain on a timeout are those of the BF16 kernel in
// dense.cu: clusters of two CTAs on one 256-row tile (M = 256, cta_group::2), the leader issuing the MMAs
// (here K = 32 per instruction, four per 128-byte K-block), TMEM holding one FP32 column per probe.

#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sme_internal.cuh"
#include "tc_common.cuh"

namespace sme {

constexpr int F8_BM = 128;                   // rows per CTA
constexpr int F8_BK = 128;                   // K per block: 128 E4M3 = one 128-byte swizzle row
constexpr int F8_A_SLOT = F8_BM * F8_BK;     // 16 KB: one K-block of this CTA's 128 rows of A (or A^T)
constexpr int F8_THREADS = 192;              // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2..5 epilogue

template <int KP>
struct F8Cfg {
    static constexpr int B_SLOT = (KP / 2) * F8_BK;      // this CTA's half of the N = KP operand rows
    static constexpr int SLOT = F8_A_SLOT + B_SLOT;      // A part then B part, one barrier pair per slot
    static constexpr int STAGES = KP == 256 ? 6 : 8;
    static constexpr int BYTES = STAGES * SLOT;
};
static_assert(F8Cfg<256>::BYTES + 1024 <= 227 * 1024 && F8Cfg<128>::BYTES + 1024 <= 227 * 1024,
              "FP8 ring exceeds the shared memory of one CTA");

// Layout of DenseOp::f8_small (32-bit words).
constexpr int F8_Q = 0;      // q[slot 0..2][side 0..1]: ordered keys of max (x + log|c|)
constexpr int F8_BMAX = 6;   // bmax[side]: float bits of max |e^{x} c| (exact, for a call's first operand)
constexpr int F8_EXP = 8;    // S[parity 0..1][side 0..1]
constexpr int F8_WORDS = 12;

// Float -> unsigned key whose unsigned order is the float order (for atomicMax over signed values).
__host__ __device__ __forceinline__ uint32_t f8_key(float f)
{
    uint32_t b;
#if defined(__CUDA_ARCH__)
    b = __float_as_uint(f);
#else
    memcpy(&b, &f, 4);
#endif
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float f8_unkey(uint32_t k)
{
    if (k == 0u) return -INFINITY;  // nothing recorded
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Exponent S with B 2^S <= 256 for the largest operand magnitude B: S = 8 - ceil(log2 B), exact (from the
// binary exponent of B).
__device__ __forceinline__ int f8_scale_exp(float B)
{
    if (!(B > 0.f) || !isfinite(B)) return 0;
    int e;
    const float f = frexpf(B, &e);  // B = f 2^e, f in [0.5, 1)
    const int c = (f == 0.5f) ? e - 1 : e;
    return min(max(8 - c, -120), 120);
}

// S for a bound U on the log of the largest magnitude; the small margin covers the rounding of the step
// and of expf.
__device__ __forceinline__ int f8_scale_exp_log(float U)
{
    return f8_scale_exp(expf(fminf(U, 80.f)) * 1.0078125f);
}

__device__ __forceinline__ uint8_t f8_code(float v)
{
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// E4M3 code -> value (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; 0x7f / 0xff are NaN).
__device__ __forceinline__ double f8_decode(uint32_t b)
{
    const int e = (b >> 3) & 15, f = b & 7;
    double v = e == 0 ? ldexp((double)f, -9) : ldexp((double)(8 + f), e - 10);
    if ((b & 0x7f) == 0x7f) v = NAN;
    return (b & 0x80) ? -v : v;
}

// Instruction descriptor, kind::f8f6f4: D FP32, A and B E4M3 (format 0), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N)
{
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

struct DenseMaps8 {
    CUtensorMap X[2];  // [0] A, [1] A^T (E4M3, K-blocked)
    CUtensorMap B[2];  // [0] forward operand (current), [1] backward operand (current)
};

struct DenseArgs8 {
    int64_t m, n;
    int kp;                    // probes (128 or 256): the MMA's N
    int row_tiles, col_tiles;  // m / 128, n / 128
    int row_ctas;              // CTAs of the forward product: row_tiles rounded up to whole clusters
    float *x[2], *xb[2];       // [0] u, ubar (rows)   [1] v, vbar (columns)
    float *z[2];               // estimate-only outputs
    uint8_t *bnext[2];         // [0] next backward operand (written by rows), [1] next forward operand
    float target2[2];
    float gamma, M, eta, avg_new, avg_old;
    uint32_t t_next, key0, key1, sid_out[2];
    int mode;                  // 0 step, 1 estimate only
    const float *row_scale;    // c_i, or null
    float logc[2];             // max log|c| per side (0 on the column side)
    const int *s_cur;          // [side] exponents of the current operands (side 0 backward, 1 forward)
    int *s_next;               // [side] exponents of the operands this launch writes
    const uint32_t *q_prev;    // [side] keys of max (x^{t-1} + log|c|)
    uint32_t *q_cur;           // [side] keys of max (x^t + log|c|), filled here
    uint32_t *q_clear;         // [side] the ring slot the next launch fills, cleared here
    uint32_t pipe_limit;       // TC_WAIT_LIMIT, or 0 to launch the EXPIRE instantiation (see dense.cu)
    int *status;
};

// Bound on max (x^t + log|c|) of one side from the previous iterate's maximum (see the file comment).
__device__ __forceinline__ float f8_next_bound(const DenseArgs8 &a, int side)
{
    const float q = f8_unkey(a.q_prev[side]);
    const float eg = a.eta * a.gamma;  // <= 1
    float U = (1.f - eg) * q + eg * a.logc[side] + a.eta * a.target2[side];
    return fminf(U, a.M + a.logc[side]);
}

// EXPIRE: the instantiation for the test of the timeout path (see dense.cu).
// Remote arrive (release, cluster scope) on an mbarrier given by its cluster-window address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// Work item w of a launch: the products' 256-row pair tiles, the forward product's first.  This CTA's tile
// is tile 2p + rank of its side; with an odd tile count the second CTA of the last pair repeats its
// partner's tile and writes nothing.
struct F8Item {
    bool cols, active;
    int tile, nk;
};

__device__ __forceinline__ F8Item f8_item(const DenseArgs8 &a, int w, uint32_t crank)
{
    F8Item it;
    const int row_pairs = (a.row_tiles + 1) / 2;
    it.cols = w >= row_pairs;
    const int p = it.cols ? w - row_pairs : w;
    const int ntiles = it.cols ? a.col_tiles : a.row_tiles;
    const int t = 2 * p + (int)crank;
    it.active = t < ntiles;
    it.tile = it.active ? t : ntiles - 1;
    it.nk = (int)((it.cols ? a.m : a.n) / F8_BK);
    return it;
}

// Persistent: cluster c of the grid takes work items c, c + clusters, ...  TMEM holds two accumulators of KP
// columns, so the epilogue of one item overlaps the copies and MMAs of the next; the ring of K-blocks runs on
// across items.  Barriers: full / empty per ring slot (copies -> MMAs -> slot free), acc_full[2] (the
// leader's commit after an item's MMAs, in both CTAs), acc_empty[2] (in the leader: one arrival per epilogue
// warp of the pair once it has read the accumulator), mma_done (after the issuer's last MMA: TMEM may be
// freed).  Every wait is bounded; a role that gives up sets ST_TIMEOUT, and the issuer then still walks the
// accumulator protocol (without MMAs) so that every epilogue wait ends and no barrier skips a phase.
// EXPIRE: the instantiation for the test of the timeout path (see dense.cu).
template <int KP, bool EXPIRE = false>
__global__ void __launch_bounds__(F8_THREADS, 1) dense_iteration_f8(const __grid_constant__ DenseMaps8 maps, DenseArgs8 a)
{
    constexpr uint32_t PIPE_LIMIT = EXPIRE ? 0u : TC_WAIT_LIMIT;
    using C = F8Cfg<KP>;
    constexpr int NS = C::STAGES;
    constexpr uint32_t IDESC = idesc_e4m3(2 * F8_BM, KP);
    constexpr uint16_t PAIR = 0x3;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_rank();
    const bool leader = crank == 0;
    const int cluster = (int)blockIdx.x / 2, nclusters = (int)gridDim.x / 2;
    const int nitems = (a.row_tiles + 1) / 2 + (a.col_tiles + 1) / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);  // four epilogue warps in each CTA of the pair
        }
        mbar_init(&mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (blockIdx.x == 0 && a.mode == 0) {
            a.q_clear[0] = 0u;  // the slot the next iteration fills (nothing reads it in this launch)
            a.q_clear[1] = 0u;
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"((uint32_t)(2 * KP)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster_sync();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0 && lane == 0) {
        // TMA producer (both CTAs): the K-blocks of this cluster's items through one continuous ring; per
        // K-block this CTA's 128 rows of X and its KP/2 operand rows, counted on the leader's full barrier.
        bool bad = false;
        uint32_t g = 0;  // K-blocks issued so far
        for (int w = cluster; w < nitems && !bad; w += nclusters) {
            const F8Item it = f8_item(a, w, crank);
            const CUtensorMap *mapX = it.cols ? &maps.X[1] : &maps.X[0];
            const CUtensorMap *mapB = it.cols ? &maps.B[1] : &maps.B[0];
            for (int kb = 0; kb < it.nk; ++kb, ++g) {
                const uint32_t s = g % NS;
                if (g >= NS && !mbar_wait_n(&empty[s], ((g / NS) - 1) & 1, PIPE_LIMIT)) {
                    bad = true;
                    break;
                }
                if (leader) mbar_expect_tx(&full[s], 2 * C::SLOT);
                uint8_t *slot = smem + s * C::SLOT;
                const uint32_t bar = cluster_addr(&full[s], 0);
                tma_load_2d_pair(slot, mapX, 0, (it.tile * it.nk + kb) * F8_BM, bar);
                tma_load_2d_pair(slot + F8_A_SLOT, mapB, kb * F8_BK, (int)crank * (KP / 2), bar);
            }
        }
        if (bad) atomicOr(a.status, ST_TIMEOUT);
    } else if (warp == 1 && lane == 0 && leader) {
        // MMA issuer (leader only): per item, once the epilogue has released its accumulator, four K = 32 MMAs
        // (M = 256 over the pair, N = KP) per K-block, then a commit that the accumulator is complete.
        const uint32_t sbase = smem_u32(smem);
        bool bad = false, flagged = false;
        uint32_t g = 0;
        int itn = 0;
        for (int w = cluster; w < nitems; w += nclusters, ++itn) {
            const F8Item it = f8_item(a, w, 0);
            const int buf = itn & 1;
            if (itn >= 2 && !mbar_wait(&acc_empty[buf], ((itn / 2) - 1) & 1)) bad = true;
            if (!bad) {
                const uint32_t acc = tmem + (uint32_t)(buf * KP);
                for (int kb = 0; kb < it.nk; ++kb, ++g) {
                    const uint32_t s = g % NS;
                    if (!mbar_wait_n(&full[s], (g / NS) & 1, PIPE_LIMIT)) {
                        bad = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ad0 = smem_desc_sw128_u32(sbase + (uint32_t)(s * C::SLOT));
                    const uint64_t bd0 = smem_desc_sw128_u32(sbase + (uint32_t)(s * C::SLOT + F8_A_SLOT));
#pragma unroll
                    for (int kk = 0; kk < F8_BK / 32; ++kk)  // +32 bytes along K per step
                        mma_e4m3(acc, ad0 + (uint64_t)(kk * 2), bd0 + (uint64_t)(kk * 2), IDESC,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit_multicast(&empty[s], PAIR);
                }
            }
            if (bad && !flagged) {
                atomicOr(a.status, ST_TIMEOUT);  // seen by the epilogues, which then write nothing
                __threadfence();
                flagged = true;
            }
            mma_commit_multicast(&acc_full[buf], PAIR);  // in both CTAs once this item's MMAs have completed
        }
        mma_commit_multicast(&mma_done, PAIR);
    }

    if (warp >= 2) {
        // Epilogue: warps 2..5, one TMEM lane (one row of the tile) per thread.
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        int itn = 0;
        for (int w = cluster; w < nitems; w += nclusters, ++itn) {
            const F8Item it = f8_item(a, w, crank);
            const int buf = itn & 1;
            const bool ok = mbar_wait(&acc_full[buf], (itn / 2) & 1);
            if (!ok) atomicOr(a.status, ST_TIMEOUT);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem + (uint32_t)(buf * KP) + ((uint32_t)(quad * 32) << 16);
            float ss = 0.f;
#pragma unroll 1
            for (int c = 0; c < KP / 32; ++c) {
                float y[32];
                tmem_ld32(taddr + c * 32, y);
#pragma unroll
                for (int i = 0; i < 32; ++i) ss += y[i] * y[i];
            }
            // The accumulator is in registers: release it to the issuer for the item after next.
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(cluster_addr(&acc_empty[buf], 0));
            const bool cols = it.cols;
            const int side = cols ? 1 : 0;
            const int64_t r = (int64_t)it.tile * F8_BM + row;
            uint32_t qkey = 0u;
            if (ok && it.active && !(*(volatile int *)a.status & ST_TIMEOUT)) {
                float *X = a.x[side];
                const float xo = X[r];
                const float ex = expf(xo);
                const float ci = (!cols && a.row_scale) ? a.row_scale[r] : 1.f;
                // The accumulators carry the other side's operand scale 2^S twice after squaring.
                const float z = ex * ex * ci * ci * ldexpf(ss, -2 * a.s_cur[1 - side]) * (1.f / (float)KP);
                if (a.mode == 1) {
                    a.z[side][r] = z;
                } else {
                    float xn = xo - a.eta * (z - a.target2[side] + a.gamma * xo);
                    if (!isfinite(xn)) atomicOr(a.status, ST_NONFINITE);
                    xn = fminf(fmaxf(xn, -a.M), a.M);
                    X[r] = xn;
                    float *XB = a.xb[side];
                    XB[r] = a.avg_new * xn + a.avg_old * XB[r];
                    const int S = f8_scale_exp_log(f8_next_bound(a, side));
                    const uint8_t mag = f8_code(ldexpf(expf(xn) * ci, S));
                    qkey = f8_key(xn + logf(fabsf(ci)));
                    const int64_t ld = cols ? a.n : a.m;
                    uint8_t *Bn = a.bnext[side];
                    for (int gg = 0; gg < KP / 128; ++gg) {
                        const U4 o = philox10(U4{(uint32_t)r, a.t_next, a.sid_out[side], (uint32_t)gg}, a.key0, a.key1);
                        const uint32_t words[4] = {o.x, o.y, o.z, o.w};
#pragma unroll 8
                        for (int p = 0; p < 128; ++p) {
                            const uint32_t neg = (words[p >> 5] >> (p & 31)) & 1u;
                            Bn[(int64_t)(gg * 128 + p) * ld + r] = (uint8_t)(mag ^ (neg << 7));
                        }
                    }
                }
            }
            if (a.mode == 0) {
                qkey = __reduce_max_sync(0xffffffffu, qkey);
                if (lane == 0 && qkey) atomicMax(&a.q_cur[side], qkey);
            }
        }
        if (a.mode == 0 && blockIdx.x == 0 && threadIdx.x == 64) {
            a.s_next[0] = f8_scale_exp_log(f8_next_bound(a, 0));
            a.s_next[1] = f8_scale_exp_log(f8_next_bound(a, 1));
        }
    }
    __syncthreads();
    if (warp == 1) {
        // Every MMA must have completed before TMEM is released (bounded; immediate normally).
        if (lane == 0) mbar_wait(&mma_done, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * KP)));
    }
    // Neither CTA leaves while copies, commits or arrivals of the pair may still target its shared memory;
    // after an abandoned wait anywhere, copies already issued are given time to land.
    cluster_sync();
    if (threadIdx.x == 0 && (*(volatile int *)a.status & ST_TIMEOUT))
        for (int i = 0; i < 2000; ++i) __nanosleep(1000);
}
// ------------------------------------------------------------------ set-up kernels

// Maxima of one side's operand over a state vector: key of max (x_i + log|c_i|) and max |e^{x_i} c_i|.
__global__ void f8_side_max(int64_t len, const float *x, const float *c, uint32_t *qkey, uint32_t *bmax)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t q = 0u, b = 0u;
    if (i < len) {
        const float ci = c ? c[i] : 1.f;
        q = f8_key(x[i] + logf(fabsf(ci)));
        const float B = fabsf(expf(x[i]) * ci);
        b = isfinite(B) ? __float_as_uint(B) : 0x7f7fffffu;
    }
    q = __reduce_max_sync(0xffffffffu, q);
    b = __reduce_max_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0) {
        if (q) atomicMax(qkey, q);
        atomicMax(bmax, b);
    }
}

// Operand of iteration t from a state vector, scaled from the exact maximum: B[p][i] = e4m3(2^S e^{x_i} c_i) s_ip.
__global__ void f8_build_operand(int64_t len, int kp, const float *x, const float *c, uint32_t t, uint32_t sid,
                                 uint32_t k0, uint32_t k1, const uint32_t *bmax, int *s_out, uint8_t *B)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int S = f8_scale_exp(__uint_as_float(*bmax));
    if (i == 0) *s_out = S;
    if (i >= len) return;
    const float ci = c ? c[i] : 1.f;
    const uint8_t mag = f8_code(ldexpf(expf(x[i]) * ci, S));
    for (int g = 0; g < kp / 128; ++g) {
        const U4 o = philox10(U4{(uint32_t)i, t, sid, (uint32_t)g}, k0, k1);
        const uint32_t words[4] = {o.x, o.y, o.z, o.w};
        for (int p = 0; p < 128; ++p) {
            const uint32_t neg = (words[p >> 5] >> (p & 31)) & 1u;
            B[(int64_t)(g * 128 + p) * len + i] = (uint8_t)(mag ^ (neg << 7));
        }
    }
}

// One 128 x 128 tile of row-major E4M3 codes (rows x cols, leading dimension lda) into the K-blocked orders
// of A (block (i0/128, j0/128)) and of A^T (block (j0/128, i0/128)); NaN codes set ST_BAD_VALUE.
__global__ void f8_block_tiles(const uint8_t *in, int64_t lda, int64_t rows, int64_t cols, uint8_t *A, uint8_t *At,
                               int *status)
{
    __shared__ __align__(16) uint8_t t[128][144];
    const int64_t ct = cols / 128;  // one CTA per tile, tiles in row-major order
    const int64_t j0 = ((int64_t)blockIdx.x % ct) * 128, i0 = ((int64_t)blockIdx.x / ct) * 128;
    bool bad = false;
    for (int c = threadIdx.x; c < 128 * 8; c += blockDim.x) {  // 16-byte chunks: row c / 8, bytes (c % 8) * 16
        const int ii = c >> 3, jj = (c & 7) * 16;
        const int4 w = *reinterpret_cast<const int4 *>(in + (i0 + ii) * lda + j0 + jj);
        *reinterpret_cast<int4 *>(&t[ii][jj]) = w;
        const uint8_t *b = reinterpret_cast<const uint8_t *>(&w);
#pragma unroll
        for (int q = 0; q < 16; ++q) bad |= (b[q] & 0x7f) == 0x7f;
    }
    if (bad) atomicOr(status, ST_BAD_VALUE);
    __syncthreads();
    uint8_t *dA = A + (((i0 / 128) * (cols / 128) + j0 / 128) * 128) * 128;
    uint8_t *dAt = At + (((j0 / 128) * (rows / 128) + i0 / 128) * 128) * 128;
    for (int c = threadIdx.x; c < 128 * 8; c += blockDim.x) {
        const int ii = c >> 3, jj = (c & 7) * 16;
        *reinterpret_cast<int4 *>(dA + ii * 128 + jj) = *reinterpret_cast<const int4 *>(&t[ii][jj]);
        // Row ii of the A^T block is column ii of the tile, entries jj .. jj + 15 of it.
        uint8_t v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = t[jj + q][ii];
        *reinterpret_cast<int4 *>(dAt + ii * 128 + jj) = *reinterpret_cast<const int4 *>(v);
    }
}

__global__ void f8_scale_stats(int64_t m, const float *c, uint32_t *logc_key, int *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t q = 0u;
    if (i < m) {
        if (!isfinite(c[i])) atomicOr(status, ST_BAD_VALUE);
        else if (c[i] != 0.f) q = f8_key(logf(fabsf(c[i])));
    }
    q = __reduce_max_sync(0xffffffffu, q);
    if ((threadIdx.x & 31) == 0 && q) atomicMax(logc_key, q);
}

// out_i = own_i sum_j q_ij^2 sq_j for E4M3 X in its K-blocked order (rows x cols), one warp per row,
// 16-byte loads, FP64 accumulation; own_i = e^{2 x_i} (times c_i^2 for scaled rows).
__global__ void f8_row_norms(const uint8_t *X, int64_t rows, int64_t cols, const double *sq, const double *own,
                             double *out)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    double acc = 0.0;
    const int64_t base = ((r / 128) * (cols / 128)) * 128 * 128 + (r % 128) * 128;
    for (int64_t q = lane; q < cols / 16; q += 32) {
        const int64_t j = q * 16;
        const int4 w = *reinterpret_cast<const int4 *>(X + base + (j / 128) * 128 * 128 + j % 128);
        const uint8_t *e = reinterpret_cast<const uint8_t *>(&w);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const double a = f8_decode(e[t]);
            acc += a * a * sq[j + t];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = own[r] * acc;
}

// ------------------------------------------------------------------ host side

static inline unsigned nblk8(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <int KP, bool EXPIRE>
static sme_status launch_f8(const DenseMaps8 &maps, const DenseArgs8 &a, int grid, cudaStream_t s)
{
    const size_t smem = (size_t)F8Cfg<KP>::BYTES + 1024;
    static bool attr_set = false;
    if (!attr_set) {
        SME_CUDA(cudaFuncSetAttribute(dense_iteration_f8<KP, EXPIRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(F8_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SME_CUDA(cudaLaunchKernelEx(&cfg, dense_iteration_f8<KP, EXPIRE>, maps, a));
    return SME_OK;
}

sme_status dense_f8_create(sme_op op, const uint8_t *src, int64_t lda, cudaStream_t s)
{
    DenseOp *D = op->dense;
    const int64_t m = D->m, n = D->n;
    SME_TRY(dev_alloc(op, (void **)&D->A8, (size_t)m * n));
    SME_TRY(dev_alloc(op, (void **)&D->At8, (size_t)m * n));
    SME_TRY(dev_alloc(op, (void **)&D->f8_small, F8_WORDS * 4));
    SME_CUDA(cudaMemsetAsync(D->f8_small, 0, F8_WORDS * 4, s));
    f8_block_tiles<<<(unsigned)((m / 128) * (n / 128)), 256, 0, s>>>(src, lda, m, n, D->A8, D->At8, op->d_status);
    if (D->row_scale) f8_scale_stats<<<nblk8(m), 256, 0, s>>>(m, D->row_scale, D->f8_small, op->d_status);
    SME_CUDA(cudaGetLastError());
    SME_TRY(tc_make_map(&D->mapA8, CU_TENSOR_MAP_DATA_TYPE_UINT8, D->A8, m * n / F8_BK, F8_BK, 1, F8_BK, F8_BM));
    SME_TRY(tc_make_map(&D->mapAt8, CU_TENSOR_MAP_DATA_TYPE_UINT8, D->At8, m * n / F8_BK, F8_BK, 1, F8_BK, F8_BM));
    return SME_OK;
}

// Called after the creation's stream synchronisation: reads back max log|c| and clears the small block.
sme_status dense_f8_finish_create(sme_op op, cudaStream_t s)
{
    DenseOp *D = op->dense;
    uint32_t key = 0;
    SME_CUDA(cudaMemcpyAsync(&key, D->f8_small, 4, cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    D->logc_max = 0.f;
    if (D->row_scale && key) {
        const uint32_t b = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
        memcpy(&D->logc_max, &b, 4);
    }
    SME_CUDA(cudaMemsetAsync(D->f8_small, 0, F8_WORDS * 4, s));
    return SME_OK;
}

static sme_status ensure_f8_workspace(sme_op op, int kp)
{
    DenseOp *D = op->dense;
    if (D->kcap8 >= kp) return SME_OK;
    for (int b = 0; b < 2; ++b) {
        dev_free(op, D->Bf8[b], D->Bf8[b] ? (size_t)D->kcap8 * D->n : 0);
        dev_free(op, D->Bb8[b], D->Bb8[b] ? (size_t)D->kcap8 * D->m : 0);
        D->Bf8[b] = D->Bb8[b] = nullptr;
    }
    D->kcap8 = 0;
    for (int b = 0; b < 2; ++b) {
        SME_TRY(dev_alloc(op, (void **)&D->Bf8[b], (size_t)kp * D->n));
        SME_TRY(dev_alloc(op, (void **)&D->Bb8[b], (size_t)kp * D->m));
        SME_TRY(tc_make_map(&D->mapBf8[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, D->Bf8[b], kp, D->n, 1, F8_BK, kp / 2));
        SME_TRY(tc_make_map(&D->mapBb8[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, D->Bb8[b], kp, D->m, 1, F8_BK, kp / 2));
    }
    if (!D->x[0]) SME_TRY(dev_alloc(op, (void **)&D->x[0], D->m * 4));
    if (!D->xb[0]) SME_TRY(dev_alloc(op, (void **)&D->xb[0], D->m * 4));
    if (!D->x[1]) SME_TRY(dev_alloc(op, (void **)&D->x[1], D->n * 4));
    if (!D->xb[1]) SME_TRY(dev_alloc(op, (void **)&D->xb[1], D->n * 4));
    D->kcap8 = kp;
    return SME_OK;
}

static sme_status run_f8(sme_op op, const DenseArgs8 &a, int buf, cudaStream_t s)
{
    DenseOp *D = op->dense;
    DenseMaps8 maps;
    maps.X[0] = D->mapA8;
    maps.X[1] = D->mapAt8;
    maps.B[0] = D->mapBf8[buf];
    maps.B[1] = D->mapBb8[buf];
    // Persistent clusters of two CTAs: one per SM pair, at most one per work item.
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        SME_CUDA(cudaGetDevice(&dev));
        SME_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int items = (a.row_tiles + 1) / 2 + (a.col_tiles + 1) / 2;
    const int grid = 2 * std::max(1, std::min(items, sms / 2));
    if (a.pipe_limit == 0) {
        if (a.kp == 256) return launch_f8<256, true>(maps, a, grid, s);
        return launch_f8<128, true>(maps, a, grid, s);
    }
    if (a.kp == 256) return launch_f8<256, false>(maps, a, grid, s);
    return launch_f8<128, false>(maps, a, grid, s);
}

static DenseArgs8 f8_base(sme_op op, double alpha, double beta, double gamma, double M, uint64_t seed, int kp)
{
    DenseOp *D = op->dense;
    DenseArgs8 a{};
    a.m = D->m;
    a.n = D->n;
    a.row_tiles = (int)(D->m / F8_BM);
    a.col_tiles = (int)(D->n / F8_BM);
    a.row_ctas = (a.row_tiles + 1) & ~1;
    a.kp = kp;
    for (int i = 0; i < 2; ++i) {
        a.x[i] = D->x[i];
        a.xb[i] = D->xb[i];
    }
    a.target2[0] = (float)(alpha * alpha);
    a.target2[1] = (float)(beta * beta);
    a.gamma = (float)gamma;
    a.M = (float)M;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.row_scale = D->row_scale;
    a.logc[0] = D->logc_max;
    a.logc[1] = 0.f;
    a.pipe_limit = TC_WAIT_LIMIT;
    a.status = op->d_status;
    return a;
}

// Maxima of both sides of (u, v) into ring slot `slot` and bmax, then the operands of iteration t into
// buffer `buf` with their exponents at parity `par`.
static sme_status f8_first_operands(sme_op op, int kp, uint32_t t, uint32_t sid_s, uint64_t seed, int slot, int buf,
                                    int par, cudaStream_t s)
{
    DenseOp *D = op->dense;
    uint32_t *q = D->f8_small + F8_Q, *bm = D->f8_small + F8_BMAX;
    int *ex = reinterpret_cast<int *>(D->f8_small + F8_EXP);
    SME_CUDA(cudaMemsetAsync(D->f8_small, 0, F8_WORDS * 4, s));
    f8_side_max<<<nblk8(D->m), 256, 0, s>>>(D->m, D->x[0], D->row_scale, q + slot * 2 + 0, bm + 0);
    f8_side_max<<<nblk8(D->n), 256, 0, s>>>(D->n, D->x[1], nullptr, q + slot * 2 + 1, bm + 1);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    f8_build_operand<<<nblk8(D->n), 256, 0, s>>>(D->n, kp, D->x[1], nullptr, t, sid_s, k0, k1, bm + 1,
                                                 ex + par * 2 + 1, D->Bf8[buf]);
    f8_build_operand<<<nblk8(D->m), 256, 0, s>>>(D->m, kp, D->x[0], D->row_scale, t, sid_s + 1u, k0, k1, bm + 0,
                                                 ex + par * 2 + 0, D->Bb8[buf]);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

sme_status dense_f8_equilibrate(sme_op op, const sme_equil_params *p, double alpha, double beta, double gamma,
                                double M, float *u, float *v, float *ub, float *vb, cudaStream_t s)
{
    const int kp = p->k;
    SME_TRY(ensure_f8_workspace(op, kp));
    DenseOp *D = op->dense;
    const uint32_t sid_s = (uint32_t)p->stream_base, sid_w = sid_s + 1u;
    const int tb = p->t_begin;
    SME_CUDA(cudaMemcpyAsync(D->x[0], u, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->xb[0], ub, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->x[1], v, D->n * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->xb[1], vb, D->n * 4, cudaMemcpyDeviceToDevice, s));
    SME_TRY(f8_first_operands(op, kp, (uint32_t)tb, sid_s, p->seed, (tb - 1) % 3, tb & 1, tb & 1, s));
    uint32_t *q = D->f8_small + F8_Q;
    int *ex = reinterpret_cast<int *>(D->f8_small + F8_EXP);
    const bool timed = (p->flags & SME_EQ_TIMED) != 0;
    if (timed) {
        for (int i = 0; i < 2; ++i)
            if (!op->ev_loop[i]) SME_CUDA(cudaEventCreate(&op->ev_loop[i]));
        SME_CUDA(cudaEventRecord(op->ev_loop[0], s));
    }
    for (int t = tb; t < tb + p->T; ++t) {
        DenseArgs8 a = f8_base(op, alpha, beta, gamma, M, p->seed, kp);
        const int cur = t & 1, nxt = cur ^ 1;
        a.bnext[0] = D->Bb8[nxt];
        a.bnext[1] = D->Bf8[nxt];
        a.eta = (float)(2.0 / (gamma * ((double)t + (double)p->t0 + 1.0)));
        a.avg_new = (float)(2.0 / ((double)t + 2.0));
        a.avg_old = (float)((double)t / ((double)t + 2.0));
        a.t_next = (uint32_t)(t + 1);
        a.sid_out[0] = sid_w;
        a.sid_out[1] = sid_s;
        a.mode = 0;
        a.s_cur = ex + cur * 2;
        a.s_next = ex + nxt * 2;
        a.q_prev = q + ((t - 1) % 3) * 2;
        a.q_cur = q + (t % 3) * 2;
        a.q_clear = q + ((t + 1) % 3) * 2;
        if (p->flags & SME_EQ_EXPIRE_PIPELINE_WAITS) a.pipe_limit = 0;
        SME_TRY(run_f8(op, a, cur, s));
    }
    if (timed) {
        SME_CUDA(cudaEventRecord(op->ev_loop[1], s));
        op->loop_timed = true;
        op->loop_iters = p->T;
    }
    SME_CUDA(cudaMemcpyAsync(u, D->x[0], D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(ub, D->xb[0], D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(v, D->x[1], D->n * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(vb, D->xb[1], D->n * 4, cudaMemcpyDeviceToDevice, s));
    return SME_OK;
}

sme_status dense_f8_estimate(sme_op op, const float *u, const float *v, int t, int k, uint64_t seed, int sb, double alpha,
                             double beta, double gamma, double M, float *zu, float *zv, cudaStream_t s)
{
    SME_TRY(ensure_f8_workspace(op, k));
    DenseOp *D = op->dense;
    SME_CUDA(cudaMemcpyAsync(D->x[0], u, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->x[1], v, D->n * 4, cudaMemcpyDeviceToDevice, s));
    SME_TRY(f8_first_operands(op, k, (uint32_t)t, (uint32_t)sb, seed, 0, 0, 0, s));
    DenseArgs8 a = f8_base(op, alpha, beta, gamma, M, seed, k);
    a.mode = 1;
    a.z[0] = zu ? zu : D->xb[0];
    a.z[1] = zv ? zv : D->xb[1];
    a.s_cur = reinterpret_cast<int *>(D->f8_small + F8_EXP);
    return run_f8(op, a, 0, s);
}

sme_status dense_f8_exact_norms(sme_op op, const double *sq_u, const double *sq_v, double *r2, double *c2,
                                cudaStream_t s)
{
    DenseOp *D = op->dense;
    f8_row_norms<<<nblk8(D->m * 32), 256, 0, s>>>(D->A8, D->m, D->n, sq_v, sq_u, r2);
    f8_row_norms<<<nblk8(D->n * 32), 256, 0, s>>>(D->At8, D->n, D->m, sq_u, sq_v, c2);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

}  // namespace sme
