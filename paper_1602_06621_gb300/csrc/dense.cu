// Dense operator: the probe products of Algorithm 1 on the tcgen05 tensor cores.
//
// For dense A (m x n) one iteration needs Y = A (E S) and Y' = A^T (D W) with S (n x k), W (m x k)
// of +-1 probes (Section 3.1 estimator).  The +-1 entries are exact in BF16, but e^{v_j} s_jp is not,
// so each B operand holds two BF16 terms: B = [hi | lo] with hi = bf16(x), lo = bf16(x - hi), and the
// two accumulators are added in the epilogue (relative error of the scaling ~2^-17 instead of 2^-9).
//
// Both products are the same GEMM, X (M x K, BF16) times B^T (N x K, row-major BF16): the op keeps A
// and a transposed copy A^T, so every operand is K-major, both stored K-blocked (each 128 x 64 tile one
// contiguous 16 KB run).  One launch performs one iteration: the first CTAs take tiles of A (forward),
// the others tiles of A^T.  CTAs run in clusters of two, one per SM of a pair, on 256 rows of one
// product: the leader issues M = 256 tcgen05.mma (cta_group::2), each CTA holding its 128 rows of X and
// one half of every 256-row operand unit, and each CTA's TMEM receiving its 128 rows x 2k FP32
// (2k <= 512 columns).  K streams in blocks of 64 through two rings of shared-memory slots filled by TMA
// (128-byte swizzle), one for X, one for the operand halves, each slot released in both CTAs as soon as
// its own MMAs complete.  The producer and MMA-issue loops are kept to a few instructions per slot: the
// issuing thread runs only slightly ahead of the tensor core, so anything more on that path shows up
// directly as idle tensor cycles.  Four epilogue warps per CTA read TMEM and finish each row in
// registers: z = e^{2x} (1/k) sum_p (hi_p + lo_p)^2, the projected step, the running average, and the
// row's slice of the NEXT iteration's B operand (its scale and Philox probe bits), double-buffered like
// the sparse path's gather tables.
//
// Every wait on an mbarrier is bounded: on expiry the kernel sets ST_TIMEOUT in the op's status word
// (the epilogue then writes nothing), waits (bounded) for the MMAs in flight, frees its TMEM, and leaves
// after a cluster barrier that keeps both CTAs resident until neither can still be written to.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "sme_internal.cuh"
#include "tc_common.cuh"

namespace sme {

constexpr int DN_BM = 128;                  // rows per CTA (the pair's MMA has M = 256)
constexpr int DN_BK = 64;                   // K per block: 64 BF16 = one 128-byte swizzle row
constexpr int DN_ROWB = DN_BK * 2;          // bytes per operand row in shared memory
constexpr int DN_A_SLOT = DN_BM * DN_ROWB;  // 16 KB: one K-block of this CTA's 128 rows of A (or A^T)
constexpr int DN_B_SLOT = 128 * DN_ROWB;    // 16 KB: one K-block of this CTA's half of a 256-row operand unit

// Ring depths: four K-blocks in flight (k = 256: one A slot and two operand halves, hi and lo, per
// K-block; k = 128: hi and lo together are one 256-row unit).
template <int KP>
struct DenseCfg {
    static constexpr int NT = 2 * KP;
    static constexpr int UNITS = NT / 256;  // operand units (one MMA's N = 256) per K-block
    static constexpr int A_SLOTS = KP == 256 ? 4 : 6;
    static constexpr int B_SLOTS = KP == 256 ? 8 : 6;
    static constexpr int BYTES = A_SLOTS * DN_A_SLOT + B_SLOTS * DN_B_SLOT;
};
static_assert(DenseCfg<256>::BYTES + 1024 <= 227 * 1024 && DenseCfg<128>::BYTES + 1024 <= 227 * 1024,
              "dense rings exceed the shared memory of one CTA");
constexpr int DN_THREADS = 192;      // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2..5 epilogue


// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// ------------------------------------------------------------------ the iteration kernel

struct DenseArgs {
    int64_t m, n;
    int row_tiles, col_tiles; // m / 128, n / 128
    int row_ctas;             // CTAs of the forward product: row_tiles rounded up to whole clusters
    int kp;                   // probes (128 or 256)
    float *x[2], *xb[2];      // [0] u, ubar (rows)   [1] v, vbar (columns)
    float *z[2];              // estimate-only outputs, or null
    __nv_bfloat16 *bnext[2];  // [0] next backward operand (written by rows), [1] next forward operand
    float target2[2];
    float gamma, M, eta, avg_new, avg_old;
    uint32_t t_next, key0, key1, sid_out[2];
    int mode;                 // 0 step, 1 estimate only
    const float *row_scale;   // A_ij = row_scale[i] * Abf16_ij (FP8 input), or null
    uint32_t pipe_limit;      // TC_WAIT_LIMIT, or 0 to launch the EXPIRE instantiation (test of the timeout
                              // path); the drain waits always use TC_WAIT_LIMIT
    int *status;
};

struct DenseMaps {
    CUtensorMap X[2];  // [0] A, [1] A^T
    CUtensorMap B[2];  // [0] forward operand (current), [1] backward operand (current)
};

// EXPIRE: the instantiation for the test of the timeout path (producer and MMA-issuer waits bounded by zero
// polls); the bound is a compile-time constant so that the normal kernel's issuing loops stay minimal.
template <int KP, bool EXPIRE = false>
__global__ void __launch_bounds__(DN_THREADS, 1) dense_iteration(const __grid_constant__ DenseMaps maps, DenseArgs a)
{
    constexpr uint32_t PIPE_LIMIT = EXPIRE ? 0u : TC_WAIT_LIMIT;
    using C = DenseCfg<KP>;
    constexpr int NT = C::NT;  // accumulator columns: hi then lo
    constexpr int UNITS = C::UNITS, NA = C::A_SLOTS, NB = C::B_SLOTS;
    constexpr uint32_t IDESC = idesc_bf16(2 * DN_BM, 256);
    constexpr uint16_t PAIR = 0x3;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring_a = smem;                    // NA slots of DN_A_SLOT bytes
    uint8_t *ring_b = smem + NA * DN_A_SLOT;   // NB slots of DN_B_SLOT bytes
    // The full barriers of the leader (rank 0) count both CTAs' copies; the empty barriers of each CTA and
    // its acc_bar are signalled by the leader's MMA commits.
    __shared__ uint64_t a_full[NA], a_empty[NA], b_full[NB], b_empty[NB], acc_bar;
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // A cluster of two CTAs (one per SM of a pair) computes 256 rows of one product with M = 256 MMAs
    // (cta_group::2): each CTA holds its 128 rows of A and one half of every 256-row operand unit, the
    // leader issues the MMAs, and each CTA's TMEM receives its own rows.  With an odd tile count the
    // second CTA of the last cluster repeats its partner's rows and writes nothing.
    const bool cols = (int)blockIdx.x >= a.row_ctas;
    const int idx = cols ? (int)blockIdx.x - a.row_ctas : (int)blockIdx.x;
    const int ntiles = cols ? a.col_tiles : a.row_tiles;
    const bool active = idx < ntiles;
    const int tile = active ? idx : ntiles - 1;
    const uint32_t crank = cluster_rank();
    const bool leader = crank == 0;
    const int64_t K = cols ? a.m : a.n;              // reduction length
    const int nk = (int)(K / DN_BK);
    const CUtensorMap *mapX = cols ? &maps.X[1] : &maps.X[0];
    const CUtensorMap *mapB = cols ? &maps.B[1] : &maps.B[0];

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        mbar_init(&acc_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // one warp of each CTA of the pair allocates, collectively
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"((uint32_t)NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster_sync();  // both CTAs' barriers are initialised before the pair signals them
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0 && lane == 0) {
        // TMA producer (both CTAs): for each K-block this CTA's A slot, then its halves of the operand units,
        // in the order the leader consumes them; completion is counted on the leader's full barriers.  The
        // loop is kept minimal: the MMA issuer runs only a few instructions ahead of the tensor core.
        bool bad = false;
        for (int kb = 0; kb < nk && !bad; ++kb) {
            const int sa = kb % NA;
            if (kb >= NA && !mbar_wait_n(&a_empty[sa], ((kb / NA) - 1) & 1, PIPE_LIMIT)) {
                bad = true;
                break;
            }
            if (leader) mbar_expect_tx(&a_full[sa], 2 * DN_A_SLOT);
            tma_load_2d_pair(ring_a + sa * DN_A_SLOT, mapX, 0, (tile * nk + kb) * DN_BM, cluster_addr(&a_full[sa], 0));
            for (int j = 0; j < UNITS; ++j) {
                const int q = kb * UNITS + j, sb = q % NB;
                if (q >= NB && !mbar_wait_n(&b_empty[sb], ((q / NB) - 1) & 1, PIPE_LIMIT)) {
                    bad = true;
                    break;
                }
                if (leader) mbar_expect_tx(&b_full[sb], 2 * DN_B_SLOT);
                tma_load_2d_pair(ring_b + sb * DN_B_SLOT, mapB, kb * DN_BK, j * 256 + (int)crank * 128,
                                 cluster_addr(&b_full[sb], 0));
            }
        }
        if (bad) atomicOr(a.status, ST_TIMEOUT);
    } else if (warp == 1 && lane == 0 && leader) {
        // MMA issuer (leader only): four K=16 MMAs (M = 256 over the pair, N = 256) per operand unit into
        // that unit's 256 accumulator columns; each slot is released in both CTAs as soon as its MMAs
        // complete, the A slot after the block's last unit.
        const uint32_t sbase = smem_u32(smem);
        bool bad = false;
        for (int kb = 0; kb < nk && !bad; ++kb) {
            const int sa = kb % NA;
            if (!mbar_wait_n(&a_full[sa], (kb / NA) & 1, PIPE_LIMIT)) {
                bad = true;
                break;
            }
            const uint64_t ad0 = smem_desc_sw128_u32(sbase + (uint32_t)(sa * DN_A_SLOT));
            for (int j = 0; j < UNITS; ++j) {
                const int q = kb * UNITS + j, sb = q % NB;
                if (!mbar_wait_n(&b_full[sb], (q / NB) & 1, PIPE_LIMIT)) {
                    bad = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t bd0 = smem_desc_sw128_u32(sbase + (uint32_t)(NA * DN_A_SLOT + sb * DN_B_SLOT));
#pragma unroll
                for (int kk = 0; kk < DN_BK / 16; ++kk)  // +32 bytes along K per step
                    mma_bf16(tmem + j * 256, ad0 + (uint64_t)(kk * 2), bd0 + (uint64_t)(kk * 2), IDESC,
                             (kb > 0 || kk > 0) ? 1u : 0u);
                mma_commit_multicast(&b_empty[sb], PAIR);
            }
            if (!bad) mma_commit_multicast(&a_empty[sa], PAIR);
        }
        if (bad) {
            atomicOr(a.status, ST_TIMEOUT);  // seen by the epilogue, which then writes nothing
            __threadfence();
        }
        mma_commit_multicast(&acc_bar, PAIR);  // arrives in both CTAs once every MMA above has completed
    }

    // Epilogue: warps 2..5, one TMEM lane (one row of the tile) per thread.
    if (warp >= 2) {
        const bool ok = mbar_wait(&acc_bar, 0);
        if (!ok) atomicOr(a.status, ST_TIMEOUT);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int64_t r = (int64_t)tile * DN_BM + row;
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16);
        float ss = 0.f;
#pragma unroll 1
        for (int c = 0; c < KP / 32; ++c) {
            float hi[32], lo[32];
            tmem_ld32(taddr + c * 32, hi);
            tmem_ld32(taddr + KP + c * 32, lo);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float y = hi[i] + lo[i];
                ss += y * y;
            }
        }
        const int side = cols ? 1 : 0;
        if (ok && active && !(*(volatile int *)a.status & ST_TIMEOUT)) {
            float *X = a.x[side];
            const float xo = X[r];
            const float ex = expf(xo);
            // With row scales A = diag(c) A', row i of D A E is c_i times row i of D A' E, and the
            // backward operand carries c_i (see below), so only the rows' estimate needs c_i^2.
            const float ci = (!cols && a.row_scale) ? a.row_scale[r] : 1.f;
            const float z = ex * ex * ci * ci * ss * (1.f / (float)KP);
            if (a.mode == 1) {
                a.z[side][r] = z;
            } else {
                float xn = xo - a.eta * (z - a.target2[side] + a.gamma * xo);
                if (!isfinite(xn)) atomicOr(a.status, ST_NONFINITE);
                xn = fminf(fmaxf(xn, -a.M), a.M);
                X[r] = xn;
                float *XB = a.xb[side];
                XB[r] = a.avg_new * xn + a.avg_old * XB[r];
                // This row's entries of the next iteration's operand: scale e^{x^t} times probes of t+1.
                const float sc = expf(xn) * ((!cols && a.row_scale) ? a.row_scale[r] : 1.f);
                const __nv_bfloat16 hi = __float2bfloat16_rn(sc);
                const __nv_bfloat16 lo = __float2bfloat16_rn(sc - __bfloat162float(hi));
                const int64_t ld = cols ? a.n : a.m;
                __nv_bfloat16 *Bn = a.bnext[side];
                for (int g = 0; g < KP / 128; ++g) {
                    const U4 o = philox10(U4{(uint32_t)r, a.t_next, a.sid_out[side], (uint32_t)g}, a.key0, a.key1);
                    const uint32_t words[4] = {o.x, o.y, o.z, o.w};
#pragma unroll 4
                    for (int p = 0; p < 128; ++p) {
                        const bool neg = (words[p >> 5] >> (p & 31)) & 1u;
                        const int pp = g * 128 + p;
                        Bn[(int64_t)pp * ld + r] = neg ? __hneg(hi) : hi;
                        Bn[(int64_t)(KP + pp) * ld + r] = neg ? __hneg(lo) : lo;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        // MMAs still in flight must finish before their TMEM is released (bounded; completes at once normally).
        if (lane == 0) mbar_wait(&acc_bar, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT));
    }
    // Neither CTA leaves while copies or commits of the pair may still target its shared memory.  After an
    // abandoned wait anywhere (the status bit is set before the CTA that gave up reaches this barrier),
    // copies already issued are given time to land.
    cluster_sync();
    if (threadIdx.x == 0 && (*(volatile int *)a.status & ST_TIMEOUT))
        for (int i = 0; i < 2000; ++i) __nanosleep(1000);
}

// Operand of iteration t from a state vector: B[p][i] = s_ip * hi(e^{x_i}), B[k+p][i] = s_ip * lo(e^{x_i}).
__global__ void dense_build_operand(int64_t len, int kp, const float *x, const float *mult, uint32_t t, uint32_t sid,
                                    uint32_t k0, uint32_t k1, __nv_bfloat16 *B)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const float sc = expf(x[i]) * (mult ? mult[i] : 1.f);
    const __nv_bfloat16 hi = __float2bfloat16_rn(sc);
    const __nv_bfloat16 lo = __float2bfloat16_rn(sc - __bfloat162float(hi));
    for (int g = 0; g < kp / 128; ++g) {
        const U4 o = philox10(U4{(uint32_t)i, t, sid, (uint32_t)g}, k0, k1);
        const uint32_t words[4] = {o.x, o.y, o.z, o.w};
        for (int p = 0; p < 128; ++p) {
            const bool neg = (words[p >> 5] >> (p & 31)) & 1u;
            const int pp = g * 128 + p;
            B[(int64_t)pp * len + i] = neg ? __hneg(hi) : hi;
            B[(int64_t)(kp + pp) * len + i] = neg ? __hneg(lo) : lo;
        }
    }
}

// Element offset of (i, j) in the K-blocked order of a rows x cols matrix (cols a multiple of 64).
__host__ __device__ __forceinline__ int64_t blocked_offset(int64_t i, int64_t j, int64_t cols)
{
    return (((i / DN_BM) * (cols / DN_BK) + j / DN_BK) * DN_BM + i % DN_BM) * DN_BK + j % DN_BK;
}

// Row-major (rows x cols) -> K-blocked order; one thread per 16-byte group of 8 elements.
__global__ void block_k64(const __nv_bfloat16 *in, int64_t rows, int64_t cols, __nv_bfloat16 *out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rows * cols / 8) return;
    const int64_t i = g / (cols / 8), j = (g % (cols / 8)) * 8;
    *reinterpret_cast<int4 *>(out + blocked_offset(i, j, cols)) = *reinterpret_cast<const int4 *>(in + i * cols + j);
}

// 32x32 tiled transpose of a BF16 matrix (rows x cols) into (cols x rows).
__global__ void transpose_bf16(const __nv_bfloat16 *in, int64_t rows, int64_t cols, __nv_bfloat16 *out)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[j][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][j];
    }
}

__global__ void bf16_check_finite(const __nv_bfloat16 *a, int64_t count, int *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(__bfloat162float(a[i]))) atomicOr(status, ST_BAD_VALUE);
}

// ------------------------------------------------------------------ host side

// Row-major BF16 matrix (rows x cols) viewed with boxes of DN_BK columns (128 bytes) x box_rows rows.
static sme_status make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int box_rows)
{
    return tc_make_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, rows, cols, 2, DN_BK, box_rows);
}

// K-blocked matrix (rows x cols) viewed as (rows * cols / 64) rows of 64 elements, boxes of 128 such rows:
// box y = (t * cols/64 + kb) * 128 is the 128 x 64 block of row tile t and K-block kb.
static sme_status make_map_blocked(CUtensorMap *map, const void *base, int64_t rows, int64_t cols)
{
    return make_map(map, base, rows * cols / DN_BK, DN_BK, DN_BM);
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <int KP>
static size_t dense_smem() { return (size_t)DenseCfg<KP>::BYTES + 1024; }

static sme_status ensure_dense_workspace(sme_op op, int kp)
{
    DenseOp *D = op->dense;
    if (D->kcap >= kp) return SME_OK;
    for (int b = 0; b < 2; ++b) {
        dev_free(op, D->Bf[b], D->Bf[b] ? (size_t)2 * D->kcap * D->n * 2 : 0);
        dev_free(op, D->Bb[b], D->Bb[b] ? (size_t)2 * D->kcap * D->m * 2 : 0);
        D->Bf[b] = D->Bb[b] = nullptr;
        SME_TRY(dev_alloc(op, (void **)&D->Bf[b], (size_t)2 * kp * D->n * 2));
        SME_TRY(dev_alloc(op, (void **)&D->Bb[b], (size_t)2 * kp * D->m * 2));
        SME_TRY(make_map(&D->mapBf[b], D->Bf[b], 2 * kp, D->n, 128));
        SME_TRY(make_map(&D->mapBb[b], D->Bb[b], 2 * kp, D->m, 128));
    }
    // Each buffer on its own, so that a call after a failed allocation completes the set.
    if (!D->x[0]) SME_TRY(dev_alloc(op, (void **)&D->x[0], D->m * 4));
    if (!D->xb[0]) SME_TRY(dev_alloc(op, (void **)&D->xb[0], D->m * 4));
    if (!D->x[1]) SME_TRY(dev_alloc(op, (void **)&D->x[1], D->n * 4));
    if (!D->xb[1]) SME_TRY(dev_alloc(op, (void **)&D->xb[1], D->n * 4));
    D->kcap = kp;
    return SME_OK;
}

template <int KP, bool EXPIRE>
static sme_status launch_dense(const DenseMaps &maps, const DenseArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = dense_smem<KP>();
    static bool attr_set = false;
    if (!attr_set) {
        SME_CUDA(cudaFuncSetAttribute(dense_iteration<KP, EXPIRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(DN_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SME_CUDA(cudaLaunchKernelEx(&cfg, dense_iteration<KP, EXPIRE>, maps, a));
    return SME_OK;
}

static sme_status run_dense(sme_op op, const DenseArgs &a, int buf, cudaStream_t s)
{
    DenseOp *D = op->dense;
    DenseMaps maps;
    maps.X[0] = D->mapA;
    maps.X[1] = D->mapAt;
    maps.B[0] = D->mapBf[buf];
    maps.B[1] = D->mapBb[buf];
    const int grid = a.row_ctas + ((a.col_tiles + 1) & ~1);  // whole clusters of two on each product
    if (a.pipe_limit == 0) {
        if (a.kp == 256) return launch_dense<256, true>(maps, a, grid, s);
        return launch_dense<128, true>(maps, a, grid, s);
    }
    if (a.kp == 256) return launch_dense<256, false>(maps, a, grid, s);
    return launch_dense<128, false>(maps, a, grid, s);
}

static DenseArgs dense_base(sme_op op, double alpha, double beta, double gamma, double M, uint64_t seed, int kp)
{
    DenseOp *D = op->dense;
    DenseArgs a{};
    a.m = D->m;
    a.n = D->n;
    a.row_tiles = (int)(D->m / DN_BM);
    a.col_tiles = (int)(D->n / DN_BM);
    a.row_ctas = (a.row_tiles + 1) & ~1;
    a.kp = kp;
    a.x[0] = D->x[0];
    a.x[1] = D->x[1];
    a.xb[0] = D->xb[0];
    a.xb[1] = D->xb[1];
    a.target2[0] = (float)(alpha * alpha);
    a.target2[1] = (float)(beta * beta);
    a.gamma = (float)gamma;
    a.M = (float)M;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.row_scale = D->row_scale;
    a.pipe_limit = TC_WAIT_LIMIT;
    a.status = op->d_status;
    return a;
}

// E4M3 storage (dense_f8.cu).
sme_status dense_f8_create(sme_op op, const uint8_t *src, int64_t lda, cudaStream_t s);
sme_status dense_f8_finish_create(sme_op op, cudaStream_t s);
sme_status dense_f8_equilibrate(sme_op op, const sme_equil_params *p, double alpha, double beta, double gamma,
                                double M, float *u, float *v, float *ub, float *vb, cudaStream_t s);
sme_status dense_f8_estimate(sme_op op, const float *u, const float *v, int t, int k, uint64_t seed, int sb,
                             double alpha, double beta, double gamma, double M, float *zu, float *zv, cudaStream_t s);
sme_status dense_f8_exact_norms(sme_op op, const double *sq_u, const double *sq_v, double *r2, double *c2,
                                cudaStream_t s);

void dense_destroy(sme_op op)
{
    DenseOp *D = op->dense;
    if (!D) return;
    for (void *p : {(void *)D->A, (void *)D->At, (void *)D->row_scale, (void *)D->Bf[0], (void *)D->Bf[1],
                    (void *)D->Bb[0], (void *)D->Bb[1], (void *)D->x[0], (void *)D->x[1], (void *)D->xb[0],
                    (void *)D->xb[1], (void *)D->A8, (void *)D->At8, (void *)D->Bf8[0], (void *)D->Bf8[1],
                    (void *)D->Bb8[0], (void *)D->Bb8[1], (void *)D->f8_small})
        dev_release(p);
    delete D;
    op->dense = nullptr;
}

static void resolve_params(sme_op op, double &alpha, double &beta, double &gamma, double &M)
{
    if (alpha <= 0) alpha = std::pow((double)op->n / (double)op->m, 0.25);
    if (beta <= 0) beta = std::pow((double)op->m / (double)op->n, 0.25);
    if (gamma <= 0) gamma = 0.1;
    if (M <= 0) M = std::log(1e4);
}

sme_status dense_equilibrate(sme_op op, const sme_equil_params *p, float *u, float *v, float *ub, float *vb,
                             cudaStream_t s)
{
    const int kp = p->k;
    if (kp != 128 && kp != 256) {
        set_error("dense operators support k = 128 or 256");
        return SME_ERR_UNSUPPORTED;
    }
    double alpha = p->alpha, beta = p->beta, gamma = p->gamma, M = p->M;
    resolve_params(op, alpha, beta, gamma, M);
    if (op->dense->fp8) return dense_f8_equilibrate(op, p, alpha, beta, gamma, M, u, v, ub, vb, s);
    SME_TRY(ensure_dense_workspace(op, kp));
    DenseOp *D = op->dense;
    const uint32_t sid_s = (uint32_t)p->stream_base, sid_w = sid_s + 1u;
    const int tb = p->t_begin;
    SME_CUDA(cudaMemcpyAsync(D->x[0], u, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->xb[0], ub, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->x[1], v, D->n * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->xb[1], vb, D->n * 4, cudaMemcpyDeviceToDevice, s));
    const uint32_t k0 = (uint32_t)p->seed, k1 = (uint32_t)(p->seed >> 32);
    dense_build_operand<<<nblk(D->n), 256, 0, s>>>(D->n, kp, D->x[1], nullptr, (uint32_t)tb, sid_s, k0, k1,
                                                   D->Bf[tb & 1]);
    dense_build_operand<<<nblk(D->m), 256, 0, s>>>(D->m, kp, D->x[0], D->row_scale, (uint32_t)tb, sid_w, k0, k1,
                                                   D->Bb[tb & 1]);
    SME_CUDA(cudaGetLastError());
    const bool timed = (p->flags & SME_EQ_TIMED) != 0;
    if (timed) {
        for (int i = 0; i < 2; ++i)
            if (!op->ev_loop[i]) SME_CUDA(cudaEventCreate(&op->ev_loop[i]));
        SME_CUDA(cudaEventRecord(op->ev_loop[0], s));
    }
    for (int t = tb; t < tb + p->T; ++t) {
        DenseArgs a = dense_base(op, alpha, beta, gamma, M, p->seed, kp);
        const int cur = t & 1, nxt = cur ^ 1;
        a.bnext[0] = D->Bb[nxt];
        a.bnext[1] = D->Bf[nxt];
        a.eta = (float)(2.0 / (gamma * ((double)t + (double)p->t0 + 1.0)));
        a.avg_new = (float)(2.0 / ((double)t + 2.0));
        a.avg_old = (float)((double)t / ((double)t + 2.0));
        a.t_next = (uint32_t)(t + 1);
        a.sid_out[0] = sid_w;
        a.sid_out[1] = sid_s;
        a.mode = 0;
        if (p->flags & SME_EQ_EXPIRE_PIPELINE_WAITS) a.pipe_limit = 0;
        SME_TRY(run_dense(op, a, cur, s));
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

// sq[j] = e^{2 x_j} (times c_j^2 when per-row scales are given).
__global__ void dense_sq(int64_t n, const float *x, const float *scale, double *sq)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double e = exp(2.0 * (double)x[j]);
    const double c = scale ? (double)scale[j] : 1.0;
    sq[j] = e * c * c;
}

// out_i = own_i * sum_j X_ij^2 sq_j for X in K-blocked order (rows x cols, cols a multiple of 128), one warp
// per row, 16-byte loads, FP64 accumulation; own_i = e^{2 x_i} (times c_i^2 for scaled rows).
__global__ void dense_row_norms(const __nv_bfloat16 *X, int64_t rows, int64_t cols, const double *sq,
                                const double *own, double *out)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    double acc = 0.0;
    for (int64_t q = lane; q < cols / 8; q += 32) {
        const int4 w = *reinterpret_cast<const int4 *>(X + blocked_offset(r, q * 8, cols));
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&w);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const double a = (double)__bfloat162float(e[t]);
            acc += a * a * sq[q * 8 + t];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = own[r] * acc;
}

sme_status dense_exact_norms(sme_op op, const float *u, const float *v, double *sq_u, double *sq_v, double *r2,
                             double *c2, cudaStream_t s)
{
    DenseOp *D = op->dense;
    const int64_t m = D->m, n = D->n;
    dense_sq<<<nblk(m), 256, 0, s>>>(m, u, D->row_scale, sq_u);
    dense_sq<<<nblk(n), 256, 0, s>>>(n, v, nullptr, sq_v);
    if (D->fp8) return dense_f8_exact_norms(op, sq_u, sq_v, r2, c2, s);
    dense_row_norms<<<nblk(m * 32), 256, 0, s>>>(D->A, m, n, sq_v, sq_u, r2);
    dense_row_norms<<<nblk(n * 32), 256, 0, s>>>(D->At, n, m, sq_u, sq_v, c2);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

sme_status dense_estimate(sme_op op, const float *u, const float *v, int t, int k, uint64_t seed, int sb, float *zu,
                          float *zv, cudaStream_t s)
{
    if (k != 128 && k != 256) {
        set_error("dense operators support k = 128 or 256");
        return SME_ERR_UNSUPPORTED;
    }
    if (op->dense->fp8) {
        double alpha = 0, beta = 0, gamma = 0, M = 0;
        resolve_params(op, alpha, beta, gamma, M);
        return dense_f8_estimate(op, u, v, t, k, seed, sb, alpha, beta, gamma, M, zu, zv, s);
    }
    SME_TRY(ensure_dense_workspace(op, k));
    DenseOp *D = op->dense;
    SME_CUDA(cudaMemcpyAsync(D->x[0], u, D->m * 4, cudaMemcpyDeviceToDevice, s));
    SME_CUDA(cudaMemcpyAsync(D->x[1], v, D->n * 4, cudaMemcpyDeviceToDevice, s));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    dense_build_operand<<<nblk(D->n), 256, 0, s>>>(D->n, k, D->x[1], nullptr, (uint32_t)t, (uint32_t)sb, k0, k1,
                                                   D->Bf[0]);
    dense_build_operand<<<nblk(D->m), 256, 0, s>>>(D->m, k, D->x[0], D->row_scale, (uint32_t)t, (uint32_t)sb + 1u,
                                                   k0, k1, D->Bb[0]);
    double alpha = 0, beta = 0, gamma = 0, M = 0;
    resolve_params(op, alpha, beta, gamma, M);
    DenseArgs a = dense_base(op, alpha, beta, gamma, M, seed, k);
    a.mode = 1;
    a.z[0] = zu ? zu : D->xb[0];  // a NULL output is written into scratch and ignored
    a.z[1] = zv ? zv : D->xb[1];
    return run_dense(op, a, 0, s);
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_op_create_dense(sme_op *out, int64_t m, int64_t n, const void *A, int64_t lda,
                                          sme_dtype dtype, const float *row_scales, int on_device, void *stream)
{
    NvtxRange range("sme dense build");
    if (!out) return SME_ERR_ARG;
    *out = nullptr;
    if (m < 128 || n < 128 || m % 128 || n % 128 || !A || lda < n || m > (1 << 30) || n > (1 << 30)) {
        set_error("sme_op_create_dense: m and n must be positive multiples of 128, lda >= n");
        return SME_ERR_ARG;
    }
    if (m * n / DN_BK > (int64_t)INT32_MAX) {
        set_error("sme_op_create_dense: m * n must be below 2^37 (tile coordinates are 32-bit)");
        return SME_ERR_UNSUPPORTED;
    }
    if (dtype != SME_BF16 && dtype != SME_FP8E4M3) {
        set_error("sme_op_create_dense: dtype must be SME_BF16 or SME_FP8E4M3");
        return SME_ERR_ARG;
    }
    if (dtype == SME_BF16 && row_scales) {
        set_error("sme_op_create_dense: row_scales apply to SME_FP8E4M3 only");
        return SME_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sme_op op = new sme_op_s();
    op->m = m;
    op->n = n;
    op->nnz = m * n;
    op->dtype = dtype;
    op->dbl = false;
    op->dense = new DenseOp();
    DenseOp *D = op->dense;
    D->m = m;
    D->n = n;
    D->fp8 = dtype == SME_FP8E4M3;
    sme_status st = SME_OK;
    auto fail = [&](sme_status e) {
        sme_op_destroy(op);
        return e;
    };
    if ((st = dev_alloc(op, (void **)&op->d_status, sizeof(int))) != SME_OK) return fail(st);
    if (cudaMemsetAsync(op->d_status, 0, sizeof(int), s) != cudaSuccess) return fail(SME_ERR_CUDA);
    if (D->fp8) {
        // E4M3 codes stay E4M3: staged densely (pitch n) on the device, then blocked into A and A^T.
        void *staging = nullptr;
        if (cudaMalloc(&staging, (size_t)m * n) != cudaSuccess) {
            cudaGetLastError();
            return fail(SME_ERR_OOM);
        }
        auto done = [&](sme_status e) {
            cudaStreamSynchronize(s);
            cudaFree(staging);
            return e == SME_OK ? e : fail(e);
        };
        if (cudaMemcpy2DAsync(staging, (size_t)n, A, (size_t)lda, (size_t)n, (size_t)m,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
            return done(SME_ERR_CUDA);
        if (row_scales) {
            if ((st = dev_alloc(op, (void **)&D->row_scale, (size_t)m * 4)) != SME_OK) return done(st);
            if (cudaMemcpyAsync(D->row_scale, row_scales, (size_t)m * 4,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
                return done(SME_ERR_CUDA);
        }
        if ((st = dense_f8_create(op, (const uint8_t *)staging, n, s)) != SME_OK) return done(st);
        int st8 = 0;
        cudaMemcpyAsync(&st8, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e8 = cudaStreamSynchronize(s);
        if (e8 != cudaSuccess) {
            cuda_fail(e8, "sme_op_create_dense", __LINE__);
            return done(SME_ERR_CUDA);
        }
        if (st8 & ST_BAD_VALUE) {
            set_error("sme_op_create_dense: NaN code or non-finite row scale");
            return done(SME_ERR_NONFINITE);
        }
        if ((st = dense_f8_finish_create(op, s)) != SME_OK) return done(st);
        done(SME_OK);
        *out = op;
        return SME_OK;
    }
    if ((st = dev_alloc(op, (void **)&D->A, (size_t)m * n * 2)) != SME_OK) return fail(st);
    if ((st = dev_alloc(op, (void **)&D->At, (size_t)m * n * 2)) != SME_OK) return fail(st);
    const size_t esz = 2;
    const void *src = A;
    void *staging = nullptr;
    if (!on_device || lda != n) {
        // Stage the input densely on the device (copy from host, or repack a strided device matrix).
        if (cudaMalloc(&staging, (size_t)m * lda * esz) != cudaSuccess) {
            cudaGetLastError();
            return fail(SME_ERR_OOM);
        }
        if (cudaMemcpyAsync(staging, A, (size_t)m * lda * esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s) != cudaSuccess) {
            cudaFree(staging);
            return fail(SME_ERR_CUDA);
        }
        src = staging;
    }
    if (lda != n) {
        cudaMemcpy2DAsync(D->A, (size_t)n * 2, src, (size_t)lda * 2, (size_t)n * 2, (size_t)m, cudaMemcpyDeviceToDevice,
                          s);
    } else {
        cudaMemcpyAsync(D->A, src, (size_t)m * n * 2, cudaMemcpyDeviceToDevice, s);
    }
    bf16_check_finite<<<152 * 4, 256, 0, s>>>(D->A, m * n, op->d_status);
    transpose_bf16<<<dim3((unsigned)(n / 32), (unsigned)(m / 32)), dim3(32, 8), 0, s>>>(D->A, m, n, D->At);
    {
        // Both copies into K-blocked order (each TMA tile one contiguous run): A into a new buffer, then A^T
        // into A's old buffer; the row-major A^T is released.
        __nv_bfloat16 *blk = nullptr;
        if ((st = dev_alloc(op, (void **)&blk, (size_t)m * n * 2)) != SME_OK) {
            cudaStreamSynchronize(s);
            if (staging) cudaFree(staging);
            return fail(st);
        }
        block_k64<<<nblk(m * n / 8), 256, 0, s>>>(D->A, m, n, blk);
        block_k64<<<nblk(m * n / 8), 256, 0, s>>>(D->At, n, m, D->A);
        __nv_bfloat16 *row_major_t = D->At;
        D->At = D->A;
        D->A = blk;
        cudaStreamSynchronize(s);
        dev_free(op, row_major_t, (size_t)m * n * 2);
    }
    int st_h = 0;
    cudaMemcpyAsync(&st_h, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (staging) cudaFree(staging);
    if (e != cudaSuccess) {
        cuda_fail(e, "sme_op_create_dense", __LINE__);
        return fail(SME_ERR_CUDA);
    }
    if (st_h & ST_BAD_VALUE) {
        set_error("sme_op_create_dense: non-finite matrix value");
        return fail(SME_ERR_NONFINITE);
    }
    if ((st = make_map_blocked(&D->mapA, D->A, m, n)) != SME_OK) return fail(st);
    if ((st = make_map_blocked(&D->mapAt, D->At, n, m)) != SME_OK) return fail(st);
    *out = op;
    return SME_OK;
}
