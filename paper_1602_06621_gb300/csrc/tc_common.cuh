// Internal helpers of the tensor-core operators (dense.cu: BF16 operands, dense_f8.cu: E4M3 operands):
// mbarrier waits with a bound, TMA copies counted on a barrier of either CTA of a two-SM pair, shared-memory
// matrix descriptors (128-byte swizzle), tcgen05 commits and TMEM loads, tensor-map encoding, and the
// dense operator's state.  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sme_internal.cuh"

namespace sme {

constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;  // polls of a try_wait before a wait is abandoned
constexpr int TC_ROW_BYTES = 128;             // every operand row in shared memory: one 128-byte swizzle row

struct DenseOp {
    bool fp8 = false;
    int64_t m = 0, n = 0;
    // BF16 storage.  A (m x n) and A^T (n x m) in K-blocked order: the 128 x 64 block (row tile t, K-block
    // kb) is one contiguous 16 KB run at ((t * cols/64 + kb) * 128) * 64 elements, rows of 64 inside it.
    __nv_bfloat16 *A = nullptr, *At = nullptr;
    float *row_scale = nullptr;                 // FP8 input: per-row scales (applied in the epilogue)
    __nv_bfloat16 *Bf[2] = {nullptr, nullptr};  // [2k][n]: forward operand (columns' scale x probes)
    __nv_bfloat16 *Bb[2] = {nullptr, nullptr};  // [2k][m]: backward operand
    int kcap = 0;
    float *x[2] = {nullptr, nullptr}, *xb[2] = {nullptr, nullptr};  // u, ubar / v, vbar
    CUtensorMap mapA, mapAt, mapBf[2], mapBb[2];
    // E4M3 storage (fp8): A and A^T as E4M3 codes in K-blocked order with 128-byte K-blocks (the 128 x 128
    // block of row tile t and K-block kb is one contiguous 16 KB run), and single-term E4M3 operands
    // [k][n] / [k][m] holding 2^S e^{x} s (times the row scale on the backward side).
    uint8_t *A8 = nullptr, *At8 = nullptr;
    uint8_t *Bf8[2] = {nullptr, nullptr}, *Bb8[2] = {nullptr, nullptr};
    // Small device block: ordered-key maxima q[3][2] (ring of three iterations, per side), exact operand
    // maxima bmax[2], and the operands' scale exponents S[2][2] (by iteration parity, per side).
    uint32_t *f8_small = nullptr;
    float logc_max = 0.f;  // max_i log|c_i| over the row scales (0 without row scales)
    int kcap8 = 0;
    CUtensorMap mapA8, mapAt8, mapBf8[2], mapBb8[2];
};

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `limit` polls; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bounded wait for phase `parity` of `bar`; false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Shared-memory address, in the cluster window, of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// Copy into this CTA's shared memory whose completion is counted on an mbarrier of either CTA of the
// pair (`bar_cluster`: a cluster-window address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t bar_cluster)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128_u32(uint32_t saddr)
{
    const uint64_t addr = saddr;
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;              // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * TC_ROW_BYTES) >> 4) << 32; // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                    // swizzle mode: 128 bytes
    return d;
}

// Arrives on the mbarrier at `bar`'s offset in every CTA of `mask` once this thread's MMAs have completed.
__device__ __forceinline__ void mma_commit_multicast(uint64_t *bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// ------------------------------------------------------------------ tensor maps (host)

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static inline EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Row-major matrix (rows x cols elements of elem_bytes) viewed with boxes of box_cols x box_rows, 128-byte
// swizzle (box_cols * elem_bytes must be 128).
static inline sme_status tc_make_map(CUtensorMap *map, CUtensorMapDataType dt, const void *base, int64_t rows,
                                     int64_t cols, int elem_bytes, int box_cols, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return SME_ERR_CUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, (void *)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return SME_ERR_CUDA;
    }
    return SME_OK;
}

}  // namespace sme
