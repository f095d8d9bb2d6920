// Internal declarations shared by the CUDA translation units of libsme.
// Nothing here is part of the C ABI (see include/sme.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "sme.h"

namespace sme {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
sme_status cuda_fail(cudaError_t e, const char *what, int line);

#define SME_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return ::sme::cuda_fail(_e, #call, __LINE__); \
    } while (0)

#define SME_TRY(call)                        \
    do {                                     \
        sme_status _s = (call);              \
        if (_s != SME_OK) return _s;         \
    } while (0)

// Device memory (api.cu).  cache_alloc / cache_retire: blocks reused by exact size once retired (only
// after their last use has completed); scratch_alloc: stream-ordered memory from the library's pool.
cudaError_t cache_alloc(void **p, size_t bytes);
void cache_retire(void *p);
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);

// Stream-ordered scratch that is released when its scope ends, on every return path (including the early
// returns of SME_CUDA / SME_TRY).
struct AsyncScratch {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    explicit AsyncScratch(cudaStream_t st) : s(st) {}
    ~AsyncScratch()
    {
        if (p) cudaFreeAsync(p, s);
    }
    AsyncScratch(const AsyncScratch &) = delete;
    AsyncScratch &operator=(const AsyncScratch &) = delete;
    cudaError_t alloc(size_t bytes) { return scratch_alloc(&p, bytes, s); }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// A pair of timing events destroyed with their scope.
struct EventPair {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~EventPair()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
    cudaError_t create()
    {
        cudaError_t r = cudaEventCreate(&e[0]);
        return r == cudaSuccess ? cudaEventCreate(&e[1]) : r;
    }
};

// An NVTX range around one phase of a call ("sme build", "sme equilibrate", ...), visible to profilers;
// without a profiler attached the calls are no-ops.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device status word bits (set by kernels, read by sme_op_check).
enum : int {
    ST_NONFINITE = 1,
    ST_BAD_CSR = 2,
    ST_BAD_VALUE = 4,
    ST_TIMEOUT = 8,
};

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of
// two 32x32->64 multiplies with a Weyl-sequence key schedule.
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#if defined(__CUDA_ARCH__)
    lo = a * b;
    hi = __umulhi(a, b);
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mulhilo32(0xD2511F53u, c.x, h0, l0);
        mulhilo32(0xCD9E8D57u, c.z, h1, l1);
        c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// First two 32-bit probe words (probes 0..63) at `index` for iteration t and Philox stream `sid`.
__host__ __device__ __forceinline__ void probe_words2(uint32_t index, uint32_t t, uint32_t sid, uint32_t k0,
                                                      uint32_t k1, uint32_t &w0, uint32_t &w1)
{
    U4 o = philox10(U4{index, t, sid, 0u}, k0, k1);
    w0 = o.x;
    w1 = o.y;
}

// ------------------------------------------------------------------ operator

// Sliced ELL with 32-row slices, rows in descending-length order ("sorted position").
// Entries of slice s are stored in pairs of consecutive steps so that one 16-byte
// load serves two steps of one row:
//   pair q of lane r of slice s  ->  pair index slice_off[s]/2 + q*32 + r
// FP32: int4 {col0, val0_bits, col1, val1_bits};  FP64: int2 {col0, col1} + double2 {val0, val1}.
// Column (row) indices stored are SORTED positions of the other dimension.
struct Sell {
    int64_t rows = 0;       // logical rows (m for A, n for A^T)
    int64_t nslices = 0;
    int64_t entries = 0;    // incl. padding
    int64_t *slice_off = nullptr;  // [nslices + 1], entry offsets (multiples of 64)
    int32_t *slice_w = nullptr;    // [nslices], even widths
    int32_t *perm = nullptr;       // sorted position -> original index
    int32_t *iperm = nullptr;      // original index -> sorted position
    int32_t *len = nullptr;        // [rows] length at each sorted position
    void *ent = nullptr;           // see above
    double *val64 = nullptr;       // FP64 values (double2 pairs), FP64 ops only
    bool grouped = false;          // rows ordered group-major (see build_sparse)
};

struct Workspace {
    // Equilibration state in sorted order and the double-buffered gather tables.
    void *u = nullptr, *v = nullptr, *ub = nullptr, *vb = nullptr;
    void *tab_u[2] = {nullptr, nullptr};
    void *tab_v[2] = {nullptr, nullptr};
    int64_t tab_bytes_u = 0, tab_bytes_v = 0;
    // LSQR vectors and FP64 reduction scratch.
    void *lsqr = nullptr;
    int64_t lsqr_bytes = 0;
    double *red = nullptr;
    int64_t red_len = 0;
    // Varying-norm targets (sorted order) and the symmetric row -> column map.
    void *tgt[2] = {nullptr, nullptr};
    bool use_tgt = false;
    int32_t *sym_pos = nullptr;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    int64_t key[12] = {0};       // parameters of the captured graph
    int64_t last_direct[12] = {0};  // parameters of the last call launched directly
    bool have_direct = false;
};

struct DenseOp;  // tensor-core operator (dense A)

// One part of a matrix split over several devices (shard.cu, build_kernels.cu): rows and columns are cut into
// `parts` contiguous blocks, block q = [n q / parts, n (q + 1) / parts).  This part owns row block `part` of A
// (its forward products) and column block `part` of A^T (its backward products).  The gather tables of the
// whole matrix are laid out block-major in chunks of row_chunk (col_chunk) entries, chunk q at q * chunk, each
// block's rows in descending-length order inside its chunk; the sliced-ELL copies of the part store these
// global table positions.  The op's m, n are the part's block sizes.
struct ShardInfo {
    int32_t parts = 1, part = 0;
    int64_t gm = 0, gn = 0, gnnz = 0;       // the whole matrix
    int64_t r0 = 0, r1 = 0, c0 = 0, c1 = 0;  // this part's rows [r0, r1) and columns [c0, c1)
    int64_t rchunk = 0, cchunk = 0;          // table entries per part (the largest block)
    int32_t begun_kw = 0;                    // probe words per table entry of the last sme_shard_begin (0: none)
};

// A batch of matrices held as one block-diagonal operator (batch.cu).
struct BatchInfo {
    int32_t count = 0;
    int32_t *mid[2] = {nullptr, nullptr};  // matrix id per sorted row [0] / sorted column [1]
    int32_t *loc[2] = {nullptr, nullptr};  // index inside its matrix
    void *tgt2[2] = {nullptr, nullptr};    // per matrix alpha^2 [0], beta^2 [1] (state type)
    uint32_t sid_base = 0;                 // Philox stream of matrix b: sid_base + 2b (s), + 2b + 1 (w)
    int64_t *row_off = nullptr, *col_off = nullptr;  // host, count + 1
    // One group per matrix on both sides: matrix b's rows then occupy sorted positions row_off[b] ..
    // row_off[b+1]-1 (columns likewise), so its slices form one contiguous range.
    bool matrix_major = false;
};

}  // namespace sme

struct sme_op_s {
    int64_t m = 0, n = 0, nnz = 0;
    sme_dtype dtype = SME_F32;
    bool dbl = false;  // state vectors in double
    sme::Sell fwd, bwd;
    sme::Workspace ws;
    sme::GraphCache graph;
    sme::DenseOp *dense = nullptr;
    sme::BatchInfo *batch = nullptr;
    sme::ShardInfo *shard = nullptr;
    int *d_status = nullptr;
    int64_t device_bytes = 0;
    struct {
        int spc = 0, cols_first = 0;
    } tuned[8];                                    // launch shape per log2(k), 0 = default
    cudaEvent_t ev_loop[2] = {nullptr, nullptr};  // SME_EQ_TIMED
    bool loop_timed = false;
    int64_t loop_iters = 0;
};

struct sme_batch_s {
    sme_op op = nullptr;  // the block-diagonal operator (owned)
};

namespace sme {

// Device allocation bookkeeping for an op.
sme_status dev_alloc(sme_op op, void **p, size_t bytes);
void dev_free(sme_op op, void *p, size_t bytes);
// Releases a dev_alloc block without accounting (the operator is being destroyed, or the caller keeps
// the count): kept for reuse inside sme_op_destroy, freed at once elsewhere.
void dev_release(void *p);

// Build-time device utilities (build_kernels.cu).
sme_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);  // out[n] = total
sme_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);  // out[n] = total
sme_status radix_sort_pairs(uint32_t *keys, int32_t *vals, uint32_t *keys_alt, int32_t *vals_alt, int64_t n,
                            int key_bits, cudaStream_t s, bool *result_in_alt);
// Builds both sliced-ELL copies.  row_group / col_group (device, optional, one id per original row / column,
// ids < 2^group_bits): rows are ordered group-major (ascending id), then by descending length.
sme_status build_sparse(sme_op op, const int32_t *d_row_ptr, const int32_t *d_col, const void *d_vals,
                        cudaStream_t s, const uint32_t *row_group = nullptr, const uint32_t *col_group = nullptr,
                        int group_bits = 0);
// Builds the two sliced-ELL copies of one part of a split matrix (see ShardInfo) from the whole matrix's CSR
// (m x n, nnz on the device); fills op->shard's blocks and chunks and sets op->m, op->n to the part's sizes.
sme_status build_shard(sme_op op, int64_t m, int64_t n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                       const void *d_vals, cudaStream_t s);
// sme_op_create_csr with optional host group ids (see build_sparse); used for batches.
sme_status create_csr_grouped(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                              const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device, void *stream,
                              const uint32_t *row_group_host, const uint32_t *col_group_host, int group_bits,
                              int32_t shard_parts = 0, int32_t shard_part = 0);

// Equilibration / estimation launches (equilibrate.cu).
sme_status ensure_equil_workspace(sme_op op, int kw);
sme_status equilibrate_sparse(sme_op op, const sme_equil_params *p, void *u, void *v, void *ub, void *vb,
                              cudaStream_t s);
sme_status estimate_sparse(sme_op op, const void *u, const void *v, int t, int k, uint64_t seed, int sb, void *zu,
                           void *zv, cudaStream_t s);
bool probes_supported(int k);
sme_status autotune_sparse(sme_op op, int k, cudaStream_t s, int *spc, int *cols_first, float *ms);

// Host-side CSR validation (api.cu).
sme_status validate_csr_host(int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                             const void *vals, sme_dtype dtype);

// LSQR and evaluation (lsqr.cu).
void release_lsqr(sme_op op);

// Dense tensor-core operator (dense.cu).
void dense_destroy(sme_op op);
sme_status dense_equilibrate(sme_op op, const sme_equil_params *p, float *u, float *v, float *ub, float *vb,
                             cudaStream_t s);
// Exact squared row / column norms of D A E (FP64 accumulation) for a dense operator; sq_u[m], sq_v[n] scratch.
sme_status dense_exact_norms(sme_op op, const float *u, const float *v, double *sq_u, double *sq_v, double *r2,
                             double *c2, cudaStream_t s);
sme_status dense_estimate(sme_op op, const float *u, const float *v, int t, int k, uint64_t seed, int sb,
                          float *zu, float *zv, cudaStream_t s);

// Entry points that run the whole-matrix kernels refuse one part of a split matrix: its sliced-ELL indices are
// positions in the whole matrix's tables, which only the sme_shard_* calls provide.
inline sme_status no_shard(sme_op op, const char *where)
{
    if (op && op->shard) {
        set_error("%s: the operator is one part of a split matrix (drive it with sme_shard_*)", where);
        return SME_ERR_UNSUPPORTED;
    }
    return SME_OK;
}

inline int bit_length(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

}  // namespace sme
