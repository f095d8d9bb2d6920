// One-time device construction of the operator: the transposed copy of A (a stable
// radix sort of the nonzeros by column, so rows stay ascending inside each column)
// and the two sliced-ELL layouts used by the products with A and A^T.
//
// Counting uses shared-memory atomics only inside histograms (the counts do not
// depend on the order of the increments); every placement is computed from exact
// prefix sums, so the result is bitwise deterministic.

#include <cuda_runtime.h>

#include <vector>

#include "sme_internal.cuh"

namespace sme {

// ------------------------------------------------------------------ exclusive scan

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix, *total the sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total)
{
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(x);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) warp_tot[SCAN_THREADS / 32] = wi;
    }
    __syncthreads();
    T res = warp_tot[warp] + inc - x;
    *total = warp_tot[SCAN_THREADS / 32];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void scan_tile_sums(const T *in, int64_t n, T *sums)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    T tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block scans the tile sums in place (exclusive), chunk by chunk; sums[ntiles] = total.
template <typename T>
__global__ void scan_sums_single(T *sums, int64_t ntiles)
{
    T carry = 0;
    for (int64_t base = 0; base < ntiles; base += SCAN_THREADS) {
        const int64_t i = base + threadIdx.x;
        T x = i < ntiles ? sums[i] : T(0);
        T tot;
        T ex = block_exclusive_scan<T>(x, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[ntiles] = carry;
}

template <typename T>
__global__ void scan_apply(const T *in, int64_t n, const T *sums, T *out, int64_t ntiles)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : T(0);
        s += v[i];
    }
    T tot;
    T ex = block_exclusive_scan<T>(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) out[n] = sums[ntiles];
}

template <typename T>
static sme_status scan_exclusive(const T *in, T *out, int64_t n, cudaStream_t s)
{
    if (n == 0) {
        SME_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return SME_OK;
    }
    const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc((ntiles + 1) * sizeof(T)));
    T *sums = scratch.as<T>();
    scan_tile_sums<T><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, sums);
    scan_sums_single<T><<<1, SCAN_THREADS, 0, s>>>(sums, ntiles);
    scan_apply<T><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, sums, out, ntiles);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

sme_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s)
{
    return scan_exclusive<int32_t>(in, out, n, s);
}

sme_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_exclusive<int64_t>(in, out, n, s);
}

// ------------------------------------------------------------------ stable LSD radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void rs_histogram(const uint32_t *keys, int64_t n, int shift, int32_t *hist, int64_t ntiles)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Items are ranked in index order (round, then warp, then lane), so equal digits keep their order.
__global__ void rs_scatter(const uint32_t *keys, const int32_t *vals, int64_t n, int shift, const int32_t *offs,
                           int64_t ntiles, uint32_t *keys_out, int32_t *vals_out)
{
    __shared__ int base_cnt[256];
    __shared__ int warp_cnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base_cnt[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) warp_cnt[w][threadIdx.x] = 0;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? keys[i] : 0u;
        const int d = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = base_cnt[d] + rank;
            for (int w = 0; w < warp; ++w) pos += warp_cnt[w][d];
            keys_out[pos] = key;
            vals_out[pos] = vals[i];
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            add += warp_cnt[w][threadIdx.x];
            warp_cnt[w][threadIdx.x] = 0;
        }
        base_cnt[threadIdx.x] += add;
        __syncthreads();
    }
}

sme_status radix_sort_pairs(uint32_t *keys, int32_t *vals, uint32_t *keys_alt, int32_t *vals_alt, int64_t n,
                            int key_bits, cudaStream_t s, bool *result_in_alt)
{
    *result_in_alt = false;
    if (n <= 1 || key_bits <= 0) return SME_OK;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc((256 * ntiles + 1) * sizeof(int32_t)));
    int32_t *hist = scratch.as<int32_t>();
    uint32_t *ki = keys, *ko = keys_alt;
    int32_t *vi = vals, *vo = vals_alt;
    for (int shift = 0; shift < key_bits; shift += 8) {
        rs_histogram<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, n, shift, hist, ntiles);
        SME_TRY(scan_exclusive_i32(hist, hist, 256 * ntiles, s));
        rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, vi, n, shift, hist, ntiles, ko, vo);
        SME_CUDA(cudaGetLastError());
        std::swap(ki, ko);
        std::swap(vi, vo);
        *result_in_alt = !*result_in_alt;
    }
    return SME_OK;
}

// ------------------------------------------------------------------ CSR checks and transposition

template <typename real>
__global__ void validate_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                             const real *val, int *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > m) return;
    if (i == 0 && rp[0] != 0) atomicOr(status, ST_BAD_CSR);
    if (i == m) {
        if (rp[m] != nnz) atomicOr(status, ST_BAD_CSR);
        return;
    }
    const int64_t b = rp[i], e = rp[i + 1];
    if (e < b || b < 0 || e > nnz) {
        atomicOr(status, ST_BAD_CSR);
        return;
    }
    int32_t prev = -1;
    for (int64_t q = b; q < e; ++q) {
        const int32_t c = col[q];
        if (c <= prev || c >= n) atomicOr(status, ST_BAD_CSR);
        prev = c;
        if (!isfinite(val[q])) atomicOr(status, ST_BAD_VALUE);
    }
}

__global__ void row_lengths(const int32_t *rp, int64_t m, int32_t *len, int32_t *row_of)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t b = rp[i], e = rp[i + 1];
    len[i] = e - b;
    for (int32_t q = b; q < e; ++q) row_of[q] = (int32_t)i;
}

__global__ void iota_u32(uint32_t *k, const int32_t *src, int32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    k[i] = (uint32_t)src[i];
    v[i] = (int32_t)i;
}

// col_ptr from column-sorted keys: col_ptr[j] = first sorted position with key >= j.
__global__ void col_ptr_from_sorted(const uint32_t *skeys, int64_t nnz, int64_t n, int32_t *col_ptr)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q > nnz) return;
    const int64_t lo = q == 0 ? 0 : (int64_t)skeys[q - 1] + 1;
    const int64_t hi = q == nnz ? n : (int64_t)skeys[q];
    for (int64_t j = lo; j <= hi; ++j) col_ptr[j] = (int32_t)q;
}

__global__ void lengths_from_ptr(const int32_t *ptr, int64_t n, int32_t *len)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) len[j] = ptr[j + 1] - ptr[j];
}

template <typename real>
__global__ void gather_transpose(const int32_t *sorted_e, const int32_t *row_of, const real *val, int64_t nnz,
                                 int32_t *t_idx, real *t_val)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    const int32_t e = sorted_e[q];
    t_idx[q] = row_of[e];
    t_val[q] = val[e];
}

__global__ void max_i32(const int32_t *x, int64_t n, int *out)
{
    int best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// Sort keys that put longer rows first: key = maxlen - len.
// Sort keys: descending length, optionally after an ascending group id in the high bits (group-major).
__global__ void length_keys(const int32_t *len, int64_t n, int maxlen, const uint32_t *group, int len_bits,
                            uint32_t *k, int32_t *v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = (uint32_t)(maxlen - len[i]);
    k[i] = group ? (group[i] << len_bits) | key : key;
    v[i] = (int32_t)i;
}

__global__ void invert_perm(const int32_t *perm, int64_t n, int32_t *iperm, const int32_t *len_orig,
                            int32_t *len_sorted)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t i = perm[p];
    iperm[i] = (int32_t)p;
    len_sorted[p] = len_orig[i];
}

__global__ void slice_sizes(const int32_t *len_sorted, int64_t rows, int64_t nslices, int32_t *slice_w,
                            int64_t *slice_entries)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    // The longest row of the slice (the first one unless rows are grouped: then a slice that straddles two
    // groups need not start with its longest row).
    int w = 0;
    for (int l = 0; l < 32; ++l) w = max(w, len_sorted[s * 32 + l]);
    w = (w + 1) & ~1;
    slice_w[s] = w;
    slice_entries[s] = (int64_t)w * 32;
}

// Fill the paired sliced-ELL layout from a compressed source (CSR of A or of A^T).
// Padding entries repeat a valid index of the same row (or 0) with value 0.
template <typename real>
__global__ void fill_sell(int64_t rows, const int32_t *perm, const int32_t *src_ptr, const int32_t *src_idx,
                          const real *src_val, const int32_t *other_iperm, const int64_t *slice_off,
                          const int32_t *slice_w, void *ent, double *val64)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nslices = (rows + 31) / 32;
    if (p >= nslices * 32) return;
    const int64_t s = p >> 5;
    const int lane = (int)(p & 31);
    const int w = slice_w[s];
    const int64_t pair_base = slice_off[s] / 2 + lane;
    int32_t b = 0, len = 0;
    if (p < rows) {
        const int32_t i = perm[p];
        b = src_ptr[i];
        len = src_ptr[i + 1] - b;
    }
    int32_t last = 0;
    for (int q = 0; q < w / 2; ++q) {
        int32_t c[2];
        real a[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = 2 * q + h;
            if (l < len) {
                c[h] = other_iperm[src_idx[b + l]];
                a[h] = src_val[b + l];
                last = c[h];
            } else {
                c[h] = last;
                a[h] = real(0);
            }
        }
        const int64_t pi = pair_base + (int64_t)q * 32;
        if (sizeof(real) == 4) {
            int4 e;
            e.x = c[0];
            e.y = __float_as_int((float)a[0]);
            e.z = c[1];
            e.w = __float_as_int((float)a[1]);
            ((int4 *)ent)[pi] = e;
        } else {
            ((int2 *)ent)[pi] = make_int2(c[0], c[1]);
            ((double2 *)val64)[pi] = make_double2((double)a[0], (double)a[1]);
        }
    }
}

static inline unsigned nblk(int64_t n, int t = 256)
{
    return (unsigned)((n + t - 1) / t);
}

// Order rows of a compressed structure by length (descending, stable) and build the sliced ELL.
template <typename real>
static sme_status make_sell(sme_op op, Sell &S, int64_t rows, const int32_t *ptr, const int32_t *idx,
                            const real *val, const int32_t *len_orig, const uint32_t *group, int group_bits,
                            cudaStream_t s)
{
    S.rows = rows;
    S.nslices = (rows + 31) / 32;
    SME_TRY(dev_alloc(op, (void **)&S.perm, rows * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.iperm, rows * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.len, S.nslices * 32 * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.slice_w, S.nslices * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.slice_off, (S.nslices + 1) * sizeof(int64_t)));
    SME_CUDA(cudaMemsetAsync(S.len, 0, S.nslices * 32 * sizeof(int32_t), s));

    AsyncScratch s_max(s), s_k0(s), s_k1(s), s_v1(s), s_sl(s);
    SME_CUDA(s_max.alloc(sizeof(int)));
    int *d_max = s_max.as<int>();
    SME_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), s));
    max_i32<<<152 * 4, 256, 0, s>>>(len_orig, rows, d_max);
    int maxlen = 0;
    SME_CUDA(cudaMemcpyAsync(&maxlen, d_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));

    SME_CUDA(s_k0.alloc(rows * sizeof(uint32_t)));
    SME_CUDA(s_k1.alloc(rows * sizeof(uint32_t)));
    SME_CUDA(s_v1.alloc(rows * sizeof(int32_t)));
    uint32_t *k0 = s_k0.as<uint32_t>(), *k1 = s_k1.as<uint32_t>();
    int32_t *v1 = s_v1.as<int32_t>();
    // Rows in descending length (stable), group-major when groups are given and the key fits 32 bits.
    const int len_bits = std::max(1, bit_length((uint64_t)maxlen));
    if (group && len_bits + group_bits > 32) group = nullptr;
    S.grouped = group != nullptr;
    length_keys<<<nblk(rows), 256, 0, s>>>(len_orig, rows, maxlen, group, len_bits, k0, S.perm);
    bool alt = false;
    SME_TRY(radix_sort_pairs(k0, S.perm, k1, v1, rows, group ? len_bits + group_bits : bit_length((uint64_t)maxlen),
                             s, &alt));
    if (alt) SME_CUDA(cudaMemcpyAsync(S.perm, v1, rows * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    invert_perm<<<nblk(rows), 256, 0, s>>>(S.perm, rows, S.iperm, len_orig, S.len);

    SME_CUDA(s_sl.alloc(S.nslices * sizeof(int64_t)));
    int64_t *sl_entries = s_sl.as<int64_t>();
    slice_sizes<<<nblk(S.nslices), 256, 0, s>>>(S.len, rows, S.nslices, S.slice_w, sl_entries);
    SME_TRY(scan_exclusive_i64(sl_entries, S.slice_off, S.nslices, s));
    SME_CUDA(cudaMemcpyAsync(&S.entries, S.slice_off + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    (void)ptr;
    (void)idx;
    (void)val;
    return SME_OK;
}

template <typename real>
static sme_status fill(sme_op op, Sell &S, const int32_t *ptr, const int32_t *idx, const real *val,
                       const int32_t *other_iperm, cudaStream_t s)
{
    const int64_t pairs = std::max<int64_t>(S.entries / 2, 1);
    if (sizeof(real) == 4) {
        SME_TRY(dev_alloc(op, &S.ent, pairs * sizeof(int4)));
    } else {
        SME_TRY(dev_alloc(op, &S.ent, pairs * sizeof(int2)));
        SME_TRY(dev_alloc(op, (void **)&S.val64, pairs * sizeof(double2)));
    }
    fill_sell<real><<<nblk(S.nslices * 32), 256, 0, s>>>(S.rows, S.perm, ptr, idx, val, other_iperm, S.slice_off,
                                                         S.slice_w, S.ent, S.val64);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

template <typename real>
static sme_status build_sparse_t(sme_op op, const int32_t *rp, const int32_t *col, const real *val,
                                 const uint32_t *row_group, const uint32_t *col_group, int group_bits, cudaStream_t s)
{
    const int64_t m = op->m, n = op->n, nnz = op->nnz;
    SME_CUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
    validate_csr<real><<<nblk(m + 1), 256, 0, s>>>(m, n, nnz, rp, col, val, op->d_status);
    int st = 0;
    SME_CUDA(cudaMemcpyAsync(&st, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    if (st & ST_BAD_CSR) {
        set_error("invalid CSR structure");
        return SME_ERR_INVALID_CSR;
    }
    if (st & ST_BAD_VALUE) {
        set_error("non-finite matrix value");
        return SME_ERR_NONFINITE;
    }

    // Transposed copy: stable sort of the nonzeros by column.
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    AsyncScratch g_row_len(s), g_row_of(s), g_col_len(s), g_col_ptr(s), g_t_idx(s), g_t_val(s), g_k0(s), g_k1(s),
        g_e0(s), g_e1(s);
    SME_CUDA(g_row_len.alloc(m * sizeof(int32_t)));
    SME_CUDA(g_row_of.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_col_len.alloc(n * sizeof(int32_t)));
    SME_CUDA(g_col_ptr.alloc((n + 1) * sizeof(int32_t)));
    SME_CUDA(g_t_idx.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_t_val.alloc(nz1 * sizeof(real)));
    SME_CUDA(g_k0.alloc(nz1 * sizeof(uint32_t)));
    SME_CUDA(g_k1.alloc(nz1 * sizeof(uint32_t)));
    SME_CUDA(g_e0.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_e1.alloc(nz1 * sizeof(int32_t)));
    int32_t *row_len = g_row_len.as<int32_t>(), *row_of = g_row_of.as<int32_t>(), *col_len = g_col_len.as<int32_t>(),
            *col_ptr = g_col_ptr.as<int32_t>(), *t_idx = g_t_idx.as<int32_t>();
    real *t_val = g_t_val.as<real>();
    uint32_t *k0 = g_k0.as<uint32_t>(), *k1 = g_k1.as<uint32_t>();
    int32_t *e0 = g_e0.as<int32_t>(), *e1 = g_e1.as<int32_t>();
    row_lengths<<<nblk(m), 256, 0, s>>>(rp, m, row_len, row_of);
    if (nnz > 0) iota_u32<<<nblk(nnz), 256, 0, s>>>(k0, col, e0, nnz);
    bool alt = false;
    SME_TRY(radix_sort_pairs(k0, e0, k1, e1, nnz, bit_length((uint64_t)(n - 1)), s, &alt));
    const uint32_t *skeys = alt ? k1 : k0;
    const int32_t *se = alt ? e1 : e0;
    col_ptr_from_sorted<<<nblk(nnz + 1), 256, 0, s>>>(skeys, nnz, n, col_ptr);
    lengths_from_ptr<<<nblk(n), 256, 0, s>>>(col_ptr, n, col_len);
    if (nnz > 0) gather_transpose<real><<<nblk(nnz), 256, 0, s>>>(se, row_of, val, nnz, t_idx, t_val);
    SME_CUDA(cudaGetLastError());

    // Length orderings of rows and columns, then the two sliced-ELL copies with renumbered indices.
    SME_TRY(make_sell<real>(op, op->fwd, m, rp, col, val, row_len, row_group, group_bits, s));
    SME_TRY(make_sell<real>(op, op->bwd, n, col_ptr, t_idx, t_val, col_len, col_group, group_bits, s));
    SME_TRY(fill<real>(op, op->fwd, rp, col, val, op->bwd.iperm, s));
    SME_TRY(fill<real>(op, op->bwd, col_ptr, t_idx, t_val, op->fwd.iperm, s));

    SME_CUDA(cudaStreamSynchronize(s));
    return SME_OK;
}

// ------------------------------------------------------------------ one part of a split matrix

// Block of each index: block q holds [len q / parts, len (q + 1) / parts), so block(i) = ((i + 1) parts - 1) / len.
__global__ void block_ids(int64_t len, int32_t parts, uint32_t *blk)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) blk[i] = (uint32_t)(((i + 1) * (int64_t)parts - 1) / len);
}

// Global table position of every index: its block's chunk plus its rank inside the block (the block-major,
// descending-length order `iperm`, whose block q starts at q's first index).
__global__ void global_positions(int64_t len, int32_t parts, int64_t chunk, const int32_t *iperm, int32_t *gpos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int64_t q = ((i + 1) * (int64_t)parts - 1) / len;
    const int64_t start = len * q / parts;
    gpos[i] = (int32_t)(q * chunk + (iperm[i] - start));
}

// The part's rows of the block-major order: perm[r] = order[base + r] (original indices), their lengths and
// the local inverse (iperm[perm[r] - base] = r).
__global__ void sub_order(int64_t rows, int64_t base, const int32_t *order, const int32_t *len_orig, int32_t *perm,
                          int32_t *iperm, int32_t *len_sorted)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = order[base + r];
    perm[r] = i;
    iperm[i - base] = (int32_t)r;
    len_sorted[r] = len_orig[i];
}

// Block-major, descending-length (stable) order of `len` indices: order[p] = original index at position p, and
// its inverse.  Every block's indices form one contiguous range of positions starting at the block's first index.
static sme_status block_major_order(int64_t len, int32_t parts, const int32_t *lens, int32_t *order, int32_t *inv,
                                    cudaStream_t s)
{
    AsyncScratch s_max(s), s_blk(s), s_k0(s), s_k1(s), s_v1(s), s_ls(s);
    SME_CUDA(s_max.alloc(sizeof(int)));
    int *d_max = s_max.as<int>();
    SME_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), s));
    max_i32<<<152 * 4, 256, 0, s>>>(lens, len, d_max);
    int maxlen = 0;
    SME_CUDA(cudaMemcpyAsync(&maxlen, d_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    const int len_bits = std::max(1, bit_length((uint64_t)maxlen));
    const int blk_bits = std::max(1, bit_length((uint64_t)(parts - 1)));
    if (len_bits + blk_bits > 32) {
        set_error("split matrix: row length and part count exceed a 32-bit sort key");
        return SME_ERR_UNSUPPORTED;
    }
    SME_CUDA(s_blk.alloc(len * sizeof(uint32_t)));
    SME_CUDA(s_k0.alloc(len * sizeof(uint32_t)));
    SME_CUDA(s_k1.alloc(len * sizeof(uint32_t)));
    SME_CUDA(s_v1.alloc(len * sizeof(int32_t)));
    SME_CUDA(s_ls.alloc(len * sizeof(int32_t)));
    uint32_t *blk = s_blk.as<uint32_t>(), *k0 = s_k0.as<uint32_t>(), *k1 = s_k1.as<uint32_t>();
    int32_t *v1 = s_v1.as<int32_t>();
    block_ids<<<nblk(len), 256, 0, s>>>(len, parts, blk);
    length_keys<<<nblk(len), 256, 0, s>>>(lens, len, maxlen, blk, len_bits, k0, order);
    bool alt = false;
    SME_TRY(radix_sort_pairs(k0, order, k1, v1, len, len_bits + blk_bits, s, &alt));
    if (alt) SME_CUDA(cudaMemcpyAsync(order, v1, len * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    invert_perm<<<nblk(len), 256, 0, s>>>(order, len, inv, lens, s_ls.as<int32_t>());
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

// Sliced-ELL copy of rows [base, base + rows) of a block-major order.
template <typename real>
static sme_status make_sell_part(sme_op op, Sell &S, int64_t rows, int64_t base, const int32_t *order,
                                 const int32_t *len_orig, cudaStream_t s)
{
    S.rows = rows;
    S.nslices = (rows + 31) / 32;
    SME_TRY(dev_alloc(op, (void **)&S.perm, rows * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.iperm, rows * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.len, S.nslices * 32 * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.slice_w, S.nslices * sizeof(int32_t)));
    SME_TRY(dev_alloc(op, (void **)&S.slice_off, (S.nslices + 1) * sizeof(int64_t)));
    SME_CUDA(cudaMemsetAsync(S.len, 0, S.nslices * 32 * sizeof(int32_t), s));
    sub_order<<<nblk(rows), 256, 0, s>>>(rows, base, order, len_orig, S.perm, S.iperm, S.len);
    AsyncScratch s_sl(s);
    SME_CUDA(s_sl.alloc(S.nslices * sizeof(int64_t)));
    slice_sizes<<<nblk(S.nslices), 256, 0, s>>>(S.len, rows, S.nslices, S.slice_w, s_sl.as<int64_t>());
    SME_TRY(scan_exclusive_i64(s_sl.as<int64_t>(), S.slice_off, S.nslices, s));
    SME_CUDA(cudaMemcpyAsync(&S.entries, S.slice_off + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    return SME_OK;
}

template <typename real>
static sme_status build_shard_t(sme_op op, int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                                const real *val, cudaStream_t s)
{
    ShardInfo &I = *op->shard;
    const int32_t P = I.parts, p = I.part;
    SME_CUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
    validate_csr<real><<<nblk(m + 1), 256, 0, s>>>(m, n, nnz, rp, col, val, op->d_status);
    int st = 0;
    SME_CUDA(cudaMemcpyAsync(&st, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    if (st & ST_BAD_CSR) {
        set_error("invalid CSR structure");
        return SME_ERR_INVALID_CSR;
    }
    if (st & ST_BAD_VALUE) {
        set_error("non-finite matrix value");
        return SME_ERR_NONFINITE;
    }
    // The whole matrix's transpose (the same stable sort by column as an unsplit operator).
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    AsyncScratch g_row_len(s), g_row_of(s), g_col_len(s), g_col_ptr(s), g_t_idx(s), g_t_val(s), g_k0(s), g_k1(s),
        g_e0(s), g_e1(s), g_ord(s), g_inv(s), g_gpos(s);
    SME_CUDA(g_row_len.alloc(m * sizeof(int32_t)));
    SME_CUDA(g_row_of.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_col_len.alloc(n * sizeof(int32_t)));
    SME_CUDA(g_col_ptr.alloc((n + 1) * sizeof(int32_t)));
    SME_CUDA(g_t_idx.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_t_val.alloc(nz1 * sizeof(real)));
    SME_CUDA(g_k0.alloc(nz1 * sizeof(uint32_t)));
    SME_CUDA(g_k1.alloc(nz1 * sizeof(uint32_t)));
    SME_CUDA(g_e0.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_e1.alloc(nz1 * sizeof(int32_t)));
    SME_CUDA(g_ord.alloc((m + n) * sizeof(int32_t)));
    SME_CUDA(g_inv.alloc((m + n) * sizeof(int32_t)));
    SME_CUDA(g_gpos.alloc((m + n) * sizeof(int32_t)));
    int32_t *row_len = g_row_len.as<int32_t>(), *row_of = g_row_of.as<int32_t>(), *col_len = g_col_len.as<int32_t>(),
            *col_ptr = g_col_ptr.as<int32_t>(), *t_idx = g_t_idx.as<int32_t>();
    real *t_val = g_t_val.as<real>();
    uint32_t *k0 = g_k0.as<uint32_t>(), *k1 = g_k1.as<uint32_t>();
    int32_t *e0 = g_e0.as<int32_t>(), *e1 = g_e1.as<int32_t>();
    row_lengths<<<nblk(m), 256, 0, s>>>(rp, m, row_len, row_of);
    if (nnz > 0) iota_u32<<<nblk(nnz), 256, 0, s>>>(k0, col, e0, nnz);
    bool alt = false;
    SME_TRY(radix_sort_pairs(k0, e0, k1, e1, nnz, bit_length((uint64_t)(n - 1)), s, &alt));
    const uint32_t *skeys = alt ? k1 : k0;
    const int32_t *se = alt ? e1 : e0;
    col_ptr_from_sorted<<<nblk(nnz + 1), 256, 0, s>>>(skeys, nnz, n, col_ptr);
    lengths_from_ptr<<<nblk(n), 256, 0, s>>>(col_ptr, n, col_len);
    if (nnz > 0) gather_transpose<real><<<nblk(nnz), 256, 0, s>>>(se, row_of, val, nnz, t_idx, t_val);
    SME_CUDA(cudaGetLastError());

    // Block-major orders of all rows and all columns, and every index's global table position.
    int32_t *ord_r = g_ord.as<int32_t>(), *ord_c = ord_r + m;
    int32_t *inv_r = g_inv.as<int32_t>(), *inv_c = inv_r + m;
    int32_t *gpos_r = g_gpos.as<int32_t>(), *gpos_c = gpos_r + m;
    SME_TRY(block_major_order(m, P, row_len, ord_r, inv_r, s));
    SME_TRY(block_major_order(n, P, col_len, ord_c, inv_c, s));
    global_positions<<<nblk(m), 256, 0, s>>>(m, P, I.rchunk, inv_r, gpos_r);
    global_positions<<<nblk(n), 256, 0, s>>>(n, P, I.cchunk, inv_c, gpos_c);

    // This part: its row block of A and its column block of A^T, indices renumbered to global table positions.
    SME_TRY(make_sell_part<real>(op, op->fwd, I.r1 - I.r0, I.r0, ord_r, row_len, s));
    SME_TRY(make_sell_part<real>(op, op->bwd, I.c1 - I.c0, I.c0, ord_c, col_len, s));
    SME_TRY(fill<real>(op, op->fwd, rp, col, val, gpos_c, s));
    SME_TRY(fill<real>(op, op->bwd, col_ptr, t_idx, t_val, gpos_r, s));
    SME_CUDA(cudaStreamSynchronize(s));
    (void)p;
    return SME_OK;
}

sme_status build_shard(sme_op op, int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                       const void *vals, cudaStream_t s)
{
    if (op->dtype == SME_F64) return build_shard_t<double>(op, m, n, nnz, rp, col, (const double *)vals, s);
    return build_shard_t<float>(op, m, n, nnz, rp, col, (const float *)vals, s);
}

sme_status build_sparse(sme_op op, const int32_t *rp, const int32_t *col, const void *vals, cudaStream_t s,
                        const uint32_t *row_group, const uint32_t *col_group, int group_bits)
{
    if (op->dtype == SME_F64)
        return build_sparse_t<double>(op, rp, col, (const double *)vals, row_group, col_group, group_bits, s);
    return build_sparse_t<float>(op, rp, col, (const float *)vals, row_group, col_group, group_bits, s);
}

}  // namespace sme
