// Allocation-free variant of the row-side norm estimator.
//
// Who needs it: code that must not call cudaMalloc/cudaFree on the path where it
// estimates row norms -- for example a caller whose device memory is already
// owned by a caching allocator (a framework pool that reserved the free memory),
// a latency-critical loop that cannot take the device-wide synchronisation an
// allocation or a free may imply, or a plug-in that is handed fixed device
// buffers by a host application that keeps the memory budget to itself.  Such a
// caller passes its own CSR, scalings and output in device memory, and the only
// scratch the computation needs (a gather table with one entry per column:
// e^{v_j} and the probe word of column j) lives in a fixed array inside this
// library instead of being allocated.
//
// The table holds at most SME_STATIC_MAX_COLS entries (8 bytes each, 8 MiB);
// every GPU that loads the library keeps that array for the life of the process.
// Every call on a device shares it and it keeps the last call's contents; each
// call rewrites entries [0, n) before reading them, so nothing has to start at
// zero.  Calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on the array.  A column index outside [0, n) is never used
// to address the table: the row that holds it gets NaN.

#include <cuda_runtime.h>

#include <mutex>

#include "sme_internal.cuh"

namespace sme {

static __device__ __align__(256) uint2 g_static_col_table[SME_STATIC_MAX_COLS];

// Device address of g_static_col_table, per device, resolved on the first call made with that device
// current.  In host code the array's name only stands in for the symbol; it is not a device address.
constexpr int kMaxDevices = 64;
static uint2 *g_table_addr[kMaxDevices] = {};
static std::mutex g_table_mu;

static sme_status static_table_address(uint2 **out)
{
    int dev = 0;
    SME_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("sme_estimate_rows_static: device index %d out of range", dev);
        return SME_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_table_mu);
    if (!g_table_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_col_table);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress for the static table failed: %s", cudaGetErrorString(e));
            return SME_ERR_CUDA;
        }
        g_table_addr[dev] = (uint2 *)p;
    }
    *out = g_table_addr[dev];
    return SME_OK;
}

__global__ void static_fill_table(int64_t n, const float *v, uint32_t t, uint32_t sid, uint32_t k0, uint32_t k1,
                                  uint2 *tab)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t w0, w1;
    probe_words2((uint32_t)j, t, sid, k0, k1, w0, w1);
    tab[j] = make_uint2(__float_as_uint(expf(v[j])), w0);
}

// One thread per row, straight from the caller's CSR: z_u[i] = e^{2 u_i} (1/k) sum_p (sum_j A_ij e^{v_j} s_jp)^2.
// A column index outside [0, n) is skipped (it would address a stale entry, or memory past the array) and
// marks the row: z_u[i] = NaN.
template <int K>
__global__ void static_rows(int64_t m, int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                            const float *u, const uint2 *tab, float *z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float P[K];
#pragma unroll
    for (int p = 0; p < K; ++p) P[p] = 0.f;
    float C = 0.f;
    bool bad = false;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
        const uint32_t j = (uint32_t)col[q];
        if (j >= (uint64_t)n) {
            bad = true;
            continue;
        }
        const uint2 e = tab[j];
        const float y = val[q] * __uint_as_float(e.x);
        C += y;
#pragma unroll
        for (int p = 0; p < K; ++p)
            if (e.y & (1u << p)) P[p] += y;
    }
    float ss = 0.f;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const float yp = C - 2.f * P[p];
        ss += yp * yp;
    }
    const float ex = expf(u[i]);
    z[i] = bad ? __int_as_float(0x7fc00000) : ex * ex * ss * (1.f / (float)K);
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_estimate_rows_static(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                               const float *vals, const float *u, const float *v, int32_t t,
                                               int32_t k, uint64_t seed, int32_t stream_base, float *z_u,
                                               void *stream)
{
    if (m < 1 || n < 1 || !row_ptr || !col_idx || !vals || !u || !v || !z_u || t < 0) {
        set_error("sme_estimate_rows_static: bad arguments");
        return SME_ERR_ARG;
    }
    if (n > SME_STATIC_MAX_COLS) {
        set_error("sme_estimate_rows_static: n = %lld exceeds the static table of %d columns", (long long)n,
                  (int)SME_STATIC_MAX_COLS);
        return SME_ERR_ARG;
    }
    if (k != 1 && k != 2 && k != 4 && k != 8 && k != 16 && k != 32) {
        set_error("sme_estimate_rows_static: k=%d not supported (1,2,4,...,32)", k);
        return SME_ERR_UNSUPPORTED;
    }
    uint2 *tab = nullptr;
    SME_TRY(static_table_address(&tab));
    cudaStream_t s = (cudaStream_t)stream;
    static_fill_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, (uint32_t)t, (uint32_t)stream_base,
                                                                   (uint32_t)seed, (uint32_t)(seed >> 32), tab);
    const unsigned grid = (unsigned)((m + 255) / 256);
    switch (k) {
        case 1: static_rows<1><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
        case 2: static_rows<2><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
        case 4: static_rows<4><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
        case 8: static_rows<8><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
        case 16: static_rows<16><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
        default: static_rows<32><<<grid, 256, 0, s>>>(m, n, row_ptr, col_idx, vals, u, tab, z_u); break;
    }
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}
