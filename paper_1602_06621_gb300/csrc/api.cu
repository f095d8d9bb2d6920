// C ABI glue: error reporting, operator lifetime, status checks.

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <thread>
#include <vector>

#include "sme_internal.cuh"

namespace sme {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sme_status cuda_fail(cudaError_t e, const char *what, int line)
{
    set_error("CUDA error %d (%s) in %s at line %d", (int)e, cudaGetErrorString(e), what, line);
    return e == cudaErrorMemoryAllocation ? SME_ERR_OOM : SME_ERR_CUDA;
}

// Failure injection for tests: with SME_FAIL_DEV_ALLOC=N in the environment, the (N+1)-th operator allocation
// after the variable was set (or changed) fails as if the device were out of memory.
static bool injected_alloc_failure()
{
    static std::mutex mu;
    static std::string armed;
    static long long calls = 0;
    const char *env = std::getenv("SME_FAIL_DEV_ALLOC");
    std::lock_guard<std::mutex> lock(mu);
    const std::string now = env ? env : "";
    if (now != armed) {
        armed = now;
        calls = 0;
    }
    if (armed.empty()) return false;
    return calls++ == std::atoll(armed.c_str());
}

// ------------------------------------------------------------------ device memory
// Operators are often created and destroyed once per solve, and cudaMalloc / cudaFree of a large
// operator's buffers cost milliseconds.  Blocks of destroyed operators (and the host-input staging of
// operator creation) are therefore kept, by exact size, for the next operator; stream-ordered scratch
// comes from a library memory pool that keeps its memory between calls.  Only blocks whose last use has
// completed enter the cache.  sme_release_cached_memory() returns both to the system, and an allocation
// that fails first releases them and tries again.
namespace {
struct BlockCache {
    using Key = std::pair<int, size_t>;          // (device, bytes)
    std::mutex mu;
    std::unordered_map<void *, Key> live;        // blocks handed out by cache_alloc
    std::multimap<Key, void *> idle;             // retired blocks
    size_t idle_bytes = 0;
};
int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}
BlockCache &block_cache()
{
    static BlockCache *c = new BlockCache();  // never destroyed: blocks may be retired during process exit
    return *c;
}
constexpr size_t CACHE_CAP = size_t(32) << 30;  // idle bytes kept at most
thread_local bool g_retiring = false;           // set by sme_op_destroy after its device synchronisation
}  // namespace

cudaMemPool_t scratch_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

static void release_cached_blocks()
{
    BlockCache &c = block_cache();
    std::vector<void *> blocks;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        for (auto &kv : c.idle) blocks.push_back(kv.second);
        c.idle.clear();
        c.idle_bytes = 0;
    }
    for (void *p : blocks) cudaFree(p);
    if (cudaMemPool_t pool = scratch_pool()) {
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(pool, 0);
    }
}

cudaError_t cache_alloc(void **p, size_t bytes)
{
    BlockCache &c = block_cache();
    const BlockCache::Key key(current_device(), bytes);
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.idle.find(key);
        if (it != c.idle.end()) {
            *p = it->second;
            c.idle.erase(it);
            c.idle_bytes -= bytes;
            c.live[*p] = key;
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        release_cached_blocks();
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lock(c.mu);
    c.live[*p] = key;
    return cudaSuccess;
}

void cache_retire(void *p)
{
    if (!p) return;
    BlockCache &c = block_cache();
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.live.find(p);
        if (it != c.live.end()) {
            const BlockCache::Key key = it->second;
            c.live.erase(it);
            if (c.idle_bytes + key.second <= CACHE_CAP) {
                c.idle.emplace(key, p);
                c.idle_bytes += key.second;
                return;
            }
        }
    }
    cudaFree(p);
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s)
{
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return cudaMallocAsync(p, bytes, s);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        release_cached_blocks();
        e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    }
    return e;
}

sme_status dev_alloc(sme_op op, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_alloc_failure()) {
        set_error("device allocation of %zu bytes failed: injected (SME_FAIL_DEV_ALLOC)", bytes);
        return SME_ERR_OOM;
    }
    cudaError_t e = cache_alloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SME_ERR_OOM;
    }
    op->device_bytes += (int64_t)bytes;
    return SME_OK;
}

// Releases an operator block: kept for reuse while its operator is being destroyed (the device is idle
// then), freed at once otherwise.
void dev_release(void *p)
{
    if (!p) return;
    if (g_retiring) {
        cache_retire(p);
        return;
    }
    {
        BlockCache &c = block_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        c.live.erase(p);
    }
    cudaFree(p);
}

void dev_free(sme_op op, void *p, size_t bytes)
{
    if (!p) return;
    dev_release(p);
    op->device_bytes -= (int64_t)(bytes == 0 ? 16 : bytes);
}

static void free_sell(sme_op op, Sell &S)
{
    for (void *p : {(void *)S.slice_off, (void *)S.slice_w, (void *)S.perm, (void *)S.iperm, (void *)S.len, S.ent,
                    (void *)S.val64})
        dev_release(p);
    S = Sell{};
    (void)op;
}

// Host-side CSR validation (for host input), mirrors the device check.  Rows are checked in parallel
// chunks (threads only for large inputs); the error reported is the one of the lowest failing row.
template <typename real>
static void validate_rows(int64_t r0, int64_t r1, int64_t n, const int32_t *rp, const int32_t *col, const real *val,
                          int64_t *bad_row, int *bad_kind)
{
    for (int64_t i = r0; i < r1; ++i) {
        if (rp[i + 1] < rp[i]) {
            *bad_row = i;
            *bad_kind = 1;
            return;
        }
        int32_t prev = -1;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            if (col[q] <= prev || col[q] >= n) {
                *bad_row = i;
                *bad_kind = 2;
                return;
            }
            prev = col[q];
            if (!std::isfinite((double)val[q])) {
                *bad_row = i;
                *bad_kind = 3;
                return;
            }
        }
    }
}

template <typename real>
static sme_status validate_host(int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                                const real *val)
{
    if (rp[0] != 0 || rp[m] != nnz) {
        set_error("row_ptr must start at 0 and end at nnz");
        return SME_ERR_INVALID_CSR;
    }
    // row_ptr must stay within [0, nnz] before any thread follows it.
    for (int64_t i = 0; i <= m; ++i)
        if (rp[i] < 0 || rp[i] > nnz) {
            set_error("row_ptr out of range at row %lld", (long long)i);
            return SME_ERR_INVALID_CSR;
        }
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = nnz < (1 << 20) ? 1 : (int)std::min<unsigned>(16u, hw);
    std::vector<int64_t> bad_row(nt, -1);
    std::vector<int> bad_kind(nt, 0);
    if (nt == 1) {
        validate_rows<real>(0, m, n, rp, col, val, &bad_row[0], &bad_kind[0]);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) {
            const int64_t r0 = m * t / nt, r1 = m * (t + 1) / nt;
            th.emplace_back(validate_rows<real>, r0, r1, n, rp, col, val, &bad_row[t], &bad_kind[t]);
        }
        for (auto &t : th) t.join();
    }
    for (int t = 0; t < nt; ++t) {
        if (bad_row[t] < 0) continue;
        const long long i = (long long)bad_row[t];
        if (bad_kind[t] == 1) set_error("row_ptr decreases at row %lld", i);
        if (bad_kind[t] == 2) set_error("column index out of range or not increasing in row %lld", i);
        if (bad_kind[t] == 3) set_error("non-finite value in row %lld", i);
        return bad_kind[t] == 3 ? SME_ERR_NONFINITE : SME_ERR_INVALID_CSR;
    }
    return SME_OK;
}

sme_status validate_csr_host(int64_t m, int64_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                             const void *vals, sme_dtype dtype)
{
    return dtype == SME_F64 ? validate_host<double>(m, n, nnz, rp, col, (const double *)vals)
                            : validate_host<float>(m, n, nnz, rp, col, (const float *)vals);
}

// A host check running on its own thread; result() waits for it, report() re-raises its message on the
// calling thread (error messages are per thread).
class HostValidation {
  public:
    template <typename F>
    void start(F &&check)
    {
        running_ = true;
        worker_ = std::thread([this, check] {
            status_ = check();
            if (status_ != SME_OK) message_ = sme_last_error();
        });
    }
    sme_status result()
    {
        if (running_) {
            worker_.join();
            running_ = false;
        }
        return status_;
    }
    sme_status report()
    {
        const sme_status st = result();
        set_error("%s", message_.c_str());
        return st;
    }
    ~HostValidation() { result(); }

  private:
    std::thread worker_;
    bool running_ = false;
    sme_status status_ = SME_OK;
    std::string message_;
};

}  // namespace sme

using namespace sme;

extern "C" const char *sme_status_string(sme_status s)
{
    switch (s) {
        case SME_OK: return "ok";
        case SME_ERR_ARG: return "invalid argument";
        case SME_ERR_INVALID_CSR: return "invalid CSR";
        case SME_ERR_OOM: return "out of device memory";
        case SME_ERR_CUDA: return "CUDA error";
        case SME_ERR_NONFINITE: return "non-finite value";
        case SME_ERR_TIMEOUT: return "device wait timed out";
        case SME_ERR_NOT_CONVERGED: return "not converged";
        case SME_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

extern "C" const char *sme_last_error(void) { return g_err; }

extern "C" sme_status sme_release_cached_memory(void)
{
    release_cached_blocks();
    return SME_OK;
}

extern "C" sme_status sme_op_destroy(sme_op op)
{
    if (!op) return SME_OK;
    cudaDeviceSynchronize();
    g_retiring = true;  // nothing on the device uses this operator's memory any more
    free_sell(op, op->fwd);
    free_sell(op, op->bwd);
    Workspace &W = op->ws;
    for (void *p : {W.u, W.v, W.ub, W.vb, W.tab_u[0], W.tab_u[1], W.tab_v[0], W.tab_v[1], (void *)W.red, W.tgt[0],
                    W.tgt[1], (void *)W.sym_pos})
        dev_release(p);
    release_lsqr(op);
    if (op->graph.exec) cudaGraphExecDestroy(op->graph.exec);
    if (op->graph.stream) cudaStreamDestroy(op->graph.stream);
    if (op->dense) dense_destroy(op);
    delete op->shard;
    if (op->batch) {
        for (int side = 0; side < 2; ++side)
            for (void *p : {(void *)op->batch->mid[side], (void *)op->batch->loc[side], op->batch->tgt2[side]})
                dev_release(p);
        delete[] op->batch->row_off;
        delete[] op->batch->col_off;
        delete op->batch;
    }
    dev_release(op->d_status);
    g_retiring = false;
    for (cudaEvent_t e : op->ev_loop)
        if (e) cudaEventDestroy(e);
    delete op;
    return SME_OK;
}

extern "C" sme_status sme_op_create_csr(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                        const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device,
                                        void *stream)
{
    return create_csr_grouped(out, m, n, nnz, row_ptr, col_idx, vals, dtype, on_device, stream, nullptr, nullptr, 0);
}

extern "C" sme_status sme_op_create_csr_shard(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                              const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device,
                                              int32_t parts, int32_t part, void *stream)
{
    if (parts < 1 || part < 0 || part >= parts || parts > m || parts > n) {
        if (out) *out = nullptr;
        set_error("sme_op_create_csr_shard: need 1 <= parts <= min(m, n) and 0 <= part < parts");
        return SME_ERR_ARG;
    }
    return create_csr_grouped(out, m, n, nnz, row_ptr, col_idx, vals, dtype, on_device, stream, nullptr, nullptr, 0,
                              parts, part);
}

extern "C" sme_status sme_shard_get_info(sme_op op, int32_t k, sme_shard_info *info)
{
    if (!op || !info || k < 1) return SME_ERR_ARG;
    if (!op->shard) {
        set_error("sme_shard_get_info: the operator is not a part of a split matrix");
        return SME_ERR_ARG;
    }
    const ShardInfo &I = *op->shard;
    info->parts = I.parts;
    info->part = I.part;
    info->m = I.gm;
    info->n = I.gn;
    info->row_begin = I.r0;
    info->row_end = I.r1;
    info->col_begin = I.c0;
    info->col_end = I.c1;
    info->row_chunk = I.rchunk;
    info->col_chunk = I.cchunk;
    // Gather-table entries: {e^x, probe words}, 8 bytes for FP32 state with k <= 32, 16 otherwise.
    info->entry_bytes = (!op->dbl && k <= 32) ? 8 : 16;
    return SME_OK;
}

sme_status sme::create_csr_grouped(sme_op *out, int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                   const int32_t *col_idx, const void *vals, sme_dtype dtype, int on_device,
                                   void *stream, const uint32_t *row_group_host, const uint32_t *col_group_host,
                                   int group_bits, int32_t shard_parts, int32_t shard_part)
{
    NvtxRange range("sme build");
    if (!out) return SME_ERR_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || nnz < 0 || nnz > 0x7fffffffLL - 64 || m > 0x7fffffffLL || n > 0x7fffffffLL || !row_ptr ||
        (nnz > 0 && (!col_idx || !vals))) {
        set_error("sme_op_create_csr: bad sizes or null pointers");
        return SME_ERR_ARG;
    }
    if (dtype != SME_F64 && dtype != SME_F32) {
        set_error("sme_op_create_csr: dtype must be SME_F64 or SME_F32");
        return SME_ERR_ARG;
    }
    const size_t vsz = dtype == SME_F64 ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    // Host input is checked on a host thread while the device copies and builds it (the device build
    // checks the same structure first and stops on a violation); an invalid input is reported with the
    // host check's message, also when the device setup fails.
    HostValidation validation;
    if (!on_device)
        validation.start([=] {
            return dtype == SME_F64 ? validate_host<double>(m, n, nnz, row_ptr, col_idx, (const double *)vals)
                                    : validate_host<float>(m, n, nnz, row_ptr, col_idx, (const float *)vals);
        });
    sme_op op = new sme_op_s();
    op->m = m;
    op->n = n;
    op->nnz = nnz;
    op->dtype = dtype;
    op->dbl = dtype == SME_F64;
    if (shard_parts > 0) {
        ShardInfo *I = new ShardInfo();
        I->parts = shard_parts;
        I->part = shard_part;
        I->gm = m;
        I->gn = n;
        I->gnnz = nnz;
        I->r0 = m * shard_part / shard_parts;
        I->r1 = m * (shard_part + 1) / shard_parts;
        I->c0 = n * shard_part / shard_parts;
        I->c1 = n * (shard_part + 1) / shard_parts;
        I->rchunk = (m + shard_parts - 1) / shard_parts;
        I->cchunk = (n + shard_parts - 1) / shard_parts;
        op->shard = I;
    }
    sme_status st = dev_alloc(op, (void **)&op->d_status, sizeof(int));
    if (st != SME_OK) {
        sme_op_destroy(op);
        return validation.result() != SME_OK ? validation.report() : st;
    }
    const int32_t *d_rp = row_ptr, *d_col = col_idx;
    const void *d_val = vals;
    void *tmp[3] = {nullptr, nullptr, nullptr};
    if (!on_device) {
        const size_t bytes[3] = {(size_t)(m + 1) * 4, (size_t)std::max<int64_t>(nnz, 1) * 4,
                                 (size_t)std::max<int64_t>(nnz, 1) * vsz};
        const void *src[3] = {row_ptr, col_idx, vals};
        for (int i = 0; i < 3; ++i) {
            if (cache_alloc(&tmp[i], bytes[i]) != cudaSuccess) {
                cudaGetLastError();
                cudaStreamSynchronize(s);
                for (void *p : tmp) cache_retire(p);
                sme_op_destroy(op);
                if (validation.result() != SME_OK) return validation.report();
                set_error("sme_op_create_csr: staging allocation failed");
                return SME_ERR_OOM;
            }
            if (i == 0 || nnz > 0) cudaMemcpyAsync(tmp[i], src[i], i == 0 ? bytes[0] : (size_t)nnz * (i == 1 ? 4 : vsz),
                                                   cudaMemcpyHostToDevice, s);
        }
        d_rp = (const int32_t *)tmp[0];
        d_col = (const int32_t *)tmp[1];
        d_val = tmp[2];
        // The copies are in flight, and the build below starts without waiting for the host check: the
        // build's first step is the same check on the device, which gates every later kernel, so nothing
        // reads out of bounds on invalid input.  The host check's verdict (its message names the row and
        // the fault) is taken after the build.
    }
    uint32_t *groups[2] = {nullptr, nullptr};
    if (row_group_host && col_group_host) {
        const int64_t len[2] = {m, n};
        const uint32_t *src[2] = {row_group_host, col_group_host};
        for (int i = 0; i < 2; ++i) {
            if (cudaMalloc(&groups[i], (size_t)len[i] * 4) != cudaSuccess) {
                // Without room for the ids the build proceeds ungrouped (same results, other order).
                cudaGetLastError();
                if (groups[0]) cudaFree(groups[0]);
                groups[0] = groups[1] = nullptr;
                break;
            }
            cudaMemcpyAsync(groups[i], src[i], (size_t)len[i] * 4, cudaMemcpyHostToDevice, s);
        }
    }
    if (op->shard) {
        st = build_shard(op, m, n, nnz, d_rp, d_col, d_val, s);
        op->m = op->shard->r1 - op->shard->r0;
        op->n = op->shard->c1 - op->shard->c0;
    } else {
        st = build_sparse(op, d_rp, d_col, d_val, s, groups[0], groups[1], groups[0] && groups[1] ? group_bits : 0);
    }
    cudaStreamSynchronize(s);
    for (void *p : tmp) cache_retire(p);  // the copies and the build that read them have completed
    for (void *p : groups)
        if (p) cudaFree(p);
    if (validation.result() != SME_OK) {
        sme_op_destroy(op);
        return validation.report();
    }
    if (st != SME_OK) {
        sme_op_destroy(op);
        return st;
    }
    *out = op;
    return SME_OK;
}

extern "C" sme_status sme_op_get_info(sme_op op, sme_op_info *info)
{
    if (!op || !info) return SME_ERR_ARG;
    info->m = op->m;
    info->n = op->n;
    info->nnz = op->nnz;
    info->dtype = (int32_t)op->dtype;
    info->state_is_double = op->dbl ? 1 : 0;
    info->device_bytes = op->device_bytes;
    info->padded_entries_fwd = op->fwd.entries;
    info->padded_entries_bwd = op->bwd.entries;
    info->last_loop_ms = 0.0;
    info->last_loop_iters = 0;
    if (op->loop_timed) {
        float ms = 0.f;
        SME_CUDA(cudaEventSynchronize(op->ev_loop[1]));
        SME_CUDA(cudaEventElapsedTime(&ms, op->ev_loop[0], op->ev_loop[1]));
        info->last_loop_ms = ms;
        info->last_loop_iters = op->loop_iters;
    }
    return SME_OK;
}

extern "C" sme_status sme_op_check(sme_op op, void *stream)
{
    if (!op) return SME_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    SME_CUDA(cudaMemcpyAsync(&st, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    SME_CUDA(cudaStreamSynchronize(s));
    if (st) SME_CUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
    if (st & ST_TIMEOUT) {
        set_error("a device-side wait timed out");
        return SME_ERR_TIMEOUT;
    }
    if (st & ST_NONFINITE) {
        set_error("an iterate became non-finite");
        return SME_ERR_NONFINITE;
    }
    return SME_OK;
}
