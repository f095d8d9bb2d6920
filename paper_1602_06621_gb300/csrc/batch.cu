// Batches of sparse matrices equilibrated together.
//
// The batch is held as ONE block-diagonal operator diag(A_0, ..., A_{B-1}): its rows (and columns) are
// sorted by length across all matrices, so one launch per iteration (and one captured graph for all T
// iterations) serves every matrix, and matrices of very different sizes share the same slices instead
// of each leaving the GPU mostly idle.  Per sorted row and column the operator keeps the matrix id and
// the index inside that matrix; the iteration kernel uses them for the matrix's own alpha^2 / beta^2 and
// for the Philox counter, so matrix b draws exactly the probes a separate run with stream_base = 2b
// (plus the batch's own base) would draw, and its result is the same bit for bit.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sme_internal.cuh"

namespace sme {

__global__ void gather_meta(int64_t rows, const int32_t *perm, const int32_t *mid_orig, const int32_t *loc_orig,
                            int32_t *mid, int32_t *loc)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = perm[r];
    mid[r] = mid_orig[i];
    loc[r] = loc_orig[i];
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_batch_destroy(sme_batch b)
{
    if (!b) return SME_OK;
    sme_op_destroy(b->op);
    delete b;
    return SME_OK;
}

extern "C" sme_status sme_batch_create(sme_batch *out, int32_t count, const int64_t *m, const int64_t *n,
                                       const int32_t *const *row_ptr, const int32_t *const *col_idx,
                                       const void *const *vals, sme_dtype dtype, void *stream)
{
    NvtxRange range("sme batch build");
    if (!out) return SME_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !m || !n || !row_ptr || !col_idx || !vals || (dtype != SME_F32 && dtype != SME_F64)) {
        set_error("sme_batch_create: bad arguments");
        return SME_ERR_ARG;
    }
    const size_t vsz = dtype == SME_F64 ? 8 : 4;
    std::vector<int64_t> roff(count + 1, 0), coff(count + 1, 0), zoff(count + 1, 0);
    for (int32_t b = 0; b < count; ++b) {
        if (m[b] < 1 || n[b] < 1 || !row_ptr[b]) {
            set_error("sme_batch_create: matrix %d has bad sizes", b);
            return SME_ERR_ARG;
        }
        const int64_t nnz = row_ptr[b][m[b]];
        if (nnz > 0 && (!col_idx[b] || !vals[b])) {
            set_error("sme_batch_create: matrix %d has null arrays", b);
            return SME_ERR_ARG;
        }
        sme_status st = validate_csr_host(m[b], n[b], nnz, row_ptr[b], col_idx[b], vals[b], dtype);
        if (st != SME_OK) {
            set_error("sme_batch_create: matrix %d: %s", b, sme_last_error());
            return st;
        }
        roff[b + 1] = roff[b] + m[b];
        coff[b + 1] = coff[b] + n[b];
        zoff[b + 1] = zoff[b] + nnz;
    }
    const int64_t M = roff[count], N = coff[count], NNZ = zoff[count];
    if (M > 0x7fffffffLL || N > 0x7fffffffLL || NNZ > 0x7fffffffLL - 64) {
        set_error("sme_batch_create: the batch exceeds 2^31 rows, columns or nonzeros");
        return SME_ERR_ARG;
    }
    // The block-diagonal CSR, and for every original row / column its matrix and local index.
    std::vector<int32_t> rp(M + 1), ci(std::max<int64_t>(NNZ, 1)), mid_r(M), loc_r(M), mid_c(N), loc_c(N);
    std::vector<uint8_t> va(std::max<int64_t>(NNZ, 1) * vsz);
    for (int32_t b = 0; b < count; ++b) {
        for (int64_t i = 0; i < m[b]; ++i) {
            rp[roff[b] + i] = (int32_t)(zoff[b] + row_ptr[b][i]);
            mid_r[roff[b] + i] = b;
            loc_r[roff[b] + i] = (int32_t)i;
        }
        const int64_t nnz = zoff[b + 1] - zoff[b];
        for (int64_t q = 0; q < nnz; ++q) ci[zoff[b] + q] = (int32_t)(col_idx[b][q] + coff[b]);
        if (nnz) std::memcpy(va.data() + zoff[b] * vsz, vals[b], (size_t)nnz * vsz);
        for (int64_t j = 0; j < n[b]; ++j) {
            mid_c[coff[b] + j] = b;
            loc_c[coff[b] + j] = (int32_t)j;
        }
    }
    rp[M] = (int32_t)NNZ;
    // Rows and columns are laid out group-major (then by length), so the CTAs running at any moment gather
    // from one group's tables and those stay cached.  By default every matrix is its own group: its slices
    // then form one contiguous range (at most one partially filled slice per matrix), which also lets
    // per-matrix work such as LSQR skip finished matrices' slices altogether.  SME_BATCH_GROUP_BYTES > 0
    // packs consecutive matrices into groups whose gather tables (8 bytes per row and per column) fit that
    // many bytes instead.
    int64_t group_bytes = 0;
    if (const char *env = std::getenv("SME_BATCH_GROUP_BYTES")) {
        const long long v = std::atoll(env);
        if (v > 0) group_bytes = v;
    }
    std::vector<uint32_t> gr(M), gc(N);
    uint32_t g = 0;
    int64_t acc = 0;
    for (int32_t b = 0; b < count; ++b) {
        const int64_t bytes = 8 * (m[b] + n[b]);
        if (b > 0 && (group_bytes == 0 || acc + bytes > group_bytes)) {
            ++g;
            acc = 0;
        }
        acc += bytes;
        for (int64_t i = roff[b]; i < roff[b + 1]; ++i) gr[i] = g;
        for (int64_t j = coff[b]; j < coff[b + 1]; ++j) gc[j] = g;
    }
    int gbits = 0;
    while ((1u << gbits) <= g) ++gbits;
    sme_op op = nullptr;
    sme_status st = g > 0 ? create_csr_grouped(&op, M, N, NNZ, rp.data(), ci.data(), va.data(), dtype, 0, stream,
                                               gr.data(), gc.data(), gbits)
                          : sme_op_create_csr(&op, M, N, NNZ, rp.data(), ci.data(), va.data(), dtype, 0, stream);
    if (st != SME_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    BatchInfo *B = new BatchInfo();
    op->batch = B;
    B->count = count;
    B->matrix_major = group_bytes == 0 && count > 1 && op->fwd.grouped && op->bwd.grouped;
    B->row_off = new int64_t[count + 1];
    B->col_off = new int64_t[count + 1];
    std::memcpy(B->row_off, roff.data(), (count + 1) * sizeof(int64_t));
    std::memcpy(B->col_off, coff.data(), (count + 1) * sizeof(int64_t));
    auto fail = [&](sme_status e) {
        sme_op_destroy(op);
        return e;
    };
    const int64_t len[2] = {M, N};
    const std::vector<int32_t> *mo[2] = {&mid_r, &mid_c}, *lo[2] = {&loc_r, &loc_c};
    for (int side = 0; side < 2; ++side) {
        if ((st = dev_alloc(op, (void **)&B->mid[side], len[side] * 4)) != SME_OK) return fail(st);
        if ((st = dev_alloc(op, (void **)&B->loc[side], len[side] * 4)) != SME_OK) return fail(st);
        if ((st = dev_alloc(op, &B->tgt2[side], (size_t)count * vsz)) != SME_OK) return fail(st);
        int32_t *tm = nullptr, *tl = nullptr;
        if (cudaMalloc(&tm, len[side] * 4) != cudaSuccess || cudaMalloc(&tl, len[side] * 4) != cudaSuccess) {
            cudaGetLastError();
            if (tm) cudaFree(tm);
            return fail(SME_ERR_OOM);
        }
        cudaMemcpyAsync(tm, mo[side]->data(), len[side] * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(tl, lo[side]->data(), len[side] * 4, cudaMemcpyHostToDevice, s);
        const Sell &S = side == 0 ? op->fwd : op->bwd;
        gather_meta<<<nblk(len[side]), 256, 0, s>>>(len[side], S.perm, tm, tl, B->mid[side], B->loc[side]);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(tm);
        cudaFree(tl);
        if (e != cudaSuccess) {
            cuda_fail(e, "sme_batch_create", __LINE__);
            return fail(SME_ERR_CUDA);
        }
    }
    sme_batch bt = new sme_batch_s();
    bt->op = op;
    *out = bt;
    return SME_OK;
}

extern "C" sme_status sme_batch_get_info(sme_batch b, int32_t *count, int64_t *row_off, int64_t *col_off)
{
    if (!b) return SME_ERR_ARG;
    const BatchInfo *B = b->op->batch;
    if (count) *count = B->count;
    if (row_off) std::memcpy(row_off, B->row_off, (B->count + 1) * sizeof(int64_t));
    if (col_off) std::memcpy(col_off, B->col_off, (B->count + 1) * sizeof(int64_t));
    return SME_OK;
}

extern "C" sme_status sme_batch_equilibrate(sme_batch b, const sme_equil_params *p, void *u, void *v, void *u_bar,
                                            void *v_bar, void *stream)
{
    NvtxRange range("sme batch equilibrate");
    if (!b || !p || !u || !v || !u_bar || !v_bar || p->T < 0 || p->t_begin < 1 || p->t0 < 0) {
        set_error("sme_batch_equilibrate: bad arguments");
        return SME_ERR_ARG;
    }
    if (!probes_supported(p->k)) {
        set_error("sme_batch_equilibrate: k=%d not supported (1,2,4,...,64)", p->k);
        return SME_ERR_UNSUPPORTED;
    }
    sme_op op = b->op;
    BatchInfo *B = op->batch;
    cudaStream_t s = (cudaStream_t)stream;
    // Targets per matrix: the given alpha / beta for all, or each matrix's (n/m)^(1/4), (m/n)^(1/4).
    std::vector<double> t2[2];
    for (int side = 0; side < 2; ++side) t2[side].resize(B->count);
    for (int32_t i = 0; i < B->count; ++i) {
        const double mi = (double)(B->row_off[i + 1] - B->row_off[i]), ni = (double)(B->col_off[i + 1] - B->col_off[i]);
        const double al = p->alpha > 0 ? p->alpha : std::pow(ni / mi, 0.25);
        const double be = p->beta > 0 ? p->beta : std::pow(mi / ni, 0.25);
        t2[0][i] = al * al;
        t2[1][i] = be * be;
    }
    for (int side = 0; side < 2; ++side) {
        if (op->dbl) {
            SME_CUDA(cudaMemcpyAsync(B->tgt2[side], t2[side].data(), B->count * 8, cudaMemcpyHostToDevice, s));
        } else {
            std::vector<float> f(t2[side].begin(), t2[side].end());
            SME_CUDA(cudaMemcpyAsync(B->tgt2[side], f.data(), B->count * 4, cudaMemcpyHostToDevice, s));
            SME_CUDA(cudaStreamSynchronize(s));
        }
    }
    // First call with this k: choose the launch shape for this batch (sme_op_autotune).
    int slot = 0;
    while ((1 << slot) < p->k) ++slot;
    if (op->tuned[slot].spc == 0) SME_TRY(autotune_sparse(op, p->k, s, nullptr, nullptr, nullptr));
    SME_TRY(equilibrate_sparse(op, p, u, v, u_bar, v_bar, s));
    if (p->flags & SME_EQ_ASYNC) return SME_OK;
    return sme_op_check(op, stream);
}

extern "C" sme_status sme_batch_estimate(sme_batch b, const void *u, const void *v, int32_t t, int32_t k, uint64_t seed,
                                         int32_t stream_base, void *z_u, void *z_v, void *stream)
{
    if (!b || !u || !v || t < 0) {
        set_error("sme_batch_estimate: bad arguments");
        return SME_ERR_ARG;
    }
    if (!probes_supported(k)) {
        set_error("sme_batch_estimate: k=%d not supported", k);
        return SME_ERR_UNSUPPORTED;
    }
    return estimate_sparse(b->op, u, v, t, k, seed, stream_base, z_u, z_v, (cudaStream_t)stream);
}

extern "C" sme_status sme_batch_op(sme_batch b, sme_op *op)
{
    if (!b || !op) return SME_ERR_ARG;
    *op = b->op;
    return SME_OK;
}
