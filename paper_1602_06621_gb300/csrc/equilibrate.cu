// Algorithm 1 (projected stochastic gradient for eq. (3)) on the device.
//
// One launch performs one iteration t.  Its CTAs split into two groups:
//   rows    (A, sliced ELL):    z_u[i] = (1/k) sum_p ( e^{u_i} sum_j A_ij e^{v_j} s_jp )^2
//   columns (A^T, sliced ELL):  z_v[j] = (1/k) sum_p ( e^{v_j} sum_i A_ij e^{u_i} w_ip )^2
// and every thread owns one row (one column), so the square-and-reduce over the
// k probes, the projected step, the running average and the next iteration's
// probe words all happen in registers right after the row's products.
//
// Both groups read the PREVIOUS iterate through double-buffered gather tables
// (entry = { e^{x}, probe words }) and write the next table, so the u- and v-steps
// of one iteration never see each other's new values (D and E are formed once
// at the top of the iteration in Algorithm 1).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sme_internal.cuh"

namespace sme {

constexpr int DEFAULT_SPC = 8;  // 32-row slices per CTA unless the autotuner chose otherwise

struct SellArgs {
    const int64_t *slice_off;
    const int32_t *slice_w;
    const void *ent;
    const double *val64;
    const int32_t *perm;
    int64_t rows, nslices;
};

template <typename real>
struct StepArgs {
    SellArgs A[2];          // [0] rows of A, [1] rows of A^T (columns of A)
    const void *tab_in[2];  // [0] column table (read by rows), [1] row table (read by columns)
    void *tab_out[2];       // [0] next row table (written by rows), [1] next column table
    real *x[2];             // [0] u, [1] v, sorted order
    real *xb[2];            // averages, sorted order
    real *z[2];             // estimate-only outputs, original order
    real target2[2];        // alpha^2, beta^2
    real gamma, M, eta, avg_new, avg_old;
    uint32_t t_next, key0, key1;
    uint32_t sid_out[2];    // Philox stream of the table each side writes: rows -> w, columns -> s
    int64_t blocks0;        // CTAs of the first group
    int cols_first;         // 1: the first group is the column side
    int split[2];           // warps per slice, rows [0] / columns [1] (1, 2, 4 or 8, dividing SPC)
    int mode;               // 0: full step, 1: estimate only
    int *status;
    // Batches of matrices (block-diagonal operator): per sorted row / column the matrix id and the
    // index inside that matrix, per matrix the squared targets; null for a single matrix.
    const int32_t *mid[2];
    const int32_t *loc[2];
    const real *tgt2[2];
    uint32_t sid_base;
    // Varying norms: squared targets per sorted row [0] / column [1], or null.
    const real *tgt_row[2];
    // Symmetric equilibration (mode 2): sorted column position of each sorted row's index.
    const int32_t *sym_pos;
};

// ------------------------------------------------------------------ gather tables

template <typename real, int KW>
struct TabEntry;

template <>
struct TabEntry<float, 1> {
    static constexpr int bytes = 8;
    __device__ __forceinline__ static void load(const void *t, int32_t i, float &x, uint32_t (&w)[1])
    {
        const uint2 e = __ldg((const uint2 *)t + i);
        x = __uint_as_float(e.x);
        w[0] = e.y;
    }
    __device__ __forceinline__ static void store(void *t, int64_t i, float x, uint32_t w0, uint32_t)
    {
        ((uint2 *)t)[i] = make_uint2(__float_as_uint(x), w0);
    }
};

template <>
struct TabEntry<float, 2> {
    static constexpr int bytes = 16;
    __device__ __forceinline__ static void load(const void *t, int32_t i, float &x, uint32_t (&w)[2])
    {
        const uint4 e = __ldg((const uint4 *)t + i);
        x = __uint_as_float(e.x);
        w[0] = e.y;
        w[1] = e.z;
    }
    __device__ __forceinline__ static void store(void *t, int64_t i, float x, uint32_t w0, uint32_t w1)
    {
        ((uint4 *)t)[i] = make_uint4(__float_as_uint(x), w0, w1, 0u);
    }
};

template <int KW>
struct TabEntry<double, KW> {
    static constexpr int bytes = 16;
    __device__ __forceinline__ static void load(const void *t, int32_t i, double &x, uint32_t (&w)[KW])
    {
        const uint4 e = __ldg((const uint4 *)t + i);
        x = __hiloint2double((int)e.y, (int)e.x);
        w[0] = e.z;
        if (KW > 1) w[KW - 1] = e.w;
    }
    __device__ __forceinline__ static void store(void *t, int64_t i, double x, uint32_t w0, uint32_t w1)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        ((uint4 *)t)[i] = make_uint4((uint32_t)b, (uint32_t)(b >> 32), w0, w1);
    }
};

// ------------------------------------------------------------------ entries

__device__ __forceinline__ void load_pair(const SellArgs &S, int64_t pi, int &c0, float &a0, int &c1, float &a1)
{
    const int4 e = __ldcs((const int4 *)S.ent + pi);
    c0 = e.x;
    a0 = __int_as_float(e.y);
    c1 = e.z;
    a1 = __int_as_float(e.w);
}

__device__ __forceinline__ void load_pair(const SellArgs &S, int64_t pi, int &c0, double &a0, int &c1, double &a1)
{
    const int2 c = __ldcs((const int2 *)S.ent + pi);
    const double2 v = __ldcs((const double2 *)S.val64 + pi);
    c0 = c.x;
    c1 = c.y;
    a0 = v.x;
    a1 = v.y;
}

// FP32 accumulation of the signed sums y_p = sum_l s_lp y_l (s_lp = -1 where bit p of the probe
// words is set).  It is kept as y_p = C - 2 P_p with C = sum_l y_l and P_p = sum over set bits of y_l:
// each (nonzero, probe) pair then costs one predicated add instead of a sign flip and an add.
template <int K>
struct SignAcc32 {
    float P[K];
    float C;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int p = 0; p < K; ++p) P[p] = 0.f;
        C = 0.f;
    }
    __device__ __forceinline__ void add(float y, const uint32_t *w)
    {
        C += y;
#pragma unroll
        for (int p = 0; p < K; ++p)
            if (w[p >> 5] & (1u << (p & 31))) P[p] += y;
    }
    __device__ __forceinline__ float sum_sq() const
    {
        float ss = 0.f;
#pragma unroll
        for (int p = 0; p < K; ++p) {
            const float yp = C - 2.f * P[p];
            ss += yp * yp;
        }
        return ss;
    }
    // Partial sums of one warp in shared memory, [K + 1][32] (lane-minor: no bank conflicts).
    static constexpr int WORDS = K + 1;
    __device__ __forceinline__ void store(float *sh, int lane) const
    {
#pragma unroll
        for (int p = 0; p < K; ++p) sh[p * 32 + lane] = P[p];
        sh[K * 32 + lane] = C;
    }
    __device__ __forceinline__ void add_partial(const float *sh, int lane)
    {
#pragma unroll
        for (int p = 0; p < K; ++p) P[p] += sh[p * 32 + lane];
        C += sh[K * 32 + lane];
    }
};

// FP64: direct signed accumulation (small problems; accuracy first).
template <int K>
struct SignAcc64 {
    double acc[K];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] = 0.0;
    }
    __device__ __forceinline__ void add(double y, const uint32_t *w)
    {
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] += ((w[p >> 5] >> (p & 31)) & 1u) ? -y : y;
    }
    __device__ __forceinline__ double sum_sq() const
    {
        double ss = 0.0;
#pragma unroll
        for (int p = 0; p < K; ++p) ss += acc[p] * acc[p];
        return ss;
    }
    static constexpr int WORDS = K;
    __device__ __forceinline__ void store(double *sh, int lane) const
    {
#pragma unroll
        for (int p = 0; p < K; ++p) sh[p * 32 + lane] = acc[p];
    }
    __device__ __forceinline__ void add_partial(const double *sh, int lane)
    {
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] += sh[p * 32 + lane];
    }
};

template <typename real, int K>
struct SignAcc;
template <int K>
struct SignAcc<float, K> : SignAcc32<K> {};
template <int K>
struct SignAcc<double, K> : SignAcc64<K> {};

__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dclip(float x, float M) { return fminf(fmaxf(x, -M), M); }
__device__ __forceinline__ double dclip(double x, double M) { return fmin(fmax(x, -M), M); }

// ------------------------------------------------------------------ the iteration kernel

template <typename real, int K, int SPC, bool SPLIT>
__global__ void __launch_bounds__(SPC * 32) sgd_iteration(StepArgs<real> a)
{
    constexpr int KW = (K + 31) / 32;
    using Tab = TabEntry<real, KW>;
    // Select this CTA's side with per-field selects (no dynamic indexing into the parameter block).
    const bool first = (int64_t)blockIdx.x < a.blocks0;
    const bool cols = a.cols_first ? first : !first;
    const int64_t blk = first ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - a.blocks0;
    const SellArgs S = cols ? a.A[1] : a.A[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Long rows: `split` warps share a slice, each over a contiguous range of its pair steps (loads stay
    // coalesced); their partial sums are added in warp order below.  split is the same for the whole CTA.
    const int split = SPLIT ? (cols ? a.split[1] : a.split[0]) : 1;  // SPLIT = false: the plain kernel
    const int part = warp % split;
    const int64_t slice = blk * (SPC / split) + warp / split;
    const bool valid = slice < S.nslices;
    if (split == 1 && !valid) return;
    const int64_t r = slice * 32 + lane;

    SignAcc<real, K> acc;
    acc.init();

    // Two-stage software pipeline over the row's pairs of steps: the entries of pair q+2 and the
    // table gathers of pair q+1 are in flight while pair q is accumulated.  Slice widths are
    // uniform across the warp, so every branch below is warp-uniform.
    const int np_all = valid ? S.slice_w[slice] / 2 : 0;
    const int q_begin = np_all * part / split;
    const int np = np_all * (part + 1) / split - q_begin;
    const int64_t pbase = (valid ? S.slice_off[slice] / 2 : 0) + lane + (int64_t)q_begin * 32;
    const void *tab = cols ? a.tab_in[1] : a.tab_in[0];
    int c0 = 0, c1 = 0, n0 = 0, n1 = 0;
    real a0 = real(0), a1 = real(0), b0 = real(0), b1 = real(0);
    real x0 = real(0), x1 = real(0);
    uint32_t w0[KW] = {}, w1[KW] = {};
    if (np > 0) {
        load_pair(S, pbase, c0, a0, c1, a1);
        Tab::load(tab, c0, x0, w0);
        Tab::load(tab, c1, x1, w1);
    }
    if (np > 1) load_pair(S, pbase + 32, n0, b0, n1, b1);
    for (int q = 0; q < np; ++q) {
        real y0 = real(0), y1 = real(0);
        uint32_t v0[KW] = {}, v1[KW] = {};
        if (q + 1 < np) {
            Tab::load(tab, n0, y0, v0);
            Tab::load(tab, n1, y1, v1);
        }
        int m0 = 0, m1 = 0;
        real d0 = real(0), d1 = real(0);
        if (q + 2 < np) load_pair(S, pbase + (int64_t)(q + 2) * 32, m0, d0, m1, d1);
        acc.add(a0 * x0, w0);
        acc.add(a1 * x1, w1);
        a0 = b0;
        a1 = b1;
        b0 = d0;
        b1 = d1;
        n0 = m0;
        n1 = m1;
        x0 = y0;
        x1 = y1;
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            w0[h] = v0[h];
            w1[h] = v1[h];
        }
    }
    (void)c0;
    (void)c1;
    if (SPLIT && split > 1) {
        extern __shared__ __align__(16) unsigned char sgd_partials[];
        real *sh = reinterpret_cast<real *>(sgd_partials);
        constexpr int WORDS = SignAcc<real, K>::WORDS;
        acc.store(sh + (size_t)warp * WORDS * 32, lane);
        __syncthreads();
        if (part != 0 || !valid) return;
        for (int q = 1; q < split; ++q) acc.add_partial(sh + (size_t)(warp + q) * WORDS * 32, lane);
    }
    if (r >= S.rows) return;

    const real ss = acc.sum_sq();
    real *X = cols ? a.x[1] : a.x[0];
    const real xo = X[r];
    const real ex = dexp(xo);
    const real z = ex * ex * ss * (real(1) / real(K));
    if (a.mode == 1) {
        (cols ? a.z[1] : a.z[0])[S.perm[r]] = z;
        return;
    }
    const int32_t *MID = cols ? a.mid[1] : a.mid[0];
    real t2 = cols ? a.target2[1] : a.target2[0];
    uint32_t pidx = (uint32_t)S.perm[r];
    uint32_t psid = cols ? a.sid_out[1] : a.sid_out[0];
    if (MID) {
        const int32_t b = MID[r];
        t2 = (cols ? a.tgt2[1] : a.tgt2[0])[b];
        pidx = (uint32_t)(cols ? a.loc[1] : a.loc[0])[r];
        psid = a.sid_base + 2u * (uint32_t)b + (cols ? 0u : 1u);
    }
    const real *TR = cols ? a.tgt_row[1] : a.tgt_row[0];
    if (TR) t2 = TR[r];
    real xn = xo - a.eta * (z - t2 + a.gamma * xo);
    if (!isfinite(xn)) atomicOr(a.status, ST_NONFINITE);
    xn = dclip(xn, a.M);
    X[r] = xn;
    real *XB = cols ? a.xb[1] : a.xb[0];
    XB[r] = a.avg_new * xn + a.avg_old * XB[r];
    uint32_t pw0, pw1;
    if (a.mode == 2) {
        // Symmetric: D = E, so the new e^{u_i} and the s-probes of index i feed the column table.
        probe_words2(pidx, a.t_next, a.sid_out[1], a.key0, a.key1, pw0, pw1);
        Tab::store(a.tab_out[1], a.sym_pos[r], dexp(xn), pw0, pw1);
        return;
    }
    probe_words2(pidx, a.t_next, psid, a.key0, a.key1, pw0, pw1);
    Tab::store(cols ? a.tab_out[1] : a.tab_out[0], r, dexp(xn), pw0, pw1);
}

// Load a start state (original order) into sorted order and build the tables of iteration t.
template <typename real, int KW>
__global__ void load_state(int64_t rows, const int32_t *perm, const real *x_in, const real *xb_in, real *x,
                           real *xb, void *tab, uint32_t t, uint32_t sid, uint32_t k0, uint32_t k1,
                           const int32_t *mid, const int32_t *loc, uint32_t sid_base, uint32_t side_off)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = perm[r];
    const real xi = x_in ? x_in[i] : real(0);
    if (x) x[r] = xi;
    if (xb) xb[r] = xb_in ? xb_in[i] : real(0);
    uint32_t pidx = (uint32_t)i, psid = sid;
    if (mid) {
        pidx = (uint32_t)loc[r];
        psid = sid_base + 2u * (uint32_t)mid[r] + side_off;
    }
    uint32_t w0, w1;
    probe_words2(pidx, t, psid, k0, k1, w0, w1);
    TabEntry<real, KW>::store(tab, r, dexp(xi), w0, w1);
}

template <typename real>
__global__ void store_state(int64_t rows, const int32_t *perm, const real *x, const real *xb, real *x_out,
                            real *xb_out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = perm[r];
    x_out[i] = x[r];
    xb_out[i] = xb[r];
}

__global__ void draw_probe_words(uint64_t seed, uint32_t t, uint32_t sid, int64_t len, int kw, uint32_t *out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= len) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int w = 0; w < kw; w += 4) {
        const U4 o = philox10(U4{(uint32_t)idx, t, sid, (uint32_t)(w >> 2)}, k0, k1);
        const uint32_t ws[4] = {o.x, o.y, o.z, o.w};
        for (int h = 0; h < 4 && w + h < kw; ++h) out[(int64_t)(w + h) * len + idx] = ws[h];
    }
}

// One part of a split matrix: load the part's start state (vectors of the part's own rows / columns, index
// i - base) into sorted order and write the part's chunk of the tables of iteration t (`tab` points at the
// chunk).  Probe counters use the whole matrix's index, so every part draws the probes an unsplit run draws.
template <typename real, int KW>
__global__ void shard_load(int64_t rows, int64_t base, const int32_t *perm, const real *x_in, const real *xb_in, real *x,
                           real *xb, void *tab, uint32_t t, uint32_t sid, uint32_t k0, uint32_t k1)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = perm[r];
    const real xi = x_in[i - base];
    x[r] = xi;
    xb[r] = xb_in[i - base];
    uint32_t w0, w1;
    probe_words2((uint32_t)i, t, sid, k0, k1, w0, w1);
    TabEntry<real, KW>::store(tab, r, dexp(xi), w0, w1);
}

template <typename real>
__global__ void shard_store(int64_t rows, int64_t base, const int32_t *perm, const real *x, const real *xb, real *x_out,
                            real *xb_out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = perm[r];
    x_out[i - base] = x[r];
    xb_out[i - base] = xb[r];
}

// ------------------------------------------------------------------ host side

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static bool k_supported(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32 || k == 64; }

bool probes_supported(int k) { return k_supported(k); }

static int entry_bytes(bool dbl, int kw) { return (!dbl && kw == 1) ? 8 : 16; }

sme_status ensure_equil_workspace(sme_op op, int kw)
{
    Workspace &W = op->ws;
    const size_t sz = op->dbl ? 8 : 4;
    // Each buffer on its own, so that a call after a failed allocation completes the set.
    if (!W.u) SME_TRY(dev_alloc(op, &W.u, op->m * sz));
    if (!W.ub) SME_TRY(dev_alloc(op, &W.ub, op->m * sz));
    if (!W.v) SME_TRY(dev_alloc(op, &W.v, op->n * sz));
    if (!W.vb) SME_TRY(dev_alloc(op, &W.vb, op->n * sz));
    const int64_t eb = entry_bytes(op->dbl, kw);
    const int64_t need_u = op->fwd.nslices * 32 * eb, need_v = op->bwd.nslices * 32 * eb;
    if (W.tab_bytes_u < need_u) {
        for (int b = 0; b < 2; ++b) {
            dev_free(op, W.tab_u[b], W.tab_bytes_u);
            W.tab_u[b] = nullptr;
            SME_TRY(dev_alloc(op, &W.tab_u[b], need_u));
        }
        W.tab_bytes_u = need_u;
    }
    if (W.tab_bytes_v < need_v) {
        for (int b = 0; b < 2; ++b) {
            dev_free(op, W.tab_v[b], W.tab_bytes_v);
            W.tab_v[b] = nullptr;
            SME_TRY(dev_alloc(op, &W.tab_v[b], need_v));
        }
        W.tab_bytes_v = need_v;
    }
    return SME_OK;
}

static SellArgs sell_args(const Sell &S)
{
    return SellArgs{S.slice_off, S.slice_w, S.ent, S.val64, S.perm, S.rows, S.nslices};
}

// Shared memory for the partial sums of split slices: [SPC warps][words][32 lanes].
template <typename real, int K>
static size_t split_smem(int spc)
{
    return (size_t)spc * 32 * SignAcc<real, K>::WORDS * sizeof(real);
}

// Split slices run a separate instantiation (with the shared-memory combine), so the plain kernel keeps its
// registers and occupancy; splitting is only used with the default slices per CTA.
template <typename real, int K>
static void launch_k(const StepArgs<real> &a, int spc, unsigned grid, cudaStream_t s)
{
    if (a.split[0] > 1 || a.split[1] > 1) {
        sgd_iteration<real, K, DEFAULT_SPC, true><<<grid, DEFAULT_SPC * 32, split_smem<real, K>(DEFAULT_SPC), s>>>(a);
        return;
    }
    if (sizeof(real) == 4 && (K == 16 || K == 32)) {
        if (spc == 4) {
            sgd_iteration<real, K, 4, false><<<grid, 4 * 32, 0, s>>>(a);
            return;
        }
        if (spc == 16) {
            sgd_iteration<real, K, 16, false><<<grid, 16 * 32, 0, s>>>(a);
            return;
        }
    }
    sgd_iteration<real, K, DEFAULT_SPC, false><<<grid, DEFAULT_SPC * 32, 0, s>>>(a);
}

template <typename real>
static size_t split_smem_bytes(int k, int spc)
{
    switch (k) {
        case 1: return split_smem<real, 1>(spc);
        case 2: return split_smem<real, 2>(spc);
        case 4: return split_smem<real, 4>(spc);
        case 8: return split_smem<real, 8>(spc);
        case 16: return split_smem<real, 16>(spc);
        case 32: return split_smem<real, 32>(spc);
        default: return split_smem<real, 64>(spc);
    }
}

template <typename real>
static void launch_iteration(const StepArgs<real> &a, int k, int spc, unsigned grid, cudaStream_t s)
{
    switch (k) {
        case 1: launch_k<real, 1>(a, spc, grid, s); break;
        case 2: launch_k<real, 2>(a, spc, grid, s); break;
        case 4: launch_k<real, 4>(a, spc, grid, s); break;
        case 8: launch_k<real, 8>(a, spc, grid, s); break;
        case 16: launch_k<real, 16>(a, spc, grid, s); break;
        case 32: launch_k<real, 32>(a, spc, grid, s); break;
        case 64: launch_k<real, 64>(a, spc, grid, s); break;
        default: break;
    }
}

// Launch shape chosen for probe count k: slices per CTA, which side's CTAs come first, and warps per slice.
struct Shape {
    int spc = DEFAULT_SPC;
    int cols_first = 0;
    int split[2] = {1, 1};
};

// Warps per slice: long rows are shared by several warps, so that a lane walks about 16 pair steps or fewer,
// as far as 48 KB of shared memory for the partial sums (at the default slices per CTA) allow.  The choice
// depends only on the operator and k; a split operator always runs the default slices per CTA, so that the
// tuned launch shape changes scheduling only, never the order of the sums.
static void set_split(sme_op op, int k, Shape &sh)
{
    const size_t bytes =
        op->dbl ? split_smem_bytes<double>(k, DEFAULT_SPC) : split_smem_bytes<float>(k, DEFAULT_SPC);
    for (int side = 0; side < 2; ++side) {
        const Sell &S = side ? op->bwd : op->fwd;
        const double steps = S.nslices > 0 ? (double)S.entries / (64.0 * (double)S.nslices) : 0.0;
        int sp = steps >= 96 ? 8 : steps >= 48 ? 4 : steps >= 24 ? 2 : 1;
        if (bytes > 48 * 1024) sp = 1;
        sh.split[side] = sp;
    }
    if (sh.split[0] > 1 || sh.split[1] > 1) sh.spc = DEFAULT_SPC;
}

static int64_t side_blocks(const Sell &S, const Shape &sh, int side)
{
    const int per_cta = sh.spc / sh.split[side];
    return (S.nslices + per_cta - 1) / per_cta;
}

static int k_slot(int k)
{
    int b = 0;
    while ((1 << b) < k) ++b;
    return b;
}

static Shape shape_for(sme_op op, int k)
{
    Shape sh;
    const int slot = k_slot(k);
    if (slot < 8 && op->tuned[slot].spc > 0) {
        sh.spc = op->tuned[slot].spc;
        sh.cols_first = op->tuned[slot].cols_first;
    }
    set_split(op, k, sh);
    return sh;
}

static unsigned grid_for(sme_op op, const Shape &sh)
{
    return (unsigned)(side_blocks(op->fwd, sh, 0) + side_blocks(op->bwd, sh, 1));
}

template <typename real>
static void launch_load(sme_op op, int side, int kw, const real *x_in, const real *xb_in, real *x, real *xb,
                        void *tab, uint32_t t, uint32_t sid, uint64_t seed, cudaStream_t s, uint32_t sid_base = 0)
{
    const Sell &S = side == 0 ? op->fwd : op->bwd;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int32_t *mid = op->batch ? op->batch->mid[side] : nullptr;
    const int32_t *loc = op->batch ? op->batch->loc[side] : nullptr;
    if (op->batch) sid_base = op->batch->sid_base;
    const uint32_t side_off = side == 0 ? 1u : 0u;
    if (op->dbl || kw == 2)
        load_state<real, 2><<<nblk(S.rows), 256, 0, s>>>(S.rows, S.perm, x_in, xb_in, x, xb, tab, t, sid, k0, k1, mid,
                                                         loc, sid_base, side_off);
    else
        load_state<real, 1><<<nblk(S.rows), 256, 0, s>>>(S.rows, S.perm, x_in, xb_in, x, xb, tab, t, sid, k0, k1, mid,
                                                         loc, sid_base, side_off);
}

struct Resolved {
    double alpha, beta, gamma, M;
};

static Resolved resolve(sme_op op, double alpha, double beta, double gamma, double M);

// Defaults from the whole matrix's sizes (a part of a split matrix has its blocks' sizes in op->m, op->n).
static Resolved resolve_whole(sme_op op, double alpha, double beta, double gamma, double M)
{
    const double m = op->shard ? (double)op->shard->gm : (double)op->m;
    const double n = op->shard ? (double)op->shard->gn : (double)op->n;
    Resolved r;
    r.alpha = alpha > 0 ? alpha : std::pow(n / m, 0.25);
    r.beta = beta > 0 ? beta : std::pow(m / n, 0.25);
    r.gamma = gamma > 0 ? gamma : 0.1;
    r.M = M > 0 ? M : std::log(1e4);
    return r;
}

static Resolved resolve(sme_op op, double alpha, double beta, double gamma, double M)
{
    Resolved r;
    r.alpha = alpha > 0 ? alpha : std::pow((double)op->n / (double)op->m, 0.25);
    r.beta = beta > 0 ? beta : std::pow((double)op->m / (double)op->n, 0.25);
    r.gamma = gamma > 0 ? gamma : 0.1;
    r.M = M > 0 ? M : std::log(1e4);
    return r;
}

template <typename real>
static StepArgs<real> base_args(sme_op op, int buf_in, const Resolved &R, uint64_t seed, const Shape &sh)
{
    StepArgs<real> a{};
    a.A[0] = sell_args(op->fwd);
    a.A[1] = sell_args(op->bwd);
    a.tab_in[0] = op->ws.tab_v[buf_in];
    a.tab_in[1] = op->ws.tab_u[buf_in];
    a.tab_out[0] = op->ws.tab_u[buf_in ^ 1];
    a.tab_out[1] = op->ws.tab_v[buf_in ^ 1];
    a.x[0] = (real *)op->ws.u;
    a.x[1] = (real *)op->ws.v;
    a.xb[0] = (real *)op->ws.ub;
    a.xb[1] = (real *)op->ws.vb;
    a.target2[0] = (real)(R.alpha * R.alpha);
    a.target2[1] = (real)(R.beta * R.beta);
    a.gamma = (real)R.gamma;
    a.M = (real)R.M;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    const int64_t br = side_blocks(op->fwd, sh, 0), bc = side_blocks(op->bwd, sh, 1);
    a.cols_first = sh.cols_first;
    a.blocks0 = sh.cols_first ? bc : br;
    a.split[0] = sh.split[0];
    a.split[1] = sh.split[1];
    a.status = op->d_status;
    if (op->batch) {
        for (int side = 0; side < 2; ++side) {
            a.mid[side] = op->batch->mid[side];
            a.loc[side] = op->batch->loc[side];
            a.tgt2[side] = (const real *)op->batch->tgt2[side];
        }
        a.sid_base = op->batch->sid_base;
    }
    if (op->ws.use_tgt) {
        a.tgt_row[0] = (const real *)op->ws.tgt[0];
        a.tgt_row[1] = (const real *)op->ws.tgt[1];
    }
    return a;
}


template <typename real>
static sme_status equilibrate_t(sme_op op, const sme_equil_params *p, real *u, real *v, real *ub, real *vb,
                                cudaStream_t s)
{
    const int k = p->k, kw = (k + 31) / 32;
    SME_TRY(ensure_equil_workspace(op, kw));
    const Resolved R = resolve(op, p->alpha, p->beta, p->gamma, p->M);
    if (op->batch) op->batch->sid_base = (uint32_t)p->stream_base;
    const uint32_t sid_s = (uint32_t)p->stream_base, sid_w = (uint32_t)p->stream_base + 1u;
    const int tb = p->t_begin;
    int buf = tb & 1;
    launch_load<real>(op, 0, kw, u, ub, (real *)op->ws.u, (real *)op->ws.ub, op->ws.tab_u[buf], (uint32_t)tb, sid_w,
                      p->seed, s);
    launch_load<real>(op, 1, kw, v, vb, (real *)op->ws.v, (real *)op->ws.vb, op->ws.tab_v[buf], (uint32_t)tb, sid_s,
                      p->seed, s);
    const Shape sh = shape_for(op, k);
    const unsigned grid = grid_for(op, sh);
    const bool timed = (p->flags & SME_EQ_TIMED) != 0;
    if (timed) {
        for (int i = 0; i < 2; ++i)
            if (!op->ev_loop[i]) SME_CUDA(cudaEventCreate(&op->ev_loop[i]));
        SME_CUDA(cudaEventRecord(op->ev_loop[0], s));
    }
    auto enqueue = [&](cudaStream_t q) {
        for (int t = tb; t < tb + p->T; ++t) {
            StepArgs<real> a = base_args<real>(op, t & 1, R, p->seed, sh);
            a.eta = (real)(2.0 / (R.gamma * ((double)t + (double)p->t0 + 1.0)));
            a.avg_new = (real)(2.0 / ((double)t + 2.0));
            a.avg_old = (real)((double)t / ((double)t + 2.0));
            a.t_next = (uint32_t)(t + 1);
            a.sid_out[0] = sid_w;
            a.sid_out[1] = sid_s;
            a.mode = 0;
            launch_iteration<real>(a, k, sh.spc, grid, q);
        }
    };
    if ((p->flags & SME_EQ_NO_GRAPH) || p->T < 2) {
        enqueue(s);
    } else {
        // The iteration launches depend only on these values (all buffers they touch belong to the op),
        // so one captured graph is replayed for repeated calls with the same parameters.
        const int64_t key[12] = {p->T, p->k, p->t_begin, p->t0, (int64_t)p->seed, p->stream_base,
                                 (int64_t)(R.alpha * 1e15), (int64_t)(R.beta * 1e15), (int64_t)(R.gamma * 1e15),
                                 (int64_t)(R.M * 1e15), (int64_t)op->ws.tab_bytes_u,
                                 sh.spc * 4 + sh.cols_first * 2 + (op->ws.use_tgt ? 1 : 0)};
        // A call is captured only when it repeats the previous one: a one-off call (a fresh operator, new
        // parameters) launches directly and does not pay for capture and instantiation.
        GraphCache &G = op->graph;
        const bool cached = G.exec && std::memcmp(G.key, key, sizeof(key)) == 0;
        const bool repeat = !cached && G.have_direct && std::memcmp(G.last_direct, key, sizeof(key)) == 0;
        if (!cached && !repeat) {
            enqueue(s);
            std::memcpy(G.last_direct, key, sizeof(key));
            G.have_direct = true;
        } else {
            if (!cached) {
                if (G.exec) {
                    cudaGraphExecDestroy(G.exec);
                    G.exec = nullptr;
                }
                if (!G.stream) SME_CUDA(cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking));
                cudaGraph_t graph = nullptr;
                SME_CUDA(cudaStreamBeginCapture(G.stream, cudaStreamCaptureModeThreadLocal));
                enqueue(G.stream);
                SME_CUDA(cudaStreamEndCapture(G.stream, &graph));
                cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
                cudaGraphDestroy(graph);
                SME_CUDA(e);
                std::memcpy(G.key, key, sizeof(key));
            }
            SME_CUDA(cudaGraphLaunch(G.exec, s));
        }
    }
    if (timed) {
        SME_CUDA(cudaEventRecord(op->ev_loop[1], s));
        op->loop_timed = true;
        op->loop_iters = p->T;
    }
    store_state<real><<<nblk(op->m), 256, 0, s>>>(op->m, op->fwd.perm, (real *)op->ws.u, (real *)op->ws.ub, u, ub);
    store_state<real><<<nblk(op->n), 256, 0, s>>>(op->n, op->bwd.perm, (real *)op->ws.v, (real *)op->ws.vb, v, vb);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

template <typename real>
static sme_status estimate_t(sme_op op, const real *u, const real *v, int t, int k, uint64_t seed, int sb,
                             real *zu, real *zv, cudaStream_t s)
{
    const int kw = (k + 31) / 32;
    SME_TRY(ensure_equil_workspace(op, kw));
    const Resolved R = resolve(op, 0, 0, 0, 0);
    const int buf = 0;
    launch_load<real>(op, 0, kw, u, nullptr, (real *)op->ws.u, nullptr, op->ws.tab_u[buf], (uint32_t)t,
                      (uint32_t)sb + 1u, seed, s);
    launch_load<real>(op, 1, kw, v, nullptr, (real *)op->ws.v, nullptr, op->ws.tab_v[buf], (uint32_t)t, (uint32_t)sb,
                      seed, s);
    const Shape sh = shape_for(op, k);
    StepArgs<real> a = base_args<real>(op, buf, R, seed, sh);
    a.mode = 1;
    a.z[0] = zu;
    a.z[1] = zv;
    // A NULL output skips that side by giving it no slices.
    if (!zu) a.A[0].nslices = 0;
    if (!zv) a.A[1].nslices = 0;
    launch_iteration<real>(a, k, sh.spc, grid_for(op, sh), s);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

// Squared targets in sorted order: out[r] = in[perm[r]].
template <typename real>
__global__ void permute_in(int64_t n, const int32_t *perm, const real *in, real *out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = in[perm[r]];
}

__global__ void sym_positions(int64_t n, const int32_t *perm_r, const int32_t *iperm_c, int32_t *pos)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) pos[r] = iperm_c[perm_r[r]];
}

template <typename real>
static sme_status targets_t(sme_op op, const sme_equil_params *p, const real *rt, const real *ct, real *u, real *v,
                            real *ub, real *vb, cudaStream_t s)
{
    Workspace &W = op->ws;
    const size_t sz = op->dbl ? 8 : 4;
    if (!W.tgt[0]) {
        SME_TRY(dev_alloc(op, &W.tgt[0], op->m * sz));
        SME_TRY(dev_alloc(op, &W.tgt[1], op->n * sz));
    }
    permute_in<real><<<nblk(op->m), 256, 0, s>>>(op->m, op->fwd.perm, rt, (real *)W.tgt[0]);
    permute_in<real><<<nblk(op->n), 256, 0, s>>>(op->n, op->bwd.perm, ct, (real *)W.tgt[1]);
    W.use_tgt = true;
    sme_status st = equilibrate_t<real>(op, p, u, v, ub, vb, s);
    W.use_tgt = false;
    return st;
}

template <typename real>
static sme_status symmetric_t(sme_op op, const sme_equil_params *p, real *u, real *ub, cudaStream_t s)
{
    const int k = p->k, kw = (k + 31) / 32;
    SME_TRY(ensure_equil_workspace(op, kw));
    Workspace &W = op->ws;
    if (!W.sym_pos) {
        SME_TRY(dev_alloc(op, (void **)&W.sym_pos, op->m * sizeof(int32_t)));
        sym_positions<<<nblk(op->m), 256, 0, s>>>(op->m, op->fwd.perm, op->bwd.iperm, W.sym_pos);
    }
    const Resolved R = resolve(op, p->alpha, p->alpha, p->gamma, p->M);
    const uint32_t sid_s = (uint32_t)p->stream_base;
    const int tb = p->t_begin;
    const int buf = tb & 1;
    launch_load<real>(op, 0, kw, u, ub, (real *)W.u, (real *)W.ub, W.tab_u[buf], (uint32_t)tb, sid_s + 1u, p->seed, s);
    launch_load<real>(op, 1, kw, u, nullptr, (real *)W.v, nullptr, W.tab_v[buf], (uint32_t)tb, sid_s, p->seed, s);
    Shape sh;  // rows only: the default shape
    set_split(op, k, sh);
    const unsigned grid = (unsigned)side_blocks(op->fwd, sh, 0);
    for (int t = tb; t < tb + p->T; ++t) {
        StepArgs<real> a = base_args<real>(op, t & 1, R, p->seed, sh);
        a.eta = (real)(2.0 / (R.gamma * ((double)t + (double)p->t0 + 1.0)));
        a.avg_new = (real)(2.0 / ((double)t + 2.0));
        a.avg_old = (real)((double)t / ((double)t + 2.0));
        a.t_next = (uint32_t)(t + 1);
        a.sid_out[0] = sid_s + 1u;
        a.sid_out[1] = sid_s;
        a.mode = 2;
        a.sym_pos = W.sym_pos;
        a.A[1].nslices = 0;
        launch_iteration<real>(a, k, sh.spc, grid, s);
    }
    store_state<real><<<nblk(op->m), 256, 0, s>>>(op->m, op->fwd.perm, (real *)W.u, (real *)W.ub, u, ub);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

// Block equilibration: expand block scalings to rows / columns (original order).
template <typename real>
__global__ void expand_blocks(int64_t n, const int32_t *blk, const real *xb, real *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = xb[blk[i]];
}

// One CTA per block: z_b = sum of the block's estimates (FP64, fixed order), then the projected step and
// the running average of the block variable.  Row blocks first, then column blocks.
template <typename real>
__global__ void block_step_kernel(int64_t p, const int64_t *rb, int64_t q, const int64_t *cb, const real *zu,
                                  const real *zv, real *ub, real *vb, real *ubb, real *vbb, double a2, double b2,
                                  double gamma, double M, double eta, double avg_new, double avg_old, int *status)
{
    __shared__ double sh[256];
    const int64_t g = blockIdx.x;
    const bool colb = g >= p;
    const int64_t b = colb ? g - p : g;
    const int64_t lo = colb ? cb[b] : rb[b], hi = colb ? cb[b + 1] : rb[b + 1];
    const real *z = colb ? zv : zu;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += (double)z[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    real *X = colb ? vb : ub, *XB = colb ? vbb : ubb;
    const double xo = (double)X[b];
    const double target = (colb ? b2 : a2) * (double)(hi - lo);
    double xn = xo - eta * (sh[0] - target + gamma * xo);
    if (!isfinite(xn)) atomicOr(status, ST_NONFINITE);
    xn = fmin(fmax(xn, -M), M);
    X[b] = (real)xn;
    XB[b] = (real)(avg_new * xn + avg_old * (double)XB[b]);
}

template <typename real>
static sme_status block_t(sme_op op, const sme_equil_params *p, int64_t pb, const int64_t *rb_h, int64_t qb,
                          const int64_t *cb_h, real *ub, real *vb, real *ubb, real *vbb, cudaStream_t s)
{
    const int k = p->k;
    const Resolved R = resolve(op, p->alpha, p->beta, p->gamma, p->M);
    const int64_t m = op->m, n = op->n;
    std::vector<int32_t> br(m), bc(n);
    for (int64_t b = 0; b < pb; ++b)
        for (int64_t i = rb_h[b]; i < rb_h[b + 1]; ++i) br[i] = (int32_t)b;
    for (int64_t c = 0; c < qb; ++c)
        for (int64_t j = cb_h[c]; j < cb_h[c + 1]; ++j) bc[j] = (int32_t)c;
    const size_t sz = sizeof(real);
    const size_t bytes = (size_t)(m + n) * 4 + (size_t)(pb + qb + 2) * 8 + (size_t)2 * (m + n) * sz;
    AsyncScratch scratch(s);
    SME_CUDA(scratch.alloc(bytes));
    char *buf = scratch.as<char>();
    int32_t *dbr = (int32_t *)buf, *dbc = dbr + m;
    int64_t *drb = (int64_t *)(buf + (size_t)(m + n) * 4), *dcb = drb + pb + 1;
    real *xr = (real *)(buf + (size_t)(m + n) * 4 + (size_t)(pb + qb + 2) * 8), *xc = xr + m, *zu = xc + n,
         *zv = zu + m;
    SME_CUDA(cudaMemcpyAsync(dbr, br.data(), m * 4, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemcpyAsync(dbc, bc.data(), n * 4, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemcpyAsync(drb, rb_h, (pb + 1) * 8, cudaMemcpyHostToDevice, s));
    SME_CUDA(cudaMemcpyAsync(dcb, cb_h, (qb + 1) * 8, cudaMemcpyHostToDevice, s));
    for (int t = p->t_begin; t < p->t_begin + p->T; ++t) {
        expand_blocks<real><<<nblk(m), 256, 0, s>>>(m, dbr, ub, xr);
        expand_blocks<real><<<nblk(n), 256, 0, s>>>(n, dbc, vb, xc);
        SME_TRY(estimate_t<real>(op, xr, xc, t, k, p->seed, p->stream_base, zu, zv, s));
        const double eta = 2.0 / (R.gamma * ((double)t + (double)p->t0 + 1.0));
        block_step_kernel<real><<<(unsigned)(pb + qb), 256, 0, s>>>(pb, drb, qb, dcb, zu, zv, ub, vb, ubb, vbb,
                                                                   R.alpha * R.alpha, R.beta * R.beta, R.gamma, R.M,
                                                                   eta, 2.0 / ((double)t + 2.0),
                                                                   (double)t / ((double)t + 2.0), op->d_status);
    }
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

// Times every launch shape on this operator (estimate mode, zero state) and keeps the fastest for k.
template <typename real>
static sme_status autotune_t(sme_op op, int k, cudaStream_t s, int *spc_out, int *cf_out, float *ms_out)
{
    const int kw = (k + 31) / 32;
    SME_TRY(ensure_equil_workspace(op, kw));
    const Resolved R = resolve(op, 0, 0, 0, 0);
    launch_load<real>(op, 0, kw, (const real *)nullptr, nullptr, (real *)op->ws.u, nullptr, op->ws.tab_u[0], 1u, 1u,
                      0, s);
    launch_load<real>(op, 1, kw, (const real *)nullptr, nullptr, (real *)op->ws.v, nullptr, op->ws.tab_v[0], 1u, 0u,
                      0, s);
    EventPair ev;
    SME_CUDA(ev.create());
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    const int spcs[3] = {4, 8, 16};
    float best = 1e30f;
    Shape best_sh;
    for (int cf = 0; cf < 2; ++cf)
        for (int i = 0; i < 3; ++i) {
            Shape sh;
            sh.spc = (sizeof(real) == 4 && (k == 16 || k == 32)) ? spcs[i] : DEFAULT_SPC;
            sh.cols_first = cf;
            set_split(op, k, sh);  // a split operator keeps the default slices per CTA
            if (sh.spc != spcs[i] && i != 1) continue;
            StepArgs<real> a = base_args<real>(op, 0, R, 0, sh);
            a.mode = 1;
            a.z[0] = (real *)op->ws.ub;
            a.z[1] = (real *)op->ws.vb;
            const unsigned grid = grid_for(op, sh);
            for (int w = 0; w < 2; ++w) launch_iteration<real>(a, k, sh.spc, grid, s);
            SME_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 5; ++r) launch_iteration<real>(a, k, sh.spc, grid, s);
            SME_CUDA(cudaEventRecord(e1, s));
            SME_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            SME_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_sh = sh;
            }
        }
    const int slot = k_slot(k);
    if (slot < 8) {
        op->tuned[slot].spc = best_sh.spc;
        op->tuned[slot].cols_first = best_sh.cols_first;
    }
    if (spc_out) *spc_out = best_sh.spc;
    if (cf_out) *cf_out = best_sh.cols_first;
    if (ms_out) *ms_out = best / 5.f;
    return SME_OK;
}

// ------------------------------------------------------------------ one part of a split matrix

template <typename real>
static sme_status shard_begin_t(sme_op op, const sme_equil_params *p, const real *u, const real *v, const real *ub,
                                const real *vb, void *row_table, void *col_table, cudaStream_t s)
{
    const int k = p->k, kw = (k + 31) / 32;
    SME_TRY(ensure_equil_workspace(op, kw));
    const ShardInfo &I = *op->shard;
    const int64_t eb = entry_bytes(op->dbl, kw);
    const uint32_t sid_s = (uint32_t)p->stream_base, sid_w = sid_s + 1u;
    const uint32_t k0 = (uint32_t)p->seed, k1 = (uint32_t)(p->seed >> 32), t = (uint32_t)p->t_begin;
    char *rt = (char *)row_table + I.part * I.rchunk * eb, *ct = (char *)col_table + I.part * I.cchunk * eb;
    if (op->dbl || kw == 2) {
        shard_load<real, 2><<<nblk(op->m), 256, 0, s>>>(op->m, I.r0, op->fwd.perm, u, ub, (real *)op->ws.u,
                                                        (real *)op->ws.ub, rt, t, sid_w, k0, k1);
        shard_load<real, 2><<<nblk(op->n), 256, 0, s>>>(op->n, I.c0, op->bwd.perm, v, vb, (real *)op->ws.v,
                                                        (real *)op->ws.vb, ct, t, sid_s, k0, k1);
    } else {
        shard_load<real, 1><<<nblk(op->m), 256, 0, s>>>(op->m, I.r0, op->fwd.perm, u, ub, (real *)op->ws.u,
                                                        (real *)op->ws.ub, rt, t, sid_w, k0, k1);
        shard_load<real, 1><<<nblk(op->n), 256, 0, s>>>(op->n, I.c0, op->bwd.perm, v, vb, (real *)op->ws.v,
                                                        (real *)op->ws.vb, ct, t, sid_s, k0, k1);
    }
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

// Iteration t of the part: its rows against the whole column table, its columns against the whole row table
// (both gathered from every part), writing the part's chunks of the next tables.
template <typename real>
static sme_status shard_step_t(sme_op op, const sme_equil_params *p, int t, const void *row_in, const void *col_in,
                               void *row_out, void *col_out, cudaStream_t s)
{
    const int k = p->k, kw = (k + 31) / 32;
    const ShardInfo &I = *op->shard;
    const int64_t eb = entry_bytes(op->dbl, kw);
    const Resolved R = resolve_whole(op, p->alpha, p->beta, p->gamma, p->M);
    const Shape sh = shape_for(op, k);
    StepArgs<real> a = base_args<real>(op, 0, R, p->seed, sh);
    a.tab_in[0] = col_in;
    a.tab_in[1] = row_in;
    a.tab_out[0] = (char *)row_out + I.part * I.rchunk * eb;
    a.tab_out[1] = (char *)col_out + I.part * I.cchunk * eb;
    a.eta = (real)(2.0 / (R.gamma * ((double)t + (double)p->t0 + 1.0)));
    a.avg_new = (real)(2.0 / ((double)t + 2.0));
    a.avg_old = (real)((double)t / ((double)t + 2.0));
    a.t_next = (uint32_t)(t + 1);
    a.sid_out[0] = (uint32_t)p->stream_base + 1u;
    a.sid_out[1] = (uint32_t)p->stream_base;
    a.mode = 0;
    launch_iteration<real>(a, k, sh.spc, grid_for(op, sh), s);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

sme_status autotune_sparse(sme_op op, int k, cudaStream_t s, int *spc, int *cols_first, float *ms)
{
    if (op->dbl) return autotune_t<double>(op, k, s, spc, cols_first, ms);
    return autotune_t<float>(op, k, s, spc, cols_first, ms);
}

sme_status equilibrate_sparse(sme_op op, const sme_equil_params *p, void *u, void *v, void *ub, void *vb,
                              cudaStream_t s)
{
    if (op->dbl) return equilibrate_t<double>(op, p, (double *)u, (double *)v, (double *)ub, (double *)vb, s);
    return equilibrate_t<float>(op, p, (float *)u, (float *)v, (float *)ub, (float *)vb, s);
}

sme_status estimate_sparse(sme_op op, const void *u, const void *v, int t, int k, uint64_t seed, int sb, void *zu,
                           void *zv, cudaStream_t s)
{
    if (op->batch) op->batch->sid_base = (uint32_t)sb;
    if (op->dbl)
        return estimate_t<double>(op, (const double *)u, (const double *)v, t, k, seed, sb, (double *)zu, (double *)zv, s);
    return estimate_t<float>(op, (const float *)u, (const float *)v, t, k, seed, sb, (float *)zu, (float *)zv, s);
}

}  // namespace sme

using namespace sme;

extern "C" sme_status sme_draw_probes(uint64_t seed, int32_t t, int32_t stream_id, int64_t len, int32_t k,
                                      uint32_t *words, void *stream)
{
    if (len < 0 || k < 1 || (len > 0 && !words)) {
        set_error("sme_draw_probes: bad arguments");
        return SME_ERR_ARG;
    }
    if (len == 0) return SME_OK;
    draw_probe_words<<<nblk(len), 256, 0, (cudaStream_t)stream>>>(seed, (uint32_t)t, (uint32_t)stream_id, len,
                                                                  (k + 31) / 32, words);
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}

extern "C" sme_status sme_equilibrate(sme_op op, const sme_equil_params *p, void *u, void *v, void *u_bar,
                                      void *v_bar, void *stream)
{
    NvtxRange range("sme equilibrate");
    SME_TRY(no_shard(op, "sme_equilibrate"));
    if (!op || !p || !u || !v || !u_bar || !v_bar || p->T < 0 || p->t_begin < 1 || p->t0 < 0) {
        set_error("sme_equilibrate: bad arguments");
        return SME_ERR_ARG;
    }
    if (op->batch) {
        set_error("sme_equilibrate: the operator of a batch is driven by sme_batch_equilibrate");
        return SME_ERR_ARG;
    }
    if (!op->dense && !k_supported(p->k)) {
        set_error("sme_equilibrate: k=%d not supported (1,2,4,...,64)", p->k);
        return SME_ERR_UNSUPPORTED;
    }
    if (op->dense) {
        SME_TRY(dense_equilibrate(op, p, (float *)u, (float *)v, (float *)u_bar, (float *)v_bar,
                                  (cudaStream_t)stream));
    } else if (op->dbl) {
        SME_TRY(equilibrate_t<double>(op, p, (double *)u, (double *)v, (double *)u_bar, (double *)v_bar,
                                      (cudaStream_t)stream));
    } else {
        SME_TRY(equilibrate_t<float>(op, p, (float *)u, (float *)v, (float *)u_bar, (float *)v_bar,
                                     (cudaStream_t)stream));
    }
    if (p->flags & SME_EQ_ASYNC) return SME_OK;
    return sme_op_check(op, stream);
}

extern "C" sme_status sme_equilibrate_targets(sme_op op, const sme_equil_params *p, const void *row_targets_sq,
                                              const void *col_targets_sq, void *u, void *v, void *u_bar,
                                              void *v_bar, void *stream)
{
    SME_TRY(no_shard(op, "sme_equilibrate_targets"));
    if (!op || !p || !row_targets_sq || !col_targets_sq || !u || !v || !u_bar || !v_bar || p->T < 0 ||
        p->t_begin < 1 || p->t0 < 0 || op->dense || op->batch) {
        set_error("sme_equilibrate_targets: bad arguments (sparse single operators only)");
        return SME_ERR_ARG;
    }
    if (!k_supported(p->k)) {
        set_error("sme_equilibrate_targets: k=%d not supported", p->k);
        return SME_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (op->dbl)
        SME_TRY(targets_t<double>(op, p, (const double *)row_targets_sq, (const double *)col_targets_sq, (double *)u,
                                  (double *)v, (double *)u_bar, (double *)v_bar, s));
    else
        SME_TRY(targets_t<float>(op, p, (const float *)row_targets_sq, (const float *)col_targets_sq, (float *)u,
                                 (float *)v, (float *)u_bar, (float *)v_bar, s));
    if (p->flags & SME_EQ_ASYNC) return SME_OK;
    return sme_op_check(op, stream);
}

extern "C" sme_status sme_equilibrate_symmetric(sme_op op, const sme_equil_params *p, void *u, void *u_bar,
                                                void *stream)
{
    SME_TRY(no_shard(op, "sme_equilibrate_symmetric"));
    if (!op || !p || !u || !u_bar || p->T < 0 || p->t_begin < 1 || p->t0 < 0 || op->dense || op->batch ||
        op->m != op->n) {
        set_error("sme_equilibrate_symmetric: bad arguments (square sparse single operators only)");
        return SME_ERR_ARG;
    }
    if (!k_supported(p->k)) {
        set_error("sme_equilibrate_symmetric: k=%d not supported", p->k);
        return SME_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (op->dbl)
        SME_TRY(symmetric_t<double>(op, p, (double *)u, (double *)u_bar, s));
    else
        SME_TRY(symmetric_t<float>(op, p, (float *)u, (float *)u_bar, s));
    if (p->flags & SME_EQ_ASYNC) return SME_OK;
    return sme_op_check(op, stream);
}

extern "C" sme_status sme_equilibrate_block(sme_op op, const sme_equil_params *p, int64_t p_blocks,
                                            const int64_t *row_block_ptr, int64_t q_blocks,
                                            const int64_t *col_block_ptr, void *u, void *v, void *u_bar,
                                            void *v_bar, void *stream)
{
    SME_TRY(no_shard(op, "sme_equilibrate_block"));
    if (!op || !p || !row_block_ptr || !col_block_ptr || !u || !v || !u_bar || !v_bar || p->T < 0 ||
        p->t_begin < 1 || p->t0 < 0 || op->dense || op->batch || p_blocks < 1 || q_blocks < 1) {
        set_error("sme_equilibrate_block: bad arguments (sparse single operators only)");
        return SME_ERR_ARG;
    }
    const int64_t lim[2] = {op->m, op->n};
    const int64_t *ptr[2] = {row_block_ptr, col_block_ptr};
    const int64_t cnt[2] = {p_blocks, q_blocks};
    for (int side = 0; side < 2; ++side) {
        if (ptr[side][0] != 0 || ptr[side][cnt[side]] != lim[side]) {
            set_error("sme_equilibrate_block: block offsets must run from 0 to the dimension");
            return SME_ERR_ARG;
        }
        for (int64_t b = 0; b < cnt[side]; ++b)
            if (ptr[side][b + 1] <= ptr[side][b]) {
                set_error("sme_equilibrate_block: empty or decreasing block");
                return SME_ERR_ARG;
            }
    }
    if (!k_supported(p->k)) {
        set_error("sme_equilibrate_block: k=%d not supported", p->k);
        return SME_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (op->dbl)
        SME_TRY(block_t<double>(op, p, p_blocks, row_block_ptr, q_blocks, col_block_ptr, (double *)u, (double *)v,
                                (double *)u_bar, (double *)v_bar, s));
    else
        SME_TRY(block_t<float>(op, p, p_blocks, row_block_ptr, q_blocks, col_block_ptr, (float *)u, (float *)v,
                               (float *)u_bar, (float *)v_bar, s));
    if (p->flags & SME_EQ_ASYNC) return SME_OK;
    return sme_op_check(op, stream);
}

extern "C" sme_status sme_op_autotune(sme_op op, int32_t k, int32_t *slices_per_cta, int32_t *cols_first,
                                      float *ms_per_iteration, void *stream)
{
    NvtxRange range("sme autotune");
    SME_TRY(no_shard(op, "sme_op_autotune"));
    if (!op || op->dense) {
        set_error("sme_op_autotune: sparse operators only");
        return SME_ERR_ARG;
    }
    if (!k_supported(k)) {
        set_error("sme_op_autotune: k=%d not supported", k);
        return SME_ERR_UNSUPPORTED;
    }
    int spc = 0, cf = 0;
    float ms = 0.f;
    if (op->batch) op->batch->sid_base = 0;
    SME_TRY(autotune_sparse(op, k, (cudaStream_t)stream, &spc, &cf, &ms));
    if (slices_per_cta) *slices_per_cta = spc;
    if (cols_first) *cols_first = cf;
    if (ms_per_iteration) *ms_per_iteration = ms;
    return SME_OK;
}

extern "C" sme_status sme_estimate(sme_op op, const void *u, const void *v, int32_t t, int32_t k, uint64_t seed,
                                   int32_t stream_base, void *z_u, void *z_v, void *stream)
{
    SME_TRY(no_shard(op, "sme_estimate"));
    if (!op || !u || !v || t < 0) {
        set_error("sme_estimate: bad arguments");
        return SME_ERR_ARG;
    }
    if (!op->dense && !k_supported(k)) {
        set_error("sme_estimate: k=%d not supported", k);
        return SME_ERR_UNSUPPORTED;
    }
    if (op->dense) {
        return dense_estimate(op, (const float *)u, (const float *)v, t, k, seed, stream_base, (float *)z_u,
                              (float *)z_v, (cudaStream_t)stream);
    }
    return estimate_sparse(op, u, v, t, k, seed, stream_base, z_u, z_v, (cudaStream_t)stream);
}

static sme_status shard_args(sme_op op, const sme_equil_params *p, const char *where)
{
    if (!op || !p || !op->shard || p->T < 0 || p->t_begin < 1 || p->t0 < 0) {
        set_error("%s: bad arguments (a part of a split matrix is required)", where);
        return SME_ERR_ARG;
    }
    if (!k_supported(p->k)) {
        set_error("%s: k=%d not supported (1,2,4,...,64)", where, p->k);
        return SME_ERR_UNSUPPORTED;
    }
    return SME_OK;
}

extern "C" sme_status sme_shard_begin(sme_op op, const sme_equil_params *p, const void *u, const void *v,
                                      const void *u_bar, const void *v_bar, void *row_table, void *col_table,
                                      void *stream)
{
    NvtxRange range("sme shard begin");
    SME_TRY(shard_args(op, p, "sme_shard_begin"));
    if (!u || !v || !u_bar || !v_bar || !row_table || !col_table) {
        set_error("sme_shard_begin: null pointer");
        return SME_ERR_ARG;
    }
    op->shard->begun_kw = 0;
    const sme_status st =
        op->dbl ? shard_begin_t<double>(op, p, (const double *)u, (const double *)v, (const double *)u_bar,
                                        (const double *)v_bar, row_table, col_table, (cudaStream_t)stream)
                : shard_begin_t<float>(op, p, (const float *)u, (const float *)v, (const float *)u_bar,
                                       (const float *)v_bar, row_table, col_table, (cudaStream_t)stream);
    if (st == SME_OK) op->shard->begun_kw = (p->k + 31) / 32;
    return st;
}

// A step or the end needs the state a successful sme_shard_begin set up; a step also needs table entries of
// the size that begin wrote (the tables are sized by the caller from sme_shard_get_info for one k).
static sme_status shard_begun(sme_op op, int k, const char *where)
{
    const int kw = k > 0 ? (k + 31) / 32 : op->shard->begun_kw;
    if (op->shard->begun_kw == 0 || !op->ws.u || !op->ws.v || !op->ws.ub || !op->ws.vb ||
        entry_bytes(op->dbl, kw) != entry_bytes(op->dbl, op->shard->begun_kw)) {
        set_error("%s: call sme_shard_begin first, with a k of the same table entry size", where);
        return SME_ERR_ARG;
    }
    return SME_OK;
}

extern "C" sme_status sme_shard_step(sme_op op, const sme_equil_params *p, int32_t t, const void *row_table_in,
                                     const void *col_table_in, void *row_table_out, void *col_table_out, void *stream)
{
    SME_TRY(shard_args(op, p, "sme_shard_step"));
    SME_TRY(shard_begun(op, p->k, "sme_shard_step"));
    if (t < 1 || !row_table_in || !col_table_in || !row_table_out || !col_table_out || row_table_in == row_table_out ||
        col_table_in == col_table_out) {
        set_error("sme_shard_step: bad iteration or tables (the next tables must be other buffers)");
        return SME_ERR_ARG;
    }
    if (op->dbl)
        return shard_step_t<double>(op, p, t, row_table_in, col_table_in, row_table_out, col_table_out,
                                    (cudaStream_t)stream);
    return shard_step_t<float>(op, p, t, row_table_in, col_table_in, row_table_out, col_table_out, (cudaStream_t)stream);
}

extern "C" sme_status sme_shard_end(sme_op op, void *u, void *v, void *u_bar, void *v_bar, void *stream)
{
    if (!op || !op->shard || !u || !v || !u_bar || !v_bar) {
        set_error("sme_shard_end: bad arguments");
        return SME_ERR_ARG;
    }
    SME_TRY(shard_begun(op, 0, "sme_shard_end"));
    cudaStream_t s = (cudaStream_t)stream;
    const ShardInfo &I = *op->shard;
    if (op->dbl) {
        shard_store<double><<<nblk(op->m), 256, 0, s>>>(op->m, I.r0, op->fwd.perm, (double *)op->ws.u,
                                                        (double *)op->ws.ub, (double *)u, (double *)u_bar);
        shard_store<double><<<nblk(op->n), 256, 0, s>>>(op->n, I.c0, op->bwd.perm, (double *)op->ws.v,
                                                        (double *)op->ws.vb, (double *)v, (double *)v_bar);
    } else {
        shard_store<float><<<nblk(op->m), 256, 0, s>>>(op->m, I.r0, op->fwd.perm, (float *)op->ws.u, (float *)op->ws.ub,
                                                       (float *)u, (float *)u_bar);
        shard_store<float><<<nblk(op->n), 256, 0, s>>>(op->n, I.c0, op->bwd.perm, (float *)op->ws.v, (float *)op->ws.vb,
                                                       (float *)v, (float *)v_bar);
    }
    SME_CUDA(cudaGetLastError());
    return SME_OK;
}
