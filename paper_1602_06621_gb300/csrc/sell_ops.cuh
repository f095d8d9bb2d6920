// Device helpers shared by the LSQR, CCP and evaluation kernels: FP64 block sums, deterministic grid
// reductions (the last block to arrive sums the block partials in block order), and the software-pipelined
// dot product of one sliced-ELL row with a gathered vector.
#pragma once

#include <algorithm>

#include "sme_internal.cuh"

namespace sme {

constexpr int LQ_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum; valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[LQ_THREADS / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < LQ_THREADS / 32 ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Writes this block's partial, and returns true in every thread of the block that arrives last.
__device__ __forceinline__ bool arrive_last(double part, double *partials, unsigned *counter)
{
    __shared__ bool last;
    const double b = block_sum(part);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return last;
}

// In the last block: the sum of all partials in a fixed order (deterministic).
__device__ __forceinline__ double sum_partials(const double *partials, unsigned *counter)
{
    __threadfence();
    // Loads through L2 (the partials come from other SMs), several in flight per thread; each thread still
    // adds its partials in index order.
    double v = 0.0;
#pragma unroll 4
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
    const double s = block_sum(v);
    __shared__ double res;
    if (threadIdx.x == 0) {
        res = s;
        *counter = 0u;
    }
    __syncthreads();
    return res;
}

template <typename real>
__device__ __forceinline__ void pair_load(const Sell &S, int64_t pi, int &c0, real &a0, int &c1, real &a1)
{
    if (sizeof(real) == 4) {
        const int4 e = __ldcs((const int4 *)S.ent + pi);
        c0 = e.x;
        c1 = e.z;
        a0 = (real)__int_as_float(e.y);
        a1 = (real)__int_as_float(e.w);
    } else {
        const int2 c = __ldcs((const int2 *)S.ent + pi);
        const double2 v = __ldcs((const double2 *)S.val64 + pi);
        c0 = c.x;
        c1 = c.y;
        a0 = (real)v.x;
        a1 = (real)v.y;
    }
}

// sum_l a_l * g[c_l] over pair steps [q0, q1) of the row owned by this thread (acc type `acc_t`),
// software-pipelined: the entries two steps ahead and the gathers one step ahead are in flight.
template <typename real, typename acc_t, typename G>
__device__ __forceinline__ acc_t sell_row_dot_range(const Sell &S, int64_t slice, int lane, const G *g, int q0, int q1)
{
    const int np = q1 - q0;
    const int64_t pbase = S.slice_off[slice] / 2 + lane + (int64_t)q0 * 32;
    acc_t acc = acc_t(0);
    int c0 = 0, c1 = 0, n0 = 0, n1 = 0;
    real a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    if (np > 0) pair_load<real>(S, pbase, c0, a0, c1, a1);
    if (np > 1) pair_load<real>(S, pbase + 32, n0, b0, n1, b1);
    G g0 = np > 0 ? g[c0] : G(0), g1 = np > 0 ? g[c1] : G(0);
    for (int q = 0; q < np; ++q) {
        G h0 = G(0), h1 = G(0);
        if (q + 1 < np) {
            h0 = g[n0];
            h1 = g[n1];
        }
        int m0 = 0, m1 = 0;
        real d0 = 0, d1 = 0;
        if (q + 2 < np) pair_load<real>(S, pbase + (int64_t)(q + 2) * 32, m0, d0, m1, d1);
        acc += (acc_t)a0 * (acc_t)g0;
        acc += (acc_t)a1 * (acc_t)g1;
        a0 = b0;
        a1 = b1;
        b0 = d0;
        b1 = d1;
        n0 = m0;
        n1 = m1;
        g0 = h0;
        g1 = h1;
    }
    return acc;
}

// The whole row owned by this thread.
template <typename real, typename acc_t, typename G>
__device__ __forceinline__ acc_t sell_row_dot(const Sell &S, int64_t slice, int lane, const G *g, bool active = true)
{
    // An inactive lane loads nothing and returns 0 (its row belongs to a finished problem).
    return sell_row_dot_range<real, acc_t, G>(S, slice, lane, g, 0, active ? S.slice_w[slice] / 2 : 0);
}

// Slices of long rows shared by SPLIT warps of a LQ_THREADS-thread block: warp w takes slice
// blockIdx.x * (8 / SPLIT) + w / SPLIT and the w % SPLIT-th contiguous range of its pair steps, so loads
// stay coalesced and a slice's latency chain is SPLIT times shorter.  The partial sums are added in warp
// order (deterministic) and the full row sum is returned in the slice's first warp (part 0); every thread
// of the block must call this (it synchronises the block).
template <int SPLIT>
struct SplitSlice {
    int64_t slice;
    int part, lane;
    __device__ __forceinline__ SplitSlice()
    {
        const int warp = threadIdx.x >> 5;
        lane = threadIdx.x & 31;
        slice = (int64_t)blockIdx.x * (LQ_THREADS / 32 / SPLIT) + warp / SPLIT;
        part = warp % SPLIT;
    }
    __device__ __forceinline__ bool lead() const { return part == 0; }
};

template <typename real, typename acc_t, typename G, int SPLIT>
__device__ __forceinline__ acc_t sell_row_dot_split(const Sell &S, const SplitSlice<SPLIT> &w, const G *g)
{
    acc_t acc = acc_t(0);
    if (w.slice < S.nslices) {
        const int np = S.slice_w[w.slice] / 2;
        acc = sell_row_dot_range<real, acc_t, G>(S, w.slice, w.lane, g, np * w.part / SPLIT,
                                                 np * (w.part + 1) / SPLIT);
    }
    if (SPLIT == 1) return acc;
    __shared__ acc_t partial[LQ_THREADS];
    partial[threadIdx.x] = acc;
    __syncthreads();
    acc_t tot = acc_t(0);
    if (w.part == 0)
        for (int p = 0; p < SPLIT; ++p) tot += partial[threadIdx.x + p * 32];
    __syncthreads();
    return tot;
}

// Warps per slice for a sliced-ELL copy: enough that a lane walks about 16 pair steps or fewer.
inline int split_for(const Sell &S)
{
    const double steps = S.nslices > 0 ? (double)S.entries / (64.0 * (double)S.nslices) : 0.0;
    return steps >= 96 ? 8 : steps >= 48 ? 4 : steps >= 24 ? 2 : 1;
}

// Launch geometry of one sliced-ELL pass with SPLIT warps per slice.
struct Pass {
    int split;
    unsigned blocks;
};

inline Pass pass_for(const Sell &S)
{
    const int sp = split_for(S);
    const int64_t per_block = LQ_THREADS / 32 / sp;
    return Pass{sp, (unsigned)std::max<int64_t>((S.nslices + per_block - 1) / per_block, 1)};
}

// Dispatch a kernel template over the split factor.
#define SPLIT_LAUNCH(kernel, real, pass, s, ...)                                                    \
    do {                                                                                          \
        switch ((pass).split) {                                                                   \
            case 8: kernel<real, 8><<<(pass).blocks, LQ_THREADS, 0, s>>>(__VA_ARGS__); break;     \
            case 4: kernel<real, 4><<<(pass).blocks, LQ_THREADS, 0, s>>>(__VA_ARGS__); break;     \
            case 2: kernel<real, 2><<<(pass).blocks, LQ_THREADS, 0, s>>>(__VA_ARGS__); break;     \
            default: kernel<real, 1><<<(pass).blocks, LQ_THREADS, 0, s>>>(__VA_ARGS__); break;    \
        }                                                                                         \
    } while (0)

// A CUDA graph captured once from a stream of launches (on its own stream) and destroyed with its scope;
// exec stays null when capture is not possible, and the caller then launches directly.
struct GraphOnce {
    cudaGraphExec_t exec = nullptr;
    template <typename F>
    void capture(F &&enqueue)
    {
        cudaStream_t q = nullptr;
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            enqueue(q);
            if (cudaStreamEndCapture(q, &g) == cudaSuccess && g) {
                if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();
        cudaStreamDestroy(q);
    }
    ~GraphOnce()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

}  // namespace sme
