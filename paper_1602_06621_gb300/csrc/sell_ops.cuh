// Device helpers shared by the LSQR, CCP and evaluation kernels: FP64 block sums, deterministic grid
// reductions (the last block to arrive sums the block partials in block order), and the software-pipelined
// dot product of one sliced-ELL row with a gathered vector.
#pragma once

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
    double v = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += ((volatile const double *)partials)[i];
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

// sum_l a_l * g[c_l] over the row owned by this thread (acc type `acc_t`), software-pipelined.
template <typename real, typename acc_t, typename G>
__device__ __forceinline__ acc_t sell_row_dot(const Sell &S, int64_t slice, int lane, const G *g, bool active = true)
{
    // An inactive lane loads nothing and returns 0 (its row belongs to a finished problem).
    const int np = active ? S.slice_w[slice] / 2 : 0;
    const int64_t pbase = S.slice_off[slice] / 2 + lane;
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

}  // namespace sme
