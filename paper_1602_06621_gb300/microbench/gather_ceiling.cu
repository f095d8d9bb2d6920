// Random-gather throughput on one GPU: 8-byte loads at uniform-random indices from a table in L2, in L1,
// or in shared memory.  It measures the ceiling that bounds the sparse probe products (one gather per
// nonzero per pass).  Not part of the library.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o gather_ceiling gather_ceiling.cu && ./gather_ceiling
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16; return x;
}

template <int MODE>
__device__ __forceinline__ uint2 ld8(const uint2 *p) {
    if (MODE == 0) return __ldg(p);
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}

template <int MODE>
__global__ void gather8(const uint2 *__restrict__ tab, uint32_t mask, int G, uint32_t *out) {
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(tid * 2654435761u + 1);
    uint32_t acc = 0;
#pragma unroll 8
    for (int g = 0; g < G; ++g) {
        h = h * 1664525u + 1013904223u;
        uint2 e = ld8<MODE>(tab + ((h >> 3) & mask));
        acc += e.x ^ e.y;
    }
    out[tid] = acc;
}

// Table copied to shared memory first (entries <= 24576), then random gathers from shared memory.
__global__ void gather8_smem(const uint2 *__restrict__ tab, uint32_t entries, int G, uint32_t *out) {
    extern __shared__ uint2 sm[];
    for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) sm[i] = tab[i];
    __syncthreads();
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(tid * 2654435761u + 1);
    uint32_t acc = 0;
#pragma unroll 8
    for (int g = 0; g < G; ++g) {
        h = h * 1664525u + 1013904223u;
        uint2 e = sm[(h >> 3) % entries];
        acc += e.x ^ e.y;
    }
    out[tid] = acc;
}

int main() {
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int threads = 256, blocks = 152 * 8;
    uint32_t *out; cudaMalloc(&out, (size_t)threads * blocks * sizeof(uint32_t) * 4);
    const int G = 256;
    for (int logsz : {12, 13, 14, 19, 22}) {   // 32 KB, 64 KB, 128 KB (L1-resident), 4 MB, 32 MB
        size_t entries = (size_t)1 << logsz;
        uint2 *tab; cudaMalloc(&tab, entries * sizeof(uint2)); cudaMemset(tab, 1, entries * sizeof(uint2));
        for (int mode = 0; mode < 2; ++mode) {
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0);
                if (mode == 0) gather8<0><<<blocks, threads>>>(tab, (uint32_t)(entries - 1), G, out);
                else gather8<1><<<blocks, threads>>>(tab, (uint32_t)(entries - 1), G, out);
                cudaEventRecord(e1); cudaEventSynchronize(e1);
                float ms; cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 2) {
                    double g = (double)blocks * threads * G;
                    printf("gather8 %s table %8.1f KB: %.3f ms, %.3e gathers/s\n", mode ? "no_alloc" : "ldg     ",
                           entries * 8 / 1e3, ms, g / (ms * 1e-3));
                }
            }
        }
        cudaFree(tab);
    }
    {
        const uint32_t entries = 24576;  // 192 KB
        uint2 *tab; cudaMalloc(&tab, entries * sizeof(uint2)); cudaMemset(tab, 1, entries * sizeof(uint2));
        cudaFuncSetAttribute(gather8_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, entries * 8);
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            gather8_smem<<<152, 1024, entries * 8>>>(tab, entries, G * 2, out);
            cudaEventRecord(e1); cudaEventSynchronize(e1);
            float ms; cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 2) {
                double g = 152.0 * 1024 * G * 2;
                printf("gather8 smem  table %8.1f KB: %.3f ms, %.3e gathers/s\n", entries * 8 / 1e3, ms, g / (ms * 1e-3));
            }
        }
        cudaFree(tab);
    }
    cudaError_t e = cudaDeviceSynchronize();
    printf("status: %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
