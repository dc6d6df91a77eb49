// Throughput of 8-byte (float2), 16-byte (float4), f32 and f64 reductions to
// global memory under several address patterns on one GPU: the denominators of
// the scatter's roofline.  Standalone (no library code); every index is masked
// into its buffer.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o l2_reduction_probe l2_reduction_probe.cu
//   ./l2_reduction_probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t hsh(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16; return x;
}

// pattern: 0 = each lane random; G>1 = groups of G lanes to G consecutive
// elements (group base aligned to G); window>0: warp base random, lane random
// within 'window' elements after it.
template <class T, int G>
__global__ void red_kernel(T *buf, uint32_t mask, int iters, uint32_t window, uint32_t hot) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31, warp = tid >> 5;
    T v; 
    if constexpr (sizeof(T) == 8 && alignof(T) == 8 && !std::is_same<T,double>::value) { v.x = 1.f; v.y = 1.f; }
    for (int it = 0; it < iters; ++it) {
        uint32_t idx;
        if (hot) {
            idx = hsh(tid * 131u + it) % hot;
        } else if (window) {
            const uint32_t base = hsh(warp * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask;
            idx = (base + hsh(tid * 7919u + it * 104729u) % window) & mask;
        } else if (G == 1) {
            idx = hsh(tid * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask;
        } else {
            const uint32_t grp = tid / G;
            idx = ((hsh(grp * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask) & ~(uint32_t)(G - 1)) + (lane % G);
        }
        if constexpr (std::is_same<T, double>::value) atomicAdd(buf + idx, 1.0);
        else if constexpr (std::is_same<T, float>::value) atomicAdd(buf + idx, 1.f);
        else atomicAdd(buf + idx, v);
    }
}
template <int G>
__global__ void red4_kernel(float4 *buf, uint32_t mask, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    for (int it = 0; it < iters; ++it) {
        uint32_t idx;
        if (G == 1) idx = hsh(tid * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask;
        else idx = ((hsh((tid / G) * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask) & ~(uint32_t)(G - 1)) + (lane % G);
        atomicAdd(buf + idx, make_float4(1.f, 1.f, 1.f, 1.f));
    }
}
__global__ void red_d2_kernel(double2 *buf, uint32_t mask, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        uint32_t idx = hsh(tid * 0x9E3779B9u + it * 0x85EBCA6Bu) & mask;
        atomicAdd(&buf[idx].x, 1.0);
        atomicAdd(&buf[idx].y, 1.0);
    }
}

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

int main() {
    int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const size_t big = size_t(1) << 32;   // 4 GiB buffer
    void *buf; CK(cudaMalloc(&buf, big)); CK(cudaMemset(buf, 0, big));
    const int threads = 256, blocks = sms * 16, iters = 256;
    const double ops = double(threads) * blocks * iters;
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    auto time = [&](auto launch, const char *name, double per_op_elems) {
        launch(); CK(cudaDeviceSynchronize());
        float best = 1e30f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1);
            float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
        }
        CK(cudaGetLastError());
        printf("%-44s %8.3f ms  %8.2f G red/s  %8.2f G elem/s\n", name, best, ops / best * 1e-6, ops * per_op_elems / best * 1e-6);
        return 0;
    };
    // element counts: 64 MiB region (fits L2) and 4 GiB region
    const uint32_t m2_l2 = (64u << 20) / 8 - 1, m2_hbm = uint32_t((big / 8) - 1);
    float2 *b2 = (float2 *)buf;
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 random, 64MiB", 1);
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_hbm, iters, 0, 0); }, "float2 random, 4GiB", 1);
    time([&] { red_kernel<float2, 2><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 groups of 2 (16B), 64MiB", 1);
    time([&] { red_kernel<float2, 4><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 groups of 4 (32B), 64MiB", 1);
    time([&] { red_kernel<float2, 8><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 groups of 8 (64B), 64MiB", 1);
    time([&] { red_kernel<float2, 16><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 groups of 16 (128B), 64MiB", 1);
    time([&] { red_kernel<float2, 32><<<blocks, threads>>>(b2, m2_l2, iters, 0, 0); }, "float2 groups of 32 (256B), 64MiB", 1);
    time([&] { red_kernel<float2, 4><<<blocks, threads>>>(b2, m2_hbm, iters, 0, 0); }, "float2 groups of 4 (32B), 4GiB", 1);
    time([&] { red_kernel<float2, 32><<<blocks, threads>>>(b2, m2_hbm, iters, 0, 0); }, "float2 groups of 32 (256B), 4GiB", 1);
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_l2, iters, 3200, 0); }, "float2 warp window 3200 cells, 64MiB", 1);
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_hbm, iters, 3200, 0); }, "float2 warp window 3200 cells, 4GiB", 1);
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_l2, iters, 0, 4096); }, "float2 hot 4096 cells", 1);
    time([&] { red_kernel<float2, 1><<<blocks, threads>>>(b2, m2_l2, iters, 0, 64); }, "float2 hot 64 cells", 1);
    float4 *b4 = (float4 *)buf;
    time([&] { red4_kernel<1><<<blocks, threads>>>(b4, (64u << 20) / 16 - 1, iters); }, "float4 random, 64MiB (2 cells/op)", 2);
    time([&] { red4_kernel<2><<<blocks, threads>>>(b4, (64u << 20) / 16 - 1, iters); }, "float4 groups of 2 (32B), 64MiB", 2);
    time([&] { red4_kernel<8><<<blocks, threads>>>(b4, (64u << 20) / 16 - 1, iters); }, "float4 groups of 8 (128B), 64MiB", 2);
    float *b1 = (float *)buf;
    time([&] { red_kernel<float, 1><<<blocks, threads>>>(b1, (64u << 20) / 4 - 1, iters, 0, 0); }, "f32 random, 64MiB", 1);
    time([&] { red_kernel<float, 8><<<blocks, threads>>>(b1, (64u << 20) / 4 - 1, iters, 0, 0); }, "f32 groups of 8 (32B), 64MiB", 1);
    double *bd = (double *)buf;
    time([&] { red_kernel<double, 1><<<blocks, threads>>>(bd, (64u << 20) / 8 - 1, iters, 0, 0); }, "f64 random, 64MiB", 1);
    time([&] { red_d2_kernel<<<blocks, threads>>>((double2 *)buf, (64u << 20) / 16 - 1, iters); }, "double2 as 2 x f64 random, 64MiB (per cell)", 1);
    cudaFree(buf);
    printf("probe done\n");
    return 0;
}
