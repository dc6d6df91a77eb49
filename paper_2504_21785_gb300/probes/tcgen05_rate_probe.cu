// Issue rate of tcgen05.mma.cta_group::1.kind::tf32 (M = 128, K = 8) for N =
// 64, 128 and 256, into one accumulator or two alternating ones: the clocks
// per instruction of 4096 chained MMAs on operands fixed in shared memory
// (zeros, canonical K-major layout without swizzle), measured with clock64 by
// the issuing thread up to the completion of the last one (commit + mbarrier,
// bounded wait).  One CTA, and one CTA per SM (152).  The denominator of the
// tensor-core direct sum's MMA time.  Standalone (no library code).  Build and
// run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O2 -o tcgen05_rate_probe tcgen05_rate_probe.cu
//   ./tcgen05_rate_probe
#include <cstdio>
#include <cstdint>
__device__ __forceinline__ unsigned sa(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t desc(unsigned addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}
template <int N, int NACC>
__global__ void rate(long long *out, int iters) {
    extern __shared__ __align__(1024) unsigned char sm[];   // A 128x8 (4 KB) + B Nx8 (N*32 B)
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned s_tmem;
    for (int e = threadIdx.x; e < (4096 + N * 32) / 4; e += blockDim.x) reinterpret_cast<float *>(sm)[e] = 0.0f;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    constexpr unsigned cols = N * NACC <= 32 ? 32 : (N * NACC <= 64 ? 64 : (N * NACC <= 128 ? 128 : (N * NACC <= 256 ? 256 : 512)));
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&s_tmem)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = s_tmem;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((128u >> 4) << 24);
    if (threadIdx.x == 0) {
        const uint64_t da = desc(sa(sm)), db = desc(sa(sm + 4096));
        long long t0 = clock64();
        for (int i = 0; i < iters; ++i) {
            const unsigned d = tmem + (unsigned)((i % NACC) * N);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d), "l"(da), "l"(db), "r"(idesc), "r"(i >= NACC ? 1 : 0));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&bar)));
        unsigned ok = 0;
        for (int it = 0; it < (1 << 26) && !ok; ++it)
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(sa(&bar)));
        long long t1 = clock64();
        out[blockIdx.x] = ok ? (t1 - t0) : -1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}
template <int N, int NACC>
void run(int blocks) {
    long long *d, h[152];
    cudaMalloc(&d, sizeof(h));
    const int iters = 4096;
    size_t smem = 4096 + N * 32;
    rate<N, NACC><<<blocks, 128, smem>>>(d, iters);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("err %s\n", cudaGetErrorString(e)); exit(1); }
    cudaMemcpy(h, d, blocks * 8, cudaMemcpyDeviceToHost);
    long long mx = 0;
    for (int b = 0; b < blocks; ++b) mx = h[b] > mx ? h[b] : mx;
    printf("N=%d acc=%d blocks=%d: %.1f cycles per MMA (%.0f flop/cycle/SM)\n", N, NACC, blocks, (double)mx / iters,
           2.0 * 128 * N * 8 * iters / (double)mx);
    cudaFree(d);
}
int main() {
    run<64, 1>(1); run<64, 2>(1); run<128, 1>(1); run<256, 1>(1); run<256, 2>(1);
    run<64, 1>(152); run<256, 1>(152);
    return 0;
}
