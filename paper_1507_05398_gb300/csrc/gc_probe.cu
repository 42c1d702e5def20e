// gc_probe.cu -- measured ceilings of the two strategies on this GPU.
//  - The distance test's arithmetic: every thread keeps eight candidates in
//    registers and tests them against a stream of codewords generated in
//    registers (XOR, popcount, compare, OR into a flag), so no memory traffic
//    limits it.  The denominator of the distance kernel's roofline.
//  - The ball marks' word ORs: atomic ORs (no return value) at random words
//    of a region, the bitmap strategy's marking operation.  The denominator
//    of the marks' throughput.
#include <cuda_runtime.h>

#include <cstdint>

#include "gc_internal.h"

namespace gc {

__global__ void __launch_bounds__(256) probe_popc_kernel(uint32_t seed, int iters, int d,
                                                        uint32_t* sink) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (seed + 977u * k) * (threadIdx.x + 131u * blockIdx.x + 1u);
    uint32_t c = seed ^ (threadIdx.x * 2654435761u);
    uint32_t hits = 0;
    for (int i = 0; i < iters; ++i) {
        c = c * 1664525u + 1013904223u;
#pragma unroll
        for (int k = 0; k < 8; ++k) hits += (uint32_t)(__popc(x[k] ^ c) < d);
    }
    // the count depends on every test and the seed is a run-time value, so
    // the compiler cannot drop the loop
    if (hits == seed) sink[0] = hits;
}

__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Every thread ORs one bit into `per_thread` pseudo-random words of
// buf[0..mask_words].
__global__ void __launch_bounds__(1024) probe_or_kernel(uint32_t* buf, uint32_t mask_words,
                                                       int per_thread, uint32_t seed) {
    uint32_t h = probe_mix((blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + seed);
    for (int k = 0; k < per_thread; ++k) {
        h = probe_mix(h + 0x9e3779b9u);
        atomicOr(buf + (h & mask_words), 1u << (h >> 27));
    }
}

}  // namespace gc

extern "C" int gc_probe_mark_rate(double* ors_per_second, size_t region_bytes) {
    using namespace gc;
    if (!ors_per_second) return fail(GC_ERR_INVALID, "null argument");
    if (region_bytes == 0) region_bytes = 64ull << 20;
    if (region_bytes < (1ull << 20) || region_bytes > (1ull << 30) ||
        (region_bytes & (region_bytes - 1)) != 0)
        return fail(GC_ERR_INVALID, "region must be a power of two from 1 MiB to 1 GiB");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t* buf = nullptr;
    if (cudaMalloc(&buf, region_bytes) != cudaSuccess) return fail(GC_ERR_OOM, "probe region");
    const uint32_t mask = (uint32_t)(region_bytes / 4 - 1);
    const int blocks = sms * 2, threads = 1024, per = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaMemset(buf, 0, region_bytes);
    probe_or_kernel<<<blocks, threads>>>(buf, mask, per, 17u);  // warm-up
    cudaEventRecord(a);
    probe_or_kernel<<<blocks, threads>>>(buf, mask, per, 18u);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    *ors_per_second = (double)blocks * threads * per / (ms * 1e-3);
    return GC_OK;
}

extern "C" int gc_probe_test_rate(double* tests_per_second, double* sm_clock_hz_hint) {
    using namespace gc;
    if (!tests_per_second) return fail(GC_ERR_INVALID, "null argument");
    int dev = 0, sms = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) return fail(GC_ERR_OOM, "probe sink");
    const int blocks = sms * 8, threads = 256, iters = 1 << 14;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    probe_popc_kernel<<<blocks, threads>>>(12345u, iters, 8, sink);  // warm-up
    cudaEventRecord(a);
    probe_popc_kernel<<<blocks, threads>>>(777u, iters, 8, sink);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    *tests_per_second = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
    if (sm_clock_hz_hint) *sm_clock_hz_hint = clk_khz * 1e3;
    return GC_OK;
}
