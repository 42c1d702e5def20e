// gc_probe.cu -- measured throughput of the distance test's arithmetic on
// this GPU: every thread keeps eight candidates in registers and tests them
// against a stream of codewords generated in registers (XOR, popcount,
// compare, OR into a flag), so no memory traffic limits it.  The rate it
// reports is the denominator of the distance kernel's arithmetic roofline.
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

}  // namespace gc

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
