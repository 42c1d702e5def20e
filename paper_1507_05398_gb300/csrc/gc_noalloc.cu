// gc_noalloc.cu -- gc_generate_noalloc: the whole sweep without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the moment they need a code:
// runtimes that have no device allocator of their own, hosts whose device
// memory is all handed to another framework's pool up front (so a
// cudaMalloc from this library would fail or fragment that pool), and code
// on a latency-critical path where an allocation's synchronisation is not
// acceptable.  This entry point takes only the caller's output and
// statistics buffers and keeps the sweep's scratch (control words, survivor
// segments, code store or exclusion bitmap, ball table) in one file-scope
// device array of kNoAllocScratchBytes.  Every GPU that loads the library
// holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gc_internal.h"

namespace gc {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory, so the device address is looked up once per device (with that
// device current) and cached.
static std::mutex g_mu;
static void* g_scratch_ptr[kMaxDevices] = {};

static int scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(GC_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(GC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" size_t gc_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int gc_generate_noalloc(const gc_problem* prob, const gc_plan_t* plan, uint32_t* d_out,
                                   uint64_t capacity, gc_stats* d_stats, void* stream) {
    if (!prob || !d_stats || (!d_out && capacity > 0)) return fail(GC_ERR_INVALID, "null argument");
    size_t need = 0;
    const int rc0 = workspace_bytes(prob, plan, &need);
    if (rc0) return rc0;
    if (need > kNoAllocScratchBytes)
        return fail(GC_ERR_UNSUPPORTED,
                    "problem needs " + std::to_string(need) + " bytes of scratch; the static scratch "
                    "of gc_generate_noalloc holds " + std::to_string(kNoAllocScratchBytes));
    void* ws = nullptr;
    int rc = scratch_for_current_device(&ws);
    if (rc) return rc;
    return gc_generate_async(prob, plan, d_out, capacity, d_stats, ws, kNoAllocScratchBytes, stream);
}
