// gc_server.cu -- continuous-batching request server for code generation.
//
// One persistent cooperative launch of the sweep runs in serving mode: its
// SM groups take jobs from a ring of descriptors in host-mapped memory while
// it runs.  The host side (this file) admits a request when its output fits
// in the device pool (first-fit, by the request's capacity bound) and its
// scratch fits a group, writes its descriptor, raises `tail`, and later sees
// done[slot] raised by the group that ran it.  Requests that arrive while
// others run are admitted as soon as pool space and ring slots free up, and
// their sweeps overlap on the device with the ones already running.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "gc_internal.h"

namespace gc {

struct ServerRequest {
    uint64_t id = 0;
    int state = 0;          // 0 free, 1 in flight, 2 done (not yet released)
    size_t pool_off = 0, pool_len = 0;
    uint64_t capacity = 0;
};

}  // namespace gc

struct gc_server {
    int dev = 0;
    gc_server_config cfg{};
    cudaStream_t stream = nullptr;   // the persistent kernel
    cudaStream_t copy = nullptr;     // result copies
    gc::ServeLayout L;
    void* ws = nullptr;              // device workspace (groups, flags, scratch)
    void* pool = nullptr;            // device output pool
    gc_stats* stats = nullptr;       // device, one per ring slot
    // host-mapped control block
    gc::JobDescHost* ring = nullptr;
    unsigned* tail = nullptr;
    unsigned* stop = nullptr;
    unsigned long long* done = nullptr;
    unsigned next_id = 0;            // == published count (tail)
    std::vector<gc::ServerRequest> slots;
    std::map<size_t, size_t> free_blocks;  // offset -> length
    bool running = false;
};

namespace gc {

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static bool pool_alloc(gc_server* s, size_t len, size_t* off) {
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second >= len) {
            *off = it->first;
            const size_t rest = it->second - len;
            const size_t at = it->first + len;
            s->free_blocks.erase(it);
            if (rest) s->free_blocks[at] = rest;
            return true;
        }
    }
    return false;
}

static void pool_free(gc_server* s, size_t off, size_t len) {
    auto it = s->free_blocks.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

}  // namespace gc

using namespace gc;

extern "C" {

int gc_server_create(const gc_server_config* cfg_in, gc_server** out) {
    if (!out) return fail(GC_ERR_INVALID, "null argument");
    *out = nullptr;
    gc_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_n <= 0) cfg.max_n = 28;
    if (cfg.max_n > 32) return fail(GC_ERR_INVALID, "max_n > 32");
    if (cfg.pool_bytes == 0) cfg.pool_bytes = 4ull << 30;
    if (cfg.queue_capacity <= 0) cfg.queue_capacity = 1024;
    if (cfg.store_words == 0) cfg.store_words = 1ull << 22;
    if (cfg.idle_seconds <= 0) cfg.idle_seconds = 30.0;
    gc_server* s = new gc_server();
    s->cfg = cfg;
    cudaGetDevice(&s->dev);
    std::string why;
    if (!serve_layout(cfg, &s->L, &why)) {
        delete s;
        return fail(GC_ERR_UNSUPPORTED, why);
    }
    cudaError_t e;
    const size_t Q = (size_t)cfg.queue_capacity;
    void* ctrl = nullptr;
    const size_t ctrl_bytes = align256(sizeof(JobDescHost) * Q) + 256 + align256(8 * Q);
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&s->ws, s->L.total)) != cudaSuccess ||
        (e = cudaMalloc(&s->pool, cfg.pool_bytes)) != cudaSuccess ||
        (e = cudaMalloc((void**)&s->stats, sizeof(gc_stats) * Q)) != cudaSuccess ||
        (e = cudaHostAlloc(&ctrl, ctrl_bytes, cudaHostAllocMapped)) != cudaSuccess) {
        gc_server_destroy(s);
        return fail(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA, cudaGetErrorString(e));
    }
    std::memset(ctrl, 0, ctrl_bytes);
    uint8_t* c = static_cast<uint8_t*>(ctrl);
    s->ring = reinterpret_cast<JobDescHost*>(c);
    s->tail = reinterpret_cast<unsigned*>(c + align256(sizeof(JobDescHost) * Q));
    s->stop = s->tail + 1;
    s->done = reinterpret_cast<unsigned long long*>(c + align256(sizeof(JobDescHost) * Q) + 256);
    s->slots.assign(Q, ServerRequest());
    s->free_blocks[0] = cfg.pool_bytes;
    if ((e = cudaMemset(static_cast<uint8_t*>(s->ws) + s->L.off_head, 0, 256)) != cudaSuccess) {
        gc_server_destroy(s);
        return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    s->L.ws = s->ws;
    int rc = launch_server(s->L, s->ws, s->ring, s->tail, s->stop, s->done, (uint32_t)Q,
                           cfg.idle_seconds, s->stream, &why);
    if (rc) {
        gc_server_destroy(s);
        return fail(rc, why);
    }
    s->running = true;
    *out = s;
    return GC_OK;
}

int gc_server_submit(gc_server* s, const gc_problem* prob, int strategy, uint64_t* request_id) {
    if (!s || !prob || !request_id) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why))
        return fail(GC_ERR_INVALID, why);
    if (p.n > s->cfg.max_n) return fail(GC_ERR_UNSUPPORTED, "n above the server's max_n");
    // the persistent kernel may have left after an idle period: restart it
    if (cudaStreamQuery(s->stream) == cudaSuccess) {
        int rc = launch_server(s->L, s->ws, s->ring, s->tail, s->stop, s->done,
                               (uint32_t)s->cfg.queue_capacity, s->cfg.idle_seconds, s->stream,
                               &why);
        if (rc) return fail(rc, why);
    }
    const uint32_t Q = (uint32_t)s->cfg.queue_capacity;
    const uint32_t slot = s->next_id % Q;
    if (s->slots[slot].state != 0) return fail(GC_ERR_CAPACITY, "request ring full");
    JobDescHost desc;
    const uint64_t cap = p.bound;
    const size_t len = align256(std::max<uint64_t>(cap, 1) * 4);
    size_t off = 0;
    if (len > s->cfg.pool_bytes) return fail(GC_ERR_UNSUPPORTED, "output larger than the pool");
    if (!pool_alloc(s, len, &off)) return fail(GC_ERR_CAPACITY, "output pool full");
    uint32_t* out = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(s->pool) + off);
    if (!serve_describe(s->L, p, strategy, out, cap, s->stats + slot, &desc, &why)) {
        pool_free(s, off, len);
        return fail(GC_ERR_UNSUPPORTED, why);
    }
    std::memcpy(&s->ring[slot], &desc, sizeof desc);
    s->done[slot] = 0;
    ServerRequest& r = s->slots[slot];
    r.id = s->next_id;
    r.state = 1;
    r.pool_off = off;
    r.pool_len = len;
    r.capacity = cap;
    std::atomic_thread_fence(std::memory_order_release);
    *(volatile unsigned*)s->tail = ++s->next_id;
    *request_id = r.id;
    return GC_OK;
}

int gc_server_poll(gc_server* s, uint64_t* done_ids, int max_ids, int* ndone) {
    if (!s || !ndone || (max_ids > 0 && !done_ids)) return fail(GC_ERR_INVALID, "null argument");
    *ndone = 0;
    const uint32_t Q = (uint32_t)s->cfg.queue_capacity;
    for (uint32_t k = 0; k < Q && *ndone < max_ids; ++k) {
        ServerRequest& r = s->slots[k];
        if (r.state != 1) continue;
        const unsigned long long v = *(volatile unsigned long long*)&s->done[k];
        if (v == r.id + 1) {
            std::atomic_thread_fence(std::memory_order_acquire);
            r.state = 2;
            done_ids[(*ndone)++] = r.id;
        }
    }
    // a kernel that stopped with requests in flight has failed
    if (*ndone == 0 && cudaStreamQuery(s->stream) != cudaErrorNotReady) {
        bool inflight = false;
        for (auto& r : s->slots) inflight |= r.state == 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
        if (inflight) {
            std::string why;
            int rc = launch_server(s->L, s->ws, s->ring, s->tail, s->stop, s->done, Q,
                                   s->cfg.idle_seconds, s->stream, &why);
            if (rc) return fail(rc, why);
        }
    }
    return GC_OK;
}

int gc_server_fetch(gc_server* s, uint64_t id, uint32_t* host_out, uint64_t* inout_count,
                    gc_stats* host_stats) {
    if (!s || !inout_count) return fail(GC_ERR_INVALID, "null argument");
    const uint32_t Q = (uint32_t)s->cfg.queue_capacity;
    ServerRequest& r = s->slots[id % Q];
    if (r.state != 2 || r.id != id) return fail(GC_ERR_INVALID, "request not finished or unknown");
    gc_stats st;
    cudaError_t e = cudaMemcpyAsync(&st, s->stats + id % Q, sizeof st, cudaMemcpyDeviceToHost, s->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    if (host_stats) *host_stats = st;
    const uint64_t want = std::min<uint64_t>(std::min<uint64_t>(st.codewords, r.capacity), *inout_count);
    if (want && host_out) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(static_cast<uint8_t*>(s->pool) + r.pool_off);
        e = cudaMemcpyAsync(host_out, src, want * 4, cudaMemcpyDeviceToHost, s->copy);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
        if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    const uint64_t have = st.codewords;
    const bool fits = have <= *inout_count;
    *inout_count = have;
    if (st.status != 0) return fail(st.status, "device-side error in the sweep");
    return fits ? GC_OK : fail(GC_ERR_CAPACITY, "output capacity too small");
}

int gc_server_release(gc_server* s, uint64_t id) {
    if (!s) return fail(GC_ERR_INVALID, "null argument");
    const uint32_t Q = (uint32_t)s->cfg.queue_capacity;
    ServerRequest& r = s->slots[id % Q];
    if (r.state != 2 || r.id != id) return fail(GC_ERR_INVALID, "request not finished or unknown");
    pool_free(s, r.pool_off, r.pool_len);
    r = ServerRequest();
    return GC_OK;
}

int gc_server_destroy(gc_server* s) {
    if (!s) return GC_OK;
    int rc = GC_OK;
    if (s->stop) *(volatile unsigned*)s->stop = 1u;
    if (s->stream) {
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) rc = GC_ERR_CUDA;
        cudaStreamDestroy(s->stream);
    }
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->ws) cudaFree(s->ws);
    if (s->pool) cudaFree(s->pool);
    if (s->stats) cudaFree(s->stats);
    if (s->ring) cudaFreeHost(s->ring);
    delete s;
    return rc;
}

}  // extern "C"
