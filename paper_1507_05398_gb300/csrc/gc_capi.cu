// gc_capi.cu -- the extern "C" entry points of libgc: argument checks,
// planning, workspace layout, allocation for the synchronous call, and the
// launches.  No exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gc_internal.h"

namespace gc {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

// C(n, k) for 0 <= n <= 64 (exact: the largest, C(64, 32), is below 2^61).
uint64_t binom64(int n, int k) {
    if (k < 0 || n < 0 || k > n || n > kMaxNWide) return 0;
    static const Binom64Table table = make_binom64();
    return table.c[n][k];
}

static unsigned __int128 ball_volume(int n, int r) {
    unsigned __int128 v = 0;
    for (int k = 0; k <= r && k <= n; ++k) v += binom64(n, k);
    return v;
}

// Inverts the basis over F_2 (Gauss-Jordan on [B | I], B's columns = basis
// vectors): inv[j] = row j of B^-1.  False if the vectors are dependent.
static bool invert_basis(int n, const uint32_t* basis, uint32_t* inv) {
    const uint32_t mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
    // rows of B: row i = bit i of every basis vector; augment with identity
    uint32_t row[32], aug[32];
    for (int i = 0; i < n; ++i) {
        row[i] = 0;
        for (int j = 0; j < n; ++j) row[i] |= ((basis[j] >> i) & 1u) << j;
        aug[i] = 1u << i;
    }
    for (int j = 0; j < n; ++j)
        if ((basis[j] & ~mask) != 0u) return false;
    for (int col = 0; col < n; ++col) {
        int piv = -1;
        for (int i = col; i < n; ++i)
            if ((row[i] >> col) & 1u) { piv = i; break; }
        if (piv < 0) return false;
        std::swap(row[piv], row[col]);
        std::swap(aug[piv], aug[col]);
        for (int i = 0; i < n; ++i)
            if (i != col && ((row[i] >> col) & 1u)) {
                row[i] ^= row[col];
                aug[i] ^= aug[col];
            }
    }
    // now B^-1 = aug as a matrix whose row i is aug[i] read by columns:
    // (B^-1)[i][k] = bit k of aug[i]; rank bit i of v = parity(aug[i] & v)
    for (int i = 0; i < n; ++i) inv[i] = aug[i];
    return true;
}

bool make_problem(const gc_problem& q, HostProblem* p, std::string* why, int max_n) {
    return make_problem(q.n, q.d, q.ordering, q.weight, p, why, q.constraint, q.basis, max_n);
}

Order order_of(const HostProblem& p, bool filter, bool even) {
    Order o{};
    o.n = p.n;
    o.ord = p.ord;
    o.w = p.w;
    o.filter = filter;
    o.even = even;
    o.N = p.N;
    uint64_t c = 0;
    for (int k = 0; k <= kMaxNWide + 1; ++k) {
        o.cum[k] = c;
        if (k <= p.n) c += binom64(p.n, k);
    }
    for (int j = 0; j < 32; ++j) {
        o.basis[j] = p.basis[j];
        o.inv[j] = p.inv[j];
    }
    return o;
}

bool make_problem(int n, int d, int ord, int w, HostProblem* p, std::string* why, int constraint,
                  const uint32_t* basis, int max_n) {
    if (n < 1 || n > max_n) {
        *why = max_n > kMaxN ? "n must be in [1, 64]"
                             : "n must be in [1, 32] (up to 64 through the *64 entry points)";
        return false;
    }
    if (d < 0) { *why = "d must be >= 0"; return false; }
    if (ord < GC_ORDER_LEX || ord > GC_ORDER_BASIS) { *why = "unknown ordering"; return false; }
    if (n > kMaxN && ord == GC_ORDER_BASIS) {
        *why = "B-orderings take n <= 32";
        return false;
    }
    if (n == kMaxNWide && w < 0) {
        *why = "n = 64 needs a weight (2^64 ranks do not fit a count)";
        return false;
    }
    for (int j = 0; j < 32; ++j) p->basis[j] = p->inv[j] = 0;
    if (ord == GC_ORDER_BASIS) {
        if (!basis) { *why = "GC_ORDER_BASIS needs a basis"; return false; }
        for (int j = 0; j < n; ++j) p->basis[j] = basis[j];
        if (!invert_basis(n, p->basis, p->inv)) {
            *why = "basis vectors are not linearly independent in F_2^n";
            return false;
        }
    }
    if (w < -1 || w > n) { *why = "weight must be -1 or in [0, n]"; return false; }
    if (constraint != GC_CONSTRAINT_NONE && constraint != GC_CONSTRAINT_SELF_ORTHOGONAL) {
        *why = "unknown constraint";
        return false;
    }
    p->orth = constraint == GC_CONSTRAINT_SELF_ORTHOGONAL;
    p->n = n;
    p->d = d;
    p->ord = ord;
    p->w = w;
    p->filter = (w >= 0 && ord == GC_ORDER_BASIS);
    p->N = (w < 0 || ord == GC_ORDER_BASIS) ? (1ull << n) : binom64(n, w);
    p->valid = (w < 0) ? (1ull << n) : binom64(n, w);
    // sphere packing: radius floor((d-1)/2) balls around codewords are disjoint
    const int t = d >= 1 ? (d - 1) / 2 : 0;
    const unsigned __int128 hb = ((unsigned __int128)1 << n) / ball_volume(n, t);
    p->bound = std::max<uint64_t>(
        1, hb < (unsigned __int128)p->valid ? (uint64_t)hb : p->valid);
    if (d <= 1) p->bound = p->valid;
    if (p->orth) p->bound = std::min<uint64_t>(p->bound, 1ull << (n / 2));
    return true;
}

// Strategy choice.  Distance strategy cost ~ executed popcount tests;
// bitmap strategy cost ~ words OR-ed by ball marking (each an L2 atomic,
// weighted as several tests) plus one lookup per candidate.  |C| is taken as
// half the sphere-packing bound (lexicodes sit close to it).
void plan_for(const HostProblem& p, gc_plan_t* pl) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    pl->grid = sms > 0 ? sms : 1;
    pl->block = 1024;
    pl->window_min = 256;
    pl->window_max = 0;
    pl->survivor_target = kTargetDistance;
    // orthogonality cannot be marked in a bitmap; n > 32 has no bitmap form
    if (p.d <= 1 || p.orth || p.n > kMaxN) {
        pl->strategy = GC_STRATEGY_DISTANCE;
        return;
    }
    const double N = (double)p.valid;
    const double C = std::max(1.0, 0.5 * (double)p.bound);
    const double space = std::ldexp(1.0, p.n);
    const double V = (double)ball_volume(p.n, p.d - 1);
    const double to_first_hit = std::max(1.0, std::min(C / 2.0, space / V));
    const double dist_cost = N * to_first_hit + 2.0 * C * C / 2.0;
    const double marks = C * (double)high_ball_len(p.n, p.d) / 2.0;
    const double bitmap_cost = 8.0 * marks + N;
    const double bitmap_bytes = space / 8.0;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const bool bitmap_ok = bitmap_bytes < 0.5 * (double)free_b && high_ball_len(p.n, p.d) < (1u << 24);
    const bool dist_ok = p.bound < 0xffffffffull;
    if (!dist_ok || (bitmap_ok && bitmap_cost < dist_cost))
        pl->strategy = GC_STRATEGY_BITMAP;
    else
        pl->strategy = GC_STRATEGY_DISTANCE;
    // a large bitmap sweep of one code runs on every SM in lockstep windows
    if (pl->strategy == GC_STRATEGY_BITMAP && p.valid >= (1ull << GC_GRID_MIN_LOG2))
        pl->strategy = GC_STRATEGY_BITMAP_GRID;
    pl->survivor_target = default_target(pl->strategy, p);
    if (const char* e = std::getenv("GC_STRATEGY")) {
        if (!std::strcmp(e, "distance")) pl->strategy = GC_STRATEGY_DISTANCE;
        if (!std::strcmp(e, "bitmap")) pl->strategy = GC_STRATEGY_BITMAP;
        if (!std::strcmp(e, "grid")) pl->strategy = GC_STRATEGY_BITMAP_GRID;
        pl->survivor_target = default_target(pl->strategy, p);
    }
}

static bool resolve_plan(const HostProblem& p, const gc_plan_t* in, gc_plan_t* out) {
    if (!tuned_plan(p, out)) plan_for(p, out);
    if (in) {
        if (in->strategy != GC_STRATEGY_AUTO && !p.orth) {
            out->strategy = in->strategy;
            out->survivor_target = default_target(in->strategy, p);
        }
        if (in->grid > 0) out->grid = in->grid;
        if (in->window_min) out->window_min = in->window_min;
        if (in->window_max) out->window_max = in->window_max;
        if (in->survivor_target) out->survivor_target = in->survivor_target;
    }
    return out->strategy == GC_STRATEGY_DISTANCE || out->strategy == GC_STRATEGY_BITMAP ||
           out->strategy == GC_STRATEGY_BITMAP_GRID;
}

// The plan of a wide sweep: the distance strategy (the bitmap has no wide
// form); an explicit bitmap request fails.
static bool resolve_plan_wide(const HostProblem& p, const gc_plan_t* in, gc_plan_t* out) {
    if (!resolve_plan(p, in, out)) return false;
    if (out->strategy == GC_STRATEGY_BITMAP || out->strategy == GC_STRATEGY_BITMAP_GRID) {
        if (in && (in->strategy == GC_STRATEGY_BITMAP || in->strategy == GC_STRATEGY_BITMAP_GRID))
            return false;
        out->strategy = GC_STRATEGY_DISTANCE;
        out->survivor_target =
            (in && in->survivor_target) ? in->survivor_target : kTargetDistance;
    }
    return true;
}

static bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// d <= 1 with no weight filter: every candidate is accepted, in order.
__global__ void all_accepted_stats(gc_stats* st, uint64_t N, int strategy) {
    st->codewords = N;
    st->candidates = N;
    st->dense_tests = N * (N - 1) / 2;  // candidate i meets the i before it
    st->executed_tests = 0;
    st->marks = 0;
    st->windows = 0;
    st->survivors = 0;
    st->status = 0;
    st->strategy = strategy;
    for (int k = 0; k < 12; ++k) st->phase_cycles[k] = 0;
    st->pair_windows = 0;
    st->pair_fallbacks = 0;
}

// wide: run the uint64-word kernel (n <= 64; d_out holds uint64 words).
static int generate_async_impl(const HostProblem& p, const gc_plan_t& plan, void* d_out,
                               uint64_t capacity, gc_stats* d_stats, void* ws, size_t ws_bytes,
                               cudaStream_t s, bool wide = false) {
    if (p.d <= 1 && !p.filter && !p.orth && !wide) {
        int rc = launch_unrank(p, 0, std::min(capacity, p.N), static_cast<uint32_t*>(d_out), s);
        if (rc) return rc;
        all_accepted_stats<<<1, 1, 0, s>>>(d_stats, p.N, plan.strategy);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GC_OK : fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    std::string why;
    if (plan.strategy == GC_STRATEGY_BITMAP_GRID && !wide) {
        GridLayout GL;
        if (!grid_sweep_layout(p, plan, &GL, &why)) return fail(GC_ERR_UNSUPPORTED, why);
        if (ws_bytes < GL.total) return fail(GC_ERR_INVALID, "workspace too small");
        if (((uintptr_t)ws & 255u) != 0) return fail(GC_ERR_INVALID, "workspace not 256-byte aligned");
        const int rc = launch_grid_sweep(p, GL, static_cast<uint32_t*>(d_out), capacity, d_stats,
                                         ws, s, &why);
        return rc ? fail(rc, why) : GC_OK;
    }
    BatchJob job{p, plan, d_out, capacity, d_stats, wide};
    BatchLayout L;
    if (!batch_layout(&job, 1, 1, &L, &why)) return fail(GC_ERR_UNSUPPORTED, why);
    if (ws_bytes < L.total) return fail(GC_ERR_INVALID, "workspace too small");
    if (((uintptr_t)ws & 255u) != 0) return fail(GC_ERR_INVALID, "workspace not 256-byte aligned");
    int rc = launch_batch(&job, 1, L, ws, s, &why);
    if (rc) return fail(rc, why);
    return GC_OK;
}

static size_t single_workspace(const HostProblem& p, const gc_plan_t& pl, std::string* why,
                               bool wide = false) {
    if (p.d <= 1 && !p.filter && !p.orth && !wide) return 256;
    if (pl.strategy == GC_STRATEGY_BITMAP_GRID && !wide) {
        GridLayout GL;
        return grid_sweep_layout(p, pl, &GL, why) ? GL.total : 0;
    }
    BatchJob job{p, pl, nullptr, 0, nullptr, wide};
    BatchLayout L;
    if (!batch_layout(&job, 1, 1, &L, why)) return 0;
    return L.total;
}

// Checks and plans every job of a batch.
static int make_batch(const gc_job* jobs, int njobs, std::vector<BatchJob>* out) {
    if (!jobs || njobs < 1) return fail(GC_ERR_INVALID, "no jobs");
    out->clear();
    for (int j = 0; j < njobs; ++j) {
        const gc_job& J = jobs[j];
        BatchJob B{};
        std::string why;
        if (!make_problem(J.prob, &B.p, &why))
            return fail(GC_ERR_INVALID, "job " + std::to_string(j) + ": " + why);
        gc_plan_t in{};
        in.strategy = J.strategy;
        if (!resolve_plan(B.p, &in, &B.plan))
            return fail(GC_ERR_INVALID, "job " + std::to_string(j) + ": bad strategy");
        B.plan.strategy = batch_strategy(B.plan.strategy);
        if (!J.d_stats || (!J.d_out && J.capacity > 0))
            return fail(GC_ERR_INVALID, "job " + std::to_string(j) + ": null pointer");
        B.d_out = J.d_out;
        B.capacity = J.capacity;
        B.d_stats = J.d_stats;
        out->push_back(B);
    }
    return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" {

const char* gc_strerror(int err) {
    switch (err) {
        case GC_OK: return "ok";
        case GC_ERR_INVALID: return "invalid argument";
        case GC_ERR_CAPACITY: return "output capacity too small";
        case GC_ERR_CUDA: return "CUDA error";
        case GC_ERR_OOM: return "out of memory";
        case GC_ERR_TIMEOUT: return "device-side wait timed out";
        case GC_ERR_UNSUPPORTED: return "unsupported";
        case GC_ERR_INTERNAL: return "internal error";
        default: return "unknown error";
    }
}

const char* gc_last_error(void) { return g_last_error.c_str(); }

uint64_t gc_candidate_count(int n, int w, int ordering) {
    HostProblem p;
    std::string why;
    if (ordering == GC_ORDER_BASIS)  // 2^n ranks whatever the basis
        return (n >= 1 && n <= kMaxN && w >= -1 && w <= n) ? (1ull << n) : 0;
    if (!make_problem(n, 2, ordering, w, &p, &why, GC_CONSTRAINT_NONE, nullptr, kMaxNWide))
        return 0;
    return p.N;
}

uint64_t gc_capacity_bound(int n, int d, int w) {
    HostProblem p;
    std::string why;
    if (!make_problem(n, d, GC_ORDER_LEX, w, &p, &why, GC_CONSTRAINT_NONE, nullptr, kMaxNWide))
        return 0;
    return p.bound;
}

int gc_plan(const gc_problem* prob, gc_plan_t* out) {
    if (!prob || !out) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why)) return fail(GC_ERR_INVALID, why);
    if (!tuned_plan(p, out)) plan_for(p, out);
    return GC_OK;
}

}  // extern "C"

namespace gc {
// The scratch bytes of one problem, with the reason when there are none:
// GC_ERR_INVALID for a bad problem or plan, GC_ERR_UNSUPPORTED (and the
// layout's reason) for a valid request the sweep's layout refuses.
int workspace_bytes(const gc_problem* prob, const gc_plan_t* plan, size_t* out) {
    *out = 0;
    if (!prob) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why)) return fail(GC_ERR_INVALID, why);
    gc_plan_t pl;
    if (!resolve_plan(p, plan, &pl)) return fail(GC_ERR_INVALID, "bad strategy");
    *out = single_workspace(p, pl, &why);
    return *out ? GC_OK : fail(GC_ERR_UNSUPPORTED, why);
}
}  // namespace gc

extern "C" {

size_t gc_workspace_size(const gc_problem* prob, const gc_plan_t* plan) {
    if (!prob) return 0;
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why)) return 0;
    gc_plan_t pl;
    if (!resolve_plan(p, plan, &pl)) return 0;
    return single_workspace(p, pl, &why);
}

int gc_generate_async(const gc_problem* prob, const gc_plan_t* plan, uint32_t* d_out,
                      uint64_t capacity, gc_stats* d_stats, void* workspace,
                      size_t workspace_bytes, void* stream) {
    if (!prob || !d_stats || (!d_out && capacity > 0)) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why)) return fail(GC_ERR_INVALID, why);
    gc_plan_t pl;
    if (!resolve_plan(p, plan, &pl)) return fail(GC_ERR_INVALID, "bad strategy");
    return generate_async_impl(p, pl, d_out, capacity, d_stats, workspace, workspace_bytes,
                               (cudaStream_t)stream);
}

}  // extern "C"

// The synchronous call: host or device output of `wbytes`-byte words.
static int generate_sync(const HostProblem& p, void* out, uint64_t* inout_count, bool wide) {
    std::string why;
    gc_plan_t pl;
    if (wide)
        resolve_plan_wide(p, nullptr, &pl);
    else
        resolve_plan(p, nullptr, &pl);
    const size_t wbytes = wide ? 8 : 4;
    const uint64_t cap = *inout_count;
    const bool dev_out = cap > 0 && is_device_ptr(out);
    const size_t ws_bytes = single_workspace(p, pl, &why, wide);
    if (ws_bytes == 0) return fail(GC_ERR_UNSUPPORTED, why);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(GC_ERR_CUDA, "stream create");
    void* ws = nullptr;
    gc_stats* d_stats = nullptr;
    void* d_buf = nullptr;
    const uint64_t dcap = dev_out ? 0 : std::min<uint64_t>(cap, p.bound);
    int rc = GC_OK;
    cudaError_t e;
    if ((e = cudaMallocAsync(&ws, ws_bytes, s)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&d_stats, sizeof(gc_stats), s)) != cudaSuccess ||
        (dcap && (e = cudaMallocAsync(&d_buf, dcap * wbytes, s)) != cudaSuccess)) {
        rc = fail(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!rc) rc = generate_async_impl(p, pl, dev_out ? out : d_buf, dev_out ? cap : dcap, d_stats,
                                      ws, ws_bytes, s, wide);
    gc_stats st{};
    if (!rc) {
        if ((e = cudaMemcpyAsync(&st, d_stats, sizeof st, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            rc = fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!rc && st.status != 0) rc = fail(st.status, "device-side error in the sweep");
    if (!rc && !dev_out && dcap) {
        const uint64_t ncopy = std::min<uint64_t>(st.codewords, dcap);
        if ((e = cudaMemcpy(out, d_buf, ncopy * wbytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
            rc = fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (d_buf) cudaFreeAsync(d_buf, s);
    if (d_stats) cudaFreeAsync(d_stats, s);
    if (ws) cudaFreeAsync(ws, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc) return rc;
    *inout_count = st.codewords;
    if (st.codewords > cap) return fail(GC_ERR_CAPACITY, "output capacity too small");
    return GC_OK;
}

extern "C" {

int gc_generate(int n, int d, int ordering, int w, uint32_t* out, uint64_t* inout_count) {
    if (!inout_count || (!out && *inout_count > 0)) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(n, d, ordering, w, &p, &why)) return fail(GC_ERR_INVALID, why);
    return generate_sync(p, out, inout_count, false);
}

// ---- wide vectors (uint64 words, n <= 64) ----
size_t gc_workspace_size64(const gc_problem* prob, const gc_plan_t* plan) {
    if (!prob) return 0;
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why, kMaxNWide)) return 0;
    gc_plan_t pl;
    if (!resolve_plan_wide(p, plan, &pl)) return 0;
    return single_workspace(p, pl, &why, true);
}

int gc_generate64_async(const gc_problem* prob, const gc_plan_t* plan, uint64_t* d_out,
                        uint64_t capacity, gc_stats* d_stats, void* workspace,
                        size_t workspace_bytes, void* stream) {
    if (!prob || !d_stats || (!d_out && capacity > 0)) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why, kMaxNWide)) return fail(GC_ERR_INVALID, why);
    gc_plan_t pl;
    if (!resolve_plan_wide(p, plan, &pl))
        return fail(GC_ERR_UNSUPPORTED, "the wide sweep runs the distance strategy only");
    return generate_async_impl(p, pl, d_out, capacity, d_stats, workspace, workspace_bytes,
                               (cudaStream_t)stream, true);
}

int gc_generate64(int n, int d, int ordering, int w, uint64_t* out, uint64_t* inout_count) {
    if (!inout_count || (!out && *inout_count > 0)) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(n, d, ordering, w, &p, &why, GC_CONSTRAINT_NONE, nullptr, kMaxNWide))
        return fail(GC_ERR_INVALID, why);
    return generate_sync(p, out, inout_count, true);
}

size_t gc_batch_workspace_size(const gc_job* jobs, int njobs, int ngroups) {
    std::vector<BatchJob> B;
    if (make_batch(jobs, njobs, &B)) return 0;
    BatchLayout L;
    std::string why;
    if (!batch_layout(B.data(), njobs, ngroups, &L, &why)) return 0;
    return L.total;
}

int gc_batch_generate_async(const gc_job* jobs, int njobs, int ngroups, void* workspace,
                            size_t workspace_bytes, void* stream) {
    std::vector<BatchJob> B;
    int rc = make_batch(jobs, njobs, &B);
    if (rc) return rc;
    BatchLayout L;
    std::string why;
    if (!batch_layout(B.data(), njobs, ngroups, &L, &why)) return fail(GC_ERR_UNSUPPORTED, why);
    if (!workspace || workspace_bytes < L.total) return fail(GC_ERR_INVALID, "workspace too small");
    if (((uintptr_t)workspace & 255u) != 0)
        return fail(GC_ERR_INVALID, "workspace not 256-byte aligned");
    rc = launch_batch(B.data(), njobs, L, workspace, (cudaStream_t)stream, &why);
    return rc ? fail(rc, why) : GC_OK;
}

}  // extern "C"

// A prepared batch: jobs checked and planned, workspace laid out and filled.
struct gc_batch {
    std::vector<BatchJob> jobs;
    BatchLayout L;
    void* ws = nullptr;
};

extern "C" {

int gc_batch_create(const gc_job* jobs, int njobs, int ngroups, void* workspace,
                    size_t workspace_bytes, void* stream, gc_batch** out) {
    if (!out) return fail(GC_ERR_INVALID, "null handle pointer");
    *out = nullptr;
    gc_batch* b = new (std::nothrow) gc_batch();
    if (!b) return fail(GC_ERR_OOM, "host allocation");
    int rc = make_batch(jobs, njobs, &b->jobs);
    std::string why;
    if (!rc && !batch_layout(b->jobs.data(), njobs, ngroups, &b->L, &why))
        rc = fail(GC_ERR_UNSUPPORTED, why);
    if (!rc && (!workspace || workspace_bytes < b->L.total))
        rc = fail(GC_ERR_INVALID, "workspace too small");
    if (!rc && ((uintptr_t)workspace & 255u) != 0)
        rc = fail(GC_ERR_INVALID, "workspace not 256-byte aligned");
    if (!rc) {
        b->ws = workspace;
        const int r = upload_batch(b->jobs.data(), njobs, b->L, workspace, (cudaStream_t)stream,
                                   &why);
        if (r) rc = fail(r, why);
    }
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return GC_OK;
}

int gc_batch_launch(gc_batch* b, void* stream) {
    if (!b) return fail(GC_ERR_INVALID, "null handle");
    std::string why;
    const int rc = launch_batch_kernel(b->L, b->ws, (cudaStream_t)stream, &why);
    return rc ? fail(rc, why) : GC_OK;
}

int gc_batch_destroy(gc_batch* b) {
    delete b;
    return GC_OK;
}

int gc_unrank(int n, int ordering, int w, uint64_t rank0, uint64_t count, uint32_t* d_vec,
              void* stream) {
    HostProblem p;
    std::string why;
    if (ordering == GC_ORDER_BASIS) return fail(GC_ERR_UNSUPPORTED, "gc_unrank: no basis argument");
    if (!make_problem(n, 2, ordering, w, &p, &why)) return fail(GC_ERR_INVALID, why);
    if (count > 0 && !d_vec) return fail(GC_ERR_INVALID, "null output");
    if (rank0 > p.N || count > p.N - rank0) return fail(GC_ERR_INVALID, "rank out of range");
    return launch_unrank(p, rank0, count, d_vec, (cudaStream_t)stream);
}

int gc_rank(int n, int ordering, const uint32_t* d_vec, uint64_t count, uint64_t* d_rank,
            void* stream) {
    HostProblem p;
    std::string why;
    if (ordering == GC_ORDER_BASIS) return fail(GC_ERR_UNSUPPORTED, "gc_rank: no basis argument");
    if (!make_problem(n, 2, ordering, -1, &p, &why)) return fail(GC_ERR_INVALID, why);
    if (count > 0 && (!d_vec || !d_rank)) return fail(GC_ERR_INVALID, "null pointer");
    return launch_rank(n, ordering, d_vec, count, d_rank, (cudaStream_t)stream);
}

int gc_block_test(int d, const uint32_t* d_cand, uint64_t ncand, const uint32_t* d_code,
                  uint64_t ncode, uint8_t* d_alive, void* stream) {
    if (d < 0) return fail(GC_ERR_INVALID, "d must be >= 0");
    if ((ncand && (!d_cand || !d_alive)) || (ncode && !d_code))
        return fail(GC_ERR_INVALID, "null pointer");
    return launch_block_test(d, d_cand, ncand, d_code, ncode, d_alive, (cudaStream_t)stream);
}

int gc_resolve(int d, const uint32_t* d_cand, uint32_t ncand, uint32_t* d_accepted,
               uint32_t* d_count, void* stream) {
    if (d < 0) return fail(GC_ERR_INVALID, "d must be >= 0");
    if (!d_count || (ncand && (!d_cand || !d_accepted))) return fail(GC_ERR_INVALID, "null pointer");
    return launch_resolve(d, d_cand, ncand, d_accepted, d_count, (cudaStream_t)stream);
}

int gc_bitmap_mark(int n, int d, const uint32_t* d_code, uint64_t ncode, uint32_t* d_bitmap,
                   void* stream) {
    if (n < 1 || n > 32 || d < 0) return fail(GC_ERR_INVALID, "bad n or d");
    if (ncode && (!d_code || !d_bitmap)) return fail(GC_ERR_INVALID, "null pointer");
    if (ncode == 0 || d == 0) return GC_OK;
    const uint64_t hlen = high_ball_len(n, d);
    if (hlen >= (1ull << 31)) return fail(GC_ERR_UNSUPPORTED, "ball too large");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* tmp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&tmp, hlen * 4, s);
    if (e != cudaSuccess) return fail(GC_ERR_OOM, cudaGetErrorString(e));
    int rc = launch_bitmap_mark(n, d, d_code, ncode, d_bitmap, tmp, s);
    cudaFreeAsync(tmp, s);
    return rc;
}

int gc_bitmap_scan(int n, int ordering, int w, const uint32_t* d_bitmap, uint64_t rank0,
                   uint64_t count, uint32_t* d_out, uint64_t capacity, uint64_t* d_found,
                   void* stream) {
    HostProblem p;
    std::string why;
    if (ordering == GC_ORDER_BASIS) return fail(GC_ERR_UNSUPPORTED, "gc_bitmap_scan: no basis argument");
    if (!make_problem(n, 2, ordering, w, &p, &why)) return fail(GC_ERR_INVALID, why);
    if (!d_found || (count && !d_bitmap) || (capacity && !d_out))
        return fail(GC_ERR_INVALID, "null pointer");
    if (rank0 > p.N || count > p.N - rank0) return fail(GC_ERR_INVALID, "rank out of range");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* counts = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&counts, sizeof(uint64_t) * kScanMaxBlocks, s);
    if (e != cudaSuccess) return fail(GC_ERR_OOM, cudaGetErrorString(e));
    int rc = launch_bitmap_scan(p, d_bitmap, rank0, count, d_out, capacity, d_found, counts, s);
    cudaFreeAsync(counts, s);
    return rc;
}

}  // extern "C"
