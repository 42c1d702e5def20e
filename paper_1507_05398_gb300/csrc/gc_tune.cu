// gc_tune.cu -- measured autotuning of the sweep's plan.
//
// gc_plan() picks a strategy from a cost model.  gc_autotune() measures
// instead: it runs the candidate plans (distance or bitmap strategy, window
// survivor targets, CTA counts) on the current device, keeps the fastest,
// and records it in a plain-text cache keyed by the problem and the device
// name.  When a cache is installed (gc_set_tune_cache, or the GC_TUNE_CACHE
// environment variable), gc_plan() and every sweep entry point that plans by
// itself use the cached plan for a problem it holds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gc_internal.h"

namespace gc {

namespace {

std::mutex g_tune_mu;
std::string g_cache_path;  // "" = none installed (GC_TUNE_CACHE is read lazily)
bool g_env_read = false;

struct Entry {
    int n, d, ord, w, constraint;
    std::string device;
    gc_plan_t plan;
    double ms;
};

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    std::string s = prop.name;
    for (char& c : s)
        if (c == ' ') c = '_';
    return s;
}

std::string cache_path_locked() {
    if (!g_env_read) {
        g_env_read = true;
        if (g_cache_path.empty())
            if (const char* e = std::getenv("GC_TUNE_CACHE")) g_cache_path = e;
    }
    return g_cache_path;
}

// Problems with a basis are not cached (the basis is not part of the key).
bool cacheable(const HostProblem& p) { return p.ord != GC_ORDER_BASIS; }

std::vector<Entry> read_cache(const std::string& path) {
    std::vector<Entry> out;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return out;
    char dev[256];
    Entry e;
    while (std::fscanf(f, "%d %d %d %d %d %255s %d %d %u %u %u %lf", &e.n, &e.d, &e.ord, &e.w,
                       &e.constraint, dev, &e.plan.strategy, &e.plan.grid, &e.plan.window_min,
                       &e.plan.window_max, &e.plan.survivor_target, &e.ms) == 12) {
        e.device = dev;
        e.plan.block = 1024;
        out.push_back(e);
    }
    std::fclose(f);
    return out;
}

bool append_cache(const std::string& path, const Entry& e) {
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return false;
    std::fprintf(f, "%d %d %d %d %d %s %d %d %u %u %u %.6f\n", e.n, e.d, e.ord, e.w, e.constraint,
                 e.device.c_str(), e.plan.strategy, e.plan.grid, e.plan.window_min,
                 e.plan.window_max, e.plan.survivor_target, e.ms);
    std::fclose(f);
    return true;
}

}  // namespace

bool tuned_plan(const HostProblem& p, gc_plan_t* out) {
    if (!cacheable(p)) return false;
    std::string path;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        path = cache_path_locked();
    }
    if (path.empty()) return false;
    const std::string dev = device_name();
    const int cons = p.orth ? GC_CONSTRAINT_SELF_ORTHOGONAL : GC_CONSTRAINT_NONE;
    bool found = false;
    for (const Entry& e : read_cache(path))  // the last entry for a key wins
        if (e.n == p.n && e.d == p.d && e.ord == p.ord && e.w == p.w && e.constraint == cons &&
            e.device == dev) {
            *out = e.plan;
            found = true;
        }
    return found;
}

// Runs each candidate plan of a problem once to warm up and once timed, on
// its own stream and scratch; returns the fastest (GC_ERR_UNSUPPORTED if
// none ran).  A warm-up over twice the best so far is not timed again, and
// one over four times it drops the rest of that strategy's candidates
// (candidates come grouped by strategy, the planner's first).
static int measure_plans(const gc_problem* prob, const HostProblem& p,
                         const std::vector<gc_plan_t>& cands, gc_plan_t* best, double* best_ms) {
    if (cands.empty()) return fail(GC_ERR_UNSUPPORTED, "no admissible plan");
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(GC_ERR_CUDA, "stream create");
    uint32_t* d_out = nullptr;
    gc_stats* d_stats = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_out, std::max<uint64_t>(p.bound, 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_stats, sizeof(gc_stats));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best_t = 1e300;
    int rc = (e == cudaSuccess) ? GC_OK : fail(GC_ERR_OOM, cudaGetErrorString(e));
    int dropped = GC_STRATEGY_AUTO;  // a strategy found hopeless
    for (const gc_plan_t& c : cands) {
        if (rc) break;
        if (c.strategy == dropped) continue;
        const size_t ws_bytes = gc_workspace_size(prob, &c);
        if (ws_bytes == 0) continue;  // e.g. the bitmap would not fit
        void* ws = nullptr;
        if (cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {  // warm-up, then timed
            cudaEventRecord(a, s);
            ok = gc_generate_async(prob, &c, d_out, p.bound, d_stats, ws, ws_bytes, s) == GC_OK;
            cudaEventRecord(b, s);
            ok = ok && cudaEventSynchronize(b) == cudaSuccess;
            // a warm-up over twice the best so far cannot win: not timed again
            if (ok && rep == 0 && best_t < 1e300) {
                cudaEventElapsedTime(&ms, a, b);
                if (ms > 4.0 * best_t) dropped = c.strategy;
                if (ms > 2.0 * best_t) break;
            }
        }
        gc_stats st{};
        ok = ok && cudaMemcpy(&st, d_stats, sizeof st, cudaMemcpyDeviceToHost) == cudaSuccess &&
             st.status == 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaFree(ws);
        if (ok && ms < best_t) {
            best_t = ms;
            *best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (d_out) cudaFree(d_out);
    if (d_stats) cudaFree(d_stats);
    cudaStreamDestroy(s);
    if (rc) return rc;
    if (best_t >= 1e300) return fail(GC_ERR_UNSUPPORTED, "no plan ran");
    *best_ms = best_t;
    return GC_OK;
}

// Candidate strategies of a problem: distance and the pipelined bitmap,
// each where it applies, the planner's choice first.
static std::vector<int> tune_strategies(const HostProblem& p) {
    std::vector<int> out;
    gc_plan_t base{};
    plan_for(p, &base);
    const bool dist_ok = p.bound < 0xffffffffull;
    const bool bitmap_ok = !p.orth && high_ball_len(p.n, p.d) < (1u << 24);
    const bool bitmap_first = batch_strategy(base.strategy) == GC_STRATEGY_BITMAP;
    if (bitmap_first && bitmap_ok) out.push_back(GC_STRATEGY_BITMAP);
    if (dist_ok) out.push_back(GC_STRATEGY_DISTANCE);
    if (!bitmap_first && bitmap_ok) out.push_back(GC_STRATEGY_BITMAP);
    return out;
}

}  // namespace gc

using namespace gc;

extern "C" {

int gc_set_tune_cache(const char* path) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_env_read = true;
    g_cache_path = path ? path : "";
    return GC_OK;
}

int gc_autotune(const gc_problem* prob, gc_plan_t* best, double* best_ms) {
    if (!prob || !best) return fail(GC_ERR_INVALID, "null argument");
    HostProblem p;
    std::string why;
    if (!make_problem(*prob, &p, &why)) return fail(GC_ERR_INVALID, why);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // candidate plans
    std::vector<gc_plan_t> cands;
    gc_plan_t base{};
    plan_for(p, &base);
    const uint32_t targets[4] = {256, 512, 1024, 2048};
    const int grids[3] = {sms, std::max(1, sms / 4), std::max(1, sms / 8)};
    for (int st : tune_strategies(p))
        for (uint32_t t : targets)
            for (int g : grids) {
                gc_plan_t c = base;
                c.strategy = st;
                c.survivor_target = t;
                c.grid = g;
                cands.push_back(c);
            }
    double best_t = 0;
    const int rc = measure_plans(prob, p, cands, best, &best_t);
    if (rc) return rc;
    if (best_ms) *best_ms = best_t;
    std::string path;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        path = cache_path_locked();
    }
    if (!path.empty() && cacheable(p)) {
        Entry en{p.n, p.d, p.ord, p.w, p.orth ? 1 : 0, device_name(), *best, best_t};
        if (!append_cache(path, en)) return fail(GC_ERR_INVALID, "cannot write the tuning cache");
    }
    return GC_OK;
}

int gc_batch_autotune(const gc_job* jobs, int njobs, int ngroups, int max_jobs, int* tuned) {
    if (!jobs || njobs < 1 || !tuned) return fail(GC_ERR_INVALID, "null argument or no jobs");
    *tuned = 0;
    std::string path;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        path = cache_path_locked();
    }
    if (path.empty()) return fail(GC_ERR_INVALID, "gc_batch_autotune needs a tuning cache");
    // the batch as gc_batch_create would plan and lay it out (cost model)
    std::vector<BatchJob> B(njobs);
    std::vector<gc_problem> probs(njobs);
    for (int j = 0; j < njobs; ++j) {
        std::string why;
        if (!make_problem(jobs[j].prob, &B[j].p, &why))
            return fail(GC_ERR_INVALID, "job " + std::to_string(j) + ": " + why);
        plan_for(B[j].p, &B[j].plan);
        B[j].plan.strategy = batch_strategy(B[j].plan.strategy);
        B[j].plan.survivor_target = default_target(B[j].plan.strategy, B[j].p);
        probs[j] = jobs[j].prob;
    }
    BatchLayout L;
    std::string why;
    if (!batch_layout(B.data(), njobs, ngroups, &L, &why)) return fail(GC_ERR_UNSUPPORTED, why);
    // CTAs each job gets: its group's (with dynamic claiming, the smallest)
    std::vector<int> ctas(njobs, L.ncta.empty() ? 1 : L.ncta[0]);
    if (L.dynamic) {
        const int m = *std::min_element(L.ncta.begin(), L.ncta.end());
        std::fill(ctas.begin(), ctas.end(), m);
    } else {
        for (int g = 0; g < L.ngroups; ++g)
            for (int q = L.job_begin[g]; q < L.job_end[g]; ++q) ctas[L.job_order[q]] = L.ncta[g];
    }
    // the costliest distinct problems first
    std::vector<int> idx(njobs);
    for (int j = 0; j < njobs; ++j) idx[j] = j;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return job_cost(B[x].p, B[x].plan.strategy) > job_cost(B[y].p, B[y].plan.strategy);
    });
    std::vector<int> done;
    for (int j : idx) {
        if (max_jobs >= 0 && *tuned >= max_jobs) break;
        const HostProblem& p = B[j].p;
        if (!cacheable(p)) continue;
        bool seen = false;
        for (int k : done)
            seen = seen || (B[k].p.n == p.n && B[k].p.d == p.d && B[k].p.ord == p.ord &&
                             B[k].p.w == p.w && B[k].p.orth == p.orth);
        if (seen) continue;
        done.push_back(j);
        std::vector<gc_plan_t> cands;
        const uint32_t targets[4] = {256, 512, 1024, 2048};
        for (int st : tune_strategies(p))
            for (uint32_t t : targets) {
                gc_plan_t c = B[j].plan;
                c.strategy = st;
                c.survivor_target = t;
                c.grid = ctas[j];
                cands.push_back(c);
            }
        gc_plan_t best{};
        double best_t = 0;
        const int rc = measure_plans(&probs[j], p, cands, &best, &best_t);
        if (rc) return rc;
        // recorded for every launch size: a batch takes its grid from the
        // SMs, and a cached grid would shrink the whole launch
        best.grid = 0;
        Entry en{p.n, p.d, p.ord, p.w, p.orth ? 1 : 0, device_name(), best, best_t};
        if (!append_cache(path, en)) return fail(GC_ERR_INVALID, "cannot write the tuning cache");
        ++*tuned;
    }
    return GC_OK;
}

}  // extern "C"
