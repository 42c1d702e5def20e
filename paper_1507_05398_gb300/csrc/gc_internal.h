// gc_internal.h -- host-side interfaces between the C ABI (gc_capi.cu) and
// the kernel launchers (gc_sweep.cu, gc_steps.cu).  Not installed.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdlib>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gc.h"
#include "gc_device.cuh"

namespace gc {

// Fully checked problem description shared by the launchers.  n <= 32, or
// n <= 64 for the wide entry points (uint64 words).
struct HostProblem {
    int n, d, ord, w;
    bool orth;         // self-orthogonal constraint (Section 4.4)
    uint32_t basis[32];  // B-ordering basis and the rows of its inverse
    uint32_t inv[32];
    bool filter;       // GRAY with a weight: ranks of the wrong weight skipped
    uint64_t N;        // rank-space size
    uint64_t valid;    // number of candidates (C(n,w) or 2^n)
    uint64_t bound;    // gc_capacity_bound
};

// Default survivors per window (the window size adapts to about this many):
// the bitmap windows carry no old-code scan, so they take more survivors per
// group exchange; measured on GB300 (n = 20, d = 4 in four orders and
// n = 24, d = 8 lex, with 16-152 CTAs per code).  Bitmap sweeps of 2^28 or
// more candidates take larger windows: n = 31, d = 3 and n = 32, d = 4 ran
// 1.1-1.4x faster in lex and Gray with 4096, in the graded orders with 2048.
constexpr uint32_t kTargetDistance = 512;
constexpr uint32_t kTargetBitmap = 1024;
constexpr uint64_t kLargeSweep = 1ull << 28;
// GC_TARGET_BITMAP overrides the bitmap target of sweeps below kLargeSweep
// candidates (measurements).
// The grid bitmap sweep decides at most 8192 survivors per window and cuts
// the window after them; it aims a little above that, so that windows end at
// the cut and little of the generated window is thrown away (windows whose
// survivors conflict densely aim lower, by their pair density).
constexpr uint32_t kTargetGrid = 8800;
inline uint32_t default_target(int strategy, const HostProblem& p) {
    if (strategy == GC_STRATEGY_BITMAP_GRID) return kTargetGrid;
    if (strategy != GC_STRATEGY_BITMAP) return kTargetDistance;
    if (p.valid < kLargeSweep) {
        const char* e = std::getenv("GC_TARGET_BITMAP");
        const int v = e ? std::atoi(e) : 0;
        return v >= 64 && v <= 4096 ? (uint32_t)v : kTargetBitmap;
    }
    return (p.ord == GC_ORDER_LEX || p.ord == GC_ORDER_GRAY) ? 4096u : 2048u;
}


uint64_t binom64(int n, int k);
bool make_problem(int n, int d, int ord, int w, HostProblem* out, std::string* why,
                  int constraint = GC_CONSTRAINT_NONE, const uint32_t* basis = nullptr,
                  int max_n = kMaxN);
// make_problem from the ABI struct
bool make_problem(const gc_problem& q, HostProblem* out, std::string* why, int max_n = kMaxN);
// Fills an Order for the device from a checked problem.
Order order_of(const HostProblem& p, bool filter, bool even);
// Strategy and launch shape for a problem (gc_plan).
void plan_for(const HostProblem& p, gc_plan_t* pl);
// The plan the installed tuning cache holds for a problem, if any (gc_tune.cu).
bool tuned_plan(const HostProblem& p, gc_plan_t* out);

// Word-grouped ball: entries (e_high << 3) | radius for every high part of
// weight <= d-1 over the n-5 word-index bits; radius = d-1-weight(e_high),
// clipped to 7.  Its length:
uint64_t high_ball_len(int n, int d);
int launch_high_ball(int nh, int rad, uint32_t* d_out, uint32_t len, cudaStream_t s);

// One code to generate, as the sweep kernel reads it (device memory for
// batches, host-mapped memory for the server's ring).
struct JobDesc {
    Order ord;
    int d;
    int strategy;          // 1 distance, 2 bitmap
    void* out;             // uint32 words (narrow kernel) or uint64 words (wide)
    uint64_t cap;
    gc_stats* stats;
    const uint32_t* hball;
    uint32_t hball_len;
    uint32_t wmin, wmax, target;
    int orth;              // self-orthogonal constraint
    int pipelined;         // bitmap job: resolver CTA + generator CTAs
};
using JobDescHost = JobDesc;

// Server: groups of equal size, scratch sized for the largest admissible
// job, ball tables filled from the host on demand.
struct ServeLayout {
    int grid = 0, ngroups = 0, group_ctas = 0;
    uint32_t cache_words = 0;
    size_t smem_bytes = 0;
    uint64_t store_words = 0;      // per group
    uint64_t bitmap_bits = 0;      // per group
    size_t off_err = 0, off_head = 0, off_groups = 0, off_hball = 0, hball_bytes = 0;
    std::vector<size_t> g_flags, g_segx, g_segoff, g_store, g_bitmap, g_slice, g_pipe;
    size_t total = 0;
    // ball tables already uploaded: key (n << 8 | d) -> (offset, length)
    std::vector<std::pair<uint32_t, std::pair<size_t, uint32_t>>> hball_tables;
    size_t hball_used = 0;
    void* ws = nullptr;            // set once the workspace exists
};

bool serve_layout(const gc_server_config& cfg, ServeLayout* L, std::string* why);
// Fills the descriptor of one request (uploads its ball table if needed).
bool serve_describe(ServeLayout& L, const HostProblem& p, int strategy, uint32_t* d_out,
                    uint64_t cap, gc_stats* d_stats, JobDesc* desc, std::string* why);
int launch_server(ServeLayout& L, void* ws, JobDesc* ring, unsigned* tail, unsigned* stop,
                  unsigned long long* done, uint32_t capacity, double idle_seconds,
                  cudaStream_t stream, std::string* why);

// One job of a batch, checked and planned on the host.
struct BatchJob {
    HostProblem p;
    gc_plan_t plan;     // strategy is DISTANCE or BITMAP here
    void* d_out;        // uint32 words, or uint64 words for a wide job
    uint64_t capacity;
    gc_stats* d_stats;
    bool wide = false;  // run on the wide kernel (uint64 words, n <= 64)
};

// Where everything of a batched sweep lives: CTA groups, their jobs, and
// the workspace offsets of the descriptors and scratch.
struct BatchLayout {
    int grid = 0, ngroups = 0;
    bool wide = false;          // the uint64-word kernel
    bool dynamic = false;       // groups claim jobs (longest first) as they free up
    bool dense = false;         // pipelined windows may use whole-window matrices
    uint32_t cache_words = 0;   // shared-memory code cache (distance jobs; whole-window
                                // matrices when dense)
    size_t smem_bytes = 0;
    std::vector<int> first_cta, ncta, job_begin, job_end, job_order;
    size_t off_err = 0, off_jobs = 0, off_order = 0, off_groups = 0;
    std::vector<size_t> g_flags, g_segx, g_segoff, g_store, g_bitmap, g_slice, g_pipe, hball_off;
    std::vector<uint64_t> g_store_words;
    size_t total = 0;
};

// Rough device cost of one job (used to balance and order batch jobs).
double job_cost(const HostProblem& p, int strategy);

// Splits the SMs into groups (ngroups <= 0: one per job, up to the SM count),
// assigns jobs to groups (longest first) and lays out the workspace.
bool batch_layout(const BatchJob* jobs, int njobs, int ngroups, BatchLayout* L, std::string* why);

// Launches the batched sweep (descriptor copies, set-up kernels, the
// cooperative sweep) on stream; returns a GC_* code.  It is upload_batch
// (descriptors, ball tables, kernel attributes: once per batch) followed by
// launch_batch_kernel (per-launch state reset and the persistent kernel:
// stream operations only, so it can be captured into a CUDA graph).
int launch_batch(const BatchJob* jobs, int njobs, const BatchLayout& L, void* workspace,
                 cudaStream_t stream, std::string* why);
int upload_batch(const BatchJob* jobs, int njobs, const BatchLayout& L, void* workspace,
                 cudaStream_t stream, std::string* why);
int launch_batch_kernel(const BatchLayout& L, void* workspace, cudaStream_t stream,
                        std::string* why);

// The grid bitmap sweep (gc_gridsweep.cu): one code on every SM, lockstep
// windows.  Workspace offsets and launch shape.
struct GridLayout {
    int grid = 0;
    size_t smem_bytes = 0;
    size_t off_ctrl = 0, off_slot = 0, off_pslot = 0, off_segx = 0, off_segoff = 0;
    size_t off_pairs = 0, off_kill = 0, off_hball = 0, off_bitmap = 0;
    size_t off_cnt = 0;        // d = 3: 2^n byte counters (0: none)
    size_t total = 0;
    uint32_t wmin = 0, wmax = 0, target = 0;
};
bool grid_sweep_layout(const HostProblem& p, const gc_plan_t& plan, GridLayout* L,
                       std::string* why);
// Ball table, control words and the cooperative launch, all on stream s.
int launch_grid_sweep(const HostProblem& p, const GridLayout& L, uint32_t* d_out,
                      uint64_t capacity, gc_stats* d_stats, void* workspace, cudaStream_t s,
                      std::string* why);
// A batch or a server runs a grid-strategy job with the pipelined bitmap.
inline int batch_strategy(int strategy) {
    return strategy == GC_STRATEGY_BITMAP_GRID ? GC_STRATEGY_BITMAP : strategy;
}

// Step launchers (gc_steps.cu); each returns a GC_* code.
int launch_unrank(const HostProblem& p, uint64_t rank0, uint64_t count, uint32_t* d_vec,
                  cudaStream_t s);
int launch_rank(int n, int ord, const uint32_t* d_vec, uint64_t count, uint64_t* d_rank,
                cudaStream_t s);
int launch_block_test(int d, const uint32_t* d_cand, uint64_t ncand, const uint32_t* d_code,
                      uint64_t ncode, uint8_t* d_alive, cudaStream_t s);
int launch_resolve(int d, const uint32_t* d_cand, uint32_t ncand, uint32_t* d_acc,
                   uint32_t* d_count, cudaStream_t s);
int launch_bitmap_mark(int n, int d, const uint32_t* d_code, uint64_t ncode, uint32_t* d_bitmap,
                       uint32_t* d_hball_scratch, cudaStream_t s);
constexpr int kScanMaxBlocks = 1024;  // d_counts must hold this many uint64
int launch_bitmap_scan(const HostProblem& p, const uint32_t* d_bitmap, uint64_t rank0,
                       uint64_t count, uint32_t* d_out, uint64_t capacity, uint64_t* d_found,
                       uint64_t* d_counts, cudaStream_t s);

// Scratch bytes of one problem (gc_workspace_size), or the error and its
// reason: GC_ERR_INVALID (bad problem or plan), GC_ERR_UNSUPPORTED (valid,
// but the sweep's layout refuses it).
int workspace_bytes(const gc_problem* prob, const gc_plan_t* plan, size_t* out);

// Records a message for gc_last_error() and returns code.
int fail(int code, const std::string& msg);

}  // namespace gc
