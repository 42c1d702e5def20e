// gc_sweep.cu -- the persistent windowed sweep: the ordered greedy
// construction of Section 4 for one code or a batch of codes in one
// cooperative launch.
//
// The CTAs (one per SM) are split into groups; each group sweeps its own
// list of jobs (codes) one after the other.  For one job the rank space is
// cut into windows of W consecutive ranks, and for window t:
//  1. (all CTAs of the group, in parallel) every candidate of the window is
//     generated from its rank (Section 4.2 orders, closed form) and tested
//     against the code committed before the window:
//       distance strategy: popcount(x ^ c) >= d against every codeword,
//         most recent first, from shared memory, with warp-wide early exit
//         (Sections 4.1, 5.2); first every warp scans the newest codewords
//         for its own candidates, then the few candidates left are scanned
//         against the rest with the codeword range split across warps;
//       bitmap strategy: one bit lookup in the exclusion bitmap, which holds
//         the radius-(d-1) balls of every codeword accepted two or more
//         windows ago, plus the distance test against the previous window's
//         accepts, whose balls the group marks meanwhile.
//     Survivors are written, in rank order, to the CTA's segment, and the CTA
//     publishes (sequence number, count) in its flag word.
//  2. each CTA waits until every flag of its group carries the window's
//     sequence number (acquire loads, bounded wait).
//  3. (every CTA of the group, redundantly and identically) the survivors are
//     gathered in rank order and resolved in order (block_resolve), which
//     reproduces the serial decisions; the accepts are appended to the code.
//     Every CTA keeps its own copy of the accepts, so no second wait is needed.
// The window size adapts so that about `target` candidates survive step 1; if
// more than kSurvCap survive, the window is cut after the kSurvCap-th one.
// Refinements of this scheme:
//  - distance jobs with a long code deal the window out in kSlice-rank
//    slices round-robin instead of one chunk per CTA, because the test cost
//    per candidate is very uneven along the order;
//  - bitmap jobs on three or more CTAs run pipelined: the group's first CTA
//    resolves window t while the others generate and filter window t+1;
//  - in pipelined groups of 64 or more generators, after a window that
//    accepted at least 7/8 of its survivors, the generators also list the
//    next window's conflicting pairs between them, and the resolver decides
//    it in rounds over that list (pair_resolve) instead of conflict matrices;
//  - otherwise, pipelined jobs of small survivor targets (in launches with
//    a group of kDenseMinGenerators or more generators) have the generators
//    build the window's whole conflict matrix, which the resolver copies
//    into shared memory and decides in rounds (dense_build, dense_resolve);
//    such windows are cut after as many survivors as the matrix holds.
// The kernel is instantiated for narrow vectors (uint32 words, n <= 32, both
// strategies) and wide ones (uint64 words, n <= 64, distance strategy only).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "gc_block.cuh"
#include "gc_internal.h"

namespace gc {

constexpr int kChunk = 4096;       // candidates per CTA per window
constexpr int kSlice = 128;        // distance jobs: ranks per interleaved slice
constexpr int kMaxSlices = kChunk / kSlice;   // slices per CTA per window (32)
constexpr int kMaxInterleaveCtas = 256;       // larger groups use contiguous chunks
// Interleave only once the committed code is this long: below it the tests
// are cheap and even, and the gather's fixed cost (about 3 us a window at
// 152 CTAs) outweighs the balance it buys (measured on GB300).
constexpr uint64_t kInterleaveMinCode = 1024;
static_assert(kChunk <= 4096, "the interleaved gather packs segment indices in 12 bits");
static_assert(kMaxSlices % 4 == 0 && kMaxSlices <= 32, "slice counts: one warp lane each");
constexpr int kSurvCap = 4096;     // survivors resolved per window
// Pipelined windows: conflicting pairs one generator may publish, and pairs
// the resolver takes into shared memory (behind 8 KiB of round flags in the
// resolver matrix); more and the window goes to the conflict matrices.
// (Rounds that read longer lists from the generators' buffers in L2 were
// latency-bound: ~160 us per window against ~34 us for the matrices.)
constexpr uint32_t kPairCap = 2048;
constexpr uint32_t kPairShared = 6144;
// Generators list the conflicts only in groups with at least this many of
// them: in smaller groups the generators' own work per window already
// paces the pipeline, and the search lengthens it by more than the
// resolver saves (measured on the n = 20, d = 4 codes in groups of ~30).
constexpr int kPairMinGenerators = 64;
// A batch launch uses whole-window conflict matrices only if one of its
// groups has at least this many generators: the 512 mixed codes of
// n = 14-24 on groups of 3 generators took 122 ms per batch with them and
// 113 ms without.
constexpr int kDenseMinGenerators = 8;
constexpr int kMaxGroupCtas = 1024;
constexpr int kMinGroup = 8;       // CTAs of the smallest group when sizes follow cost
enum : int { kStratDistance = 1, kStratBitmap = 2 };

// A group of CTAs and the scratch it owns.
struct GroupDesc {
    int first_cta, ncta;
    int job_begin, job_end;       // range of job_order
    unsigned long long* flags;    // [2][ncta]: (sequence << 32) | survivor count
    void* seg_x;                  // [2][ncta][kChunk] vectors (the kernel's word type)
    uint32_t* seg_off;            // [2][ncta][kChunk]
    void* store;                  // distance jobs: code beyond the shared cache
    uint64_t store_words;
    uint32_t* bitmap;             // bitmap jobs: 2^n bits, vector-indexed
    uint8_t* slice_cnt;           // [2][ncta][kMaxSlices] survivors per slice (or null)
    // pipelined bitmap jobs (or null): generator survivor flags [2][ncta],
    // the resolver's flag, generator pair flags [2][ncta]; the resolver's
    // accepts [2][kSurvCap]; the generators' conflicting pairs
    // [2][ncta][kPairCap]
    unsigned long long* pflags;
    uint32_t* accbuf;
    uint32_t* pairbuf;
    uint32_t* densebuf;           // pipelined: whole-window conflict matrices [2][kDenseTriMax]
};

// Serving mode: jobs arrive while the kernel runs.  The host writes a job
// descriptor into a ring in host-mapped memory, then raises `tail`; a group
// claims the next published job with a compare-and-swap on `head`, runs it,
// and raises done[slot] to (job index + 1).
struct ServeQueue {
    const JobDesc* descs;         // host-mapped ring [capacity]
    const unsigned* tail;         // host-mapped: number of jobs published
    const unsigned* stop;         // host-mapped: 1 = leave once idle
    unsigned long long* done;     // host-mapped [capacity]
    unsigned* head;               // device: number of jobs claimed
    uint32_t capacity;
    long long idle_cycles;        // bound on one wait for a new job
};

struct BatchArgs {
    const JobDesc* jobs;
    const int* job_order;
    const GroupDesc* groups;
    int ngroups;
    unsigned* err;
    uint32_t cache_words;
    long long timeout_cycles;
    uint32_t resolve_block;       // entries per conflict matrix (<= kResolveBlock)
    uint32_t pairs;               // pipelined generators list each window's conflicts:
                                  // 0 never, 1 when it pays, 2 always
    uint32_t dense_rows;          // pipelined windows: most entries of a whole-window
                                  // conflict matrix (0: blocked matrices only)
    uint32_t dense_cut;           // 1: cut such windows at dense_rows survivors
    uint32_t timing_cta;          // CTA of each group whose phases are timed
    unsigned* claim;              // dynamic batches: jobs of job_order handed out so far
    int njobs;                    // dynamic batches: length of job_order
    ServeQueue queue;             // used when queue.descs != nullptr
};

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Serving mode, thread 0 of a group's first CTA: claim the next published
// job.  Returns its index + 1, or 0 when asked to stop (or idle too long).
__device__ uint32_t serve_claim(const ServeQueue& q) {
    const long long t0 = clock64();
    for (;;) {
        const unsigned t = ld_acquire_sys(q.tail);
        unsigned h = ld_acquire_gpu(q.head);
        while (h < t) {
            const unsigned prev = atomicCAS(q.head, h, h + 1u);
            if (prev == h) return h + 1u;
            h = prev;
        }
        if (ld_acquire_sys(q.stop) != 0u) return 0u;
        if (clock64() - t0 > q.idle_cycles) return 0u;
        __nanosleep(256);
    }
}

template <typename W>
struct __align__(16) SweepSmem;
// the interleaved gather's count and prefix tables live in the resolver matrix
static_assert(kMaxSlices * kMaxInterleaveCtas * 3 <= kResolveWords * kResolveBlock * 4,
              "gather tables must fit the resolver matrix");

template <typename W>
struct __align__(16) SweepSmem {
    uint32_t C[kMaxN + 1][kMaxN + 1];
    uint32_t pad0[3];
    uint32_t lowball[8][32];  // lowball[r][c]: bits y < 32 with popc(y ^ c) <= r
    uint32_t lowlight[8];     // lowlight[k]: bits y < 32 with popc(y) < k (k >= 6: all)
    __align__(16) W list_x[kChunk];
    __align__(16) uint32_t list_off[kChunk];
    __align__(16) W accA[kSurvCap];
    __align__(16) W accB[kSurvCap];
    __align__(16) uint32_t acc_off[kSurvCap];
    uint32_t pref[kMaxGroupCtas + 1];
    uint8_t dead[kChunk];
    JobDesc job;
    GroupDesc grp;
    uint32_t slice_cnt[kMaxSlices];  // distance jobs: survivors per local slice
    unsigned long long phase[12];  // phase timers (thread 0 of the group's first CTA)
    // the current job's windows, survivors, pair-decided and pair-overflow
    // windows: kept by thread 0 (uniform values, out of the registers)
    unsigned long long jstat[4];
    long long tprev;
    BlockScratch bs;
    __align__(16) uint32_t dund[kDenseWords];  // whole-window resolver: undecided /
    __align__(16) uint32_t dacc[kDenseWords];  // accepted bits
    // Last, so that it runs on into the dynamic code cache: a pipelined
    // resolver holds a whole-window conflict matrix in M and the cache.
    __align__(16) uint32_t M[kResolveWords][kResolveBlock];
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// CTA-wide.  Publishes this CTA's count for sequence number seq and waits
// until every CTA of the group has published seq; then s.pref holds the
// exclusive prefix of the counts and the total is returned.  Bounded: on
// timeout (or when another CTA reported one) sets *ok = false.
// CTA-wide.  Waits until flags[0..nf) all carry sequence number seq (acquire
// loads, bounded like group_exchange); then s.pref holds the exclusive prefix
// of their counts and the total is returned.
template <typename W>
__device__ uint32_t await_counts(SweepSmem<W>& s, const unsigned long long* flags, int nf,
                                 uint32_t seq, unsigned* err, long long timeout, bool* ok) {
    uint32_t v = 0;
    bool fine = true;
    if ((int)threadIdx.x < nf) {
        const long long t0 = clock64();
        for (;;) {
            const unsigned long long f = ld_acquire_u64(flags + threadIdx.x);
            if ((uint32_t)(f >> 32) == seq) {
                v = (uint32_t)f;
                break;
            }
            if (ld_acquire_gpu(err) != 0u) { fine = false; break; }
            if (clock64() - t0 > timeout) {
                atomicExch(err, 1u);
                fine = false;
                break;
            }
        }
    }
    if (threadIdx.x == 0) s.bs.flag_any = 1u;
    __syncthreads();
    if (!fine) s.bs.flag_any = 0u;
    uint32_t total = 0;
    const uint32_t ex = block_exclusive_scan(s.bs, v, &total);  // has barriers
    if ((int)threadIdx.x < nf) s.pref[threadIdx.x] = ex;
    if (threadIdx.x == 0) s.pref[nf] = total;
    *ok = *ok && s.bs.flag_any != 0u;
    __syncthreads();
    return total;
}

template <typename W>
__device__ uint32_t group_exchange(SweepSmem<W>& s, unsigned long long* flags, int lb, int gsize,
                                   uint32_t seq, uint32_t count, unsigned* err, long long timeout,
                                   bool* ok) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        st_release_u64(flags + lb, ((unsigned long long)seq << 32) | count);
    uint32_t v = 0;
    bool fine = true;
    if ((int)threadIdx.x < gsize) {
        const long long t0 = clock64();
        for (;;) {
            const unsigned long long f = ld_acquire_u64(flags + threadIdx.x);
            if ((uint32_t)(f >> 32) == seq) {
                v = (uint32_t)f;
                break;
            }
            if (ld_acquire_gpu(err) != 0u) { fine = false; break; }
            if (clock64() - t0 > timeout) {
                atomicExch(err, 1u);
                fine = false;
                break;
            }
        }
    }
    if (threadIdx.x == 0) s.bs.flag_any = 1u;
    __syncthreads();
    if (!fine) s.bs.flag_any = 0u;
    uint32_t total = 0;
    const uint32_t ex = block_exclusive_scan(s.bs, v, &total);  // has barriers
    if ((int)threadIdx.x < gsize) s.pref[threadIdx.x] = ex;
    if (threadIdx.x == 0) s.pref[gsize] = total;
    *ok = s.bs.flag_any != 0u;
    __syncthreads();
    return total;
}

// C(p, k) for p, k <= 64, for the wide kernel's graded orders.
__device__ const Binom64Table g_binom64 = make_binom64();

template <typename Word>
__global__ void __launch_bounds__(kBlock, 1) sweep_kernel(const __grid_constant__ BatchArgs a) {
    constexpr bool kWide = sizeof(Word) == 8;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    SweepSmem<Word>& s = *reinterpret_cast<SweepSmem<Word>*>(smem_raw);
    Word* cache = reinterpret_cast<Word*>(smem_raw + sizeof(SweepSmem<Word>));
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();

    // which group this CTA belongs to
    if (tid == 0) {
        int g = 0;
        while (g + 1 < a.ngroups && a.groups[g + 1].first_cta <= (int)blockIdx.x) ++g;
        s.grp = a.groups[g];
    }
    if constexpr (!kWide)
        for (int q = tid; q < (kMaxN + 1) * (kMaxN + 1); q += kBlock) {
            const int p = q / (kMaxN + 1), k = q % (kMaxN + 1);
            uint64_t r = (k <= p) ? 1u : 0u;
            for (int i = 1; i <= k && k <= p; ++i) r = r * (uint64_t)(p - k + i) / (uint64_t)i;
            s.C[p][k] = (uint32_t)r;
        }
    __syncthreads();
    const GroupDesc& grp = s.grp;
    Word* const seg_x = static_cast<Word*>(grp.seg_x);
    Word* const store = static_cast<Word*>(grp.store);
    const int lb = (int)blockIdx.x - grp.first_cta;
    const int G = grp.ncta;
    const uint32_t(*C)[kMaxN + 1] = s.C;
    // phase timers: thread 0 of one CTA of the group (the first, unless the
    // launch names another)
    const bool timing = (lb == (a.timing_cta < (uint32_t)grp.ncta ? (int)a.timing_cta : 0) &&
                         tid == 0);
    uint32_t seq = 0;
    uint32_t pseq = 0;  // pipelined jobs: sequence numbers used so far
    bool ok = true;
    // every job's statistics start at zero (ordered before any other CTA's
    // update by the first group exchange)
    if (lb == 0 && tid == 0)
        for (int jq = grp.job_begin; jq < grp.job_end; ++jq) {
            gc_stats* st = a.jobs[a.job_order[jq]].stats;
            st->codewords = 0; st->candidates = 0; st->dense_tests = 0; st->executed_tests = 0;
            st->marks = 0; st->windows = 0; st->survivors = 0; st->status = 0; st->strategy = 0;
            for (int k = 0; k < 12; ++k) st->phase_cycles[k] = 0;
            st->pair_windows = 0; st->pair_fallbacks = 0;
        }

    const bool serving = a.queue.descs != nullptr;
    // Dynamic batches (more jobs than groups): job_order lists the jobs
    // longest first, and a group claims the next one whenever it is free, so
    // a wrong cost estimate cannot leave one group with too much work.
    const bool dynamic = !serving && a.claim != nullptr;
    uint32_t claimed = 0;  // dynamic: this group's last claim + 1 (first CTA only)
    for (int jq = grp.job_begin; ok && (serving || dynamic || jq < grp.job_end); ++jq) {
        uint32_t serve_idx = 0;  // serving mode: job index + 1
        if (dynamic) {
            const uint32_t mine = (lb == 0 && tid == 0) ? atomicAdd(a.claim, 1u) + 1u : 0u;
            if (lb == 0 && tid == 0) claimed = mine;
            const uint32_t idx = group_exchange(s, grp.flags + (size_t)(seq & 1) * G, lb, G, seq,
                                                mine, a.err, a.timeout_cycles, &ok);
            ++seq;
            if (!ok || idx > (uint32_t)a.njobs) break;
            if (tid == 0) s.job = a.jobs[a.job_order[idx - 1]];
        } else if (serving) {
            const uint32_t mine = (lb == 0 && tid == 0) ? serve_claim(a.queue) : 0u;
            // every CTA of the group learns the claim (the sum of the counts)
            serve_idx = group_exchange(s, grp.flags + (size_t)(seq & 1) * G, lb, G, seq, mine,
                                       a.err, a.timeout_cycles + a.queue.idle_cycles, &ok);
            ++seq;
            if (!ok || serve_idx == 0) break;
            if (tid == 0) {
                // the descriptor was written before tail was raised (release),
                // and serve_claim read tail with acquire; volatile loads keep
                // stale cache lines of an earlier use of the slot out
                const volatile uint32_t* src = reinterpret_cast<const volatile uint32_t*>(
                    a.queue.descs + (serve_idx - 1) % a.queue.capacity);
                uint32_t* dst = reinterpret_cast<uint32_t*>(&s.job);
                for (uint32_t w = 0; w < sizeof(JobDesc) / 4; ++w) dst[w] = src[w];
            }
        } else if (tid == 0) {
            s.job = a.jobs[a.job_order[jq]];
        }
        __syncthreads();
        if ((serving || dynamic) && lb == 0 && tid == 0) {
            gc_stats* st = s.job.stats;
            st->codewords = 0; st->candidates = 0; st->dense_tests = 0; st->executed_tests = 0;
            st->marks = 0; st->windows = 0; st->survivors = 0; st->status = 0; st->strategy = 0;
            for (int k = 0; k < 12; ++k) st->phase_cycles[k] = 0;
            st->pair_windows = 0; st->pair_fallbacks = 0;
        }
        const JobDesc& job = s.job;
        const Order& o = job.ord;
        const int d = job.d;
        const int n = o.n;
        if (!kWide && job.strategy == kStratBitmap) {
            const int nl = n < 5 ? n : 5;
            for (int q = tid; q < 8 * 32; q += kBlock) {
                const int r = q / 32, c = q % 32;
                uint32_t m = 0;
                for (int y = 0; y < (1 << nl); ++y)
                    if (__popc((unsigned)(y ^ c)) <= r) m |= 1u << y;
                s.lowball[r][c] = m;
            }
            for (int k = tid; k < 8; k += kBlock) {
                uint32_t m = 0;
                for (int y = 0; y < (1 << nl); ++y)
                    if (__popc((unsigned)y) < k) m |= 1u << y;
                s.lowlight[k] = m;
            }
        }
        // job start: clear this CTA's share of the bitmap
        if (!kWide && job.strategy == kStratBitmap) {
            const uint64_t words = ((1ull << n) + 31) / 32;
            const uint64_t per = (words + G - 1) / G;
            const uint64_t w0 = min((uint64_t)lb * per, words), w1 = min(w0 + per, words);
            for (uint64_t w = w0 + tid; w < w1; w += kBlock) grp.bitmap[w] = 0u;
        }
        group_exchange(s, grp.flags + (size_t)(seq & 1) * G, lb, G, seq, 0, a.err,
                       a.timeout_cycles, &ok);
        ++seq;
        if (!ok) break;

        uint64_t R0 = 0, K = 0, Kprev = 0;
        uint32_t W = job.wmin;
        Word* cur = s.accA;
        Word* prev = s.accB;
        uint32_t nprev = 0;
        uint64_t my_tests = 0, my_marks = 0, dense = 0, resolve_tests = 0;
        if (tid == 0) s.jstat[0] = s.jstat[1] = s.jstat[2] = s.jstat[3] = 0;
        if (timing)
            for (int k = 0; k < 12; ++k) s.phase[k] = 0;
        // adds the cycles since the last mark to phase k (first CTA, thread 0)
        auto mark_phase = [&](int k) {
            if (timing) {
                const long long t = clock64();
                s.phase[k] += (unsigned long long)(t - s.tprev);
                s.tprev = t;
            }
        };
        // resolves the gathered window in order with conflict matrices

        auto resolve = [&](uint32_t Suse, uint64_t& rt) -> uint32_t {
            return job.orth ? block_resolve<true>(s.bs, s.list_x, s.list_off, s.dead, Suse, d, cur,
                                                  s.acc_off, s.M, rt,
                                                  timing ? s.phase + 8 : nullptr, a.resolve_block)
                            : block_resolve<false>(s.bs, s.list_x, s.list_off, s.dead, Suse, d,
                                                   cur, s.acc_off, s.M, rt,
                                                   timing ? s.phase + 8 : nullptr,
                                                   a.resolve_block);
        };

        // bitmap strategy: share `share` of `nshares` of the ball marks of
        // the accepts accs[0..nacc)
        auto mark_share = [&](const Word* accs, uint32_t nacc, int share, int nshares) {
            if (kWide || job.strategy != kStratBitmap || nacc == 0) return;
            {
                const uint32_t hl = job.hball_len;
                const uint64_t total = (uint64_t)nacc * hl;
                const uint64_t per = (total + nshares - 1) / nshares;
                const uint64_t q0 = min((uint64_t)share * per, total), q1 = min(q0 + per, total);
                // (i, j) = divmod(q, hl), advanced by kBlock without dividing
                const uint64_t qs = q0 + tid;
                uint32_t i = (uint32_t)(qs / hl), j = (uint32_t)(qs - (uint64_t)i * hl);
                const uint32_t di = kBlock / hl, dj = kBlock - di * hl;
                for (uint64_t q = qs; q < q1; q += kBlock) {
                    const uint32_t c = (uint32_t)accs[i];
                    const uint32_t e = __ldg(job.hball + j);
                    const uint32_t cw = c >> 5, word = cw ^ (e >> 3);
                    uint32_t mask = s.lowball[e & 7u][c & 31u];
                    bool skip = false;
                    // only ranks after c matter; skip words wholly before it
                    if (o.ord == kLex) {
                        skip = word < cw;
                        if (word == cw) mask &= ~((2u << (c & 31u)) - 1u);
                    } else if (o.ord == kGray) {
                        skip = gray_inverse(word) < gray_inverse(cw);
                    } else if (o.ord == kGrlex || o.ord == kGrevlex) {
                        // graded orders: every vector lighter than c is behind it
                        const int below = __popc(c) - __popc(word);  // low bits must weigh >= this
                        if (below > 0) mask &= ~s.lowlight[below < 7 ? below : 7];
                    }
                    if (!skip && mask) {
                        atomicOr(grp.bitmap + word, mask);
                        ++my_marks;
                    }
                    i += di;
                    j += dj;
                    if (j >= hl) {
                        j -= hl;
                        ++i;
                    }
                }
            }
        };
        // Bitmap jobs of a group of three or more CTAs run pipelined.  The
        // group's first CTA resolves window t while the others (generators)
        // mark the balls of window t-2's accepts and generate window t+1.
        // When a generator generates window t, the bitmap is complete up to
        // window t-3 (the marks of window t-3 were made during window t-1
        // and the generators' exchange after it ordered them), so it also
        // tests its candidates against window t-2's accepts and -- once the
        // resolver has published them -- window t-1's.  Every CTA computes
        // the windows by the rules of the sequential loop below, from the
        // generators' counts.  Flags carry job-unique sequence numbers
        // (pseq), and every wait is bounded.
        const bool piped = !kWide && job.strategy == kStratBitmap && job.pipelined != 0 &&
                           G >= 3 && grp.pflags != nullptr && grp.accbuf != nullptr;
        if (piped) {
            const int nG = G - 1, gi = lb - 1;
            unsigned long long* gflag = grp.pflags;                  // [2][G]
            unsigned long long* rflag = grp.pflags + 2 * (size_t)G;  // the resolver's
            unsigned long long* eflag = rflag + 1;                   // [2][G] pair counts
            const uint32_t wmax_p = (uint32_t)min((uint64_t)job.wmax, (uint64_t)nG * kChunk);
            W = min(W, wmax_p);
            Word* acc_pp = s.accA;  // generators: accepts of window t-2
            Word* acc_p = s.accB;   // generators: accepts of window t-1
            uint32_t n_pp = 0, n_p = 0;
            // whether window t's conflicts are listed as pairs: the resolver
            // decides it at the end of window t-1 (mostly accepted: few
            // conflicts) and hands it to the generators in its flag
            bool pairs_on = false;
            uint32_t t = 0;
            for (; ok && R0 < o.N; ++t) {
                if (timing) s.tprev = clock64();
                const uint32_t wseq = pseq + t + 1;
                const int par = t & 1;
                const uint64_t span = min((uint64_t)W, o.N - R0);
                if (lb > 0) {
                    mark_share(acc_pp, n_pp, gi, nG);
                    mark_phase(0);
                    const uint64_t chunk = (span + nG - 1) / nG;
                    const uint64_t c0 = min(R0 + (uint64_t)gi * chunk, R0 + span);
                    const uint64_t c1 = min(c0 + chunk, R0 + span);
                    uint32_t na = 0;
                    for (uint64_t t0 = c0; t0 < c1; t0 += kBlock) {
                        const uint64_t r = t0 + tid;
                        uint32_t x = 0;
                        bool keep = false;
                        if (r < c1) {
                            keep = unrank(o, C, r, x);
                            if (keep) keep = !((ld_cg(grp.bitmap + (x >> 5)) >> (x & 31u)) & 1u);
                        }
                        na = block_append(s.bs, keep, (Word)x, (uint32_t)(r - R0), s.list_x,
                                          s.list_off, na);
                    }
                    mark_phase(1);
                    na = block_filter<false>(s.bs, s.list_x, s.list_off, s.dead, na,
                                             (const Word*)acc_pp, 0u, n_pp, d, my_tests);
                    mark_phase(2);
                    n_p = 0;
                    if (t > 0) {
                        // window t-1's accepts, once the resolver has them
                        if (tid == 0) {
                            const long long tw = clock64();
                            uint32_t cnt = 0, fine = 1;
                            for (;;) {
                                const unsigned long long f = ld_acquire_u64(rflag);
                                if ((uint32_t)(f >> 32) == wseq - 1) {
                                    cnt = (uint32_t)f;  // bit 31: pairs for window t
                                    break;
                                }
                                if (ld_acquire_gpu(a.err) != 0u) { fine = 0; break; }
                                if (clock64() - tw > a.timeout_cycles) {
                                    atomicExch(a.err, 1u);
                                    fine = 0;
                                    break;
                                }
                            }
                            s.bs.bcast[0] = cnt;
                            s.bs.bcast[1] = fine;
                        }
                        __syncthreads();
                        if (s.bs.bcast[1] == 0u) {
                            ok = false;
                            break;
                        }
                        n_p = s.bs.bcast[0] & 0x7fffffffu;
                        pairs_on = (s.bs.bcast[0] >> 31) != 0u;
                        mark_phase(4);
                        for (uint32_t i = tid; i < n_p; i += kBlock)
                            acc_p[i] = (Word)ld_cg(grp.accbuf + (size_t)(par ^ 1) * kSurvCap + i);
                        __syncthreads();
                        na = block_filter<false>(s.bs, s.list_x, s.list_off, s.dead, na,
                                                 (const Word*)acc_p, 0u, n_p, d, my_tests);
                        mark_phase(3);
                    }
                    // publish this generator's survivors
                    Word* sx = seg_x + ((size_t)par * G + gi) * kChunk;
                    uint32_t* so = grp.seg_off + ((size_t)par * G + gi) * kChunk;
                    for (uint32_t i = tid; i < na; i += kBlock) {
                        sx[i] = s.list_x[i];
                        so[i] = s.list_off[i];
                    }
                    __threadfence();
                    __syncthreads();
                    if (tid == 0)
                        st_release_u64(gflag + (size_t)par * G + gi,
                                       ((unsigned long long)wseq << 32) | na);
                }
                // every CTA: the generators' counts for window t
                const uint32_t S = await_counts(s, gflag + (size_t)par * G, nG, wseq, a.err,
                                                a.timeout_cycles, &ok);
                if (!ok) break;
                mark_phase(4);
                // Jobs whose survivor target is below the rows of a
                // whole-window matrix decide their windows from one (unless a
                // pair list does).  Such a window is cut after as many
                // survivors as the matrix takes, any other after kSurvCap; the
                // rest of its ranks start the next window.  (Jobs with larger
                // targets, the sweeps of 2^28 or more candidates, measured
                // slower with a matrix of their first survivors only.)
                const bool dense_job = a.dense_rows != 0u && job.target < a.dense_rows;
                const uint32_t cut = (dense_job && a.dense_cut != 0u && !pairs_on)
                                         ? a.dense_rows : (uint32_t)kSurvCap;
                const uint32_t Suse = min(S, cut);
                // the next window starts after the cut-th survivor when the
                // window is cut (generator order is rank order)
                if (tid == 0) {
                    uint64_t rn = R0 + span;
                    if (S > cut) {
                        int j = 0;
                        while (j + 1 < nG && s.pref[j + 1] <= cut - 1u) ++j;
                        rn = R0 + ld_cg(grp.seg_off + ((size_t)par * G + j) * kChunk +
                                        (cut - 1u - s.pref[j])) + 1;
                    }
                    s.bs.bcast64 = rn;
                }
                // The generators list the window's conflicting pairs: each
                // gathers the window and tests entry i against every earlier
                // entry for i = gi (mod nG), and publishes what it found.
                // The resolver then only runs the decision rounds (or, when
                // the pairs overflow, its own conflict matrices).
                const bool by_pairs = pairs_on && Suse >= 2u;
                if (lb > 0 && by_pairs) {
                    for (int g = warp; g < nG; g += kWarps) {
                        const uint32_t p0 = s.pref[g];
                        if (p0 >= Suse) continue;
                        const uint32_t cnt = min(s.pref[g + 1] - p0, Suse - p0);
                        const Word* gx = seg_x + ((size_t)par * G + g) * kChunk;
                        for (uint32_t i = lane; i < cnt; i += 32) s.list_x[p0 + i] = ld_cg(gx + i);
                    }
                    if (tid == 0) s.bs.sp_edges = 0u;
                    __syncthreads();
                    mark_phase(5);
                    uint32_t* pb = grp.pairbuf + ((size_t)par * G + gi) * kPairCap;
                    volatile uint32_t* found = &s.bs.sp_edges;
                    for (uint32_t i = (uint32_t)gi; i < Suse && *found <= kPairCap; i += nG) {
                        const Word xi = s.list_x[i];
                        for (uint32_t k = tid; k < i; k += kBlock) {
                            ++my_tests;
                            if (popc(xi ^ s.list_x[k]) < d) {
                                const uint32_t e = atomicAdd(&s.bs.sp_edges, 1u);
                                if (e < kPairCap) pb[e] = (k << 16) | i;
                            }
                        }
                    }
                    __threadfence();
                    __syncthreads();
                    if (tid == 0) {
                        const uint32_t np = s.bs.sp_edges;
                        st_release_u64(eflag + (size_t)par * G + gi,
                                       ((unsigned long long)wseq << 32) |
                                           (np > kPairCap ? kPairCap + 1u : np));
                    }
                    mark_phase(6);
                }
                // A window of more survivors than one conflict matrix takes
                // is decided from the conflict matrix of its first Pd entries
                // (all of them unless GC_DENSE_CUT=0), which the generators
                // build: each gathers those entries and writes the rows of its
                // share of the 4-row quads, then publishes with its pair flag.
                const uint32_t Pd = (dense_job && !by_pairs && Suse > a.resolve_block)
                                        ? min(Suse, a.dense_rows) : 0u;
                if (lb > 0 && Pd > 0u) {
                    for (int g = warp; g < nG; g += kWarps) {
                        const uint32_t p0 = s.pref[g];
                        if (p0 >= Pd) continue;
                        const uint32_t cnt = min(s.pref[g + 1] - p0, Pd - p0);
                        const Word* gx = seg_x + ((size_t)par * G + g) * kChunk;
                        for (uint32_t i = lane; i < cnt; i += 32) s.list_x[p0 + i] = ld_cg(gx + i);
                    }
                    __syncthreads();
                    mark_phase(5);
                    if constexpr (!kWide)
                        dense_build(s.list_x, Pd, d, grp.densebuf + (size_t)par * kDenseTriMax,
                                    (uint32_t)gi + (uint32_t)nG * (uint32_t)warp,
                                    (uint32_t)nG * (uint32_t)kWarps, my_tests);
                    __threadfence();
                    __syncthreads();
                    if (tid == 0)
                        st_release_u64(eflag + (size_t)par * G + gi, (unsigned long long)wseq << 32);
                    mark_phase(6);
                }
                if (lb == 0) {
                    // the resolver: gather, resolve, commit, publish
                    for (int g = warp; g < nG; g += kWarps) {
                        const uint32_t p0 = s.pref[g];
                        if (p0 >= Suse) continue;
                        const uint32_t cnt = min(s.pref[g + 1] - p0, Suse - p0);
                        const Word* gx = seg_x + ((size_t)par * G + g) * kChunk;
                        const uint32_t* go = grp.seg_off + ((size_t)par * G + g) * kChunk;
                        for (uint32_t i = lane; i < cnt; i += 32) {
                            s.list_x[p0 + i] = ld_cg(gx + i);
                            s.list_off[p0 + i] = ld_cg(go + i);
                        }
                    }
                    __syncthreads();
                    mark_phase(5);
                    uint64_t rt = 0;
                    uint32_t nacc = 0;
                    bool decided = false;
                    if (by_pairs) {
                        const uint32_t np = await_counts(s, eflag + (size_t)par * G, nG, wseq,
                                                         a.err, a.timeout_cycles, &ok);
                        if (!ok) break;
                        mark_phase(4);
                        // a generator whose pairs overflowed its buffer, or more
                        // pairs than shared memory takes: conflict matrices
                        bool over = false;
                        for (int g = tid; g < nG; g += kBlock)
                            over |= s.pref[g + 1] - s.pref[g] > kPairCap;
                        over = __syncthreads_or(over) || np > kPairShared;
                        if (!over) {
                            uint32_t* pr = &s.M[0][0] + 2048;  // after 8 KiB of round flags
                            const uint32_t* pbuf = grp.pairbuf + (size_t)par * G * kPairCap;
                            for (int g = warp; g < nG; g += kWarps) {
                                const uint32_t p0 = s.pref[g], c = s.pref[g + 1] - p0;
                                const uint32_t* src = pbuf + (size_t)g * kPairCap;
                                for (uint32_t i = lane; i < c; i += 32) pr[p0 + i] = ld_cg(src + i);
                            }
                            __syncthreads();
                            if constexpr (!kWide)  // pipelining is for narrow words
                                nacc = pair_resolve(
                                    s.bs, s.list_x, s.list_off, s.dead, Suse,
                                    [&](auto&& f) {
                                        for (uint32_t e = tid; e < np; e += kBlock)
                                            f(pr[e] >> 16, pr[e] & 0xffffu);
                                    },
                                    reinterpret_cast<uint8_t*>(&s.M[0][0]), cur, s.acc_off,
                                    timing ? s.phase + 8 : nullptr);
                            decided = true;
                            if (tid == 0) ++s.jstat[2];
                        } else {
                            if (tid == 0) ++s.jstat[3];
                        }
                    }
                    if (Pd > 0u) {
                        await_counts(s, eflag + (size_t)par * G, nG, wseq, a.err,
                                     a.timeout_cycles, &ok);
                        if (!ok) break;
                        mark_phase(4);
                        uint32_t* T = &s.M[0][0];  // runs on into the code cache
                        const uint4* src = reinterpret_cast<const uint4*>(
                            grp.densebuf + (size_t)par * kDenseTriMax);
                        const uint32_t nq = (dense_tri_words(Pd) + 3u) / 4u;
                        for (uint32_t q = tid; q < nq; q += kBlock)
                            reinterpret_cast<uint4*>(T)[q] = __ldcg(src + q);
                        __syncthreads();
                        if constexpr (!kWide) {
                            nacc = dense_resolve(s.bs, s.dund, s.dacc, s.list_x, s.list_off, Pd,
                                                 T, cur, s.acc_off,
                                                 timing ? s.phase + 8 : nullptr);
                            if (Suse > Pd) {
                                // the rest: drop what the accepts exclude, then
                                // the conflict matrices
                                const uint32_t left = block_filter<false>(
                                    s.bs, s.list_x + Pd, s.list_off + Pd, s.dead, Suse - Pd, cur,
                                    0u, nacc, d, rt);
                                if (left > 0u)
                                    nacc = block_resolve<false>(
                                        s.bs, s.list_x + Pd, s.list_off + Pd, s.dead, left, d,
                                        cur, s.acc_off, s.M, rt,
                                        timing ? s.phase + 8 : nullptr, a.resolve_block, nacc);
                            }
                        }
                        decided = true;
                    }
                    if (!decided) nacc = resolve(Suse, rt);
                    resolve_tests += rt;
                    mark_phase(6);
                    for (uint32_t i = tid; i < nacc; i += kBlock) {
                        const uint64_t pos = K + i;
                        if (pos < job.cap) static_cast<Word*>(job.out)[pos] = cur[i];
                        if (!o.filter && !o.even) dense += o.N - 1 - (R0 + s.acc_off[i]);
                        grp.accbuf[(size_t)par * kSurvCap + i] = (uint32_t)cur[i];
                    }
                    __threadfence();
                    __syncthreads();
                    pairs_on = a.pairs == 2u ||
                               (a.pairs == 1u && nG >= kPairMinGenerators &&
                                8u * (Suse - nacc) <= Suse);
                    if (tid == 0)
                        st_release_u64(rflag, ((unsigned long long)wseq << 32) |
                                                  (pairs_on ? 0x80000000ull : 0ull) | nacc);
                    K += nacc;
                    if (tid == 0) s.jstat[1] += Suse;
                } else {
                    __syncthreads();
                }
                const uint64_t Rnext = s.bs.bcast64;
                if (S > 2u * job.target)
                    W = max(W / 2u, job.wmin);
                else if (S < job.target / 2u)
                    W = min(W * 2u, wmax_p);
                W = min(W, wmax_p);
                R0 = Rnext;
                if (tid == 0) ++s.jstat[0];
                if (lb > 0) {  // window t-1's accepts are window t+1's "t-2"
                    Word* tmp = acc_pp;
                    acc_pp = acc_p;
                    acc_p = tmp;
                    n_pp = n_p;
                }
                __syncthreads();  // bcast64 is read before thread 0 writes it again
                mark_phase(7);
            }
            pseq += t + 1;
        } else
        while (R0 < o.N) {
            if (timing) s.tprev = clock64();
            const uint64_t span = min((uint64_t)W, o.N - R0);
            const uint64_t chunk = (span + G - 1) / G;
            const uint64_t c0 = min(R0 + (uint64_t)lb * chunk, R0 + span);
            const uint64_t c1 = min(c0 + chunk, R0 + span);

            // bitmap strategy: this CTA's share of the previous window's marks
            mark_share(prev, nprev, lb, G);
            mark_phase(0);
            // candidates of this CTA, in rank order.  Distance jobs deal the
            // window out in slices of kSlice ranks, round-robin: local slice
            // q of this CTA is slice q * G + lb of the window.  The test cost
            // of a candidate varies by orders of magnitude along the order,
            // and contiguous chunks left whole CTAs with the expensive ones.
            // Bitmap jobs (cheap, even tests) and short codes keep one
            // contiguous chunk per CTA.
            const bool inter = job.strategy == kStratDistance && G > 1 &&
                               G <= kMaxInterleaveCtas && grp.slice_cnt != nullptr &&
                               K >= kInterleaveMinCode;
            const uint64_t nslices = (span + kSlice - 1) / kSlice;
            const uint32_t qmax =
                inter ? (nslices > (uint64_t)lb ? (uint32_t)((nslices - lb + G - 1) / G) : 0u) : 0u;
            const uint64_t gen_end = inter ? (uint64_t)qmax * kSlice : c1 - c0;
            uint32_t na = 0;
            for (uint64_t t0 = 0; t0 < gen_end; t0 += kBlock) {
                uint64_t r;
                bool in_range;
                if (inter) {
                    const uint64_t q = (t0 + tid) / kSlice;
                    r = R0 + (q * G + lb) * kSlice + (t0 + tid) % kSlice;
                    in_range = q < qmax && r < R0 + span;
                } else {
                    r = c0 + t0 + tid;
                    in_range = r < c1;
                }
                Word x = 0;
                bool keep = false;
                if (in_range) {
                    if constexpr (kWide) {
                        keep = unrank_wide(o, g_binom64, r, x);
                    } else {
                        keep = unrank(o, C, r, x);
                        if (keep && job.strategy == kStratBitmap)
                            keep = !((ld_cg(grp.bitmap + (x >> 5)) >> (x & 31u)) & 1u);
                    }
                }
                na = block_append(s.bs, keep, x, (uint32_t)(r - R0), s.list_x, s.list_off, na);
            }

            // test against the code committed before the window, newest first:
            // prev (the previous window's accepts), then for the distance
            // strategy the older code (global store above the cache, then the
            // cache)
            mark_phase(1);
            if ((d >= 2 || job.orth) && na > 0) {
                // the committed code in newest-first order: prev (the previous
                // window's accepts), then for the distance strategy the global
                // store above the shared cache, then the cache.  It is scanned
                // in slices of growing length; after each slice the survivors
                // are compacted so lanes stay busy with live candidates.
                const uint32_t ncached =
                    job.strategy == kStratDistance ? (uint32_t)min(Kprev, (uint64_t)a.cache_words) : 0u;
                const uint32_t nglob = (job.strategy == kStratDistance && Kprev > a.cache_words)
                                           ? (uint32_t)(Kprev - a.cache_words) : 0u;
                const uint32_t total = nprev + nglob + ncached;
                uint32_t u = 0;
                while (na > 0 && u < total) {
                    // short list: the rest in one slice (block_test splits the
                    // codeword range across warps); else 16, then up to 256
                    uint32_t u1 = total;
                    if (na > 8u * 32u) u1 = min(total, u < 16u ? 16u : (u < 256u ? 256u : total));
                    for (uint32_t i = tid; i < na; i += kBlock) s.dead[i] = 0;
                    __syncthreads();
                    // prev: unified [0, nprev) -> prev[nprev-1 .. 0]
                    if (u < nprev) {
                        const uint32_t hi = min(u1, nprev);
                        if (job.orth)
                            block_test<false, true>(s.list_x, na, s.dead, prev, nprev - hi,
                                                    nprev - u, d, my_tests);
                        else
                            block_test<false, false>(s.list_x, na, s.dead, prev, nprev - hi,
                                                     nprev - u, d, my_tests);
                    }
                    // global store: unified [nprev, nprev+nglob) -> store[Kprev-1 ..]
                    if (nglob && u1 > nprev && u < nprev + nglob) {
                        const uint32_t lo = max(u, nprev) - nprev, hi = min(u1, nprev + nglob) - nprev;
                        if (job.orth)
                            block_test<true, true>(s.list_x, na, s.dead, store,
                                                   (uint32_t)Kprev - hi, (uint32_t)Kprev - lo, d,
                                                   my_tests);
                        else
                            block_test<true, false>(s.list_x, na, s.dead, store,
                                                    (uint32_t)Kprev - hi, (uint32_t)Kprev - lo, d,
                                                    my_tests);
                    }
                    // cache: unified [nprev+nglob, total) -> cache[ncached-1 .. 0]
                    if (ncached && u1 > nprev + nglob) {
                        const uint32_t base = nprev + nglob;
                        const uint32_t lo = max(u, base) - base, hi = u1 - base;
                        if (job.orth)
                            block_test<false, true>(s.list_x, na, s.dead, cache, ncached - hi,
                                                    ncached - lo, d, my_tests);
                        else
                            block_test<false, false>(s.list_x, na, s.dead, cache, ncached - hi,
                                                     ncached - lo, d, my_tests);
                    }
                    __syncthreads();
                    na = block_compact(s.bs, s.list_x, s.list_off, s.dead, na);
                    u = u1;
                    if (u == 16u || u1 == total) mark_phase(2);
                }
            }
            mark_phase(3);

            // publish this CTA's survivors (and, interleaved, how many each
            // local slice kept) and wait for the group
            {
                const int par = seq & 1;
                Word* sx = seg_x + ((size_t)par * G + lb) * kChunk;
                uint32_t* so = grp.seg_off + ((size_t)par * G + lb) * kChunk;
                for (uint32_t i = tid; i < na; i += kBlock) {
                    sx[i] = s.list_x[i];
                    so[i] = s.list_off[i];
                }
                if (inter) {
                    if (tid < kMaxSlices) s.slice_cnt[tid] = 0u;
                    __syncthreads();
                    for (uint32_t i = tid; i < na; i += kBlock)
                        atomicAdd(&s.slice_cnt[(s.list_off[i] / kSlice - lb) / G], 1u);
                    __syncthreads();
                    if (tid < kMaxSlices)
                        grp.slice_cnt[((size_t)par * G + lb) * kMaxSlices + tid] =
                            (uint8_t)s.slice_cnt[tid];
                }
            }
            const int par = seq & 1;
            const uint32_t S = group_exchange(s, grp.flags + (size_t)par * G, lb, G, seq, na,
                                              a.err, a.timeout_cycles, &ok);
            ++seq;
            if (!ok) break;
            mark_phase(4);

            // gather every CTA's survivors in rank order
            const uint32_t Suse = min(S, (uint32_t)kSurvCap);
            if (!inter) {  // contiguous chunks: CTA order is rank order
                for (int g = warp; g < G; g += kWarps) {
                    const uint32_t p0 = s.pref[g];
                    if (p0 >= Suse) continue;
                    const uint32_t cnt = min(s.pref[g + 1] - p0, Suse - p0);
                    const Word* gx = seg_x + ((size_t)par * G + g) * kChunk;
                    const uint32_t* go = grp.seg_off + ((size_t)par * G + g) * kChunk;
                    for (uint32_t i = lane; i < cnt; i += 32) {
                        s.list_x[p0 + i] = ld_cg(gx + i);
                        s.list_off[p0 + i] = ld_cg(go + i);
                    }
                }
            } else {
                // slice (q, g) -- local slice q of CTA g -- is window slice
                // q * G + g, so rank order is row-major order over (q, g):
                // its survivors start at the exclusive prefix T[q][g] of the
                // counts in that order, and sit in CTA g's segment after the
                // survivors of its slices q' < q.  The tables reuse the
                // resolver's matrix space (free until the resolve).
                uint8_t* cnt8 = reinterpret_cast<uint8_t*>(&s.M[0][0]);          // [q][g]
                uint16_t* T = reinterpret_cast<uint16_t*>(cnt8 + kMaxSlices * kMaxInterleaveCtas);
                const uint32_t cells = (uint32_t)kMaxSlices * G;
                // counts: CTA g published kMaxSlices bytes, read four at a time
                for (uint32_t e = tid; e < (uint32_t)G * (kMaxSlices / 4); e += kBlock) {
                    const uint32_t g = e / (kMaxSlices / 4), q4 = (e % (kMaxSlices / 4)) * 4;
                    const uint32_t v = __ldcg(reinterpret_cast<const unsigned*>(
                        grp.slice_cnt + ((size_t)par * G + g) * kMaxSlices + q4));
#pragma unroll
                    for (uint32_t k = 0; k < 4; ++k) cnt8[(q4 + k) * G + g] = (uint8_t)(v >> (8 * k));
                }
                __syncthreads();
                // exclusive prefix in (q, g) order: each thread owns
                // kPerThread consecutive cells
                constexpr uint32_t kPerThread = kMaxSlices * kMaxInterleaveCtas / kBlock;
                const uint32_t e0 = tid * kPerThread;
                uint32_t mine = 0;
                for (uint32_t k = 0; k < kPerThread; ++k)
                    if (e0 + k < cells) mine += cnt8[e0 + k];
                uint32_t tot = 0;
                uint32_t run = block_exclusive_scan(s.bs, mine, &tot);
                for (uint32_t k = 0; k < kPerThread; ++k)
                    if (e0 + k < cells) {
                        // positions past the resolver's capacity are not used
                        T[e0 + k] = (uint16_t)min(run, 65535u);
                        run += cnt8[e0 + k];
                    }
                __syncthreads();
                // source map: one warp per source CTA g, lane q holds slice
                // (q, g); the map entry (g << 12 | index in g's segment) of
                // every output position goes into list_off first (shared
                // memory only), then one pass fetches all entries at once
                for (int g = warp; g < G; g += kWarps) {
                    const uint32_t c = cnt8[(uint32_t)lane * G + g];
                    uint32_t incl = c;
#pragma unroll
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const uint32_t t = __shfl_up_sync(kFull, incl, o2);
                        if (lane >= o2) incl += t;
                    }
                    const uint32_t src = incl - c;  // in CTA g's segment
                    const uint32_t dst = T[(uint32_t)lane * G + g];
                    unsigned any = __ballot_sync(kFull, c != 0u && dst < Suse);
                    while (any) {
                        const int q = __ffs(any) - 1;
                        any &= any - 1u;
                        const uint32_t cq = __shfl_sync(kFull, c, q);
                        const uint32_t sq = __shfl_sync(kFull, src, q);
                        const uint32_t dq = __shfl_sync(kFull, dst, q);
                        for (uint32_t k = lane; k < cq && dq + k < Suse; k += 32)
                            s.list_off[dq + k] = ((uint32_t)g << 12) | (sq + k);
                    }
                }
                __syncthreads();
                for (uint32_t pidx = tid; pidx < Suse; pidx += kBlock) {
                    const uint32_t m = s.list_off[pidx];
                    const uint32_t g = m >> 12, ix = m & 4095u;
                    s.list_x[pidx] = ld_cg(seg_x + ((size_t)par * G + g) * kChunk + ix);
                    s.list_off[pidx] = ld_cg(grp.seg_off + ((size_t)par * G + g) * kChunk + ix);
                }
            }
            __syncthreads();
            const uint64_t Rnext = (S > (uint32_t)kSurvCap) ? R0 + s.list_off[kSurvCap - 1] + 1
                                                            : R0 + span;
            mark_phase(5);

            // resolve in order; identical in every CTA of the group
            uint64_t rt = 0;
            const uint32_t nacc = resolve(Suse, rt);
            if (lb == 0) resolve_tests += rt;
            mark_phase(6);

            // commit
            if (lb == 0) {
                for (uint32_t i = tid; i < nacc; i += kBlock) {
                    const uint64_t pos = K + i;
                    if (pos < job.cap) static_cast<Word*>(job.out)[pos] = cur[i];
                    if (!o.filter && !o.even) dense += o.N - 1 - (R0 + s.acc_off[i]);
                }
            }
            if (job.strategy == kStratDistance) {
                for (uint32_t i = tid; i < nacc; i += kBlock) {
                    const uint64_t pos = K + i;
                    if (lb == 0 && pos < grp.store_words) store[pos] = cur[i];
                    if (pos < a.cache_words) cache[pos] = cur[i];
                }
            }
            if (tid == 0) {
                ++s.jstat[0];
                s.jstat[1] += Suse;
            }
            if (S > 2u * job.target)
                W = max(W / 2u, job.wmin);
            else if (S < job.target / 2u)
                W = min(W * 2u, job.wmax);
            Kprev = K;
            K += nacc;
            Word* t = cur;
            cur = prev;
            prev = t;
            nprev = nacc;
            R0 = Rnext;
            __syncthreads();
            mark_phase(7);
        }

        // statistics: warp-reduce then one atomic per warp
        uint64_t tt = my_tests + resolve_tests, m = my_marks, dn = dense;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            tt += __shfl_down_sync(kFull, tt, off);
            m += __shfl_down_sync(kFull, m, off);
            dn += __shfl_down_sync(kFull, dn, off);
        }
        if (lane == 0) {
            if (tt) atomicAdd((unsigned long long*)&job.stats->executed_tests, (unsigned long long)tt);
            if (m) atomicAdd((unsigned long long*)&job.stats->marks, (unsigned long long)m);
            if (dn) atomicAdd((unsigned long long*)&job.stats->dense_tests, (unsigned long long)dn);
        }
        if (tid == 0 && lb == 0) {
            job.stats->codewords = K;
            job.stats->candidates = o.N;
            job.stats->windows = s.jstat[0];
            job.stats->survivors = s.jstat[1];
            job.stats->strategy = job.strategy;
            job.stats->pair_windows = s.jstat[2];
            job.stats->pair_fallbacks = s.jstat[3];
        }
        if (timing)
            for (int k = 0; k < 12; ++k) job.stats->phase_cycles[k] = s.phase[k];
        // the next job reuses the statistics-free scratch; make sure every CTA
        // of the group is done with this job's shared state first
        __syncthreads();
        if (serving && ok) {
            // every CTA's statistics are in before the host is told
            group_exchange(s, grp.flags + (size_t)(seq & 1) * G, lb, G, seq, 0, a.err,
                           a.timeout_cycles, &ok);
            ++seq;
            if (lb == 0 && tid == 0) {
                __threadfence_system();
                st_release_sys_u64(a.queue.done + (serve_idx - 1) % a.queue.capacity,
                                   (unsigned long long)serve_idx);
            }
        }
    }
    if (!serving && tid == 0 && (!ok || ld_acquire_gpu(a.err) != 0u)) {
        // report on every job this group owns (the failing one is among them)
        for (int jq = grp.job_begin; jq < grp.job_end; ++jq)
            atomicMax((int*)&a.jobs[a.job_order[jq]].stats->status, (int)GC_ERR_TIMEOUT);
        if (dynamic) {
            // the job this group claimed last, and every job nobody claimed
            if (lb == 0 && claimed >= 1u && claimed <= (uint32_t)a.njobs)
                atomicMax((int*)&a.jobs[a.job_order[claimed - 1]].stats->status,
                          (int)GC_ERR_TIMEOUT);
            for (uint32_t i = atomicAdd(a.claim, 1u); i < (uint32_t)a.njobs;
                 i = atomicAdd(a.claim, 1u))
                atomicMax((int*)&a.jobs[a.job_order[i]].stats->status, (int)GC_ERR_TIMEOUT);
        }
    }
}

// Word-grouped ball entries: (e_high << 3) | min(d-1-weight(e_high), 7) for
// every e_high over nh bits with weight <= d-1, weight classes ascending.
__global__ void high_ball_kernel(int nh, int rad, uint32_t* out, uint32_t len) {
    __shared__ uint32_t C[kMaxN + 1][kMaxN + 1];
    for (int q = threadIdx.x; q < (kMaxN + 1) * (kMaxN + 1); q += blockDim.x) {
        const int p = q / (kMaxN + 1), k = q % (kMaxN + 1);
        uint64_t r = (k <= p) ? 1u : 0u;
        for (int i = 1; i <= k && k <= p; ++i) r = r * (uint64_t)(p - k + i) / (uint64_t)i;
        C[p][k] = (uint32_t)r;
    }
    __syncthreads();
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < len; q += gridDim.x * blockDim.x) {
        uint32_t i = q;
        int k = 0;
        while (k < rad && k < nh && i >= C[nh][k]) {
            i -= C[nh][k];
            ++k;
        }
        const uint32_t eh = comb_unrank(C, nh, k, i);
        const int r = rad - k;
        out[q] = (eh << 3) | (uint32_t)(r > 7 ? 7 : r);
    }
}

int launch_high_ball(int nh, int rad, uint32_t* d_out, uint32_t len, cudaStream_t s) {
    if (len == 0) return GC_OK;
    const int blocks = (int)std::min<uint64_t>(1024, (len + 255) / 256);
    high_ball_kernel<<<blocks, 256, 0, s>>>(nh, rad, d_out, len);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GC_OK : fail(GC_ERR_CUDA, std::string("high_ball: ") + cudaGetErrorString(e));
}

uint64_t high_ball_len(int n, int d) {
    const int nh = n > 5 ? n - 5 : 0;
    uint64_t len = 0;
    for (int k = 0; k <= d - 1 && k <= nh; ++k) len += binom64(nh, k);
    return len;
}

// ------------------------------------------------------------------ host side
static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Dynamic job claiming for batches with more jobs than groups;
// GC_BATCH_DYNAMIC=0 turns it off (measurements).
static bool dynamic_enabled() {
    const char* e = std::getenv("GC_BATCH_DYNAMIC");
    return !(e && std::strcmp(e, "0") == 0);
}

// Pipelined bitmap jobs, per group of G CTAs: flags [4G + 1] u64, the
// accepts [2][kSurvCap] u32, the whole-window conflict matrices
// [2][kDenseTriMax] u32, the conflicting pairs [2][G][kPairCap] u32.
static size_t pipe_flag_bytes(int G) {
    return align_up(sizeof(unsigned long long) * (4 * (size_t)G + 1));
}
static size_t pipe_bytes(int G) {
    return pipe_flag_bytes(G) + align_up(sizeof(uint32_t) * 2 * (size_t)kSurvCap) +
           align_up(sizeof(uint32_t) * 2 * (size_t)kDenseTriMax) +
           align_up(sizeof(uint32_t) * 2 * (size_t)G * kPairCap);
}
static void set_pipe(GroupDesc& D, uint8_t* base) {
    uint8_t* at = base + pipe_flag_bytes(D.ncta);
    D.pflags = reinterpret_cast<unsigned long long*>(base);
    D.accbuf = reinterpret_cast<uint32_t*>(at);
    at += align_up(sizeof(uint32_t) * 2 * (size_t)kSurvCap);
    D.densebuf = reinterpret_cast<uint32_t*>(at);
    at += align_up(sizeof(uint32_t) * 2 * (size_t)kDenseTriMax);
    D.pairbuf = reinterpret_cast<uint32_t*>(at);
}

// GC_PIPELINE=0 runs bitmap jobs with the sequential window loop (for
// measurements); pipelining is on by default.
static bool pipeline_enabled() {
    const char* e = std::getenv("GC_PIPELINE");
    return !(e && std::strcmp(e, "0") == 0);
}

// Pipelined windows of more survivors than one conflict matrix takes are
// decided from a whole-window matrix that the generators build (GC_DENSE=0
// turns this off, for measurements).  Its rows are limited by the resolver's
// shared memory: the matrix area plus the code cache behind it.
static bool dense_enabled() {
    const char* e = std::getenv("GC_DENSE");
    return !(e && std::strcmp(e, "0") == 0);
}
// GC_DENSE_CUT=0 keeps windows whole (up to kSurvCap survivors) and decides
// the survivors beyond the matrix with the blocked matrices (measurements).
static uint32_t dense_cut_mode() {
    const char* e = std::getenv("GC_DENSE_CUT");
    return (e && std::strcmp(e, "0") == 0) ? 0u : 1u;
}
static uint32_t dense_rows_for(uint32_t cache_words) {
    if (!dense_enabled()) return 0u;
    const uint64_t room = (uint64_t)kResolveWords * kResolveBlock + cache_words;
    uint32_t P = kDenseMaxRows;
    while (P > 0 && dense_tri_words(P) > room) P -= 32;
    return P >= 128 ? P : 0u;
}

static Order make_order_host(const HostProblem& p) { return order_of(p, p.filter, p.orth); }

// Entries per resolver conflict matrix: smaller blocks build smaller
// matrices but take more block steps.  GC_RESOLVE_BLOCK overrides (tuning).
static uint32_t resolve_block_size() {
    uint32_t b = 384;
    if (const char* e = std::getenv("GC_RESOLVE_BLOCK")) b = (uint32_t)std::atoi(e);
    b = (b + 31u) & ~31u;
    return std::max<uint32_t>(32u, std::min<uint32_t>(b, kResolveBlock));
}

// Rough device cost of one job, used to balance jobs over groups.
double job_cost(const HostProblem& p, int strategy) {
    const double N = (double)p.valid;
    const double C = std::max(1.0, 0.5 * (double)p.bound);
    if (strategy == GC_STRATEGY_BITMAP) return N + 8.0 * C * (double)high_ball_len(p.n, p.d);
    return N * 32.0 + C * C;
}

bool batch_layout(const BatchJob* jobs, int njobs, int ngroups_req, BatchLayout* L,
                  std::string* why) {
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        *why = "cannot query the CUDA device";
        return false;
    }
    if (njobs < 1) {
        *why = "no jobs";
        return false;
    }
    // one wide job makes the whole launch wide (uint64 words, distance only)
    bool wide = false;
    for (int j = 0; j < njobs; ++j) wide = wide || jobs[j].wide;
    for (int j = 0; j < njobs; ++j)
        if (wide && jobs[j].plan.strategy != GC_STRATEGY_DISTANCE) {
            *why = "the wide sweep (uint64 words) runs the distance strategy only";
            return false;
        }
    L->wide = wide;
    const size_t wbytes = wide ? 8 : 4;
    const size_t base = wide ? sizeof(SweepSmem<uint64_t>) : sizeof(SweepSmem<uint32_t>);
    if ((size_t)optin < base + 16) {
        *why = "not enough shared memory per block";
        return false;
    }
    int grid = sms;
    for (int j = 0; j < njobs; ++j)
        if (jobs[j].plan.grid > 0) grid = std::min(grid, jobs[j].plan.grid);
    // default: one group per job; a batch of more jobs than a quarter of the
    // SMs runs on groups of four CTAs that claim jobs dynamically (512 mixed
    // n = 14-24 codes: 114 ms, against 295 ms with 152 one-CTA groups and
    // 157 ms with the best static assignment)
    int ng = ngroups_req > 0 ? ngroups_req
                             : (dynamic_enabled() && njobs > grid / 4 ? std::max(1, grid / 4)
                                                                    : std::min(njobs, grid));
    ng = std::max(1, std::min(ng, std::min(njobs, grid)));
    L->grid = grid;
    L->ngroups = ng;
    // shared-memory code cache for distance jobs
    uint64_t need_cache = 0;
    for (int j = 0; j < njobs; ++j)
        if (jobs[j].plan.strategy == GC_STRATEGY_DISTANCE)
            need_cache = std::max<uint64_t>(need_cache, jobs[j].p.bound);
    uint64_t room = (((size_t)optin - base) / wbytes) & ~(uint64_t)31;
    uint32_t cache = (uint32_t)std::min<uint64_t>(room, (need_cache + 31) & ~(uint64_t)31);
    L->cache_words = cache;
    L->smem_bytes = base + (size_t)cache * wbytes;
    std::vector<double> cost(njobs);
    for (int j = 0; j < njobs; ++j) cost[j] = job_cost(jobs[j].p, jobs[j].plan.strategy);
    L->first_cta.assign(ng, 0);
    L->ncta.assign(ng, 0);
    std::vector<std::vector<int>> per(ng);
    if (ng == njobs && ng > 1) {
        // one job per group: CTAs in proportion to the job's estimated work,
        // at least kMinGroup (or an equal share if the SMs are too few);
        // distance jobs weigh 1.5x their estimate: the bitmap jobs' time is
        // mostly their resolver's chain, which more CTAs do not shorten (the
        // five codes of n = 24, d = 8 and n = 20, d = 4: 2.445 ms per launch
        // with 1x, 2.409 with 1.5x, 2.413 with 2x, 2.581 with 3x);
        // GC_DIST_SHARE overrides it (measurements)
        const int minc = std::max(1, std::min(kMinGroup, grid / ng));
        double dist_share = 1.5;
        if (const char* e = std::getenv("GC_DIST_SHARE")) dist_share = std::atof(e);
        if (!(dist_share > 0.0 && dist_share < 100.0)) dist_share = 1.5;
        std::vector<double> share(cost);
        for (int j = 0; j < njobs; ++j)
            if (jobs[j].plan.strategy == GC_STRATEGY_DISTANCE) share[j] *= dist_share;
        double total = 0;
        for (double c : share) total += c;
        int left = grid - minc * ng;
        std::vector<int> extra(ng, 0);
        int given = 0;
        for (int g = 0; g < ng; ++g) {
            extra[g] = (int)std::floor(left * share[g] / std::max(total, 1e-30));
            given += extra[g];
        }
        for (int g = 0; given < left; g = (g + 1) % ng, ++given) extra[g] += 1;
        int at = 0;
        for (int g = 0; g < ng; ++g) {
            L->first_cta[g] = at;
            L->ncta[g] = minc + extra[g];
            at += L->ncta[g];
            per[g].push_back(g);
        }
    } else {
        // equal CTA counts; jobs longest first onto the least-loaded group
        for (int g = 0; g < ng; ++g) {
            L->first_cta[g] = g * grid / ng;
            L->ncta[g] = (g + 1) * grid / ng - L->first_cta[g];
        }
        std::vector<int> idx(njobs);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<double> load(ng, 0.0);
        for (int j : idx) {
            const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            per[g].push_back(j);
            load[g] += cost[j] / std::max(1, L->ncta[g]);
        }
    }
    for (int g = 0; g < ng; ++g)
        if (L->ncta[g] > kMaxGroupCtas || L->ncta[g] < 1) {
            *why = "bad group size";
            return false;
        }
    L->job_order.clear();
    L->job_begin.assign(ng, 0);
    L->job_end.assign(ng, 0);
    L->dynamic = ng < njobs && dynamic_enabled();
    if (L->dynamic) {
        // one list, longest first; the groups claim from it at run time
        L->job_order.resize(njobs);
        std::iota(L->job_order.begin(), L->job_order.end(), 0);
        std::stable_sort(L->job_order.begin(), L->job_order.end(),
                         [&](int x, int y) { return cost[x] > cost[y]; });
    } else {
        for (int g = 0; g < ng; ++g) {
            // keep each group's jobs in submission order
            std::sort(per[g].begin(), per[g].end());
            L->job_begin[g] = (int)L->job_order.size();
            for (int j : per[g]) L->job_order.push_back(j);
            L->job_end[g] = (int)L->job_order.size();
        }
    }
    // Pipelined bitmap jobs that decide windows from whole-window matrices
    // (survivor target below the matrix's rows, a group of at least
    // kDenseMinGenerators + 1 CTAs) hold them in the cache area too.  Only
    // then: a larger shared-memory carve-out leaves less L1 for the kernel's
    // spills (sweeps of n = 32 ran up to 1.4x slower with it).
    const uint32_t dense_rows_max = dense_rows_for((uint32_t)room);
    bool dense_any = false;
    for (int g = 0; g < ng && pipeline_enabled(); ++g) {
        if (L->ncta[g] - 1 < kDenseMinGenerators) continue;
        const int q0 = L->dynamic ? 0 : L->job_begin[g], q1 = L->dynamic ? njobs : L->job_end[g];
        for (int q = q0; q < q1; ++q) {
            const BatchJob& J = jobs[L->job_order[q]];
            const uint32_t tgt = J.plan.survivor_target ? J.plan.survivor_target
                                                        : default_target(J.plan.strategy, J.p);
            dense_any |= J.plan.strategy == GC_STRATEGY_BITMAP && tgt < dense_rows_max;
        }
    }
    L->dense = dense_any;
    if (dense_any) {
        cache = (uint32_t)room;
        L->cache_words = cache;
        L->smem_bytes = base + (size_t)cache * wbytes;
    }
    // workspace
    size_t off = 0;
    L->off_err = off;        off += align_up(256);
    L->off_jobs = off;       off += align_up(sizeof(JobDesc) * njobs);
    L->off_order = off;      off += align_up(sizeof(int) * njobs);
    L->off_groups = off;     off += align_up(sizeof(GroupDesc) * ng);
    L->g_flags.assign(ng, 0); L->g_segx.assign(ng, 0); L->g_segoff.assign(ng, 0);
    L->g_store.assign(ng, 0); L->g_store_words.assign(ng, 0); L->g_bitmap.assign(ng, 0);
    L->g_slice.assign(ng, 0);
    L->g_pipe.assign(ng, 0);
    for (int g = 0; g < ng; ++g) {
        uint64_t store = 0, bits = 0;
        // a dynamic group may run any job of the batch
        const int q0 = L->dynamic ? 0 : L->job_begin[g], q1 = L->dynamic ? njobs : L->job_end[g];
        for (int q = q0; q < q1; ++q) {
            const BatchJob& J = jobs[L->job_order[q]];
            if (J.plan.strategy == GC_STRATEGY_DISTANCE && J.p.bound > cache)
                store = std::max<uint64_t>(store, J.p.bound);
            if (J.plan.strategy == GC_STRATEGY_BITMAP)
                bits = std::max<uint64_t>(bits, 1ull << J.p.n);
        }
        if (store > 0xffffffffull) {
            *why = "code too large for the distance strategy";
            return false;
        }
        const int G = L->ncta[g];
        // one spare flag pair per group (used only by the wait-fault injection)
        L->g_flags[g] = off;  off += align_up(sizeof(unsigned long long) * 2 * (G + 1));
        L->g_segx[g] = off;   off += align_up(wbytes * 2 * (size_t)G * kChunk);
        L->g_segoff[g] = off; off += align_up(sizeof(uint32_t) * 2 * (size_t)G * kChunk);
        L->g_store[g] = off;  off += align_up(wbytes * store);
        L->g_store_words[g] = store;
        L->g_bitmap[g] = off; off += align_up((bits + 31) / 32 * 4);
        L->g_slice[g] = off;  off += align_up((size_t)2 * G * kMaxSlices);
        // pipelined bitmap jobs (sized, like the flags, for one spare CTA)
        L->g_pipe[g] = 0;
        if (bits > 0) {
            L->g_pipe[g] = off;
            off += pipe_bytes(G + 1);
        }
    }
    // ball tables, one per distinct (n, d) among bitmap jobs
    L->hball_off.assign(njobs, 0);
    for (int j = 0; j < njobs; ++j) {
        if (jobs[j].plan.strategy != GC_STRATEGY_BITMAP) continue;
        int same = -1;
        for (int i = 0; i < j; ++i)
            if (jobs[i].plan.strategy == GC_STRATEGY_BITMAP && jobs[i].p.n == jobs[j].p.n &&
                jobs[i].p.d == jobs[j].p.d) { same = i; break; }
        if (same >= 0) { L->hball_off[j] = L->hball_off[same]; continue; }
        L->hball_off[j] = off;
        off += align_up(4 * high_ball_len(jobs[j].p.n, jobs[j].p.d));
    }
    L->total = off;
    return true;
}

// Host-side fault injection for tests of the failure path: GC_FAULT=wait
// makes group 0 wait for one CTA that does not exist, with a 0.2 s limit, so
// its bounded waits expire and every job reports GC_ERR_TIMEOUT.
// Pipelined windows: the generators list the window's conflicting pairs for
// the resolver when that pays; GC_PAIRS=0 turns it off, GC_PAIRS=2 makes it
// unconditional (measurements, tests).
static uint32_t pairs_mode() {
    const char* e = std::getenv("GC_PAIRS");
    if (!e) return 1u;
    return std::strcmp(e, "0") == 0 ? 0u : std::strcmp(e, "2") == 0 ? 2u : 1u;
}

// CTA of each group whose phase cycles the statistics report: the first,
// or GC_TIMING_CTA (diagnostics: a pipelined job's CTA 1 is a generator).
static uint32_t timing_cta() {
    const char* e = std::getenv("GC_TIMING_CTA");
    return e ? (uint32_t)std::atoi(e) : 0u;
}

static bool inject_wait_fault() {
    const char* fault = std::getenv("GC_FAULT");
    return fault && std::strcmp(fault, "wait") == 0;
}

int upload_batch(const BatchJob* jobs, int njobs, const BatchLayout& L, void* workspace,
                 cudaStream_t stream, std::string* why) {
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    const bool inject_wait = inject_wait_fault();
    std::vector<JobDesc> jd(njobs);
    for (int j = 0; j < njobs; ++j) {
        const BatchJob& J = jobs[j];
        JobDesc& D = jd[j];
        D.ord = make_order_host(J.p);
        D.d = J.p.d;
        D.strategy = J.plan.strategy == GC_STRATEGY_BITMAP ? kStratBitmap : kStratDistance;
        D.orth = J.p.orth ? 1 : 0;
        D.pipelined = (D.strategy == kStratBitmap && pipeline_enabled()) ? 1 : 0;
        D.out = J.d_out;
        D.cap = J.capacity;
        D.stats = J.d_stats;
        D.hball = D.strategy == kStratBitmap ? reinterpret_cast<const uint32_t*>(ws + L.hball_off[j])
                                             : nullptr;
        D.hball_len = D.strategy == kStratBitmap ? (uint32_t)high_ball_len(J.p.n, J.p.d) : 0u;
        D.target = J.plan.survivor_target ? J.plan.survivor_target
                                          : default_target(J.plan.strategy, J.p);
        // a window never holds more candidates than the group's chunks (in a
        // dynamic batch, the smallest group's)
        int g = 0;
        if (L.dynamic) {
            for (int q = 1; q < L.ngroups; ++q)
                if (L.ncta[q] < L.ncta[g]) g = q;
        } else {
            for (int q = 0; q < L.ngroups; ++q)
                for (int i = L.job_begin[q]; i < L.job_end[q]; ++i)
                    if (L.job_order[i] == j) g = q;
        }
        const uint64_t wcap = (uint64_t)L.ncta[g] * kChunk;
        D.wmax = (uint32_t)std::min<uint64_t>(J.plan.window_max ? J.plan.window_max : wcap, wcap);
        D.wmin = std::max<uint32_t>(
            1, std::min<uint32_t>(J.plan.window_min ? J.plan.window_min : 256, D.wmax));
    }
    std::vector<GroupDesc> gd(L.ngroups);
    for (int g = 0; g < L.ngroups; ++g) {
        GroupDesc& G = gd[g];
        G.first_cta = L.first_cta[g];
        G.ncta = L.ncta[g] + ((inject_wait && g == 0) ? 1 : 0);
        G.job_begin = L.job_begin[g];
        G.job_end = L.job_end[g];
        G.flags = reinterpret_cast<unsigned long long*>(ws + L.g_flags[g]);
        G.seg_x = ws + L.g_segx[g];
        G.seg_off = reinterpret_cast<uint32_t*>(ws + L.g_segoff[g]);
        G.store = ws + L.g_store[g];
        G.store_words = L.g_store_words[g];
        G.bitmap = reinterpret_cast<uint32_t*>(ws + L.g_bitmap[g]);
        G.slice_cnt = ws + L.g_slice[g];
        G.pflags = nullptr;
        G.accbuf = nullptr;
        G.pairbuf = nullptr;
        G.densebuf = nullptr;
        if (L.g_pipe[g]) set_pipe(G, ws + L.g_pipe[g]);
    }
    cudaError_t e;
    auto cuda_fail = [&](const char* what) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        return GC_ERR_CUDA;
    };
    // descriptors (pageable host memory: staged before the call returns)
    if ((e = cudaMemcpyAsync(ws + L.off_jobs, jd.data(), sizeof(JobDesc) * njobs,
                             cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail("job descriptors");
    if ((e = cudaMemcpyAsync(ws + L.off_order, L.job_order.data(), sizeof(int) * njobs,
                             cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail("job order");
    if ((e = cudaMemcpyAsync(ws + L.off_groups, gd.data(), sizeof(GroupDesc) * L.ngroups,
                             cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail("group descriptors");
    for (int j = 0; j < njobs; ++j) {
        if (jd[j].strategy != kStratBitmap) continue;
        bool first = true;
        for (int i = 0; i < j; ++i)
            if (jd[i].strategy == kStratBitmap && L.hball_off[i] == L.hball_off[j]) first = false;
        if (!first) continue;
        const int nh = jobs[j].p.n > 5 ? jobs[j].p.n - 5 : 0;
        const int rc = launch_high_ball(nh, jobs[j].p.d - 1, const_cast<uint32_t*>(jd[j].hball),
                                        jd[j].hball_len, stream);
        if (rc) {
            *why = "ball table";
            return rc;
        }
    }
    const void* kernel = L.wide ? (const void*)sweep_kernel<uint64_t>
                                : (const void*)sweep_kernel<uint32_t>;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_bytes)) != cudaSuccess)
        return cuda_fail("shared memory attribute");
    return GC_OK;
}

int launch_batch_kernel(const BatchLayout& L, void* workspace, cudaStream_t stream,
                        std::string* why) {
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    const bool inject_wait = inject_wait_fault();
    cudaError_t e;
    auto cuda_fail = [&](const char* what) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        return GC_ERR_CUDA;
    };
    if ((e = cudaMemsetAsync(ws + L.off_err, 0, 256, stream)) != cudaSuccess)
        return cuda_fail("error word");
    for (int g = 0; g < L.ngroups; ++g) {
        // flags start at sequence 0xffffffff so no stale value matches
        if ((e = cudaMemsetAsync(ws + L.g_flags[g], 0xff,
                                 sizeof(unsigned long long) * 2 * (L.ncta[g] + 1), stream)) !=
            cudaSuccess)
            return cuda_fail("group flags");
        if (L.g_pipe[g] &&
            (e = cudaMemsetAsync(ws + L.g_pipe[g], 0xff, pipe_flag_bytes(L.ncta[g] + 1),
                                 stream)) != cudaSuccess)
            return cuda_fail("pipeline flags");
    }
    const void* kernel = L.wide ? (const void*)sweep_kernel<uint64_t>
                                : (const void*)sweep_kernel<uint32_t>;
    BatchArgs a{};
    a.jobs = reinterpret_cast<const JobDesc*>(ws + L.off_jobs);
    a.job_order = reinterpret_cast<const int*>(ws + L.off_order);
    // the claim counter shares the error word's 256 bytes, zeroed per launch
    a.claim = L.dynamic ? reinterpret_cast<unsigned*>(ws + L.off_err + 64) : nullptr;
    a.njobs = (int)L.job_order.size();
    a.groups = reinterpret_cast<const GroupDesc*>(ws + L.off_groups);
    a.ngroups = L.ngroups;
    a.err = reinterpret_cast<unsigned*>(ws + L.off_err);
    a.cache_words = L.cache_words;
    a.timeout_cycles = inject_wait ? 400000000ll : 20000000000ll;  // ~0.2 s / ~10 s at 2 GHz
    a.resolve_block = resolve_block_size();
    a.pairs = pairs_mode();
    a.dense_rows = L.dense ? dense_rows_for(L.cache_words) : 0u;
    a.dense_cut = dense_cut_mode();
    a.timing_cta = timing_cta();
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel(kernel, dim3(L.grid), dim3(kBlock), args, L.smem_bytes,
                                    stream);
    if (e != cudaSuccess) return cuda_fail("sweep launch");
    return GC_OK;
}

int launch_batch(const BatchJob* jobs, int njobs, const BatchLayout& L, void* workspace,
                 cudaStream_t stream, std::string* why) {
    const int rc = upload_batch(jobs, njobs, L, workspace, stream, why);
    return rc ? rc : launch_batch_kernel(L, workspace, stream, why);
}

}  // namespace gc

namespace gc {

// ------------------------------------------------------------------ server
bool serve_layout(const gc_server_config& cfg, ServeLayout* L, std::string* why) {
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        *why = "cannot query the CUDA device";
        return false;
    }
    const size_t base = sizeof(SweepSmem<uint32_t>);
    if ((size_t)optin < base + 16) {
        *why = "not enough shared memory per block";
        return false;
    }
    int ng = cfg.ngroups > 0 ? cfg.ngroups : std::max(1, sms / 8);
    ng = std::max(1, std::min(ng, sms));
    L->ngroups = ng;
    L->group_ctas = sms / ng;
    L->grid = L->group_ctas * ng;
    uint64_t room = (((size_t)optin - base) / 4) & ~(uint64_t)31;
    L->cache_words = (uint32_t)std::min<uint64_t>(room, 16384);
    L->smem_bytes = base + (size_t)L->cache_words * 4;
    L->store_words = cfg.store_words;
    L->bitmap_bits = 1ull << cfg.max_n;
    size_t off = 0;
    L->off_err = off;    off += align_up(256);
    L->off_head = off;   off += align_up(256);
    L->off_groups = off; off += align_up(sizeof(GroupDesc) * ng);
    L->g_flags.assign(ng, 0); L->g_segx.assign(ng, 0); L->g_segoff.assign(ng, 0);
    L->g_store.assign(ng, 0); L->g_bitmap.assign(ng, 0);
    L->g_slice.assign(ng, 0); L->g_pipe.assign(ng, 0);
    const int G = L->group_ctas;
    for (int g = 0; g < ng; ++g) {
        L->g_flags[g] = off;  off += align_up(sizeof(unsigned long long) * 2 * (G + 1));
        L->g_segx[g] = off;   off += align_up(sizeof(uint32_t) * 2 * (size_t)G * kChunk);
        L->g_segoff[g] = off; off += align_up(sizeof(uint32_t) * 2 * (size_t)G * kChunk);
        L->g_store[g] = off;  off += align_up(sizeof(uint32_t) * L->store_words);
        L->g_bitmap[g] = off; off += align_up((L->bitmap_bits + 31) / 32 * 4);
        L->g_slice[g] = off;  off += align_up((size_t)2 * G * kMaxSlices);
        L->g_pipe[g] = off;
        off += pipe_bytes(G);
    }
    L->off_hball = off;
    L->hball_bytes = 64ull << 20;
    off += L->hball_bytes;
    L->total = off;
    return true;
}

// The word-grouped ball of radius d-1 (see high_ball_kernel), built on the
// host so no kernel has to run beside the persistent one.
static std::vector<uint32_t> host_high_ball(int n, int d) {
    const int nh = n > 5 ? n - 5 : 0;
    std::vector<uint32_t> out;
    for (int k = 0; k <= d - 1 && k <= nh; ++k) {
        const int r = std::min(d - 1 - k, 7);
        if (k == 0) {
            out.push_back((uint32_t)r);
            continue;
        }
        // every nh-bit integer with k bits set, in increasing order
        uint64_t y = (1ull << k) - 1;
        while (y < (1ull << nh)) {
            out.push_back(((uint32_t)y << 3) | (uint32_t)r);
            const uint64_t low = y & (~y + 1);
            const uint64_t up = y + low;
            y = (((up ^ y) >> 2) / low) | up;
        }
    }
    return out;
}

bool serve_describe(ServeLayout& L, const HostProblem& p, int strategy, uint32_t* d_out,
                    uint64_t cap, gc_stats* d_stats, JobDesc* D, std::string* why) {
    gc_plan_t pl{};
    plan_for(p, &pl);
    pl.strategy = batch_strategy(pl.strategy);
    strategy = batch_strategy(strategy);
    if (strategy == GC_STRATEGY_DISTANCE || strategy == GC_STRATEGY_BITMAP) pl.strategy = strategy;
    const bool dist_fits = p.bound <= (uint64_t)L.cache_words + L.store_words;
    const bool bitmap_fits = (1ull << p.n) <= L.bitmap_bits && high_ball_len(p.n, p.d) < (1u << 24);
    if (pl.strategy == GC_STRATEGY_DISTANCE && !dist_fits && bitmap_fits)
        pl.strategy = GC_STRATEGY_BITMAP;
    if (pl.strategy == GC_STRATEGY_BITMAP && !bitmap_fits && dist_fits)
        pl.strategy = GC_STRATEGY_DISTANCE;
    if ((pl.strategy == GC_STRATEGY_DISTANCE && !dist_fits) ||
        (pl.strategy == GC_STRATEGY_BITMAP && !bitmap_fits)) {
        *why = "request does not fit the server's scratch";
        return false;
    }
    std::memset(D, 0, sizeof *D);
    D->ord = make_order_host(p);
    D->d = p.d;
    D->strategy = pl.strategy == GC_STRATEGY_BITMAP ? kStratBitmap : kStratDistance;
    D->orth = p.orth ? 1 : 0;
    D->pipelined = (D->strategy == kStratBitmap && pipeline_enabled()) ? 1 : 0;
    D->out = d_out;
    D->cap = cap;
    D->stats = d_stats;
    D->target = default_target(pl.strategy, p);
    D->wmax = (uint32_t)((uint64_t)L.group_ctas * kChunk);
    D->wmin = std::min<uint32_t>(256, D->wmax);
    if (D->strategy == kStratBitmap && p.d >= 1) {
        const uint32_t key = ((uint32_t)p.n << 8) | (uint32_t)std::min(p.d, 255);
        size_t at = 0;
        uint32_t len = 0;
        bool found = false;
        for (auto& t : L.hball_tables)
            if (t.first == key) { at = t.second.first; len = t.second.second; found = true; }
        if (!found) {
            std::vector<uint32_t> tab = host_high_ball(p.n, p.d);
            const size_t bytes = align_up(tab.size() * 4);
            if (L.hball_used + bytes > L.hball_bytes) {
                *why = "ball-table arena full";
                return false;
            }
            at = L.off_hball + L.hball_used;
            len = (uint32_t)tab.size();
            if (cudaMemcpy(static_cast<uint8_t*>(L.ws) + at, tab.data(), tab.size() * 4,
                           cudaMemcpyHostToDevice) != cudaSuccess) {
                *why = "ball-table upload";
                return false;
            }
            L.hball_used += bytes;
            L.hball_tables.push_back({key, {at, len}});
        }
        D->hball = reinterpret_cast<const uint32_t*>(static_cast<uint8_t*>(L.ws) + at);
        D->hball_len = len;
    }
    return true;
}

int launch_server(ServeLayout& L, void* workspace, JobDesc* ring, unsigned* tail, unsigned* stop,
                  unsigned long long* done, uint32_t capacity, double idle_seconds,
                  cudaStream_t stream, std::string* why) {
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    L.ws = workspace;
    std::vector<GroupDesc> gd(L.ngroups);
    for (int g = 0; g < L.ngroups; ++g) {
        GroupDesc& G = gd[g];
        G.first_cta = g * L.group_ctas;
        G.ncta = L.group_ctas;
        G.job_begin = G.job_end = 0;
        G.flags = reinterpret_cast<unsigned long long*>(ws + L.g_flags[g]);
        G.seg_x = ws + L.g_segx[g];
        G.seg_off = reinterpret_cast<uint32_t*>(ws + L.g_segoff[g]);
        G.store = ws + L.g_store[g];
        G.store_words = L.store_words;
        G.bitmap = reinterpret_cast<uint32_t*>(ws + L.g_bitmap[g]);
        G.slice_cnt = ws + L.g_slice[g];
        set_pipe(G, ws + L.g_pipe[g]);
    }
    cudaError_t e;
    auto cuda_fail = [&](const char* what) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        return GC_ERR_CUDA;
    };
    if ((e = cudaMemcpyAsync(ws + L.off_groups, gd.data(), sizeof(GroupDesc) * L.ngroups,
                             cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail("group descriptors");
    if ((e = cudaMemsetAsync(ws + L.off_err, 0, 256, stream)) != cudaSuccess)
        return cuda_fail("error word");
    for (int g = 0; g < L.ngroups; ++g) {
        if ((e = cudaMemsetAsync(ws + L.g_flags[g], 0xff,
                                 sizeof(unsigned long long) * 2 * (L.group_ctas + 1), stream)) !=
            cudaSuccess)
            return cuda_fail("group flags");
        if ((e = cudaMemsetAsync(ws + L.g_pipe[g], 0xff, pipe_flag_bytes(L.group_ctas),
                                 stream)) != cudaSuccess)
            return cuda_fail("pipeline flags");
    }
    // the claim counter (zeroed when the server is created) is left as it
    // is: a relaunch continues with the first published job no group has
    // claimed
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail("server set-up");
    if ((e = cudaFuncSetAttribute(sweep_kernel<uint32_t>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_bytes)) != cudaSuccess)
        return cuda_fail("shared memory attribute");
    BatchArgs a{};
    a.jobs = nullptr;
    a.job_order = nullptr;
    a.groups = reinterpret_cast<const GroupDesc*>(ws + L.off_groups);
    a.ngroups = L.ngroups;
    a.err = reinterpret_cast<unsigned*>(ws + L.off_err);
    a.cache_words = L.cache_words;
    a.timeout_cycles = 20000000000ll;
    a.resolve_block = resolve_block_size();
    a.pairs = pairs_mode();
    a.dense_rows = dense_rows_for(L.cache_words);
    a.dense_cut = dense_cut_mode();
    a.timing_cta = timing_cta();
    int dev = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    a.queue.descs = ring;
    a.queue.tail = tail;
    a.queue.stop = stop;
    a.queue.done = done;
    a.queue.head = reinterpret_cast<unsigned*>(ws + L.off_head);
    a.queue.capacity = capacity;
    a.queue.idle_cycles = (long long)(idle_seconds * (clk_khz > 0 ? clk_khz : 2000000) * 1e3);
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)sweep_kernel<uint32_t>, dim3(L.grid),
                                    dim3(kBlock), args,
                                    L.smem_bytes, stream);
    if (e != cudaSuccess) return cuda_fail("server launch");
    return GC_OK;
}

}  // namespace gc
