// gc_gridsweep.cu -- the exclusion-bitmap sweep of one code on the whole
// GPU in lockstep windows (the "grid" bitmap strategy).
//
// It computes what the pipelined bitmap sweep of gc_sweep.cu computes -- the
// ordered greedy code of Section 4 -- for one code at a time, with every SM
// taking part in every step of every window.  The exclusion bitmap holds the
// radius-(d-2) balls of the codewords accepted so far, and a vector is
// covered (within distance d-1 of one of them) iff a marked vector lies
// within distance 1 of it: its own word, under the in-word radius-1 mask, or
// its bit in the n - 5 words one high bit away.  The radius-(d-2) ball is
// several times smaller than the radius-(d-1) one (32 against about 350
// words per codeword at n = 31, d = 3; 379 against about 3300 at n = 32,
// d = 4), and most covered candidates show it at the first probe.  Window t
// of W consecutive ranks takes two phases, each ended by a grid-wide barrier
// (one arrival counter, polled by one thread per CTA):
//  A. every CTA writes its share of window t-1's accepts to the output, ORs
//     its share of their balls into the bitmap, then generates its
//     contiguous chunk of window t from the ranks (Section 4.2 orders,
//     closed form; a thread takes up to four consecutive ranks, and in the
//     orders that list a weight class as k-subsets in numeric order steps
//     from one to the next instead of unranking each) and drops the
//     candidates the bitmap covers -- it is complete up to window t-2 and
//     holds part of window t-1.  The survivors go to the CTA's segment, in
//     rank order.
//  B. every CTA gathers the window's survivors (the first kGwSurvCap; the
//     window is cut after them).  It probes its rows (entries i = CTA index
//     mod grid) against the bitmap, now complete up to window t-1 -- a hit
//     rejects the entry -- and tests them against every earlier entry of the
//     window, listing the conflicting pairs (Hamming distance < d).  The
//     (row, earlier entry) triangle is cut into one equal span per warp,
//     whose lanes sweep consecutive entries, four to a 16-byte load, against
//     the row word the warp holds.  For d = 3 a 2^n-byte array counts, for
//     each vector, the window's survivors within distance 1 of it (each CTA
//     adds its survivors' radius-1 balls in phase A and takes its previous
//     window's out); the counts over a row's own radius-1 ball add up to
//     n + 1 plus two for every other survivor within distance 2, so only the
//     rows above n + 1 run the tests -- in most windows, none.
//     Each CTA publishes its rows' kills and its pairs, the pairs into one
//     list for the window at offsets reserved on a counter.
// Then every CTA, from the same data, decides the window exactly as the
// serial loop would: with no pair, the entries no accept rejected are the
// accepts; otherwise rounds over the pair list (an entry is rejected once an
// earlier neighbour is accepted and accepted once every earlier neighbour is
// rejected), from shared memory, or first over the list in L2 while it is
// too long for shared memory; when it is longer still, the conflict
// matrices of block_resolve.  Every CTA keeps the accepts for the next
// window.  The next window aims at kGwSurvCap survivors at the density this
// one had, fewer where its survivors conflict densely (sized for a set
// number of pairs at this window's pair density).
// A second form (GC_GRID_EARLY=0) marks window t-1's balls between the row
// tests of phase B and tests the rows against window t-1's accepts instead
// of probing them; with GC_GRID_PROBE=0 as well, it marks radius-(d-1) balls
// and a lookup reads one bit.
// Compared with the pipelined form, no CTA waits on another's flag word
// (the flag all-gathers of that design took several microseconds each at
// 152 CTAs, the counter barrier about two), nothing runs on one SM while the
// others wait, and the pair search and the marks are spread over every SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "gc_block.cuh"
#include "gc_internal.h"

namespace gc {

constexpr int kGwSurvCap = 8192;        // survivors decided per window
constexpr int kGwChunk = 4096;          // candidates per CTA per window
constexpr uint32_t kGwPairCap = 4096;   // pairs one CTA may list per window
constexpr uint32_t kGwPairSmem = 16384; // pairs a CTA takes into shared memory
constexpr uint32_t kGwPairGlobal = 8 * kGwPairSmem;  // pairs decided by rounds over L2
constexpr int kGwMaxCtas = kBlock;      // one count per thread in the prefix scans
constexpr int kGwProbeBatch = 14;       // high-bit probes a lookup issues at once
static_assert(kGwChunk <= 4 * kBlock, "a thread generates at most four ranks of its CTA's chunk");
static_assert(kGwSurvCap <= 65536, "pairs pack two entry indices in 16 bits each");
constexpr int kGwPerThread = kGwSurvCap / kBlock;   // window entries per thread
static_assert(kGwSurvCap % (4 * kBlock) == 0, "threads take window entries four at a time");
static_assert(kGwPerThread == 8, "a thread decides eight consecutive entries");
static_assert(kGwPairSmem >= kResolveWords * kResolveBlock + kGwSurvCap,
              "the conflict-matrix fallback keeps its accepts' offsets after its matrix");
constexpr uint32_t kGwPairTargetDefault = 16000;  // pairs a window is sized for
static_assert(kGwPairCap <= kGwPairSmem, "a CTA's own pairs are staged in the pair area");
static_assert(kGwPairCap == 4 * kBlock, "a thread publishes at most four of its CTA's pairs");

struct GwArgs {
    Order ord;
    int d;
    uint32_t* out;
    uint64_t cap;
    gc_stats* stats;
    const uint32_t* hball;    // word-grouped ball table (high_ball_kernel)
    uint32_t hball_len;
    uint32_t* bitmap;         // 2^n bits, vector-indexed
    uint32_t* seg_x;          // [2][grid][kGwChunk] survivors of each CTA's chunk
    uint32_t* seg_off;        // [2][grid][kGwChunk] their offsets from the window start
    uint32_t* slot;           // [2][grid] survivor counts
    uint32_t* pslot;          // [2][grid] pair counts (kGwPairCap + 1: overflow)
    uint32_t* pairbuf;        // grid * kGwPairCap: the window's pairs, (earlier << 16) | later,
                              // packed in the order the CTAs reserve space (ctrl[2 + parity])
    uint8_t* killbuf;         // [kGwSurvCap] 1: the entry meets a previous accept
    unsigned* ctrl;           // [0] barrier arrivals, [1] error word, [2..3] pairs listed
                              // in the window of parity 0 / 1
    uint32_t wmin, wmax, target;
    long long timeout_cycles;
    uint32_t timing_cta;
    uint32_t extra_arrivals;  // fault injection: barriers wait for this many CTAs more
    uint32_t reversed;        // 1: the bitmap is indexed by the bit-reversed vector
    uint32_t probe;           // 1: radius-(d-2) balls marked, lookups probe radius 1
    uint32_t pair_smem;       // pairs decided from shared memory (<= kGwPairSmem)
    uint32_t pair_target;     // pairs the next window is sized for
    uint32_t early;           // 1 (with probe): window t-1's balls marked in phase A of
                              // window t, rows probed in phase B instead of tested
    uint32_t* cnt;            // d = 3 (with early): byte v counts the current window's
                              // survivors within distance 1 of vector v (indexed like
                              // the bitmap: bit-reversed for grevlex); null: unused
};

struct __align__(16) GwSmem;
struct __align__(16) GwSmem {
    uint32_t C[kMaxN + 1][kMaxN + 1];
    uint32_t lowball[8][32];  // lowball[r][c]: bits y < 32 with popc(y ^ c) <= r
    uint32_t lowlight[8];     // lowlight[k]: bits y < 32 with popc(y) < k
    uint32_t pref[kGwMaxCtas + 1];
    __align__(16) uint32_t wx[kGwSurvCap];      // own chunk (A), the window (B)
    __align__(16) uint32_t woff[kGwSurvCap];
    __align__(16) uint32_t ax[kGwSurvCap];      // the previous window's accepts
    __align__(16) uint32_t rx[kGwSurvCap];      // B: this CTA's rows, contiguous
    uint8_t state[kGwSurvCap];                  // 0 undecided, 1 accepted, 2 rejected
    uint8_t flags[2 * kGwSurvCap];              // row kills (B); killed / blocked (rounds)
    BlockScratch bs;
    unsigned long long phase[12];
    long long tprev;
    uint32_t npairs;
    uint32_t fine;
    union {
        uint32_t pairs[kGwPairSmem];
        uint32_t M[kResolveWords][kResolveBlock];
    } u;
};

static_assert(sizeof(GwSmem) <= 232448, "one CTA per SM: at most 227 KiB of shared memory");

// CTA-wide grid barrier: one arrival per CTA on a counter that only grows;
// the barrier of epoch e is passed once it reaches (e + 1) * arrivals.  The
// arrival is a release reduction after the CTA barrier and the wait an
// acquire load before the next one, so the CTA's writes before the barrier
// are visible to every CTA after it.  Bounded: on a timeout (or an error
// another CTA reported) returns false.
__device__ bool gw_sync(GwSmem& s, const GwArgs& a, uint32_t& epoch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_add_release_gpu(a.ctrl, 1u);
        const unsigned target = (epoch + 1u) * (gridDim.x + a.extra_arrivals);
        const long long t0 = clock64();
        uint32_t fine = 1u;
        for (uint32_t it = 1;; ++it) {
            if ((int)(ld_acquire_gpu(a.ctrl) - target) >= 0) break;
            if ((it & 15u) != 0u) continue;
            if (ld_cg(a.ctrl + 1) != 0u) { fine = 0u; break; }
            if (clock64() - t0 > a.timeout_cycles) {
                atomicExch(a.ctrl + 1, 1u);
                fine = 0u;
                break;
            }
        }
        s.fine = fine;
    }
    ++epoch;
    __syncthreads();
    return s.fine != 0u;
}

// CTA-wide.  The window's decisions from its pair list: on entry state[i]
// is 2 for entries already rejected (they meet a previous window's accept)
// and 0 for the rest; pairs[0..P) hold (k << 16) | i for conflicting pairs
// k < i.  Each round decides every undecided entry whose earlier neighbours
// are all decided (the first undecided entry always is, so the rounds end);
// then the accepts x[i] are appended in order to ax.  Returns how many;
// counts rounds in *rounds.
__device__ uint32_t gw_pair_rounds(GwSmem& s, uint32_t n, uint32_t P, uint64_t* rounds) {
    uint8_t* killed = s.flags;
    uint8_t* blocked = s.flags + kGwSurvCap;
    const int lane = lane_id();
    for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
        killed[i] = 0;
        blocked[i] = 0;
    }
    if (threadIdx.x < 3) s.bs.left[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t round = 0;; ++round) {
        ++*rounds;
        const uint32_t slot = round % 3u, next = (round + 1u) % 3u;
        if (threadIdx.x == 0) s.bs.left[next] = 0u;
        for (uint32_t e = threadIdx.x; e < P; e += kBlock) {
            const uint32_t pr = s.u.pairs[e];
            const uint32_t k = pr >> 16, i = pr & 0xffffu;
            if (s.state[i] == 0) {
                const uint8_t sk = s.state[k];
                if (sk == 1) killed[i] = 1;
                else if (sk == 0) blocked[i] = 1;
            }
        }
        __syncthreads();
        bool left = false;
        for (uint32_t i = threadIdx.x; i < n; i += kBlock)
            if (s.state[i] == 0) {
                if (killed[i]) s.state[i] = 2;
                else if (!blocked[i]) s.state[i] = 1;
                else left = true;
                killed[i] = 0;
                blocked[i] = 0;
            }
        if (__any_sync(kFull, left) && lane == 0) s.bs.left[slot] = 1u;
        __syncthreads();
        if (s.bs.left[slot] == 0u) break;
    }
    uint32_t nacc = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += kBlock) {
        const uint32_t i = t0 + threadIdx.x;
        const bool keep = i < n && s.state[i] == 1;
        nacc = block_append(s.bs, keep, keep ? s.wx[i] : 0u, 0u, s.ax, (uint32_t*)nullptr, nacc);
    }
    return nacc;
}

// CTA-wide.  Rounds as in gw_pair_rounds, over a pair list too long for
// shared memory, read from the global list pairs[0..P) in every round; a
// round counts the pairs still relevant (later entry undecided, earlier
// entry not rejected).  Once they fit in shared memory (fit <= kGwPairSmem)
// a last pass copies them there and returns their number, for gw_pair_rounds
// to carry on from.  Returns 0 once every entry is decided.  Counts rounds in
// *rounds.
__device__ uint32_t gw_pair_rounds_global(GwSmem& s, const uint32_t* pairs, uint32_t P, uint32_t n,
                                          uint32_t fit, uint64_t* rounds) {
    constexpr uint32_t kNone = 0xffffffffu;   // pairs are below 2^28
    constexpr uint32_t kDepth = 8;            // loads in flight per thread
    uint8_t* killed = s.flags;
    uint8_t* blocked = s.flags + kGwSurvCap;
    const int lane = lane_id();
    for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
        killed[i] = 0;
        blocked[i] = 0;
    }
    __syncthreads();
    for (;;) {
        ++*rounds;
        uint32_t cnt = 0;
        for (uint32_t e0 = 0; e0 < P; e0 += kDepth * kBlock) {
            uint32_t pr[kDepth];
#pragma unroll
            for (uint32_t u = 0; u < kDepth; ++u) {
                const uint32_t e = e0 + u * kBlock + threadIdx.x;
                pr[u] = e < P ? ld_cg(pairs + e) : kNone;
            }
#pragma unroll
            for (uint32_t u = 0; u < kDepth; ++u) {
                if (pr[u] == kNone) continue;
                const uint32_t k = pr[u] >> 16, i = pr[u] & 0xffffu;
                if (s.state[i] != 0) continue;
                const uint8_t sk = s.state[k];
                if (sk == 1) { killed[i] = 1; ++cnt; }
                else if (sk == 0) { blocked[i] = 1; ++cnt; }
            }
        }
        uint32_t R = 0;
        block_exclusive_scan(s.bs, cnt, &R);   // ends with a CTA barrier
        bool left = false;
        for (uint32_t i = threadIdx.x; i < n; i += kBlock)
            if (s.state[i] == 0) {
                if (killed[i]) s.state[i] = 2;
                else if (!blocked[i]) s.state[i] = 1;
                else left = true;
                killed[i] = 0;
                blocked[i] = 0;
            }
        if (!__syncthreads_or(left)) return 0u;
        if (R > fit) continue;
        // the pairs relevant now are among the R counted above: copy them
        if (threadIdx.x == 0) s.npairs = 0;
        __syncthreads();
        for (uint32_t e0 = 0; e0 < P; e0 += kDepth * kBlock) {
            uint32_t pr[kDepth];
#pragma unroll
            for (uint32_t u = 0; u < kDepth; ++u) {
                const uint32_t e = e0 + u * kBlock + threadIdx.x;
                pr[u] = e < P ? ld_cg(pairs + e) : kNone;
            }
#pragma unroll
            for (uint32_t u = 0; u < kDepth; ++u) {
                bool rel = false;
                if (pr[u] != kNone) {
                    const uint32_t k = pr[u] >> 16, i = pr[u] & 0xffffu;
                    rel = s.state[i] == 0 && s.state[k] != 2;
                }
                const unsigned bal = __ballot_sync(kFull, rel);
                uint32_t base = 0;
                if (lane == 0 && bal) base = atomicAdd(&s.npairs, (uint32_t)__popc(bal));
                base = __shfl_sync(kFull, base, 0);
                if (rel) {
                    const uint32_t q = base + __popc(bal & ((1u << lane) - 1u));
                    if (q < kGwPairSmem) s.u.pairs[q] = pr[u];
                }
            }
        }
        __syncthreads();
        return min(s.npairs, (uint32_t)kGwPairSmem);
    }
}

__global__ void __launch_bounds__(kBlock, 1) grid_sweep_kernel(const __grid_constant__ GwArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GwSmem& s = *reinterpret_cast<GwSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = lane_id();
    const uint32_t G = gridDim.x, lb = blockIdx.x;
    const Order& o = a.ord;
    const int n = o.n, d = a.d;
    for (int q = tid; q < (kMaxN + 1) * (kMaxN + 1); q += kBlock) {
        const int p = q / (kMaxN + 1), k = q % (kMaxN + 1);
        uint64_t r = (k <= p) ? 1u : 0u;
        for (int i = 1; i <= k && k <= p; ++i) r = r * (uint64_t)(p - k + i) / (uint64_t)i;
        s.C[p][k] = (uint32_t)r;
    }
    {
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
    const bool timing = lb == (a.timing_cta < G ? a.timing_cta : 0u) && tid == 0;
    if (timing) {
        for (int k = 0; k < 12; ++k) s.phase[k] = 0;
        s.tprev = clock64();
    }
    auto mark_phase = [&](int k) {
        if (timing) {
            const long long t = clock64();
            s.phase[k] += (unsigned long long)(t - s.tprev);
            s.tprev = t;
        }
    };
    if (lb == 0 && tid == 0) {
        gc_stats* st = a.stats;
        st->codewords = 0; st->candidates = 0; st->dense_tests = 0; st->executed_tests = 0;
        st->marks = 0; st->windows = 0; st->survivors = 0; st->status = 0; st->strategy = 0;
        for (int k = 0; k < 12; ++k) st->phase_cycles[k] = 0;
        st->pair_windows = 0; st->pair_fallbacks = 0;
    }
    // clear this CTA's share of the bitmap
    {
        const uint64_t words = ((1ull << n) + 31) / 32;
        const uint64_t per = (words + G - 1) / G;
        const uint64_t w0 = min((uint64_t)lb * per, words), w1 = min(w0 + per, words);
        for (uint64_t w = w0 + tid; w < w1; w += kBlock) a.bitmap[w] = 0u;
        if (a.cnt) {
            const uint64_t cw = (1ull << n) / 4 > 0 ? ((1ull << n) + 3) / 4 : 1;
            const uint64_t cper = (cw + G - 1) / G;
            const uint64_t c0 = min((uint64_t)lb * cper, cw), c1 = min(c0 + cper, cw);
            for (uint64_t w = c0 + tid; w < c1; w += kBlock) a.cnt[w] = 0u;
        }
    }
    uint32_t epoch = 0;
    bool ok = gw_sync(s, a, epoch);
    mark_phase(4);
    // bit k: the window entry tid + k * kBlock this thread gathers is one of
    // this CTA's rows (entries lb + r * G)
    uint32_t own = 0;
    for (uint32_t k = 0; k < (uint32_t)kGwPerThread; ++k) {
        const uint32_t e = tid + k * kBlock;
        if (e >= lb && (e - lb) % G == 0u) own |= 1u << k;
    }

    // ORs this CTA's share of the balls of ax[0..nacc) into the bitmap.  The
    // (ball word, codeword) pairs are taken ball-word-major, so the lanes of
    // a warp mark the same ball word around neighbouring codewords, which
    // lie close together in the bitmap: consecutive lex, Gray and grlex
    // codewords share their high bits, consecutive grevlex codewords their
    // low bits, so the grevlex bitmap is indexed by the bit-reversed vector
    // (a Hamming ball reversed is the ball around the reversed centre, and
    // weights do not change).  Only vectors after the codeword in the order
    // can still be candidates: lex and Gray skip the words wholly before it,
    // the graded orders mask the lighter vectors.  The ORs go out a few at a
    // time (mark_some) between the row tests, which keep the popcount pipe
    // busy while the atomics travel to L2.
    uint64_t my_marks = 0;
    uint64_t mq = 0, mq1 = 0;   // this thread's next pair and the share's end
    uint32_t mi = 0, mj = 0, mnacc = 0, mdi = 0, mdj = 0;
    auto mark_begin = [&](uint32_t nacc) {
        const uint32_t hl = a.hball_len;
        mnacc = nacc;
        mq = mq1 = 0;
        if (nacc == 0 || hl == 0) return;
        const uint64_t total = (uint64_t)nacc * hl;
        const uint64_t per = (total + G - 1) / G;
        const uint64_t q0 = min((uint64_t)lb * per, total);
        mq1 = min(q0 + per, total);
        mq = q0 + tid;
        mj = (uint32_t)(mq / nacc);
        mi = (uint32_t)(mq - (uint64_t)mj * nacc);
        mdj = kBlock / nacc;
        mdi = kBlock - mdj * nacc;
    };
    // this thread's ORs left
    auto mark_left = [&]() -> uint32_t {
        return mq < mq1 ? (uint32_t)((mq1 - mq + kBlock - 1) / kBlock) : 0u;
    };
    auto mark_some = [&](uint32_t count) {
        for (uint32_t k = 0; k < count && mq < mq1; ++k) {
            const uint32_t c = a.reversed ? reverse_n(s.ax[mi], n) : s.ax[mi];
            const uint32_t e = __ldg(a.hball + mj);
            const uint32_t cw = c >> 5, word = cw ^ (e >> 3);
            uint32_t mask = s.lowball[e & 7u][c & 31u];
            bool skip = false;
            if (a.probe) {
                // radius-(d-2) balls are witnesses for the probes, on either
                // side of the frontier: the whole ball is marked
            } else if (o.ord == kLex) {
                skip = word < cw;
                if (word == cw) mask &= ~((2u << (c & 31u)) - 1u);
            } else if (o.ord == kGray) {
                skip = gray_inverse(word) < gray_inverse(cw);
            } else if (o.ord == kGrlex || o.ord == kGrevlex) {
                const int below = __popc(c) - __popc(word);
                if (below > 0) mask &= ~s.lowlight[below < 7 ? below : 7];
            }
            if (!skip && mask) {
                atomicOr(a.bitmap + word, mask);
                ++my_marks;
            }
            mq += kBlock;
            mi += mdi;
            mj += mdj;
            if (mi >= mnacc) {
                mi -= mnacc;
                ++mj;
            }
        }
    };

    // d = 3: survivors' radius-1 balls in the byte counters, +1 (add) or -1.
    // Item q of m * (n + 1) is vector ys[q % m] with bit q / m flipped (bit n:
    // none), so consecutive lanes touch neighbouring survivors' balls.
    auto count_balls = [&](const uint32_t* ys, bool global_src, uint32_t m, bool add) {
        const uint32_t items = m * (uint32_t)(n + 1);
        for (uint32_t q = tid; q < items; q += kBlock) {
            const uint32_t j = q / m, i = q - j * m;
            uint32_t y = global_src ? ld_cg(ys + i) : ys[i];
            if (a.reversed) y = reverse_n(y, n);   // indexed like the bitmap
            const uint32_t v = (int)j < n ? y ^ (1u << j) : y;
            const uint32_t one = 1u << (8u * (v & 3u));
            if (add) atomicAdd(a.cnt + (v >> 2), one);
            else atomicSub(a.cnt + (v >> 2), one);
        }
    };
    uint32_t na_own = 0;   // this CTA's survivors in the current window

    uint64_t R0 = 0, K = 0, Kprev = 0;
    uint32_t W = a.wmin, nprev = 0;
    uint64_t my_tests = 0, dense = 0, windows = 0, surv_total = 0;
    uint64_t pair_windows = 0, fallbacks = 0, rounds_total = 0;
    // ax[0..nprev): the accepts of the previous window, in every CTA; this
    // CTA's share of them goes to the output
    auto emit_prev = [&]() {
        const uint32_t per = (nprev + G - 1) / G;
        const uint32_t i0 = min(lb * per, nprev), i1 = min(i0 + per, nprev);
        for (uint32_t i = i0 + tid; i < i1; i += kBlock) {
            const uint64_t pos = Kprev + i;
            if (pos < a.cap) a.out[pos] = s.ax[i];
        }
    };
    // dense-equivalent tests (statistics, CTA 0): an accept of rank R is
    // compared with every later candidate
    const bool count_dense = lb == 0 && !o.filter;
    uint32_t t = 0;
    for (; ok && R0 < o.N; ++t) {
        const int p = t & 1;
        const uint64_t span = min((uint64_t)W, o.N - R0);
        // ---- A: the previous window's output; this CTA's chunk, filtered by
        // the bitmap (complete up to window t-2)
        emit_prev();
        mark_phase(0);
        if (a.early) {
            // window t-1's balls, complete at this phase's barrier: the rows
            // of window t are probed against them in phase B
            mark_begin(nprev);
            mark_some(mark_left());
            mark_phase(2);
        }
        {
            const uint64_t chunk = (span + G - 1) / G;
            const uint64_t c0 = min(R0 + (uint64_t)lb * chunk, R0 + span);
            const uint64_t c1 = min(c0 + chunk, R0 + span);
            // thread tid takes the `per` consecutive ranks from c0 + tid * per
            // (per <= 4), so one scan puts its survivors in rank order.  In
            // the orders that list a weight class as k-subsets in numeric
            // order (grlex, lex with a weight; grevlex reversed and backwards)
            // the first rank is unranked and the next ones are stepped to
            // the next (grevlex: previous) integer of the same weight.
            const uint32_t len = (uint32_t)(c1 - c0);
            const uint32_t per = (len + kBlock - 1) / kBlock;
            const uint64_t rb = c0 + (uint64_t)tid * per;
            const bool graded = o.ord == kGrlex || o.ord == kGrevlex || (o.ord == kLex && o.w >= 0);
            const uint32_t nmask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
            uint32_t xs[4] = {0u, 0u, 0u, 0u};
            uint32_t candm = 0;
            {
                int k = 0;          // graded: weight class, index in it, subset
                uint64_t ci = 0;
                uint32_t y = 0;
                auto full = [&](uint64_t r) {
                    if (o.w >= 0) {
                        k = o.w;
                        ci = r;
                    } else {
                        k = 0;
                        while (k < n && o.cum[k + 1] <= r) ++k;
                        ci = r - o.cum[k];
                    }
                    const uint32_t m = o.ord == kGrevlex ? (uint32_t)(s.C[n][k] - 1u - ci) : (uint32_t)ci;
                    y = comb_unrank(s.C, n, k, m);
                };
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) {
                    const uint64_t r = rb + j;
                    if (j >= per || r >= c1) continue;
                    if (!graded) {
                        uint32_t x = 0;
                        if (unrank(o, s.C, r, x)) {
                            xs[j] = x;
                            candm |= 1u << j;
                        }
                        continue;
                    }
                    if (j == 0 || ci + 1 >= (uint64_t)s.C[n][k]) {
                        full(r);
                    } else {
                        ++ci;
                        if (o.ord == kGrevlex) {
                            // previous integer of weight k: the complement's
                            // next one of weight n - k, complemented
                            const uint32_t z = ~y & nmask;
                            const uint32_t low = z & (0u - z), ripple = z + low;
                            y = ~(ripple | (((z ^ ripple) >> 2) >> (__ffs(z) - 1))) & nmask;
                        } else {
                            // next integer of weight k (Gosper's rule)
                            const uint32_t low = y & (0u - y), ripple = y + low;
                            y = ripple | (((y ^ ripple) >> 2) >> (__ffs(y) - 1));
                        }
                    }
                    xs[j] = o.ord == kGrevlex ? reverse_n(y, n) : y;
                    candm |= 1u << j;
                }
            }
            const int nh = n > 5 ? n - 5 : 0;
            uint32_t keepm = 0;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                if (!((candm >> j) & 1u)) continue;
                const uint32_t x = xs[j];
                const uint32_t key = a.reversed ? reverse_n(x, n) : x;
                const uint32_t w0 = key >> 5, b = key & 31u;
                bool hit;
                if (!a.probe) {
                    hit = ((ld_cg(a.bitmap + w0) >> b) & 1u) != 0u;
                } else {
                    // covered iff a marked vector is within distance 1: in
                    // the word, or this bit of a word one high bit away
                    hit = (ld_cg(a.bitmap + w0) & s.lowball[1][b]) != 0u;
                    for (int j0 = 0; j0 < nh && !hit; j0 += kGwProbeBatch) {
                        uint32_t v[kGwProbeBatch];
#pragma unroll
                        for (int u = 0; u < kGwProbeBatch; ++u)
                            v[u] = j0 + u < nh ? ld_cg(a.bitmap + (w0 ^ (1u << (j0 + u)))) : 0u;
#pragma unroll
                        for (int u = 0; u < kGwProbeBatch; ++u) hit = hit || ((v[u] >> b) & 1u);
                    }
                }
                if (!hit) keepm |= 1u << j;
            }
            uint32_t na = 0;
            uint32_t pos = block_exclusive_scan(s.bs, (uint32_t)__popc(keepm), &na);
            const uint32_t off0 = (uint32_t)(rb - R0);
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j)
                if ((keepm >> j) & 1u) {
                    s.wx[pos] = xs[j];
                    s.woff[pos] = off0 + j;
                    ++pos;
                }
            __syncthreads();
            uint32_t* sx = a.seg_x + ((size_t)p * G + lb) * kGwChunk;
            uint32_t* so = a.seg_off + ((size_t)p * G + lb) * kGwChunk;
            if (a.cnt) {
                // this window's survivors into the counters (complete at
                // this phase's barrier; they come out after phase B's)
                count_balls(s.wx, false, na, true);
                na_own = na;
            }
            for (uint32_t i = tid; i < na; i += kBlock) {
                sx[i] = s.wx[i];
                so[i] = s.woff[i];
            }
            if (tid == 0) a.slot[(size_t)p * G + lb] = na;
        }
        mark_phase(1);
        ok = gw_sync(s, a, epoch);
        if (!ok) break;
        mark_phase(4);

        // ---- B: gather the window, test this CTA's rows
        // (every CTA has read the pair count of window t-1 before this
        // phase's barrier; window t+1 adds to it after the next one)
        if (lb == 0 && tid == 0) atomicExch(a.ctrl + 2 + (p ^ 1), 0u);
        uint32_t S = 0;
        {
            const uint32_t v = (uint32_t)tid < G ? ld_cg(a.slot + (size_t)p * G + tid) : 0u;
            const uint32_t ex = block_exclusive_scan(s.bs, v, &S);
            if ((uint32_t)tid < G) s.pref[tid] = ex;
            if (tid == 0) s.pref[G] = S;
            __syncthreads();
        }
        const uint32_t Suse = min(S, (uint32_t)kGwSurvCap);
        if (tid == 0) s.npairs = 0;
        // entry e of the window sits in the segment of the last CTA g with
        // pref[g] <= e (empty segments share their successor's prefix); a
        // thread gathers its entries four at a time
        {
            // segment address of entry e
            auto seg_at = [&](uint32_t e) -> uint32_t {
                uint32_t lo = 0, hi = G;
                while (hi - lo > 1u) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s.pref[mid] <= e) lo = mid;
                    else hi = mid;
                }
                return ((uint32_t)p * G + lo) * (uint32_t)kGwChunk + (e - s.pref[lo]);  // < 2 * grid * kGwChunk
            };
            // a thread's eight entries in two groups of four; the second
            // group's loads go out before the first group is stored
            uint32_t xa0 = 0, xa1 = 0, xa2 = 0, xa3 = 0, oa0 = 0, oa1 = 0, oa2 = 0, oa3 = 0;
            uint32_t xb0 = 0, xb1 = 0, xb2 = 0, xb3 = 0, ob0 = 0, ob1 = 0, ob2 = 0, ob3 = 0;
#define GW_LOAD(k, X, O)                                           \
            if (tid + (k) * kBlock < Suse) {                       \
                const uint32_t at_ = seg_at(tid + (k) * kBlock);   \
                X = ld_cg(a.seg_x + at_);                          \
                O = ld_cg(a.seg_off + at_);                        \
            }
            GW_LOAD(0, xa0, oa0) GW_LOAD(1, xa1, oa1) GW_LOAD(2, xa2, oa2) GW_LOAD(3, xa3, oa3)
            GW_LOAD(4, xb0, ob0) GW_LOAD(5, xb1, ob1) GW_LOAD(6, xb2, ob2) GW_LOAD(7, xb3, ob3)
#undef GW_LOAD
#define GW_STORE(k, X, O)                                          \
            {                                                      \
                const uint32_t e_ = tid + (k) * kBlock;            \
                if (e_ < Suse) {                                   \
                    s.wx[e_] = X;                                  \
                    s.woff[e_] = O;                                \
                    if ((own >> (k)) & 1u) s.rx[(e_ - lb) / G] = X; \
                }                                                  \
            }
            GW_STORE(0, xa0, oa0) GW_STORE(1, xa1, oa1) GW_STORE(2, xa2, oa2) GW_STORE(3, xa3, oa3)
            GW_STORE(4, xb0, ob0) GW_STORE(5, xb1, ob1) GW_STORE(6, xb2, ob2) GW_STORE(7, xb3, ob3)
#undef GW_STORE
        }
        // this CTA's rows: entries lb + r * G, r < rows; s.flags[r] = killed
        const uint32_t rows = Suse > lb ? (Suse - lb + G - 1) / G : 0u;
        for (uint32_t r = tid; r < rows; r += kBlock) s.flags[r] = 0;
        __syncthreads();
        // a window over kGwSurvCap survivors ends after the last one taken
        const uint64_t Rnext = S > (uint32_t)kGwSurvCap ? R0 + s.woff[kGwSurvCap - 1] + 1 : R0 + span;
        mark_phase(5);
        {
            if (a.early) {
                // the bitmap holds every earlier window's balls: a row meets
                // a previous accept iff a marked vector is within distance 1
                // of it.  One warp per row, lane j < n - 5 probing the word
                // one high bit j away, lane 31 the row's own word.
                const int nh = n > 5 ? n - 5 : 0;
                for (uint32_t r = warp_id(); r < rows; r += kWarps) {
                    const uint32_t x = s.rx[r];
                    const uint32_t key = a.reversed ? reverse_n(x, n) : x;
                    const uint32_t w0 = key >> 5, b = key & 31u;
                    bool hit = false;
                    if (lane < nh) hit = ((ld_cg(a.bitmap + (w0 ^ (1u << lane))) >> b) & 1u) != 0u;
                    else if (lane == 31) hit = (ld_cg(a.bitmap + w0) & s.lowball[1][b]) != 0u;
                    hit = __any_sync(kFull, hit);
                    if (a.cnt && !hit) {
                        // d = 3: the counts over x's radius-1 ball add up
                        // to n + 1 (x's own ball) plus two for each other
                        // survivor of the window within distance 2 of x
                        uint32_t c = 0;
                        if (lane < n) {
                            const uint32_t v = key ^ (1u << lane);
                            c = (ld_cg(a.cnt + (v >> 2)) >> (8u * (v & 3u))) & 0xffu;
                        }
                        if (lane == 0) c += (ld_cg(a.cnt + (key >> 2)) >> (8u * (key & 3u))) & 0xffu;
                        c = __reduce_add_sync(kFull, c);
                        if (lane == 0) s.flags[r] = c > (uint32_t)(n + 1) ? 2 : 0;
                    } else if (lane == 0) {
                        s.flags[r] = hit ? 1 : 0;
                    }
                }
                mark_begin(0);
                if (a.cnt) __syncthreads();   // the tests below read the flags
                mark_phase(3);
            } else {
                // window t-1's marks, spread over the tests below: a slice
                // after each column of them, the rest at the end
                mark_begin(nprev);
            }
            const uint32_t mslice = (mark_left() + 7u) / 8u;
            const uint32_t* rx = s.rx;   // this CTA's rows, contiguous
            // the previous window's accepts against every row
            for (uint32_t c = tid; c < (a.early ? 0u : nprev); c += kBlock) {
                mark_some(mslice);
                const uint32_t y = s.ax[c];
                uint32_t r = 0;
                for (; r + 4 <= rows; r += 4) {
                    const uint4 q = *reinterpret_cast<const uint4*>(rx + r);
                    const int m0 = popc(q.x ^ y), m1 = popc(q.y ^ y);
                    const int m2 = popc(q.z ^ y), m3 = popc(q.w ^ y);
                    if (min(min(m0, m1), min(m2, m3)) < d) {
                        if (m0 < d) s.flags[r] = 1;
                        if (m1 < d) s.flags[r + 1] = 1;
                        if (m2 < d) s.flags[r + 2] = 1;
                        if (m3 < d) s.flags[r + 3] = 1;
                    }
                }
                for (; r < rows; ++r)
                    if (popc(rx[r] ^ y) < d) s.flags[r] = 1;
                my_tests += rows;
            }
            auto pair = [&](uint32_t k, uint32_t i) {
                const uint32_t e = atomicAdd(&s.npairs, 1u);
                if (e < kGwPairCap) s.u.pairs[e] = (k << 16) | i;
            };
            if (a.cnt) {
                // d = 3: only the rows that meet another survivor of the
                // window, a warp per row, against every earlier entry
                for (uint32_t r = warp_id(); r < rows; r += kWarps) {
                    if (s.flags[r] != 2) continue;
                    const uint32_t i = lb + r * G, x = rx[r];
                    for (uint32_t k0 = 0; k0 < i; k0 += 128u) {
                        const uint32_t k = k0 + 4u * (uint32_t)lane;
                        const uint4 q = *reinterpret_cast<const uint4*>(s.wx + k);
                        int m0 = popc(q.x ^ x), m1 = popc(q.y ^ x);
                        int m2 = popc(q.z ^ x), m3 = popc(q.w ^ x);
                        if (k0 + 128u > i) {   // entries from i on
                            if (k >= i) m0 = 32;
                            if (k + 1u >= i) m1 = 32;
                            if (k + 2u >= i) m2 = 32;
                            if (k + 3u >= i) m3 = 32;
                        }
                        if (min(min(m0, m1), min(m2, m3)) < d) {
                            if (m0 < d) pair(k, i);
                            if (m1 < d) pair(k + 1u, i);
                            if (m2 < d) pair(k + 2u, i);
                            if (m3 < d) pair(k + 3u, i);
                        }
                    }
                    if (lane == 0) my_tests += i;
                }
            } else if (a.early) {
                // the window's entries against the later rows: pairs (k, i),
                // k < i.  Row r (entry i_r = lb + r * G) meets the i_r entries
                // before it; the (row, entry) triangle, flattened row by row
                // (tri(r) tests before row r), is cut into one equal span per
                // warp, whose lanes sweep consecutive entries, four to a
                // 16-byte load, against the row word held by the whole warp.
                auto tri = [&](uint32_t r) { return r * lb + G * (r * (r - 1u) / 2u); };
                const uint32_t T = tri(rows), w = warp_id();
                const uint32_t p0 = (uint32_t)((uint64_t)T * w / kWarps);
                const uint32_t p1 = (uint32_t)((uint64_t)T * (w + 1u) / kWarps);
                if (p0 < p1) {
                    uint32_t lo = 0, hi = rows;   // tri(lo) <= p0 < tri(hi)
                    while (hi - lo > 1u) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (tri(mid) <= p0) lo = mid;
                        else hi = mid;
                    }
                    uint32_t r = lo, pos = p0;
                    while (pos < p1) {
                        const uint32_t i = lb + r * G, x = rx[r];
                        const uint32_t ka = pos - tri(r);
                        const uint32_t kb = min(i, ka + (p1 - pos));
                        for (uint32_t k0 = ka & ~127u; k0 < kb; k0 += 128u) {
                            const uint32_t k = k0 + 4u * (uint32_t)lane;
                            const uint4 q = *reinterpret_cast<const uint4*>(s.wx + k);
                            int m0 = popc(q.x ^ x), m1 = popc(q.y ^ x);
                            int m2 = popc(q.z ^ x), m3 = popc(q.w ^ x);
                            if (k0 < ka || k0 + 128u > kb) {   // entries outside [ka, kb)
                                if (k < ka || k >= kb) m0 = 32;
                                if (k + 1u < ka || k + 1u >= kb) m1 = 32;
                                if (k + 2u < ka || k + 2u >= kb) m2 = 32;
                                if (k + 3u < ka || k + 3u >= kb) m3 = 32;
                            }
                            if (min(min(m0, m1), min(m2, m3)) < d) {
                                if (m0 < d) pair(k, i);
                                if (m1 < d) pair(k + 1u, i);
                                if (m2 < d) pair(k + 2u, i);
                                if (m3 < d) pair(k + 3u, i);
                            }
                        }
                        if (lane == 0) my_tests += kb - ka;
                        pos += kb - ka;
                        ++r;
                    }
                }
            } else {
                // the window's entries against the later rows, a thread per
                // entry (column) with window t-1's marks between them.  Entry
                // k meets the rows after it, so a thread takes columns from
                // both ends of each pair of kBlock-column blocks (tid, 2047 -
                // tid, 2048 + tid, 4095 - tid, ...) and every thread has about
                // the same tests.
#pragma unroll 1
                for (uint32_t m = 0; m < (uint32_t)kGwSurvCap / kBlock; ++m) {
                    const uint32_t k = (m & 1u) ? kBlock * (m + 1u) - 1u - tid : kBlock * m + tid;
                    mark_some(mslice);
                    if (k >= Suse) continue;
                    const uint32_t y = s.wx[k];
                    const uint32_t r0 = k < lb ? 0u : (k - lb) / G + 1u;
                    uint32_t r = r0;
                    for (; r < rows && (r & 3u); ++r)
                        if (popc(rx[r] ^ y) < d) pair(k, lb + r * G);
                    for (; r + 4 <= rows; r += 4) {
                        const uint4 q = *reinterpret_cast<const uint4*>(rx + r);
                        const int m0 = popc(q.x ^ y), m1 = popc(q.y ^ y);
                        const int m2 = popc(q.z ^ y), m3 = popc(q.w ^ y);
                        if (min(min(m0, m1), min(m2, m3)) < d) {
                            if (m0 < d) pair(k, lb + r * G);
                            if (m1 < d) pair(k, lb + (r + 1) * G);
                            if (m2 < d) pair(k, lb + (r + 2) * G);
                            if (m3 < d) pair(k, lb + (r + 3) * G);
                        }
                    }
                    for (; r < rows; ++r)
                        if (popc(rx[r] ^ y) < d) pair(k, lb + r * G);
                    if (rows > r0) my_tests += rows - r0;
                }
            }
            mark_some(mark_left());
            __syncthreads();
            mark_phase(6);
            // publish: the kills, and the pairs whose later entry survived
            for (uint32_t r = tid; r < rows; r += kBlock) a.killbuf[lb + r * G] = s.flags[r] == 1 ? 1 : 0;
            const uint32_t np = s.npairs;
            uint32_t kept = 0;
            if (np <= kGwPairCap) {
                // the pairs whose later entry survived go to the window's
                // list, at an offset reserved on its counter (the pairs'
                // order does not matter, their count does)
                uint32_t pr[4];
                uint32_t km = 0;   // bit u: pair tid + u * kBlock is kept
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    const uint32_t e = tid + u * kBlock;
                    pr[u] = e < np ? s.u.pairs[e] : 0u;
                    if (e < np && s.flags[((pr[u] & 0xffffu) - lb) / G] != 1) km |= 1u << u;
                }
                uint32_t pos = block_exclusive_scan(s.bs, (uint32_t)__popc(km), &kept);
                if (tid == 0 && kept) s.bs.bcast64 = atomicAdd(a.ctrl + 2 + p, kept);
                __syncthreads();
                if (km) {
                    const uint32_t base = (uint32_t)s.bs.bcast64;
#pragma unroll
                    for (uint32_t u = 0; u < 4; ++u)
                        if ((km >> u) & 1u) a.pairbuf[base + pos++] = pr[u];
                }
            }
            if (tid == 0) a.pslot[(size_t)p * G + lb] = np <= kGwPairCap ? kept : kGwPairCap + 1u;
        }
        mark_phase(7);
        ok = gw_sync(s, a, epoch);
        if (!ok) break;
        mark_phase(4);

        // ---- every CTA decides the window from the same data
        if (a.cnt) {
            // every CTA has probed its rows: this CTA's survivors come out
            // of the counters, drained while the window is decided
            count_balls(a.seg_x + ((size_t)p * G + lb) * kGwChunk, true, na_own, false);
        }
        const uint32_t v = (uint32_t)tid < G ? ld_cg(a.pslot + (size_t)p * G + tid) : 0u;
        // kGwPerThread (8) consecutive entries per thread: their kill bytes in
        // two 4-byte loads, their states in one 8-byte store (consecutive
        // threads 8 entries apart would otherwise meet in the same banks)
        const uint32_t e0 = (uint32_t)kGwPerThread * tid;
        uint32_t keepm = 0;   // bit k: entry e0 + k exists and no accept rejected it
        {
            uint32_t kw[2];
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const uint32_t q = 4u * h;
                kw[h] = 0;
                if (e0 + q + 4 <= Suse) {
                    kw[h] = __ldcg(reinterpret_cast<const unsigned*>(a.killbuf + e0 + q));
                } else {
                    for (uint32_t k = 0; e0 + q + k < Suse && k < 4; ++k)
                        kw[h] |= (uint32_t)__ldcg(a.killbuf + e0 + q + k) << (8 * k);
                }
            }
            uint32_t st[2] = {0u, 0u};
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                if (e0 + k >= Suse) continue;
                const bool killed = ((kw[k >> 2] >> (8 * (k & 3u))) & 0xffu) != 0u;
                if (killed) st[k >> 2] |= 2u << (8 * (k & 3u));
                else keepm |= 1u << k;
            }
            *reinterpret_cast<uint2*>(s.state + e0) = make_uint2(st[0], st[1]);
        }
        const uint32_t P = ld_cg(a.ctrl + 2 + p);
        // a CTA's list overflowed, or the window's is too long for rounds
        // over L2: the conflict matrices
        const bool over = __syncthreads_or((uint32_t)tid < G && v > kGwPairCap) ||
                          P > kGwPairGlobal;
        uint32_t nacc = 0;
        if (!over && P == 0u) {
            // no conflict inside the window: the entries no previous accept
            // rejected are the accepts
            uint32_t pos = block_exclusive_scan(s.bs, __popc(keepm), &nacc);
            if (keepm) {
                const uint4 x0 = *reinterpret_cast<const uint4*>(s.wx + e0);
                const uint4 x1 = *reinterpret_cast<const uint4*>(s.wx + e0 + 4);
                const uint4 f0 = *reinterpret_cast<const uint4*>(s.woff + e0);
                const uint4 f1 = *reinterpret_cast<const uint4*>(s.woff + e0 + 4);
                const uint32_t xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const uint32_t fs[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
                uint32_t osum = 0;   // offsets of this thread's accepts (< 8 * 2^20)
#pragma unroll
                for (uint32_t k = 0; k < 8; ++k)
                    if ((keepm >> k) & 1u) {
                        s.ax[pos++] = xs[k];
                        osum += fs[k];
                    }
                if (count_dense) dense += (uint64_t)__popc(keepm) * (o.N - 1 - R0) - osum;
            }
            __syncthreads();
        } else if (!over) {
            uint32_t Ps = P;
            if (P <= a.pair_smem) {
                for (uint32_t e = tid; e < P; e += kBlock) s.u.pairs[e] = ld_cg(a.pairbuf + e);
                __syncthreads();
            } else {
                // too many for shared memory: the first rounds from L2
                Ps = gw_pair_rounds_global(s, a.pairbuf, P, Suse, a.pair_smem, &rounds_total);
            }
            nacc = gw_pair_rounds(s, Suse, Ps, &rounds_total);
            if (count_dense)
                for (uint32_t i = tid; i < Suse; i += kBlock)
                    if (s.state[i] == 1) dense += o.N - 1 - R0 - s.woff[i];
            ++pair_windows;
            mark_phase(9);
        } else {
            // drop the entries a previous accept rejects, then the conflict
            // matrices; the accepts go straight to ax, their offsets after the
            // matrices in the pair area
            __syncthreads();
            const uint32_t m = block_compact(s.bs, s.wx, s.woff, s.state, Suse);
            uint64_t rt = 0;
            uint32_t* fb_off = &s.u.pairs[kResolveWords * kResolveBlock];
            nacc = block_resolve<false>(s.bs, s.wx, s.woff, s.flags, m, d, s.ax, fb_off,
                                        s.u.M, rt, nullptr, 384u);
            if (lb == 0) my_tests += rt;
            if (count_dense)
                for (uint32_t i = tid; i < nacc; i += kBlock) dense += o.N - 1 - R0 - fb_off[i];
            __syncthreads();
            ++fallbacks;
            mark_phase(10);
        }
        mark_phase(8);
        Kprev = K;
        K += nacc;
        nprev = nacc;
        ++windows;
        surv_total += Suse;
        // the next window aims at `target` survivors at the density this one
        // had (at most twice as long), fewer where the survivors conflict
        // densely: about a.pair_target pairs at this window's pair density
        {
            uint64_t tgt = a.target;
            const uint32_t Peff = over ? max(P, 4u * a.pair_target) : P;
            if (Peff > a.pair_target && Suse > 0) {
                const float f = sqrtf((float)a.pair_target / (float)Peff);
                const uint64_t t2 = (uint64_t)((float)Suse * f);
                if (t2 < tgt) tgt = t2 > 256u ? t2 : 256u;
            }
            const uint64_t used = Rnext - R0;
            const uint64_t grow = 2ull * (uint64_t)W;
            uint64_t want = Suse ? used * tgt / Suse : grow;
            if (want > grow) want = grow;
            if (want < (uint64_t)a.wmin) want = a.wmin;
            if (want > (uint64_t)a.wmax) want = a.wmax;
            W = (uint32_t)want;
        }
        R0 = Rnext;
    }
    // the last window's accepts go to the output
    if (ok) {
        emit_prev();
        mark_phase(0);
    }
    // statistics: warp-reduce, one atomic per warp
    uint64_t tt = my_tests, m = my_marks, dn = dense;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        tt += __shfl_down_sync(kFull, tt, off);
        m += __shfl_down_sync(kFull, m, off);
        dn += __shfl_down_sync(kFull, dn, off);
    }
    if (lane == 0) {
        if (tt) atomicAdd((unsigned long long*)&a.stats->executed_tests, (unsigned long long)tt);
        if (m) atomicAdd((unsigned long long*)&a.stats->marks, (unsigned long long)m);
        if (dn) atomicAdd((unsigned long long*)&a.stats->dense_tests, (unsigned long long)dn);
    }
    if (tid == 0 && lb == 0) {
        gc_stats* st = a.stats;
        st->codewords = K;
        st->candidates = o.N;
        st->windows = windows;
        st->survivors = surv_total;
        st->strategy = GC_STRATEGY_BITMAP_GRID;
        st->pair_windows = pair_windows;
        st->pair_fallbacks = fallbacks;
        if (!ok || ld_acquire_gpu(a.ctrl + 1) != 0u) atomicMax((int*)&st->status, (int)GC_ERR_TIMEOUT);
    }
    if (timing) {
        s.phase[11] = rounds_total;
        for (int k = 0; k < 12; ++k) a.stats->phase_cycles[k] = s.phase[k];
    }
}

// ------------------------------------------------------------------ host side
static size_t gw_align(size_t v) { return (v + 255) & ~(size_t)255; }

// The launch's forms, from the problem and the switches (the layout and the
// launch must agree): early marks for every d >= 2 unless GC_GRID_EARLY=0;
// with them, for d = 3, byte counters of the window's survivors so that only
// rows that meet another survivor are tested (GC_GRID_CONF=0: all rows).
static bool gw_early(const HostProblem& p) {
    if (p.d < 2) return false;
    const char* e = std::getenv("GC_GRID_EARLY");
    return !e || std::atoi(e) != 0;
}
static bool gw_counters(const HostProblem& p) {
    if (p.d != 3 || !gw_early(p)) return false;
    const char* e = std::getenv("GC_GRID_CONF");
    return !e || std::atoi(e) != 0;
}

bool grid_sweep_layout(const HostProblem& p, const gc_plan_t& plan, GridLayout* L,
                       std::string* why) {
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        *why = "cannot query the CUDA device";
        return false;
    }
    if (p.n > kMaxN || p.orth) {
        *why = "the grid bitmap sweep takes n <= 32 and no orthogonality constraint";
        return false;
    }
    if ((size_t)optin < sizeof(GwSmem)) {
        *why = "not enough shared memory per block for the grid bitmap sweep";
        return false;
    }
    if (high_ball_len(p.n, p.d) >= (1u << 24)) {
        *why = "ball table too large for the bitmap strategy";
        return false;
    }
    int grid = sms;
    if (plan.grid > 0) grid = std::min(grid, plan.grid);
    grid = std::max(1, std::min(grid, kGwMaxCtas));
    L->grid = grid;
    L->smem_bytes = sizeof(GwSmem);
    const size_t G = (size_t)grid;
    size_t off = 0;
    L->off_ctrl = off;    off += gw_align(256);
    L->off_slot = off;    off += gw_align(sizeof(uint32_t) * 2 * G);
    L->off_pslot = off;   off += gw_align(sizeof(uint32_t) * 2 * G);
    L->off_segx = off;    off += gw_align(sizeof(uint32_t) * 2 * G * kGwChunk);
    L->off_segoff = off;  off += gw_align(sizeof(uint32_t) * 2 * G * kGwChunk);
    L->off_pairs = off;   off += gw_align(sizeof(uint32_t) * G * kGwPairCap);
    L->off_kill = off;    off += gw_align(kGwSurvCap);
    L->off_hball = off;   off += gw_align(4 * high_ball_len(p.n, p.d));
    L->off_bitmap = off;  off += gw_align(((1ull << p.n) + 31) / 32 * 4);
    L->off_cnt = 0;
    if (gw_counters(p)) {
        L->off_cnt = off;
        off += gw_align(std::max<uint64_t>(4, 1ull << p.n));
    }
    L->total = off;
    const uint64_t wcap = (uint64_t)grid * kGwChunk;
    L->wmax = (uint32_t)std::min<uint64_t>(plan.window_max ? plan.window_max : wcap, wcap);
    L->wmin = std::max<uint32_t>(
        1, std::min<uint32_t>(plan.window_min ? plan.window_min : 256, L->wmax));
    L->target = plan.survivor_target ? plan.survivor_target
                                     : default_target(GC_STRATEGY_BITMAP_GRID, p);
    return true;
}

static bool gw_fault_wait() {
    const char* f = std::getenv("GC_FAULT");
    return f && std::strcmp(f, "wait") == 0;
}

static uint32_t gw_timing_cta() {
    const char* e = std::getenv("GC_TIMING_CTA");
    return e ? (uint32_t)std::atoi(e) : 0u;
}

int launch_grid_sweep(const HostProblem& p, const GridLayout& L, uint32_t* d_out,
                      uint64_t capacity, gc_stats* d_stats, void* workspace, cudaStream_t s,
                      std::string* why) {
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e;
    auto cuda_fail = [&](const char* what) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        return GC_ERR_CUDA;
    };
    if ((e = cudaMemsetAsync(ws + L.off_ctrl, 0, 256, s)) != cudaSuccess)
        return cuda_fail("control words");
    // default: early marks with radius-(d-2) balls and radius-1 probes.
    // GC_GRID_EARLY=0 marks during the row tests instead (radius d-2 for
    // d >= 4, d-1 below, unless GC_GRID_PROBE says otherwise)
    uint32_t probe = p.d >= 4 ? 1u : 0u;
    if (const char* e = std::getenv("GC_GRID_PROBE")) probe = std::atoi(e) != 0 && p.d >= 2 ? 1u : 0u;
    const uint32_t early = gw_early(p) ? 1u : 0u;
    if (early) probe = 1u;
    const int rad = p.d - 1 - (int)probe;
    const uint32_t hl = (uint32_t)high_ball_len(p.n, rad + 1);
    const int nh = p.n > 5 ? p.n - 5 : 0;
    int rc = launch_high_ball(nh, rad, reinterpret_cast<uint32_t*>(ws + L.off_hball), hl, s);
    if (rc) {
        *why = "ball table";
        return rc;
    }
    if ((e = cudaFuncSetAttribute(grid_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_bytes)) != cudaSuccess)
        return cuda_fail("shared memory attribute");
    const bool fault = gw_fault_wait();
    GwArgs a{};
    a.ord = order_of(p, p.filter, false);
    a.d = p.d;
    a.out = d_out;
    a.cap = capacity;
    a.stats = d_stats;
    a.hball = reinterpret_cast<const uint32_t*>(ws + L.off_hball);
    a.hball_len = hl;
    a.bitmap = reinterpret_cast<uint32_t*>(ws + L.off_bitmap);
    a.seg_x = reinterpret_cast<uint32_t*>(ws + L.off_segx);
    a.seg_off = reinterpret_cast<uint32_t*>(ws + L.off_segoff);
    a.slot = reinterpret_cast<uint32_t*>(ws + L.off_slot);
    a.pslot = reinterpret_cast<uint32_t*>(ws + L.off_pslot);
    a.pairbuf = reinterpret_cast<uint32_t*>(ws + L.off_pairs);
    a.killbuf = ws + L.off_kill;
    a.ctrl = reinterpret_cast<unsigned*>(ws + L.off_ctrl);
    a.wmin = L.wmin;
    a.wmax = L.wmax;
    a.target = L.target;
    a.timeout_cycles = fault ? 400000000ll : 20000000000ll;  // ~0.2 s / ~10 s at 2 GHz
    a.timing_cta = gw_timing_cta();
    a.extra_arrivals = fault ? 1u : 0u;
    a.reversed = p.ord == GC_ORDER_GREVLEX ? 1u : 0u;
    a.probe = probe;
    a.early = early;
    a.cnt = L.off_cnt ? reinterpret_cast<uint32_t*>(ws + L.off_cnt) : nullptr;
    // GC_GRID_PAIR_SMEM (tests): decide windows of more pairs through the
    // rounds over the global list
    a.pair_smem = kGwPairSmem;
    a.pair_target = kGwPairTargetDefault;
    if (const char* e = std::getenv("GC_GRID_PAIR_TARGET"))
        a.pair_target = (uint32_t)std::max(64, std::atoi(e));
    if (const char* e = std::getenv("GC_GRID_PAIR_SMEM"))
        a.pair_smem = (uint32_t)std::max(1, std::min((int)kGwPairSmem, std::atoi(e)));
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)grid_sweep_kernel, dim3(L.grid), dim3(kBlock),
                                    args, L.smem_bytes, s);
    if (e != cudaSuccess) return cuda_fail("grid sweep launch");
    return GC_OK;
}

}  // namespace gc
