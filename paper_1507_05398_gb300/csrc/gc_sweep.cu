// gc_sweep.cu -- the persistent windowed sweep: the whole ordered greedy
// construction of Section 3 in one cooperative launch.
//
// The rank space is cut into windows of W consecutive ranks.  For window t:
//  1. (all CTAs, in parallel) every candidate of the window is generated from
//     its rank (Section 4.2 orders, closed form) and tested against the code
//     committed before the window:
//       distance strategy: popcount(x ^ c) >= d against every codeword, most
//         recent first, in shared-memory tiles with warp-wide early exit
//         (Sections 4.1, 5.2);
//       bitmap strategy: one bit lookup in the exclusion bitmap, which holds
//         the radius-(d-1) balls of every codeword accepted two or more
//         windows ago, plus the distance test against the previous window's
//         accepts, whose balls are being marked meanwhile.
//     Survivors are written, in rank order, to a per-CTA segment.
//  2. one grid-wide barrier.
//  3. (every CTA, redundantly and identically) the survivors of the window are
//     gathered in rank order and resolved in order (block_resolve), which
//     reproduces the serial decisions; the accepts are appended to the code.
//     Every CTA keeps its own copy of the new accepts, so no second barrier is
//     needed before the next window.
// The window size adapts so that about `target` candidates survive step 1;
// if more than kSurvCap survive, the window is cut after the kSurvCap-th
// survivor and the next window starts right after it.
#include <cooperative_groups.h>

#include <algorithm>

#include "gc_block.cuh"
#include "gc_internal.h"

namespace gc {

constexpr int kChunk = 4096;    // candidates per CTA per window
constexpr int kSurvCap = 4096;  // survivors resolved per window
constexpr int kMaxGrid = 1024;  // survivor-count prefix is one block scan
enum : int { kStratDistance = 1, kStratBitmap = 2 };

struct SweepArgs {
    Order ord;
    int d;
    int strategy;
    uint32_t* out;
    uint64_t cap;
    gc_stats* stats;
    unsigned* bar;
    uint32_t* seg_cnt;   // [2][G]
    uint32_t* seg_x;     // [2][G][kChunk]
    uint32_t* seg_off;   // [2][G][kChunk]
    uint32_t* store;     // distance strategy: code beyond the shared cache
    uint64_t store_words;
    uint32_t* bitmap;    // bitmap strategy: 2^n bits, vector-indexed
    const uint32_t* hball;
    uint32_t hball_len;
    uint32_t wmin, wmax, target;
    uint32_t cache_words;
    long long timeout_cycles;
};

struct __align__(16) SweepSmem {
    uint32_t C[kMaxN + 1][kMaxN + 1];
    uint32_t pad0[3];
    uint32_t lowball[8][32];  // lowball[r][c]: bits y < 32 with popc(y ^ c) <= r
    __align__(16) uint32_t list_x[kChunk];
    __align__(16) uint32_t list_off[kChunk];
    __align__(16) uint32_t accA[kSurvCap];
    __align__(16) uint32_t accB[kSurvCap];
    __align__(16) uint32_t acc_off[kSurvCap];
    uint32_t M[kResolveBlock][kResolveWords];
    uint32_t pref[kMaxGrid + 1];
    uint8_t dead[kChunk];
    BlockScratch bs;
};

// Exclusive prefix over the CTA of one value per thread; total in *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(BlockScratch& bs, uint32_t v,
                                                         uint32_t* total) {
    const int lane = lane_id(), warp = warp_id();
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) bs.warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = bs.warp_sum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        bs.warp_sum[lane] = wi - w;
        if (lane == 31) bs.warp_sum[kWarps] = wi;
    }
    __syncthreads();
    const uint32_t ex = bs.warp_sum[warp] + incl - v;
    *total = bs.warp_sum[kWarps];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kBlock, 1) sweep_kernel(const __grid_constant__ SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    SweepSmem& s = *reinterpret_cast<SweepSmem*>(smem_raw);
    uint32_t* cache = reinterpret_cast<uint32_t*>(smem_raw + sizeof(SweepSmem));
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    const uint32_t G = gridDim.x, b = blockIdx.x;
    const Order& o = a.ord;
    const int d = a.d;
    const int n = o.n;

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
    }
    __syncthreads();
    const uint32_t(*C)[kMaxN + 1] = s.C;

    uint64_t R0 = 0, K = 0, Kprev = 0;
    uint32_t W = a.wmin;
    uint32_t* cur = s.accA;
    uint32_t* prev = s.accB;
    uint32_t nprev = 0;
    unsigned gen = 0;
    int par = 0;
    uint64_t my_tests = 0, my_marks = 0, dense = 0, resolve_tests = 0;
    uint64_t windows = 0, surv_total = 0;

    while (R0 < o.N) {
        const uint64_t span = min((uint64_t)W, o.N - R0);
        const uint64_t chunk = (span + G - 1) / G;
        const uint64_t c0 = min(R0 + (uint64_t)b * chunk, R0 + span);
        const uint64_t c1 = min(c0 + chunk, R0 + span);

        // bitmap strategy: this CTA's share of the previous window's ball marks
        if (a.strategy == kStratBitmap && nprev > 0) {
            const uint64_t total = (uint64_t)nprev * a.hball_len;
            const uint64_t per = (total + G - 1) / G;
            const uint64_t q0 = min((uint64_t)b * per, total), q1 = min(q0 + per, total);
            for (uint64_t q = q0 + tid; q < q1; q += kBlock) {
                const uint32_t i = (uint32_t)(q / a.hball_len);
                const uint32_t j = (uint32_t)(q - (uint64_t)i * a.hball_len);
                const uint32_t c = prev[i];
                const uint32_t e = __ldg(a.hball + j);
                const uint32_t cw = c >> 5, word = cw ^ (e >> 3);
                uint32_t mask = s.lowball[e & 7u][c & 31u];
                // only ranks after c matter; skip words wholly before it
                if (o.ord == kLex) {
                    if (word < cw) continue;
                    if (word == cw) mask &= ~((2u << (c & 31u)) - 1u);
                } else if (o.ord == kGray) {
                    if (gray_inverse(word) < gray_inverse(cw)) continue;
                }
                if (mask) {
                    atomicOr(a.bitmap + word, mask);
                    ++my_marks;
                }
            }
        }

        // candidates of this CTA's chunk, in rank order
        uint32_t na = 0;
        for (uint64_t t0 = c0; t0 < c1; t0 += kBlock) {
            const uint64_t r = t0 + tid;
            uint32_t x = 0;
            bool keep = false;
            if (r < c1) {
                keep = unrank(o, C, r, x);
                if (keep && a.strategy == kStratBitmap)
                    keep = !((ld_cg(a.bitmap + (x >> 5)) >> (x & 31u)) & 1u);
            }
            na = block_append(s.bs, keep, x, (uint32_t)(r - R0), s.list_x, s.list_off, na);
        }

        // test against the code committed before the window, most recent first
        if (d >= 2) {
            na = block_filter<false>(s.bs, s.list_x, s.list_off, s.dead, na, prev, 0, nprev, d,
                                     my_tests);
            if (a.strategy == kStratDistance) {
                const uint32_t cached = (uint32_t)min(Kprev, (uint64_t)a.cache_words);
                if (Kprev > a.cache_words)
                    na = block_filter<true>(s.bs, s.list_x, s.list_off, s.dead, na, a.store,
                                            a.cache_words, (uint32_t)Kprev, d, my_tests);
                na = block_filter<false>(s.bs, s.list_x, s.list_off, s.dead, na, cache, 0, cached,
                                         d, my_tests);
            }
        }

        // publish this CTA's survivors
        {
            uint32_t* sx = a.seg_x + ((size_t)par * G + b) * kChunk;
            uint32_t* so = a.seg_off + ((size_t)par * G + b) * kChunk;
            for (uint32_t i = tid; i < na; i += kBlock) {
                sx[i] = s.list_x[i];
                so[i] = s.list_off[i];
            }
            if (tid == 0) a.seg_cnt[par * G + b] = na;
        }
        if (!grid_sync(a.bar, G, gen, a.timeout_cycles, s.bs.flag_any)) break;

        // gather every CTA's survivors in CTA (= rank) order
        uint32_t S = 0;
        {
            const uint32_t v = (uint32_t)tid < G ? ld_cg(a.seg_cnt + par * G + tid) : 0u;
            const uint32_t ex = block_exclusive_scan(s.bs, v, &S);
            if ((uint32_t)tid < G) s.pref[tid] = ex;
            if (tid == 0) s.pref[G] = S;
        }
        __syncthreads();
        const uint32_t Suse = min(S, (uint32_t)kSurvCap);
        for (uint32_t g = warp; g < G; g += kWarps) {
            const uint32_t p0 = s.pref[g];
            if (p0 >= Suse) continue;
            const uint32_t cnt = min(s.pref[g + 1] - p0, Suse - p0);
            const uint32_t* gx = a.seg_x + ((size_t)par * G + g) * kChunk;
            const uint32_t* go = a.seg_off + ((size_t)par * G + g) * kChunk;
            for (uint32_t i = lane; i < cnt; i += 32) {
                s.list_x[p0 + i] = ld_cg(gx + i);
                s.list_off[p0 + i] = ld_cg(go + i);
            }
        }
        __syncthreads();
        const uint64_t Rnext = (S > (uint32_t)kSurvCap) ? R0 + s.list_off[kSurvCap - 1] + 1
                                                        : R0 + span;

        // resolve in order; identical in every CTA
        uint64_t rt = 0;
        const uint32_t nacc = block_resolve(s.bs, s.list_x, s.list_off, s.dead, Suse, d, cur,
                                            s.acc_off, s.M, rt);
        if (b == 0) resolve_tests += rt;

        // commit
        if (b == 0) {
            for (uint32_t i = tid; i < nacc; i += kBlock) {
                const uint64_t pos = K + i;
                if (pos < a.cap) a.out[pos] = cur[i];
                if (!o.filter) dense += o.N - 1 - (R0 + s.acc_off[i]);
            }
        }
        if (a.strategy == kStratDistance) {
            for (uint32_t i = tid; i < nacc; i += kBlock) {
                const uint64_t pos = K + i;
                if (b == 0 && pos < a.store_words) a.store[pos] = cur[i];
                if (pos < a.cache_words) cache[pos] = cur[i];
            }
        }
        ++windows;
        surv_total += Suse;
        if (S > 2u * a.target)
            W = max(W / 2u, a.wmin);
        else if (S < a.target / 2u)
            W = min(W * 2u, a.wmax);
        Kprev = K;
        K += nacc;
        uint32_t* t = cur;
        cur = prev;
        prev = t;
        nprev = nacc;
        R0 = Rnext;
        par ^= 1;
        __syncthreads();
    }

    // statistics: warp-reduce then one atomic per warp
    uint64_t t = my_tests + resolve_tests, m = my_marks, dn = dense;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        t += __shfl_down_sync(kFull, t, off);
        m += __shfl_down_sync(kFull, m, off);
        dn += __shfl_down_sync(kFull, dn, off);
    }
    if (lane == 0) {
        if (t) atomicAdd((unsigned long long*)&a.stats->executed_tests, (unsigned long long)t);
        if (m) atomicAdd((unsigned long long*)&a.stats->marks, (unsigned long long)m);
        if (dn) atomicAdd((unsigned long long*)&a.stats->dense_tests, (unsigned long long)dn);
    }
    if (tid == 0) {
        if (ld_acquire_gpu(&a.bar[2]) != 0u) atomicMax((int*)&a.stats->status, (int)GC_ERR_TIMEOUT);
        if (b == 0) {
            a.stats->codewords = K;
            a.stats->candidates = o.N;
            a.stats->windows = windows;
            a.stats->survivors = surv_total;
            a.stats->strategy = a.strategy;
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

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

bool sweep_layout(const HostProblem& p, const gc_plan_t& plan, SweepLayout* L, std::string* why) {
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        *why = "cannot query the CUDA device";
        return false;
    }
    int grid = plan.grid > 0 ? plan.grid : sms;
    if (grid > sms) grid = sms;  // one CTA per SM (the kernel needs most of an SM)
    if (grid > kMaxGrid) grid = kMaxGrid;
    L->grid = grid;
    const size_t base = sizeof(SweepSmem);
    if ((size_t)optin < base + 16) {
        *why = "not enough shared memory per block";
        return false;
    }
    uint32_t cache = 0;
    if (plan.strategy == GC_STRATEGY_DISTANCE) {
        uint64_t room = ((size_t)optin - base) / 4;
        cache = (uint32_t)std::min<uint64_t>(room & ~(uint64_t)31, p.bound);
        cache = (cache + 31) & ~31u;
        if ((size_t)cache * 4 + base > (size_t)optin) cache -= 32;
    }
    L->cache_words = cache;
    L->smem_bytes = base + (size_t)cache * 4;
    L->store_words = (plan.strategy == GC_STRATEGY_DISTANCE && p.bound > cache) ? p.bound : 0;
    if (L->store_words > 0xffffffffull) {
        *why = "code too large for the distance strategy";
        return false;
    }
    size_t off = 0;
    L->off_bar = off;     off += align_up(64);
    L->off_segcnt = off;  off += align_up(sizeof(uint32_t) * 2 * grid);
    L->off_segx = off;    off += align_up(sizeof(uint32_t) * 2 * (size_t)grid * kChunk);
    L->off_segoff = off;  off += align_up(sizeof(uint32_t) * 2 * (size_t)grid * kChunk);
    L->off_store = off;   off += align_up(sizeof(uint32_t) * L->store_words);
    L->off_bitmap = off;
    if (plan.strategy == GC_STRATEGY_BITMAP) {
        off += align_up(((1ull << p.n) + 31) / 32 * 4);
    }
    L->off_hball = off;
    if (plan.strategy == GC_STRATEGY_BITMAP) off += align_up(4 * high_ball_len(p.n, p.d));
    L->total = off;
    return true;
}

int launch_sweep(const HostProblem& p, const gc_plan_t& plan, const SweepLayout& L,
                 uint32_t* d_out, uint64_t capacity, gc_stats* d_stats, void* workspace,
                 cudaStream_t stream, std::string* why) {
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    SweepArgs a{};
    a.ord.n = p.n;
    a.ord.ord = p.ord;
    a.ord.w = p.w;
    a.ord.filter = p.filter;
    a.ord.N = p.N;
    {
        uint64_t c = 0;
        for (int k = 0; k <= kMaxN + 1; ++k) {
            a.ord.cum[k] = c;
            if (k <= p.n) c += binom64(p.n, k);
        }
    }
    a.d = p.d;
    a.strategy = plan.strategy == GC_STRATEGY_BITMAP ? kStratBitmap : kStratDistance;
    a.out = d_out;
    a.cap = capacity;
    a.stats = d_stats;
    a.bar = reinterpret_cast<unsigned*>(ws + L.off_bar);
    a.seg_cnt = reinterpret_cast<uint32_t*>(ws + L.off_segcnt);
    a.seg_x = reinterpret_cast<uint32_t*>(ws + L.off_segx);
    a.seg_off = reinterpret_cast<uint32_t*>(ws + L.off_segoff);
    a.store = reinterpret_cast<uint32_t*>(ws + L.off_store);
    a.store_words = L.store_words;
    a.bitmap = reinterpret_cast<uint32_t*>(ws + L.off_bitmap);
    a.hball = reinterpret_cast<const uint32_t*>(ws + L.off_hball);
    a.hball_len = (uint32_t)high_ball_len(p.n, p.d);
    a.target = plan.survivor_target ? plan.survivor_target : 256;
    const uint64_t wcap = (uint64_t)L.grid * kChunk;
    a.wmax = (uint32_t)std::min<uint64_t>(plan.window_max ? plan.window_max : wcap, wcap);
    a.wmin = std::max<uint32_t>(1, std::min<uint32_t>(plan.window_min ? plan.window_min : 256, a.wmax));
    a.cache_words = L.cache_words;
    a.timeout_cycles = 20000000000ll;  // ~10 s at 2 GHz

    cudaError_t e;
    if ((e = cudaMemsetAsync(ws + L.off_bar, 0, 64, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_stats, 0, sizeof(gc_stats), stream)) != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return GC_ERR_CUDA;
    }
    if (a.strategy == kStratBitmap) {
        const size_t bytes = ((1ull << p.n) + 31) / 32 * 4;
        if ((e = cudaMemsetAsync(a.bitmap, 0, bytes, stream)) != cudaSuccess) {
            *why = cudaGetErrorString(e);
            return GC_ERR_CUDA;
        }
        const int nh = p.n > 5 ? p.n - 5 : 0;
        const int rc = launch_high_ball(nh, p.d - 1, const_cast<uint32_t*>(a.hball), a.hball_len,
                                        stream);
        if (rc) {
            *why = "ball table";
            return rc;
        }
    }
    if ((e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_bytes)) != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return GC_ERR_CUDA;
    }
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)sweep_kernel, dim3(L.grid), dim3(kBlock), args,
                                    L.smem_bytes, stream);
    if (e != cudaSuccess) {
        *why = std::string("sweep launch: ") + cudaGetErrorString(e);
        return GC_ERR_CUDA;
    }
    return GC_OK;
}

}  // namespace gc
