// gc_block.cuh -- CTA-wide primitives of the sweep: order-preserving
// compaction, the tiled candidate-vs-codeword distance test, the in-order
// resolver, and the grid barrier.  All functions here are called by every
// thread of a CTA of kBlock threads (they contain __syncthreads).
#pragma once
#include <cstdint>

#include "gc_device.cuh"

namespace gc {

constexpr int kBlock = 1024;           // threads per CTA
constexpr int kWarps = kBlock / 32;
constexpr int kResolveBlock = 256;     // survivors resolved per conflict matrix
constexpr int kResolveWords = kResolveBlock / 32;

// Scratch every primitive below needs, placed in shared memory by the caller.
struct BlockScratch {
    uint32_t warp_sum[kWarps + 1];
    uint32_t und[kResolveWords];
    uint32_t accb[kResolveWords];
    uint32_t flag_any;
};

// ------------------------------------------------------------ compaction
// Appends the calling threads' (keep, vx, vo) items, in thread order, to
// x[base..), off[base..).  Returns the new base (uniform across the CTA).
__device__ __forceinline__ uint32_t block_append(BlockScratch& bs, bool keep, uint32_t vx,
                                                 uint32_t vo, uint32_t* x, uint32_t* off,
                                                 uint32_t base) {
    const int lane = lane_id(), warp = warp_id();
    unsigned bal = __ballot_sync(kFull, keep);
    uint32_t wpre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) bs.warp_sum[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        uint32_t v = bs.warp_sum[lane];
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        bs.warp_sum[lane] = incl - v;
        if (lane == 31) bs.warp_sum[kWarps] = incl;
    }
    __syncthreads();
    if (keep) {
        uint32_t pos = base + bs.warp_sum[warp] + wpre;
        x[pos] = vx;
        if (off) off[pos] = vo;
    }
    uint32_t total = bs.warp_sum[kWarps];
    __syncthreads();
    return base + total;
}

// Keeps the entries of x/off[0..n) whose dead flag is 0, in order, in place.
__device__ __forceinline__ uint32_t block_compact(BlockScratch& bs, uint32_t* x, uint32_t* off,
                                                  const uint8_t* dead, uint32_t n) {
    uint32_t base = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += kBlock) {
        uint32_t i = t0 + threadIdx.x;
        bool keep = i < n && !dead[i];
        uint32_t vx = keep ? x[i] : 0u, vo = (keep && off) ? off[i] : 0u;
        // every read of this tile happens before block_append's first barrier,
        // and an item never moves to a higher index, so in-place is safe
        base = block_append(bs, keep, vx, vo, x, off, base);
    }
    return base;
}

// ------------------------------------------------------------ distance test
// Marks dead[i] = 1 for every candidate xs[i] (i < na) within distance d-1
// of some codeword src[lo..hi).  Codewords are read most recent (highest
// index) first.  Warps take groups of 32 candidates; when there are fewer
// groups than warps the codeword range is split across warps as well, so the
// whole CTA stays busy on a short survivor list.  A warp leaves its range as
// soon as all its lanes are dead.  Returns the number of candidate-codeword
// tests this thread executed (for the statistics).
template <bool kGlobalSrc>
__device__ __forceinline__ uint64_t block_test(const uint32_t* xs, uint32_t na, uint8_t* dead,
                                               const uint32_t* src, uint32_t lo, uint32_t hi,
                                               int d) {
    uint64_t ntests = 0;
    if (na == 0 || hi <= lo) return 0;
    const int lane = lane_id(), warp = warp_id();
    const uint32_t ngroups = (na + 31) / 32;
    const uint32_t len = hi - lo;
    uint32_t splits = ngroups >= (uint32_t)kWarps ? 1u : (uint32_t)kWarps / ngroups;
    // no split shorter than 64 codewords
    const uint32_t max_splits = max(1u, (len + 63u) / 64u);
    if (splits > max_splits) splits = max_splits;
    // split length a multiple of 32 so every split but the first starts aligned
    const uint32_t per = (((len + splits - 1u) / splits) + 31u) & ~31u;
    const uint32_t items = ngroups * splits;
    for (uint32_t it = warp; it < items; it += kWarps) {
        const uint32_t g = it % ngroups, s = it / ngroups;
        const uint32_t i = g * 32 + lane;
        const bool have = i < na;
        const uint32_t x = have ? xs[i] : 0u;
        bool is_dead = !have || dead[i];
        const uint32_t slo = lo + s * per;
        if (slo >= hi) continue;
        const uint32_t shi = min(hi, slo + per);
        uint32_t j = shi;
        while (j > slo) {
            if (__all_sync(kFull, is_dead)) break;
            uint32_t jlo;
            if (!kGlobalSrc && (j & 31u) == 0u && j - slo >= 32u) {
                // 32 codewords as 8 broadcast 16-byte shared-memory loads
                jlo = j - 32u;
                const uint4* p4 = reinterpret_cast<const uint4*>(src + jlo);
#pragma unroll
                for (int q = 7; q >= 0; --q) {
                    const uint4 c = p4[q];
                    const bool hit = (__popc(x ^ c.w) < d) | (__popc(x ^ c.z) < d) |
                                     (__popc(x ^ c.y) < d) | (__popc(x ^ c.x) < d);
                    is_dead |= hit;
                }
            } else {
                // ragged part: down to the next multiple of 32 (or the end)
                jlo = (j & 31u) ? (j & ~31u) : j - 32u;
                if (jlo < slo || jlo > j) jlo = slo;
                for (uint32_t q = j; q > jlo; --q) {
                    const uint32_t c = kGlobalSrc ? ld_cg(src + q - 1) : src[q - 1];
                    is_dead |= (__popc(x ^ c) < d);
                }
            }
            if (have) ntests += j - jlo;
            j = jlo;
        }
        if (have && is_dead) dead[i] = 1;
    }
    return ntests;
}

// Runs block_test over src[lo..hi) (most recent first) in growing slices and
// compacts the survivors after each slice, so lanes are refilled with live
// candidates.  Returns the number of candidates left alive in x/off[0..).
template <bool kGlobalSrc>
__device__ __forceinline__ uint32_t block_filter(BlockScratch& bs, uint32_t* x, uint32_t* off,
                                                 uint8_t* dead, uint32_t na, const uint32_t* src,
                                                 uint32_t lo, uint32_t hi, int d,
                                                 uint64_t& ntests) {
    uint32_t top = hi;
    while (na > 0 && top > lo) {
        // aim for ~64 tests per thread per slice, at least 32 codewords
        uint32_t want = (uint32_t)((uint64_t)kBlock * 64u / na);
        want = max(32u, min(want, 8192u));
        want = (want + 31u) & ~31u;
        uint32_t slo = (top - lo > want) ? top - want : lo;
        // keep slice ends on 32-word boundaries for the vector loads
        if (slo > lo) slo &= ~31u;
        if (slo < lo) slo = lo;
        for (uint32_t i = threadIdx.x; i < na; i += kBlock) dead[i] = 0;
        __syncthreads();
        ntests += block_test<kGlobalSrc>(x, na, dead, src, slo, top, d);
        __syncthreads();
        na = block_compact(bs, x, off, dead, na);
        top = slo;
    }
    return na;
}

// ------------------------------------------------------------ resolver
// In-order resolution of a list of candidates that have all cleared every
// codeword committed before them: accept them exactly as the serial sweep
// would (Section 3).  Works on blocks of kResolveBlock candidates: inside a
// block a bit matrix M[i] holds the earlier block entries within distance
// d-1 of entry i, and rounds decide every entry whose earlier conflicting
// entries are all decided -- rejected if one of them was accepted, accepted
// if all were rejected.  The first undecided entry is always decided, so the
// rounds end; the accept/reject decisions match the serial order because
// each is taken only from final decisions of earlier entries.  The entries
// after the block are then tested against the block's new accepts and
// compacted.
//   x/off[0..n)   candidates in order (modified: compacted)
//   acc/acc_off   receives accepted vectors/offsets in order (capacity >= n)
//   M             kResolveBlock * kResolveWords words of shared memory
// Returns the number accepted.
__device__ __forceinline__ uint32_t block_resolve(BlockScratch& bs, uint32_t* x, uint32_t* off,
                                                  uint8_t* dead, uint32_t n, int d,
                                                  uint32_t* acc, uint32_t* acc_off,
                                                  uint32_t (*M)[kResolveWords],
                                                  uint64_t& ntests) {
    const int lane = lane_id(), warp = warp_id();
    uint32_t nacc = 0;
    if (d <= 1) {  // nothing conflicts: every candidate is accepted
        for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
            acc[i] = x[i];
            if (acc_off) acc_off[i] = off[i];
        }
        __syncthreads();
        return n;
    }
    uint32_t start = 0, end = n;
    while (start < end) {
        const uint32_t P = min((uint32_t)kResolveBlock, end - start);
        const uint32_t* bx = x + start;
        // conflict matrix, lower triangle
        for (uint32_t q = threadIdx.x; q < P * kResolveWords; q += kBlock) {
            const uint32_t i = q / kResolveWords, wd = q % kResolveWords;
            const uint32_t jb = wd * 32u;
            uint32_t bits = 0;
            if (jb < i) {
                const uint32_t xi = bx[i];
                const uint32_t jn = min(32u, i - jb);
                for (uint32_t jj = 0; jj < jn; ++jj)
                    bits |= (uint32_t)(__popc(xi ^ bx[jb + jj]) < d) << jj;
                ntests += jn;
            }
            M[i][wd] = bits;
        }
        if (threadIdx.x < kResolveWords) {
            const uint32_t wb = threadIdx.x * 32u;
            bs.und[threadIdx.x] = (wb >= P) ? 0u : (P - wb >= 32u ? kFull : ((1u << (P - wb)) - 1u));
            bs.accb[threadIdx.x] = 0u;
        }
        __syncthreads();
        const uint32_t nwords = (P + 31u) / 32u;
        for (;;) {
            unsigned ba = 0, br = 0;
            if ((uint32_t)warp < nwords) {
                const uint32_t i = warp * 32u + lane;
                const bool u = (bs.und[warp] >> lane) & 1u;
                bool a_now = false, r_now = false;
                if (u) {
                    bool killed = false, blocked = false;
                    for (uint32_t wd = 0; wd <= (uint32_t)warp; ++wd) {
                        const uint32_t m = M[i][wd];
                        killed |= (m & bs.accb[wd]) != 0u;
                        blocked |= (m & bs.und[wd]) != 0u;
                    }
                    r_now = killed;
                    a_now = !killed && !blocked;
                }
                ba = __ballot_sync(kFull, a_now);
                br = __ballot_sync(kFull, r_now);
            }
            __syncthreads();
            if (lane == 0 && (uint32_t)warp < nwords) {
                bs.accb[warp] |= ba;
                bs.und[warp] &= ~(ba | br);
            }
            __syncthreads();
            bool left = false;
            for (uint32_t wd = 0; wd < nwords; ++wd) left |= bs.und[wd] != 0u;
            if (!left) break;
        }
        // append the block's accepts in order
        const uint32_t nacc0 = nacc;
        for (uint32_t t0 = 0; t0 < P; t0 += kBlock) {
            const uint32_t i = t0 + threadIdx.x;
            const bool keep = i < P && ((bs.accb[i >> 5] >> (i & 31)) & 1u);
            nacc = block_append(bs, keep, keep ? bx[i] : 0u,
                                (keep && acc_off) ? off[start + i] : 0u, acc, acc_off, nacc);
        }
        // the rest of the list against the new accepts
        const uint32_t rest = end - (start + P);
        if (rest > 0 && nacc > nacc0) {
            uint32_t* rx = x + start + P;
            uint32_t* ro = off ? off + start + P : nullptr;
            for (uint32_t i = threadIdx.x; i < rest; i += kBlock) dead[i] = 0;
            __syncthreads();
            ntests += block_test<false>(rx, rest, dead, acc, nacc0, nacc, d);
            __syncthreads();
            const uint32_t kept = block_compact(bs, rx, ro, dead, rest);
            end = start + P + kept;
        }
        start += P;
    }
    return nacc;
}

// ------------------------------------------------------------ grid barrier
// Sense-counting barrier over all CTAs of a cooperative launch.  bar[0] is
// the arrival count, bar[1] the generation, bar[2] the error word.  Every wait
// is bounded by timeout_cycles of clock64(); on expiry the error word is set
// to 1 and the CTA returns false (callers then leave the kernel).
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned nblocks, unsigned& gen,
                                          long long timeout_cycles, uint32_t& flag_any) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = gen;
        bool ok = true;
        const unsigned old = atom_add_acqrel_gpu(&bar[0], 1u);
        if (old == nblocks - 1u) {
            bar[0] = 0u;
            st_release_gpu(&bar[1], g + 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&bar[1]) == g) {
                if (ld_acquire_gpu(&bar[2]) != 0u) { ok = false; break; }
                if (clock64() - t0 > timeout_cycles) {
                    atomicExch(&bar[2], 1u);
                    ok = false;
                    break;
                }
            }
        }
        if (ok && ld_acquire_gpu(&bar[2]) != 0u) ok = false;
        gen = g + 1u;
        flag_any = ok ? 1u : 0u;
    }
    __syncthreads();
    const bool ok = flag_any != 0u;
    __syncthreads();
    return ok;
}

}  // namespace gc
