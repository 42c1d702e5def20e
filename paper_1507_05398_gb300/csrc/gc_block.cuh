// gc_block.cuh -- CTA-wide primitives of the sweep: order-preserving
// compaction, the candidate-vs-codeword distance test (warp-level scan and
// the CTA-wide 2-D tiling of it), and the in-order resolvers (blocked
// conflict matrices, a whole-window matrix, a list of conflicting pairs,
// bucketed conflict search).  Functions
// documented as CTA-wide are called by every thread of a CTA of kBlock
// threads (they contain __syncthreads).  Every primitive takes vectors of
// either width: W = uint32_t (n <= 32) or uint64_t (n <= 64).
#pragma once
#include <cstdint>

#include "gc_device.cuh"

namespace gc {

constexpr int kBlock = 1024;           // threads per CTA
constexpr int kWarps = kBlock / 32;
constexpr int kResolveBlock = 512;     // candidates per conflict matrix
constexpr int kResolveWords = kResolveBlock / 32;
// Whole-window conflict matrices (dense_build / dense_resolve): at most
// kDenseMaxRows entries, kDenseWords 32-bit words per row.
constexpr int kDenseMaxRows = 1536;
constexpr int kDenseWords = kDenseMaxRows / 32;

// Words of the strict lower triangle of the conflict matrix of P entries in
// the column-word layout of dense_build: column word w (bits for entries
// 32w..32w+31) is stored for rows 32w..P-1, so it takes P - 32w words.
__host__ __device__ constexpr uint32_t dense_tri_words(uint32_t P) {
    return ((P + 31u) / 32u) * P - 16u * ((P + 31u) / 32u) * ((P + 31u) / 32u - 1u);
}
constexpr uint32_t kDenseTriMax = dense_tri_words(kDenseMaxRows);
static_assert(kDenseTriMax % 4 == 0, "matrices are copied in 16-byte pieces");

// Scratch the primitives below need, placed in shared memory by the caller.
struct BlockScratch {
    uint32_t warp_sum[kWarps + 1];
    __align__(16) uint32_t und[kResolveWords];
    __align__(16) uint32_t accb[kResolveWords];
    uint32_t left[3];   // resolution rounds: "some entry still undecided"
    uint32_t flag_any;
    uint32_t bcast[2];           // values thread 0 hands to the CTA
    unsigned long long bcast64;
    uint32_t sp_masks[8];        // sparse resolver: bit blocks of the varying bits
    uint32_t sp_vary;            // sparse resolver: bits that vary over the list
    uint32_t sp_pairs;           // sparse resolver: pairs the buckets hold
    uint32_t sp_edges;           // sparse resolver: conflicts found
};

// ------------------------------------------------------------ compaction
// CTA-wide.  Appends the calling threads' (keep, vx, vo) items, in thread
// order, to x[base..) and off[base..).  Returns the new base (uniform).
template <typename W>
__device__ __forceinline__ uint32_t block_append(BlockScratch& bs, bool keep, W vx, uint32_t vo,
                                                 W* x, uint32_t* off, uint32_t base) {
    const int lane = lane_id(), warp = warp_id();
    const unsigned bal = __ballot_sync(kFull, keep);
    const uint32_t wpre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) bs.warp_sum[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < kWarps ? bs.warp_sum[lane] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < kWarps) bs.warp_sum[lane] = incl - v;
        if (lane == 31) bs.warp_sum[kWarps] = incl;
    }
    __syncthreads();
    if (keep) {
        const uint32_t pos = base + bs.warp_sum[warp] + wpre;
        x[pos] = vx;
        if (off) off[pos] = vo;
    }
    const uint32_t total = bs.warp_sum[kWarps];
    __syncthreads();
    return base + total;
}

// CTA-wide.  Exclusive prefix over the CTA of one value per thread; total
// in *total.  Ends with a barrier, so bs may be reused at once.
__device__ __forceinline__ uint32_t block_exclusive_scan(BlockScratch& bs, uint32_t v,
                                                         uint32_t* total) {
    const int lane = lane_id(), warp = warp_id();
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) bs.warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kWarps ? bs.warp_sum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kWarps) bs.warp_sum[lane] = wi - w;
        if (lane == 31) bs.warp_sum[kWarps] = wi;
    }
    __syncthreads();
    const uint32_t ex = bs.warp_sum[warp] + incl - v;
    *total = bs.warp_sum[kWarps];
    __syncthreads();
    return ex;
}

// CTA-wide.  Keeps the entries of x/off[0..n) whose dead flag is 0, in
// order, in place.
template <typename W>
__device__ __forceinline__ uint32_t block_compact(BlockScratch& bs, W* x, uint32_t* off,
                                                  const uint8_t* dead, uint32_t n) {
    uint32_t base = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += kBlock) {
        const uint32_t i = t0 + threadIdx.x;
        const bool keep = i < n && !dead[i];
        const W vx = keep ? x[i] : W(0);
        const uint32_t vo = (keep && off) ? off[i] : 0u;
        // every read of this tile happens before block_append's first barrier,
        // and an item never moves to a higher index, so in-place is safe
        base = block_append(bs, keep, vx, vo, x, off, base);
    }
    return base;
}

// ------------------------------------------------------------ distance test
// Warp-level.  Each lane holds one candidate x (is_dead already set for
// lanes without one); the warp scans src[lo..hi) from the highest index down
// (most recent codeword first) and sets is_dead for every lane within
// distance d-1 of a codeword.  The warp leaves as soon as all lanes are dead.
// When shared_dead is given it is re-read every 32 codewords so that other
// warps working on the same candidate can end this scan early.  Adds this
// lane's tests to nt.
template <bool kGlobalSrc, bool kOrth = false, typename W>
__device__ __forceinline__ bool warp_scan_desc(W x, bool is_dead, const W* src,
                                               uint32_t lo, uint32_t hi, int d,
                                               const volatile uint8_t* shared_dead, bool have,
                                               uint64_t& nt) {
    uint32_t j = hi;
    while (j > lo) {
        if (shared_dead) is_dead |= (*shared_dead != 0);
        if (__all_sync(kFull, is_dead)) break;
        uint32_t jlo;
        if ((j & 31u) == 0u && j - lo >= 32u) {
            // 32 codewords as 8 (narrow) or 16 (wide) broadcast 16-byte loads
            // (shared memory, or L2 for the global store: other SMs write it
            // during the kernel)
            jlo = j - 32u;
            const uint4* p4 = reinterpret_cast<const uint4*>(src + jlo);
            constexpr int kVecs = 32 * (int)sizeof(W) / 16;
#pragma unroll
            for (int q = kVecs - 1; q >= 0; --q) {
                const uint4 c = kGlobalSrc ? __ldcg(p4 + q) : p4[q];
                bool hit;
                if constexpr (sizeof(W) == 4) {
                    hit = (__popc(x ^ c.w) < d) | (__popc(x ^ c.z) < d) |
                          (__popc(x ^ c.y) < d) | (__popc(x ^ c.x) < d);
                    if (kOrth)  // Section 4.4: also a conflict if not orthogonal
                        hit |= ((__popc(x & c.w) | __popc(x & c.z) | __popc(x & c.y) |
                                 __popc(x & c.x)) & 1u) != 0u;
                } else {
                    const uint64_t c0 = ((uint64_t)c.y << 32) | c.x;
                    const uint64_t c1 = ((uint64_t)c.w << 32) | c.z;
                    hit = (__popcll(x ^ c1) < d) | (__popcll(x ^ c0) < d);
                    if (kOrth) hit |= ((__popcll(x & c1) | __popcll(x & c0)) & 1) != 0;
                }
                is_dead |= hit;
            }
        } else {
            // ragged part: down to the next multiple of 32 (or the end)
            jlo = (j & 31u) ? (j & ~31u) : j - 32u;
            if (jlo < lo || jlo > j) jlo = lo;
            for (uint32_t q = j; q > jlo; --q) {
                const W c = kGlobalSrc ? ld_cg(src + q - 1) : src[q - 1];
                is_dead |= (popc(x ^ c) < d);
                if (kOrth) is_dead |= (popc(x & c) & 1) != 0;
            }
        }
        if (have) nt += j - jlo;
        j = jlo;
    }
    return is_dead;
}

// No barriers; called by every warp of the CTA.  Marks dead[i] = 1 for every
// candidate xs[i] (i < na) within distance d-1 of some codeword src[lo..hi).
// Warps take groups of 32 candidates; when there are fewer groups than warps
// the codeword range is split across warps as well (most recent slice to the
// lowest warps), so a short list of hard candidates still keeps the whole CTA
// busy.  Callers clear dead[] before and synchronise after.
template <bool kGlobalSrc, bool kOrth = false, typename W>
__device__ __forceinline__ void block_test(const W* xs, uint32_t na, uint8_t* dead, const W* src,
                                           uint32_t lo, uint32_t hi, int d, uint64_t& nt) {
    if (na == 0 || hi <= lo) return;
    const int lane = lane_id(), warp = warp_id();
    const uint32_t ngroups = (na + 31) / 32;
    const uint32_t len = hi - lo;
    uint32_t splits = ngroups >= (uint32_t)kWarps ? 1u : (uint32_t)kWarps / ngroups;
    const uint32_t max_splits = max(1u, (len + 63u) / 64u);  // no split under 64 words
    if (splits > max_splits) splits = max_splits;
    const uint32_t per = (((len + splits - 1u) / splits) + 31u) & ~31u;
    const uint32_t items = ngroups * splits;
    for (uint32_t it = warp; it < items; it += kWarps) {
        const uint32_t g = it % ngroups, s = it / ngroups;
        const uint32_t i = g * 32 + lane;
        const bool have = i < na;
        const W x = have ? xs[i] : W(0);
        const bool was_dead = !have || dead[i];
        const uint32_t top = (uint64_t)s * per >= len ? lo : hi - s * per;
        const uint32_t bot = (top - lo > per) ? top - per : lo;
        if (top <= bot) continue;
        const bool now_dead = warp_scan_desc<kGlobalSrc, kOrth>(
            x, was_dead, src, bot, top, d,
            (have && splits > 1) ? (const volatile uint8_t*)(dead + i) : nullptr, have, nt);
        if (have && now_dead && !was_dead) dead[i] = 1;
    }
}

// CTA-wide.  Tests x[0..na) against src[lo..hi) (block_test) and keeps the
// candidates that clear it, in order, in place.  Returns how many are left.
template <bool kGlobalSrc, typename W>
__device__ __forceinline__ uint32_t block_filter(BlockScratch& bs, W* x, uint32_t* off,
                                                 uint8_t* dead, uint32_t na, const W* src,
                                                 uint32_t lo, uint32_t hi, int d, uint64_t& nt) {
    if (na == 0 || hi <= lo) return na;
    for (uint32_t i = threadIdx.x; i < na; i += kBlock) dead[i] = 0;
    __syncthreads();
    block_test<kGlobalSrc>(x, na, dead, src, lo, hi, d, nt);
    __syncthreads();
    return block_compact(bs, x, off, dead, na);
}

// ------------------------------------------------------------ resolver
// CTA-wide.  In-order resolution of a list of candidates that have all
// cleared every codeword committed before them: accept them exactly as the
// serial sweep would (Section 4).  Works on blocks of kResolveBlock
// candidates: inside a block a bit matrix row i holds the earlier block
// entries within distance d-1 of entry i, and rounds decide every entry whose
// earlier conflicting entries are all decided -- rejected if one of them was
// accepted, accepted if all were rejected.  The first undecided entry is
// always decided, so the rounds end, and every decision is taken from final
// decisions of earlier entries, so it is the serial one.  The entries after
// the block are then tested against the block's accepts and compacted.
//   x/off[0..n)   candidates in order (modified: compacted)
//   acc/acc_off   receives accepted vectors/offsets in order after the
//                 first acc_start entries, which it leaves as they are
//                 (capacity >= acc_start + n; acc 16-byte aligned: the kill
//                 step reads it with 16-byte loads)
//   Mt            kResolveWords x kResolveBlock words of shared memory
// block (<= kResolveBlock) sets how many entries one conflict matrix takes.
// Returns acc_start + the number accepted.
// tim (optional, thread 0 only): cycles added to tim[0] matrix build,
// tim[1] rounds, tim[2] append and kill step; tim[3] counts rounds.
template <bool kOrth = false, typename W>
__device__ __forceinline__ uint32_t block_resolve(BlockScratch& bs, W* x, uint32_t* off,
                                                  uint8_t* dead, uint32_t n, int d,
                                                  W* acc, uint32_t* acc_off,
                                                  uint32_t (*Mt)[kResolveBlock], uint64_t& nt,
                                                  unsigned long long* tim = nullptr,
                                                  uint32_t block = kResolveBlock,
                                                  uint32_t acc_start = 0) {
    constexpr bool orth = kOrth;
    const int lane = lane_id(), warp = warp_id();
    const bool timing = tim && threadIdx.x == 0;
    long long t_last = timing ? clock64() : 0;
    auto tick = [&](int k) {
        if (timing) {
            const long long t = clock64();
            tim[k] += (unsigned long long)(t - t_last);
            t_last = t;
        }
    };
    if (d <= 1 && !orth) {  // nothing conflicts: every candidate is accepted
        for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
            acc[acc_start + i] = x[i];
            if (acc_off) acc_off[acc_start + i] = off[i];
        }
        __syncthreads();
        return acc_start + n;
    }
    uint32_t nacc = acc_start;
    uint32_t start = 0, end = n;
    while (start < end) {
        const uint32_t P = min(block, end - start);
        const uint32_t nwords = (P + 31u) / 32u;
        const W* bx = x + start;
        // conflict matrix, strictly lower triangle, stored transposed
        // (Mt[word][row]) so both the build and the rounds read consecutive
        // shared-memory words across a warp: a warp owns a row, lane = column
        // within a 32-column word, and the word is the warp's ballot.  Words
        // right of the diagonal are never read, so they are not built.
        // four rows per warp share each column load
        for (uint32_t i0 = warp * 4u; i0 < P; i0 += kWarps * 4u) {
            const uint32_t nr = min(4u, P - i0);
            const W x0 = bx[i0];
            const W x1 = nr > 1 ? bx[i0 + 1] : W(0);
            const W x2 = nr > 2 ? bx[i0 + 2] : W(0);
            const W x3 = nr > 3 ? bx[i0 + 3] : W(0);
            const uint32_t last = (i0 + nr - 1) >> 5;  // word holding the last row's diagonal
            for (uint32_t wd = 0; wd <= last; ++wd) {
                const uint32_t j = (wd << 5) + lane;
                const W c = bx[j < P ? j : 0];
                const unsigned b0 = __ballot_sync(
                    kFull, j < i0 && ((popc(x0 ^ c) < d) || (orth && (popc(x0 & c) & 1))));
                const unsigned b1 = __ballot_sync(
                    kFull, j < i0 + 1 && ((popc(x1 ^ c) < d) || (orth && (popc(x1 & c) & 1))));
                const unsigned b2 = __ballot_sync(
                    kFull, j < i0 + 2 && ((popc(x2 ^ c) < d) || (orth && (popc(x2 & c) & 1))));
                const unsigned b3 = __ballot_sync(
                    kFull, j < i0 + 3 && ((popc(x3 ^ c) < d) || (orth && (popc(x3 & c) & 1))));
                if (lane == 0) {
                    Mt[wd][i0] = b0;
                    if (nr > 1) Mt[wd][i0 + 1] = b1;
                    if (nr > 2) Mt[wd][i0 + 2] = b2;
                    if (nr > 3) Mt[wd][i0 + 3] = b3;
                }
            }
            if (lane == 0) nt += 4u * i0 + 6u;
        }
        if (threadIdx.x < (unsigned)kResolveWords) {
            const uint32_t wb = threadIdx.x * 32u;
            bs.und[threadIdx.x] = (wb >= P) ? 0u : (P - wb >= 32u ? kFull : ((1u << (P - wb)) - 1u));
            bs.accb[threadIdx.x] = 0u;
        }
        __syncthreads();
        tick(0);
        if (threadIdx.x < 3) bs.left[threadIdx.x] = 0u;
        __syncthreads();
        // the rounds involve only the warps that own rows (barrier 1 over
        // them); the rest wait at the CTA barrier after the loop
        if ((uint32_t)warp < nwords) {
            const unsigned nthreads = nwords * 32u;
            for (uint32_t round = 0;; ++round) {
                if (timing) tim[3] += 1;
                // slot of this round's flag; the next round's slot is cleared
                // here: it was last read two rounds ago, and every thread of
                // the rounds has passed the previous round's first barrier
                const uint32_t slot = round % 3u, next = (round + 1u) % 3u;
                if (threadIdx.x == 0) bs.left[next] = 0u;
                unsigned ba = 0, br = 0;
                if (bs.und[warp] != 0u) {
                    const uint32_t i = warp * 32u + lane;
                    const bool u = (bs.und[warp] >> lane) & 1u;
                    bool a_now = false, r_now = false;
                    if (u) {
                        bool killed = false, blocked = false;
                        const uint4* acc4 = reinterpret_cast<const uint4*>(bs.accb);
                        const uint4* und4 = reinterpret_cast<const uint4*>(bs.und);
                        for (uint32_t w4 = 0; w4 * 4u <= (uint32_t)warp; ++w4) {
                            const uint4 av = acc4[w4], uv = und4[w4];
                            const uint32_t wb = w4 * 4u;
                            const uint32_t m0 = Mt[wb][i];
                            const uint32_t m1 = wb + 1 <= (uint32_t)warp ? Mt[wb + 1][i] : 0u;
                            const uint32_t m2 = wb + 2 <= (uint32_t)warp ? Mt[wb + 2][i] : 0u;
                            const uint32_t m3 = wb + 3 <= (uint32_t)warp ? Mt[wb + 3][i] : 0u;
                            killed |= ((m0 & av.x) | (m1 & av.y) | (m2 & av.z) | (m3 & av.w)) != 0u;
                            blocked |= ((m0 & uv.x) | (m1 & uv.y) | (m2 & uv.z) | (m3 & uv.w)) != 0u;
                        }
                        r_now = killed;
                        a_now = !killed && !blocked;
                    }
                    ba = __ballot_sync(kFull, a_now);
                    br = __ballot_sync(kFull, r_now);
                }
                named_barrier(1, nthreads);
                if (lane == 0) {
                    bs.accb[warp] |= ba;
                    const uint32_t und = bs.und[warp] & ~(ba | br);
                    bs.und[warp] = und;
                    if (und) bs.left[slot] = 1u;
                }
                named_barrier(1, nthreads);
                if (bs.left[slot] == 0u) break;
            }
        }
        __syncthreads();
        tick(1);
        // append the block's accepts in order
        const uint32_t nacc0 = nacc;
        for (uint32_t t0 = 0; t0 < P; t0 += kBlock) {
            const uint32_t i = t0 + threadIdx.x;
            const bool keep = i < P && ((bs.accb[i >> 5] >> (i & 31)) & 1u);
            nacc = block_append(bs, keep, keep ? bx[i] : W(0),
                                (keep && acc_off) ? off[start + i] : 0u, acc, acc_off, nacc);
        }
        // the rest of the list against the block's accepts
        const uint32_t rest = end - (start + P);
        if (rest > 0 && nacc > nacc0) {
            W* rx = x + start + P;
            uint32_t* ro = off ? off + start + P : nullptr;
            for (uint32_t i = threadIdx.x; i < rest; i += kBlock) dead[i] = 0;
            __syncthreads();
            block_test<false, kOrth>(rx, rest, dead, acc, nacc0, nacc, d, nt);
            __syncthreads();
            const uint32_t kept = block_compact(bs, rx, ro, dead, rest);
            end = start + P + kept;
        }
        start += P;
        tick(2);
    }
    return nacc;
}

// ------------------------------------------------------------ whole-window resolver
// Word w of row i of a conflict matrix in the column-word layout: with
// cb(w) = sum over v < w of (P - 32v), minus 32w, it is T[cb(w) + i] for
// i >= 32w.  cb(0) = 0 and cb(w + 1) = cb(w) + P - 32w - 32.

// No barriers; called by every warp of a CTA.  Builds rows of the strict
// lower triangle of the conflict matrix of x[0..P) (bit j of row i set iff
// j < i and the two entries are within distance d-1) into T in the layout
// above: the row quads q = q0, q0 + qstep, ... (rows 4q..4q+3), a quad per
// warp, whose four rows share each column load.  A quad never straddles a
// 32-row word.  Adds the tests to nt.
__device__ __forceinline__ void dense_build(const uint32_t* x, uint32_t P, int d, uint32_t* T,
                                            uint32_t q0, uint32_t qstep, uint64_t& nt) {
    const int lane = lane_id();
    for (uint32_t q = q0; 4u * q < P; q += qstep) {
        const uint32_t i0 = 4u * q, nr = min(4u, P - i0);
        const uint32_t x0 = x[i0];
        const uint32_t x1 = nr > 1 ? x[i0 + 1] : 0u;
        const uint32_t x2 = nr > 2 ? x[i0 + 2] : 0u;
        const uint32_t x3 = nr > 3 ? x[i0 + 3] : 0u;
        const uint32_t last = i0 >> 5;
        uint32_t cb = 0;
        for (uint32_t wd = 0; wd <= last; ++wd) {
            const uint32_t j = (wd << 5) + lane;
            const uint32_t c = x[j < P ? j : 0];
            const unsigned b0 = __ballot_sync(kFull, j < i0 && __popc(x0 ^ c) < d);
            const unsigned b1 = __ballot_sync(kFull, j < i0 + 1 && __popc(x1 ^ c) < d);
            const unsigned b2 = __ballot_sync(kFull, j < i0 + 2 && __popc(x2 ^ c) < d);
            const unsigned b3 = __ballot_sync(kFull, j < i0 + 3 && __popc(x3 ^ c) < d);
            const unsigned bw = lane == 0 ? b0 : lane == 1 ? b1 : lane == 2 ? b2 : b3;
            if ((uint32_t)lane < nr) T[cb + i0 + lane] = bw;
            cb += P - 32u * wd - 32u;
        }
        if (lane == 0) nt += 4u * i0 + 6u;
    }
}

// CTA-wide, narrow words.  Decides x[0..P) (P <= kDenseMaxRows) in order, as
// the serial greedy would (Section 4), from the whole strict lower triangle
// of its conflict matrix T (shared memory, the layout of dense_build).  The
// rounds are those of block_resolve over one block: an undecided entry with
// an accepted earlier conflict is rejected, one whose earlier conflicts are
// all rejected is accepted.  Bits on or above the diagonal are masked, so the
// first undecided entry always decides and the rounds end whatever T holds.
// Warp k owns the entries of words k and k + 32.  und/accb: kDenseWords words
// of shared memory, 16-byte aligned.  Accepted entries are appended in order to acc/acc_off.
// Returns how many.  tim as for pair_resolve.
__device__ __forceinline__ uint32_t dense_resolve(BlockScratch& bs, uint32_t* und, uint32_t* accb,
                                                  const uint32_t* x, const uint32_t* off,
                                                  uint32_t P, const uint32_t* T, uint32_t* acc,
                                                  uint32_t* acc_off,
                                                  unsigned long long* tim = nullptr) {
    const int lane = lane_id(), warp = warp_id();
    const bool timing = tim && threadIdx.x == 0;
    long long t_last = timing ? clock64() : 0;
    const uint32_t nw = (P + 31u) / 32u;
    for (uint32_t w = threadIdx.x; w < (uint32_t)kDenseWords; w += kBlock) {
        const uint32_t wb = w * 32u;
        und[w] = wb >= P ? 0u : (P - wb >= 32u ? kFull : ((1u << (P - wb)) - 1u));
        accb[w] = 0u;
    }
    if (threadIdx.x < 3) bs.left[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t owners = min(nw, (uint32_t)kWarps);
    if ((uint32_t)warp < owners) {
        const unsigned nthreads = owners * 32u;
        for (uint32_t round = 0;; ++round) {
            if (timing) tim[3] += 1;
            // this round's flag slot; the next one was last read two rounds ago
            const uint32_t slot = round % 3u, next = (round + 1u) % 3u;
            if (threadIdx.x == 0) bs.left[next] = 0u;
            unsigned ba[2] = {0u, 0u}, br[2] = {0u, 0u};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint32_t w = (uint32_t)warp + 32u * (uint32_t)k;
                if (w >= nw) continue;
                const uint32_t uw = und[w];
                if (uw == 0u) continue;
                bool a_now = false, r_now = false;
                if ((uw >> lane) & 1u) {
                    const uint32_t i = 32u * w + (uint32_t)lane;
                    uint32_t kill = 0u, block = 0u, cb = 0u, v = 0u;
                    // four words at a time: one 16-byte load each of accb, und
                    for (; v + 4u <= w; v += 4u) {
                        const uint4 av = *reinterpret_cast<const uint4*>(accb + v);
                        const uint4 uv = *reinterpret_cast<const uint4*>(und + v);
                        const uint32_t c1 = cb + P - 32u * v - 32u;
                        const uint32_t c2 = c1 + P - 32u * v - 64u;
                        const uint32_t c3 = c2 + P - 32u * v - 96u;
                        const uint32_t m0 = T[cb + i], m1 = T[c1 + i], m2 = T[c2 + i],
                                       m3 = T[c3 + i];
                        kill |= (m0 & av.x) | (m1 & av.y) | (m2 & av.z) | (m3 & av.w);
                        block |= (m0 & uv.x) | (m1 & uv.y) | (m2 & uv.z) | (m3 & uv.w);
                        cb = c3 + P - 32u * v - 128u;
                    }
                    for (; v < w; ++v) {
                        const uint32_t m = T[cb + i];
                        kill |= m & accb[v];
                        block |= m & und[v];
                        cb += P - 32u * v - 32u;
                    }
                    const uint32_t m = T[cb + i] & ((1u << lane) - 1u);
                    kill |= m & accb[w];
                    block |= m & uw;
                    r_now = kill != 0u;
                    a_now = !r_now && block == 0u;
                }
                ba[k] = __ballot_sync(kFull, a_now);
                br[k] = __ballot_sync(kFull, r_now);
            }
            named_barrier(1, nthreads);
            if (lane == 0)
                for (int k = 0; k < 2; ++k) {
                    const uint32_t w = (uint32_t)warp + 32u * (uint32_t)k;
                    if (w >= nw) continue;
                    accb[w] |= ba[k];
                    const uint32_t nu = und[w] & ~(ba[k] | br[k]);
                    und[w] = nu;
                    if (nu) bs.left[slot] = 1u;
                }
            named_barrier(1, nthreads);
            if (bs.left[slot] == 0u) break;
        }
    }
    __syncthreads();
    if (timing) {
        const long long t = clock64();
        tim[1] += (unsigned long long)(t - t_last);
        t_last = t;
    }
    uint32_t nacc = 0;
    for (uint32_t t0 = 0; t0 < P; t0 += kBlock) {
        const uint32_t i = t0 + threadIdx.x;
        const bool keep = i < P && ((accb[i >> 5] >> (i & 31u)) & 1u);
        nacc = block_append(bs, keep, keep ? x[i] : 0u, (keep && acc_off) ? off[i] : 0u, acc,
                            acc_off, nacc);
    }
    if (timing) tim[2] += (unsigned long long)(clock64() - t_last);
    return nacc;
}

// ------------------------------------------------------------ pair resolver
// CTA-wide, narrow words.  Decides the list x[0..n) (n <= 4096) in order,
// as the serial greedy would (Section 4), from the list of its conflicting
// pairs (k, i), k < i, entries within distance d-1 (or otherwise in
// conflict); every conflicting pair must be listed, duplicates are
// harmless.  for_pairs(f) calls f(k, i) for this thread's share of the
// pairs (every pair in exactly one thread).  Rounds: an undecided entry with an accepted earlier
// neighbour is rejected, one whose earlier neighbours are all rejected is
// accepted; the first undecided entry always decides, so the rounds end, and
// every decision rests on final ones.  Accepted entries are appended in
// order to acc/acc_off (off may be null when acc_off is).  Returns how many.
//   state  n bytes, flags 2 * 4096 bytes of scratch
// tim (optional, thread 0): cycles to tim[1] rounds and tim[2] append,
// tim[3] counts rounds.
template <typename ForPairs>
__device__ __forceinline__ uint32_t pair_resolve(BlockScratch& bs, const uint32_t* x,
                                                 const uint32_t* off, uint8_t* state, uint32_t n,
                                                 ForPairs for_pairs, uint8_t* flags,
                                                 uint32_t* acc, uint32_t* acc_off,
                                                 unsigned long long* tim = nullptr) {
    const int lane = lane_id();
    const bool timing = tim && threadIdx.x == 0;
    long long t_last = timing ? clock64() : 0;
    uint8_t* killed = flags;           // an accepted earlier neighbour seen this round
    uint8_t* blocked = flags + 4096;   // an undecided earlier neighbour seen this round
    for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
        state[i] = 0;  // 0 undecided, 1 accepted, 2 rejected
        killed[i] = 0;
        blocked[i] = 0;
    }
    if (threadIdx.x < 3) bs.left[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t round = 0;; ++round) {
        if (timing) tim[3] += 1;
        // this round's flag slot; the next one was last read two rounds ago
        const uint32_t slot = round % 3u, next = (round + 1u) % 3u;
        if (threadIdx.x == 0) bs.left[next] = 0u;
        for_pairs([&](uint32_t k, uint32_t i) {
            if (state[i] == 0) {
                const uint8_t sk = state[k];
                if (sk == 1) killed[i] = 1;
                else if (sk == 0) blocked[i] = 1;
            }
        });
        __syncthreads();
        // decide, and clear the marks for the next round (the thread that
        // reads an entry's marks is the one that clears them)
        bool left = false;
        for (uint32_t i = threadIdx.x; i < n; i += kBlock)
            if (state[i] == 0) {
                if (killed[i]) state[i] = 2;
                else if (!blocked[i]) state[i] = 1;
                else left = true;
                killed[i] = 0;
                blocked[i] = 0;
            }
        if (__any_sync(kFull, left) && lane == 0) bs.left[slot] = 1u;
        __syncthreads();
        if (bs.left[slot] == 0u) break;
    }
    if (timing) {
        const long long t = clock64();
        tim[1] += (unsigned long long)(t - t_last);
        t_last = t;
    }
    uint32_t nacc = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += kBlock) {
        const uint32_t i = t0 + threadIdx.x;
        const bool keep = i < n && state[i] == 1;
        nacc = block_append(bs, keep, keep ? x[i] : 0u, (keep && acc_off) ? off[i] : 0u, acc,
                            acc_off, nacc);
    }
    if (timing) tim[2] += (unsigned long long)(clock64() - t_last);
    return nacc;
}

// ------------------------------------------------------------ sparse resolver
// CTA-wide, narrow words, no orthogonality constraint.  The same decisions as
// block_resolve, through bucketed conflict detection, for lists whose
// conflicts are few.  Two words within distance d-1 differ in at most d-1 of
// the bits that vary over the list; split those bits into d blocks and the
// two words agree on at least one of them (pigeonhole), so only pairs that
// share a block's value -- hashed into kSpBuckets buckets -- are tested.  The
// greedy then runs in rounds over the conflicting pairs: an entry is
// rejected once an earlier neighbour is accepted and accepted once every
// earlier neighbour is rejected (the first undecided entry always decides).
// Returns false, having written nothing, when d is out of range, the buckets
// hold more than pair_budget pairs or the conflicts overflow the scratch;
// the caller then runs block_resolve.
//   x/off[0..n)   candidates in order (n <= 4096; not modified)
//   state         n bytes of scratch
//   acc/acc_off   receives accepted vectors/offsets in order (acc, n words,
//                 is scratch until then)
//   scratch       8192 words of shared memory (the resolver matrix)
// tim as for block_resolve: [0] bucketed search, [1] rounds, [2] append.
constexpr uint32_t kSpBuckets = 1024;
constexpr uint32_t kSpEdges = 4096;
static_assert(kSpBuckets == (uint32_t)kBlock, "one bucket per thread in the scan");

__device__ __forceinline__ uint32_t sp_hash(uint32_t v) { return (v * 0x9E3779B1u) >> 22; }

__device__ __forceinline__ bool sparse_resolve(BlockScratch& bs, const uint32_t* x,
                                               const uint32_t* off, uint8_t* state, uint32_t n,
                                               int d, uint32_t* acc, uint32_t* acc_off,
                                               uint32_t* scratch, uint32_t pair_budget,
                                               uint64_t& nt, uint32_t* nacc_out,
                                               unsigned long long* tim = nullptr) {
    if (d < 2 || d > 8 || n < 2 || n > 4096) return false;
    const bool timing = tim && threadIdx.x == 0;
    long long t_last = timing ? clock64() : 0;
    auto tick = [&](int k) {
        if (timing) {
            const long long t = clock64();
            tim[k] += (unsigned long long)(t - t_last);
            t_last = t;
        }
    };
    uint32_t* cnt = scratch;                                            // [kSpBuckets]
    uint32_t* fill = scratch + kSpBuckets;                              // [kSpBuckets]
    uint16_t* order = reinterpret_cast<uint16_t*>(scratch + 2 * kSpBuckets);  // [n]
    uint32_t* edges = scratch + 4096;                                   // [kSpEdges]
    const int lane = lane_id();
    // the bits that vary over the list
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < n; i += kBlock) v |= x[i] ^ x[0];
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
    if (threadIdx.x == 0) {
        bs.sp_vary = 0u;
        bs.sp_pairs = 0u;
        bs.sp_edges = 0u;
    }
    __syncthreads();
    if (lane == 0 && v) atomicOr(&bs.sp_vary, v);
    __syncthreads();
    const uint32_t vary = bs.sp_vary;
    const int nv = __popc(vary);
    if (nv < d) return false;  // every pair would be tested
    if (threadIdx.x == 0) {
        // block b takes the varying bits of ranks [b nv / d, (b+1) nv / d)
        uint32_t rest = vary;
        int r = 0;
        for (int b = 0; b < 8; ++b) bs.sp_masks[b] = 0u;
        while (rest) {
            const uint32_t bit = rest & (0u - rest);
            rest ^= bit;
            bs.sp_masks[(r * d) / nv] |= bit;
            ++r;
        }
    }
    __syncthreads();
    uint64_t tests = 0;
    for (int b = 0; b < d; ++b) {
        const uint32_t mask = bs.sp_masks[b];
        for (uint32_t h = threadIdx.x; h < kSpBuckets; h += kBlock) cnt[h] = 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += kBlock) atomicAdd(&cnt[sp_hash(x[i] & mask)], 1u);
        __syncthreads();
        // pairs this blocking would test; give up when they cost too much
        uint32_t pairs = 0;
        for (uint32_t h = threadIdx.x; h < kSpBuckets; h += kBlock)
            pairs += cnt[h] * (cnt[h] - (cnt[h] ? 1u : 0u)) / 2u;
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
        if (lane == 0 && pairs) atomicAdd(&bs.sp_pairs, pairs);
        uint32_t total = 0;
        const uint32_t h0 = threadIdx.x;  // one bucket per thread (kSpBuckets == kBlock)
        const uint32_t start = block_exclusive_scan(bs, h0 < kSpBuckets ? cnt[h0] : 0u, &total);
        if (bs.sp_pairs > pair_budget) return false;  // uniform: read after the scan's barriers
        if (h0 < kSpBuckets) fill[h0] = start;
        __syncthreads();
        // bucket order: index in order[], vector in acc[] (free until the
        // accepts are appended)
        for (uint32_t i = threadIdx.x; i < n; i += kBlock) {
            const uint32_t p = atomicAdd(&fill[sp_hash(x[i] & mask)], 1u);
            order[p] = (uint16_t)i;
            acc[p] = x[i];
        }
        __syncthreads();
        // every pair of a bucket, tested once from its later entry; fill[h]
        // is now the end of bucket h and cnt[h] its size.  Threads stop once
        // the conflicts overflow the scratch.
        const volatile uint32_t* found = &bs.sp_edges;
        for (uint32_t p = threadIdx.x; p < n && *found <= kSpEdges; p += kBlock) {
            const uint32_t i = order[p];
            const uint32_t xi = acc[p];
            const uint32_t h = sp_hash(xi & mask);
            const uint32_t e1 = fill[h], e0 = e1 - cnt[h];
            for (uint32_t q = e0; q < e1; ++q) {
                const uint32_t k = order[q];
                const uint32_t xk = acc[q];
                if (k >= i) continue;
                ++tests;
                if (__popc(xi ^ xk) < d) {
                    const uint32_t e = atomicAdd(&bs.sp_edges, 1u);
                    if (e < kSpEdges) edges[e] = (k << 16) | i;
                }
            }
        }
        __syncthreads();
        if (bs.sp_edges > kSpEdges) {
            nt += tests;
            return false;  // uniform: read after the barrier
        }
    }
    nt += tests;
    const uint32_t ne = bs.sp_edges;
    if (ne > kSpEdges) return false;
    uint8_t* killed = reinterpret_cast<uint8_t*>(scratch + 2 * kSpBuckets);  // [n]
    tick(0);
    *nacc_out = pair_resolve(
        bs, x, off, state, n,
        [&](auto&& f) {
            for (uint32_t e = threadIdx.x; e < ne; e += kBlock) f(edges[e] >> 16, edges[e] & 0xffffu);
        },
        killed, acc, acc_off, tim);
    return true;
}

}  // namespace gc
