// gc_device.cuh -- device-side building blocks of the greedy sweep (sm_103a).
//
// Vectors are the low n bits of a uint32 (n <= 32) or, in the wide forms, of
// a uint64 (n <= 64), with coordinate 1 as the most significant of them.  The
// four orders of Section 4.2 are turned into closed-form rank <-> vector maps
// so that any window of ranks can be generated in parallel without
// materialising the order:
//   LEX      rank r is the vector r.
//   GRAY     rank r is r ^ (r >> 1); the inverse is a prefix XOR.  With a
//            weight w the ranks are those of the weight-w vectors only, in
//            the same order (gray_weight_unrank).
//   GRLEX    weight classes in ascending weight; inside class k the i-th
//            vector is the i-th smallest n-bit integer of weight k, found with
//            the combinatorial number system.
//   GREVLEX  weight classes ascending; inside class k vectors are ordered by
//            DECREASING bit-reversed value (the lowest differing bit decides
//            and the vector holding the 1 comes first), so the i-th one is
//            the bit-reversal of the (C(n,k)-1-i)-th smallest weight-k integer.
#pragma once
#include <cstdint>

namespace gc {

constexpr int kMaxN = 32;       // narrow vectors (uint32 words)
constexpr int kMaxNWide = 64;   // wide vectors (uint64 words)
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- binomials
// Binomial coefficients C(p, k), 0 <= p, k <= 32, fit in uint32 (the largest,
// C(32,16), is about 6.0e8).  Kept in shared memory by the kernels that use
// them because the indices diverge across a warp.
struct Binom {
    uint32_t c[kMaxN + 1][kMaxN + 1];
};

__host__ __device__ inline void fill_binom(Binom& b) {
    for (int p = 0; p <= kMaxN; ++p)
        for (int k = 0; k <= kMaxN; ++k)
            b.c[p][k] = (k == 0) ? 1u : (p == 0 ? 0u : b.c[p - 1][k - 1] + b.c[p - 1][k]);
}

// i-th (0-based) n-bit integer of weight k in ascending order.  Walking bit
// positions from the top: the C(p, k) weight-k integers below 2^p come before
// every one with bit p set, so bit p is set iff i >= C(p, k).
__device__ __forceinline__ uint32_t comb_unrank(const uint32_t (*C)[kMaxN + 1], int n, int k,
                                                uint32_t i) {
    uint32_t x = 0;
    for (int p = n - 1; p >= 0 && k > 0; --p) {
        uint32_t c = C[p][k];
        if (i >= c) {
            x |= 1u << p;
            i -= c;
            --k;
        }
    }
    return x;
}

// Position of x among the n-bit integers of its weight, ascending: with set
// bits at p_1 < p_2 < ... < p_k the position is sum_j C(p_j, j).
__device__ __forceinline__ uint32_t comb_rank(const uint32_t (*C)[kMaxN + 1], uint32_t x) {
    uint32_t r = 0;
    int j = 1;
    while (x) {
        int p = __ffs(x) - 1;
        r += C[p][j];
        ++j;
        x &= x - 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t reverse_n(uint32_t v, int n) { return __brev(v) >> (32 - n); }

// i-th (0-based) n-bit vector of weight w in Gray order.  The vector of Gray
// rank r is r ^ (r >> 1), whose weight is the number of places where r
// changes between neighbouring bits, reading down from a 0 above bit n-1.  The
// rank is built from the top bit down, 0 before 1: with t changes so far and
// the bit above equal to `prev`, putting b at bit p leaves the p bits below it,
// whose p neighbour pairs must hold the w - t - [b != prev] remaining changes:
// C(p, w - t - [b != prev]) ways.
__device__ __forceinline__ uint32_t gray_weight_unrank(const uint32_t (*C)[kMaxN + 1], int n,
                                                       int w, uint32_t i) {
    uint32_t r = 0;
    int prev = 0, t = 0;
    for (int p = n - 1; p >= 0; --p) {
        const int t0 = t + (prev != 0);
        const uint32_t c0 = (w - t0 >= 0) ? C[p][w - t0] : 0u;
        if (i < c0) {
            t = t0;
            prev = 0;
        } else {
            i -= c0;
            r |= 1u << p;
            t += (prev != 1);
            prev = 1;
        }
    }
    return r ^ (r >> 1);
}

// Wide forms: C(p, k) for p, k <= 64 (Pascal's rule; C(64, 32) < 2^61), read
// through the read-only cache from a table initialised at compile time.
struct Binom64Table {
    uint64_t c[kMaxNWide + 1][kMaxNWide + 1];
};
constexpr Binom64Table make_binom64() {
    Binom64Table t{};
    for (int p = 0; p <= kMaxNWide; ++p)
        for (int k = 0; k <= kMaxNWide; ++k)
            t.c[p][k] = (k == 0) ? 1ull : (p == 0 ? 0ull : t.c[p - 1][k - 1] + t.c[p - 1][k]);
    return t;
}

__device__ __forceinline__ uint64_t comb_unrank64(const Binom64Table& C, int n, int k,
                                                  uint64_t i) {
    uint64_t x = 0;
    for (int p = n - 1; p >= 0 && k > 0; --p) {
        const uint64_t c = __ldg(&C.c[p][k]);
        if (i >= c) {
            x |= 1ull << p;
            i -= c;
            --k;
        }
    }
    return x;
}

__device__ __forceinline__ uint64_t reverse_n64(uint64_t v, int n) {
    return __brevll(v) >> (64 - n);
}

// Wide form of gray_weight_unrank.
__device__ __forceinline__ uint64_t gray_weight_unrank64(const Binom64Table& C, int n, int w,
                                                         uint64_t i) {
    uint64_t r = 0;
    int prev = 0, t = 0;
    for (int p = n - 1; p >= 0; --p) {
        const int t0 = t + (prev != 0);
        const uint64_t c0 = (w - t0 >= 0) ? __ldg(&C.c[p][w - t0]) : 0ull;
        if (i < c0) {
            t = t0;
            prev = 0;
        } else {
            i -= c0;
            r |= 1ull << p;
            t += (prev != 1);
            prev = 1;
        }
    }
    return r ^ (r >> 1);
}

// Population counts of either word width.
__device__ __forceinline__ int popc(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc(uint64_t v) { return __popcll(v); }

__device__ __forceinline__ uint32_t gray_inverse(uint32_t g) {
    g ^= g >> 1;
    g ^= g >> 2;
    g ^= g >> 4;
    g ^= g >> 8;
    g ^= g >> 16;
    return g;
}

// ---------------------------------------------------------------- orders
enum : int { kLex = 0, kGray = 1, kGrlex = 2, kGrevlex = 3, kBasis = 4 };

// Everything the ordering maps need, small enough to pass by value.
struct Order {
    int n;
    int ord;
    int w;          // -1 = every weight
    bool filter;    // BASIS with a weight: ranks of the wrong weight are skipped
    bool even;      // only even-weight vectors are candidates (self-orthogonal)
    uint64_t N;     // rank-space size
    // graded orders without a weight: cum[k] = number of vectors of weight < k
    uint64_t cum[kMaxNWide + 2];
    // B-ordering (Section 4.3): basis[j] = b_{j+1}; inv[j] = row j of the
    // inverse, so bit j of the rank of v is the parity of (v AND inv[j])
    uint32_t basis[kMaxN];
    uint32_t inv[kMaxN];
};

// Vector of rank r (r < N).  Returns false when the rank is skipped: a
// B-ordering rank of the wrong weight, or an odd-weight vector when only even
// ones are candidates.
__device__ __forceinline__ bool unrank(const Order& o, const uint32_t (*C)[kMaxN + 1], uint64_t r,
                                       uint32_t& x) {
    const int n = o.n;
    bool ok = true;
    if (o.ord == kGray) {
        x = o.w >= 0 ? gray_weight_unrank(C, n, o.w, (uint32_t)r) : (uint32_t)(r ^ (r >> 1));
    } else if (o.ord == kBasis) {
        x = 0;
        for (uint64_t b = r; b; b &= b - 1) x ^= o.basis[__ffsll((long long)b) - 1];
        ok = !o.filter || __popc(x) == o.w;
    } else if (o.ord == kLex && o.w < 0) {
        x = (uint32_t)r;
    } else {
        int k;
        uint32_t i;
        if (o.w >= 0) {
            k = o.w;
            i = (uint32_t)r;
        } else {
            // weight class of r: the last k with cum[k] <= r (classes ascend)
            k = 0;
            while (k < n && o.cum[k + 1] <= r) ++k;
            i = (uint32_t)(r - o.cum[k]);
        }
        if (o.ord == kGrevlex) {
            const uint32_t m = C[n][k] - 1 - i;
            x = reverse_n(comb_unrank(C, n, k, m), n);
        } else {
            x = comb_unrank(C, n, k, i);  // kGrlex, or kLex restricted to weight w
        }
    }
    if (o.even && (__popc(x) & 1)) ok = false;
    return ok;
}

// Wide form of unrank for n <= 64 (LEX, GRAY, GRLEX, GREVLEX; B-orderings
// are narrow only).
__device__ __forceinline__ bool unrank_wide(const Order& o, const Binom64Table& C, uint64_t r,
                                            uint64_t& x) {
    const int n = o.n;
    bool ok = true;
    if (o.ord == kGray) {
        x = o.w >= 0 ? gray_weight_unrank64(C, n, o.w, r) : (r ^ (r >> 1));
    } else if (o.ord == kLex && o.w < 0) {
        x = r;
    } else {
        int k;
        uint64_t i;
        if (o.w >= 0) {
            k = o.w;
            i = r;
        } else {
            k = 0;
            while (k < n && o.cum[k + 1] <= r) ++k;
            i = r - o.cum[k];
        }
        if (o.ord == kGrevlex) {
            const uint64_t m = __ldg(&C.c[n][k]) - 1 - i;
            x = reverse_n64(comb_unrank64(C, n, k, m), n);
        } else {
            x = comb_unrank64(C, n, k, i);
        }
    }
    if (o.even && (__popcll(x) & 1)) ok = false;
    return ok;
}

// Rank of vector x in the full 2^n order (no weight).
__device__ __forceinline__ uint64_t rank_of(const Order& o, const uint32_t (*C)[kMaxN + 1],
                                            uint32_t x) {
    const int n = o.n;
    switch (o.ord) {
        case kLex: return x;
        case kGray: return gray_inverse(x);
        case kBasis: {
            uint64_t r = 0;
            for (int j = 0; j < n; ++j) r |= (uint64_t)(__popc(x & o.inv[j]) & 1) << j;
            return r;
        }
        default: {
            int k = __popc(x);
            uint64_t base = 0;
            for (int j = 0; j < k; ++j) base += C[n][j];
            uint32_t pos = (o.ord == kGrlex) ? comb_rank(C, x)
                                             : C[n][k] - 1 - comb_rank(C, reverse_n(x, n));
            return base + pos;
        }
    }
}

// ---------------------------------------------------------------- memory ops
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Arrival on a counter that publishes everything this thread (and, through
// a preceding CTA barrier, its CTA) wrote before it; no value comes back.
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}
// Loads of data other CTAs wrote during this kernel: L2 only (L1 is not
// coherent across SMs).
__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ld_cg(const uint64_t* p) {
    return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}

// ---------------------------------------------------------------- warp utils
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
// Barrier `id` (1..15; 0 is __syncthreads) over the first nthreads threads
// of the CTA (a multiple of 32; every one of them must call it).
__device__ __forceinline__ void named_barrier(unsigned id, unsigned nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

}  // namespace gc
