/*
 * greedy_oracle.c -- plain, slow, obviously correct CPU oracle for the ordered
 * greedy construction of binary codes (Paliwal, Tiwary, Chaudhury, Gupta,
 * "Generating Binary Optimal Codes Using Heterogeneous Parallel Computing").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (Section 4, "Greedy Algorithms and Different Orderings"):
 * order all vectors of F_2^n (optionally only those of weight w), then walk the
 * order starting from the zero vector and append a vector to the code C iff its
 * Hamming distance to every codeword already in C is at least d.  The result is
 * the code in acceptance order.  Example 1 of Section 4.1 walks this for n=3,
 * d=2 and ends with {000, 011, 101, 110}.
 *
 * Encoding (the paper does not state one): coordinate 1 of a length-n vector is
 * the most significant of the low n bits of a uint32, so the string "011" is
 * the integer 3.  With that encoding the lexicographic order of Example 1
 * (000, 001, ..., 111) is ascending integer order.
 *
 * Orderings (Section 4.2, "Ordering Implementation"; the paper names the four
 * orders but defines none of them, so each reading below is stated):
 *   LEX      ascending integer.
 *   GRAY     binary-reflected Gray code: rank r is the vector r ^ (r >> 1).
 *   GRLEX    graded lexicographic: weight ascending, then ascending integer
 *            (the textbook graded-lex monomial order, read ascending, with
 *            coordinate 1 as the most significant variable).
 *   GREVLEX  graded reverse lexicographic: weight ascending; within a weight,
 *            a comes before b iff, at the LAST coordinate (least significant
 *            bit) where they differ, a has the 1 (the textbook graded-reverse-
 *            lex monomial order, read ascending).
 * Constant weight w: the chosen order restricted to the weight-w vectors, in
 * the same relative order.  The first candidate is accepted unconditionally
 * (it is the zero vector when no weight is given).
 *
 * Three forms:
 *   O1 orc_greedy_pairwise  -- the definition written out: each candidate is
 *                              compared with every codeword so far.
 *   O2 orc_greedy_ball      -- the same decision taken through an exclusion
 *                              map over vectors: a candidate is rejected iff an
 *                              earlier codeword lies within distance d-1 of it,
 *                              i.e. iff some earlier codeword's radius-(d-1)
 *                              ball covers it.  Used where O1 is too slow.
 *   O3 orc_verify           -- checks that a given list is THE greedy output:
 *                              strictly increasing in the order, pairwise
 *                              distance >= d, and every candidate not in the
 *                              list has an earlier list member within d-1.
 *                              These three properties determine the greedy
 *                              output uniquely (induction along the order).
 * Parity pins for every function live in tests/test_oracle.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_LEX = 0, ORC_GRAY = 1, ORC_GRLEX = 2, ORC_GREVLEX = 3 };

/* Error returns (negative so they cannot be confused with a count). */
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

int orc_popcount(uint32_t v) { return __builtin_popcount(v); }

/* Hamming distance (Section 5.2): number of positions where x and y differ,
 * i.e. the weight of x XOR y. */
int orc_distance(uint32_t x, uint32_t y) { return orc_popcount(x ^ y); }

/* Reverse the low n bits of x (coordinate 1 <-> coordinate n). */
uint32_t orc_reverse_bits(uint32_t x, int n) {
    uint32_t y = 0;
    for (int i = 0; i < n; ++i)
        if (x & (1u << i)) y |= 1u << (n - 1 - i);
    return y;
}

static int valid_args(int n, int ord, int w) {
    if (n < 1 || n > 32) return 0;
    if (ord < ORC_LEX || ord > ORC_GREVLEX) return 0;
    if (w < -1 || w > n) return 0;
    return 1;
}

static uint64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

/* Number of candidates: 2^n, or C(n, w) with a constant weight. */
uint64_t orc_candidate_count(int n, int w) {
    if (n < 1 || n > 32 || w < -1 || w > n) return 0;
    return w < 0 ? (1ull << n) : binom(n, w);
}

/* Smallest n-bit integer of weight k above y with the same weight (Gosper's
 * rule: move the lowest block of ones up by one place and pack the rest of
 * the block at the bottom); returns a value >= 2^n when y is the last one. */
static uint64_t next_same_weight(uint64_t y) {
    uint64_t c = y & (~y + 1);
    uint64_t r = y + c;
    return (((r ^ y) >> 2) / c) | r;
}

/* ---- streaming enumeration of the candidates, in order ------------------ */
typedef struct {
    int n, ord, w;
    int wt, wt_end;   /* graded orders: current and last weight class */
    uint64_t r;       /* LEX / GRAY: next rank; graded: current pattern */
    int started;
    int done;
} orc_iter;

static void iter_init(orc_iter *it, int n, int ord, int w) {
    memset(it, 0, sizeof *it);
    it->n = n; it->ord = ord; it->w = w;
    it->wt = (w < 0) ? 0 : w;
    it->wt_end = (w < 0) ? n : w;
}

/* Returns 1 and stores the next candidate in *x, or 0 when exhausted. */
static int iter_next(orc_iter *it, uint32_t *x) {
    const int n = it->n;
    const uint64_t full = 1ull << n;
    if (it->done) return 0;
    if (it->ord == ORC_LEX || it->ord == ORC_GRAY) {
        while (it->r < full) {
            uint64_t r = it->r++;
            uint32_t v = (uint32_t)(it->ord == ORC_LEX ? r : (r ^ (r >> 1)));
            if (it->w < 0 || orc_popcount(v) == it->w) { *x = v; return 1; }
        }
        it->done = 1;
        return 0;
    }
    /* Graded orders: weight classes in ascending order.  Within class k,
     * GRLEX walks the weight-k integers upward.  GREVLEX must visit the
     * weight-k vectors by DESCENDING bit-reversed value; it walks the
     * weight-(n-k) integers y upward and emits rev(~y), whose bit-reversal is
     * ~y, which then descends. */
    for (;;) {
        if (it->wt > it->wt_end) { it->done = 1; return 0; }
        int k = (it->ord == ORC_GRLEX) ? it->wt : n - it->wt;
        if (!it->started) {
            it->r = (k == 0) ? 0 : ((1ull << k) - 1);
            it->started = 1;
        } else if (k == 0) {
            it->r = full; /* the only weight-0 pattern has been emitted */
        } else {
            it->r = next_same_weight(it->r);
        }
        if (it->r < full) {
            uint32_t y = (uint32_t)it->r;
            if (it->ord == ORC_GRLEX) *x = y;
            else *x = orc_reverse_bits((uint32_t)(~y & (uint32_t)(full - 1)), n);
            return 1;
        }
        it->wt++;
        it->started = 0;
    }
}

/* Fill out[0..count) with the candidates in order (streaming form).
 * Returns the number written or a negative error. */
int64_t orc_order_list(int n, int ord, int w, uint32_t *out, int64_t cap) {
    if (!valid_args(n, ord, w)) return ORC_EINVAL;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x; int64_t k = 0;
    while (iter_next(&it, &x)) {
        if (k < cap) out[k] = x;
        ++k;
    }
    return k;
}

/* ---- the orders as comparators: the definitions, used to pin the stream -- */
static int g_cmp_n;
static uint32_t gray_rank(uint32_t g) { /* r with r ^ (r>>1) == g */
    uint32_t r = 0;
    for (uint32_t s = g; s; s >>= 1) r ^= s;
    return r;
}
static int cmp_lex(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}
static int cmp_gray(const void *a, const void *b) {
    uint32_t x = gray_rank(*(const uint32_t *)a), y = gray_rank(*(const uint32_t *)b);
    return (x > y) - (x < y);
}
static int cmp_grlex(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    int wx = orc_popcount(x), wy = orc_popcount(y);
    if (wx != wy) return wx - wy;
    return (x > y) - (x < y);
}
static int cmp_grevlex(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    int wx = orc_popcount(x), wy = orc_popcount(y);
    if (wx != wy) return wx - wy;
    if (x == y) return 0;
    /* the last coordinate where they differ is the lowest differing bit */
    for (int i = 0; i < g_cmp_n; ++i) {
        uint32_t m = 1u << i;
        if ((x ^ y) & m) return (x & m) ? -1 : 1;
    }
    return 0;
}

/* Candidates in order by sorting the whole space with the order's
 * comparator.  Small n only (n <= 24).  Returns the count written. */
int64_t orc_order_sorted(int n, int ord, int w, uint32_t *out, int64_t cap) {
    if (!valid_args(n, ord, w) || n > 24) return ORC_EINVAL;
    int64_t k = 0;
    for (uint64_t v = 0; v < (1ull << n); ++v)
        if (w < 0 || orc_popcount((uint32_t)v) == w) {
            if (k >= cap) return ORC_EINVAL;
            out[k++] = (uint32_t)v;
        }
    g_cmp_n = n;
    int (*cmp)(const void *, const void *) =
        ord == ORC_LEX ? cmp_lex : ord == ORC_GRAY ? cmp_gray
        : ord == ORC_GRLEX ? cmp_grlex : cmp_grevlex;
    qsort(out, (size_t)k, sizeof(uint32_t), cmp);
    return k;
}

/* ---- O1: the greedy definition, pairwise ------------------------------- */
/* Writes up to cap codewords to out (acceptance order) and, when pos is not
 * NULL, the candidate index of each codeword to pos.  Returns |C|. */
int64_t orc_greedy_pairwise(int n, int d, int ord, int w,
                            uint32_t *out, int64_t *pos, int64_t cap) {
    if (!valid_args(n, ord, w) || d < 0) return ORC_EINVAL;
    uint64_t ncand = orc_candidate_count(n, w);
    /* |C| never exceeds the number of candidates; keep our own copy so the
     * test does not depend on the caller's capacity. */
    uint64_t room = ncand < (1ull << 26) ? ncand : (1ull << 26);
    uint32_t *C = (uint32_t *)malloc(room * sizeof(uint32_t));
    if (!C) return ORC_ENOMEM;
    int64_t size = 0, idx = 0;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x;
    while (iter_next(&it, &x)) {
        int ok = 1;
        for (int64_t j = 0; j < size; ++j)
            if (orc_distance(x, C[j]) < d) { ok = 0; break; }
        if (ok) {
            if ((uint64_t)size >= room) { free(C); return ORC_ENOMEM; }
            if (size < cap) { out[size] = x; if (pos) pos[size] = idx; }
            C[size++] = x;
        }
        ++idx;
    }
    free(C);
    return size;
}

/* ---- O2: the same greedy through exclusion balls over vectors ----------- */
/* All e with weight <= rad over n bits (the radius-rad ball around 0). */
static uint32_t *ball_list(int n, int rad, uint64_t *len) {
    uint64_t total = 0;
    for (int k = 0; k <= rad && k <= n; ++k) total += binom(n, k);
    uint32_t *b = (uint32_t *)malloc((total ? total : 1) * sizeof(uint32_t));
    if (!b) return NULL;
    uint64_t m = 0;
    /* walk each weight class (a filter over all 2^n vectors is too slow at
     * n = 32) */
    for (int k = 0; k <= rad && k <= n; ++k) {
        if (k == 0) { b[m++] = 0; continue; }
        for (uint64_t y = (1ull << k) - 1; y < (1ull << n); y = next_same_weight(y))
            b[m++] = (uint32_t)y;
    }
    *len = m;
    return b;
}

int64_t orc_greedy_ball(int n, int d, int ord, int w,
                        uint32_t *out, int64_t *pos, int64_t cap) {
    if (!valid_args(n, ord, w) || d < 0) return ORC_EINVAL;
    uint64_t words = ((1ull << n) + 63) / 64;
    uint64_t *covered = (uint64_t *)calloc(words, sizeof(uint64_t));
    if (!covered) return ORC_ENOMEM;
    uint64_t blen = 0;
    uint32_t *ball = ball_list(n, d - 1, &blen);   /* d <= 0: empty ball */
    if (!ball) { free(covered); return ORC_ENOMEM; }
    if (d <= 0) blen = 0;
    int64_t size = 0, idx = 0;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x;
    while (iter_next(&it, &x)) {
        if (!(covered[x >> 6] >> (x & 63) & 1)) {
            if (size < cap) { out[size] = x; if (pos) pos[size] = idx; }
            ++size;
            for (uint64_t j = 0; j < blen; ++j) {
                uint32_t y = x ^ ball[j];
                covered[y >> 6] |= 1ull << (y & 63);
            }
        }
        ++idx;
    }
    free(ball);
    free(covered);
    return size;
}

/* ---- O3: the characterisation check ------------------------------------ */
/* Returns 0 if L[0..len) is exactly the greedy output, else a positive code:
 *   1 an element is not a candidate or the list is not strictly in order,
 *   2 two elements are closer than d,
 *   3 a candidate outside L has no earlier element of L within d-1,
 *   4 out of memory.  Cost O(N * |L|); meant for n <= 24. */
int orc_verify(int n, int d, int ord, int w, const uint32_t *L, int64_t len) {
    if (!valid_args(n, ord, w)) return 1;
    for (int64_t i = 0; i < len; ++i)
        for (int64_t j = 0; j < i; ++j)
            if (orc_distance(L[i], L[j]) < d) return 2;
    int64_t i = 0;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x;
    while (iter_next(&it, &x)) {
        if (i < len && L[i] == x) { ++i; continue; }
        int covered = 0;
        for (int64_t j = 0; j < i; ++j)
            if (orc_distance(x, L[j]) <= d - 1) { covered = 1; break; }
        if (!covered) return 3;
    }
    return i == len ? 0 : 1;
}

/* ---- the steps of the sweep, one at a time ------------------------------ */
/* Block distance test (Sections 4.1, 5.2): alive[i] = 1 iff cand[i] is at
 * distance >= d from every code[j]. */
void orc_block_test(int d, const uint32_t *cand, int64_t nc, const uint32_t *code,
                    int64_t nk, uint8_t *alive) {
    for (int64_t i = 0; i < nc; ++i) {
        int ok = 1;
        for (int64_t j = 0; j < nk; ++j)
            if (orc_distance(cand[i], code[j]) < d) { ok = 0; break; }
        alive[i] = (uint8_t)ok;
    }
}

/* In-order resolve: the greedy of Section 4 applied to a given list (the list
 * takes the place of the ordered space).  Writes the list indices of the
 * accepted entries; returns how many. */
int64_t orc_resolve(int d, const uint32_t *cand, int64_t nc, int64_t *acc_idx) {
    int64_t na = 0;
    for (int64_t i = 0; i < nc; ++i) {
        int ok = 1;
        for (int64_t j = 0; j < na; ++j)
            if (orc_distance(cand[i], cand[acc_idx[j]]) < d) { ok = 0; break; }
        if (ok) acc_idx[na++] = i;
    }
    return na;
}

/* Exclusion-ball marking: set bit (c ^ e) for every codeword c and every e of
 * weight <= d-1; bit v of the map is word v/32, bit v%32. */
int orc_ball_mark(int n, int d, const uint32_t *code, int64_t nk, uint32_t *bitmap) {
    if (n < 1 || n > 32) return ORC_EINVAL;
    uint64_t blen = 0;
    uint32_t *ball = ball_list(n, d - 1, &blen);
    if (!ball) return ORC_ENOMEM;
    if (d <= 0) blen = 0;
    for (int64_t i = 0; i < nk; ++i)
        for (uint64_t j = 0; j < blen; ++j) {
            uint32_t y = code[i] ^ ball[j];
            bitmap[y >> 5] |= 1u << (y & 31);
        }
    free(ball);
    return 0;
}

/* Find-unmarked scan over ranks [rank0, rank0 + count) of the rank space:
 * the candidates in order (all 2^n vectors, or the C(n, w) weight-w vectors
 * of the order when a weight is given; rank i is the i-th candidate).  Writes
 * the vectors whose bit is clear, in rank order; returns how many were
 * clear. */
int64_t orc_scan(int n, int ord, int w, const uint32_t *bitmap, uint64_t rank0,
                 uint64_t count, uint32_t *out, int64_t cap) {
    if (!valid_args(n, ord, w)) return ORC_EINVAL;
    int64_t found = 0;
    uint64_t r = 0;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x;
    while (r < rank0 + count && iter_next(&it, &x)) {
        if (r >= rank0 && !(bitmap[x >> 5] >> (x & 31) & 1)) {
            if (found < cap) out[found] = x;
            ++found;
        }
        ++r;
    }
    return found;
}

/* ---- self-orthogonal greedy codes (Section 4.4) ------------------------- */
/* The greedy of Section 4 with the extra constraint of Section 4.4: a vector
 * is appended only if it is orthogonal to itself and to every codeword so
 * far (over F_2, x.y = popcount(x AND y) mod 2), besides being at distance
 * >= d from every codeword.  Pairwise form. */
int64_t orc_greedy_selforth(int n, int d, int ord, int w, uint32_t *out, int64_t *pos,
                            int64_t cap) {
    if (!valid_args(n, ord, w) || d < 0) return ORC_EINVAL;
    uint64_t ncand = orc_candidate_count(n, w);
    uint64_t room = ncand < (1ull << 26) ? ncand : (1ull << 26);
    uint32_t *C = (uint32_t *)malloc((room ? room : 1) * sizeof(uint32_t));
    if (!C) return ORC_ENOMEM;
    int64_t size = 0, idx = 0;
    orc_iter it; iter_init(&it, n, ord, w);
    uint32_t x;
    while (iter_next(&it, &x)) {
        int ok = (orc_popcount(x) % 2) == 0;          /* x.x = 0 */
        for (int64_t j = 0; ok && j < size; ++j)
            if (orc_distance(x, C[j]) < d || (orc_popcount(x & C[j]) % 2) != 0) ok = 0;
        if (ok) {
            if ((uint64_t)size >= room) { free(C); return ORC_ENOMEM; }
            if (size < cap) { out[size] = x; if (pos) pos[size] = idx; }
            C[size++] = x;
        }
        ++idx;
    }
    free(C);
    return size;
}

/* ---- B-orderings (Section 4.3) ------------------------------------------ */
/* For an ordered basis B = {b_1, ..., b_n} of F_2^n the B-ordering lists
 * 0, b_1, b_2, b_2+b_1, b_3, b_3+b_1, ...: rank r is the sum (XOR) of the b_j
 * whose index j-1 is a set bit of r.  basis[j-1] holds b_j.  Returns 1 iff
 * the n vectors are linearly independent over F_2 (plain elimination). */
static int basis_independent(int n, const uint32_t *basis) {
    uint32_t rows[32];
    for (int j = 0; j < n; ++j) rows[j] = basis[j] & (uint32_t)((n == 32) ? 0xffffffffu : ((1u << n) - 1u));
    for (int j = 0; j < n; ++j) if (rows[j] != basis[j]) return 0;
    int rank = 0;
    for (int bit = n - 1; bit >= 0; --bit) {
        int piv = -1;
        for (int j = rank; j < n; ++j)
            if (rows[j] >> bit & 1u) { piv = j; break; }
        if (piv < 0) continue;
        uint32_t t = rows[piv]; rows[piv] = rows[rank]; rows[rank] = t;
        for (int j = 0; j < n; ++j)
            if (j != rank && (rows[j] >> bit & 1u)) rows[j] ^= rows[rank];
        ++rank;
    }
    return rank == n;
}

uint32_t orc_border_vector(int n, const uint32_t *basis, uint64_t r) {
    uint32_t v = 0;
    for (int j = 0; j < n; ++j)
        if (r >> j & 1u) v ^= basis[j];
    return v;
}

/* The greedy of Section 4 over a B-ordering (optionally only weight-w
 * vectors, skipped in place like GRAY), pairwise form. */
int64_t orc_greedy_border(int n, int d, const uint32_t *basis, int w, uint32_t *out,
                          int64_t *pos, int64_t cap) {
    if (n < 1 || n > 32 || d < 0 || w < -1 || w > n || !basis_independent(n, basis))
        return ORC_EINVAL;
    uint64_t room = (w < 0 ? (1ull << n) : binom(n, w));
    if (room > (1ull << 26)) room = 1ull << 26;
    uint32_t *C = (uint32_t *)malloc((room ? room : 1) * sizeof(uint32_t));
    if (!C) return ORC_ENOMEM;
    int64_t size = 0, idx = 0;
    for (uint64_t r = 0; r < (1ull << n); ++r) {
        const uint32_t x = orc_border_vector(n, basis, r);
        if (w >= 0 && orc_popcount(x) != w) continue;
        int ok = 1;
        for (int64_t j = 0; j < size; ++j)
            if (orc_distance(x, C[j]) < d) { ok = 0; break; }
        if (ok) {
            if ((uint64_t)size >= room) { free(C); return ORC_ENOMEM; }
            if (size < cap) { out[size] = x; if (pos) pos[size] = idx; }
            C[size++] = x;
        }
        ++idx;
    }
    free(C);
    return size;
}

/* ---- vectors of up to 64 coordinates ------------------------------------ */
/* The same greedy for 1 <= n <= 64 (Section 4; the constant-weight codes of
 * Section 7 go to length 35).  Vectors are the low n bits of a uint64 with
 * coordinate 1 the most significant of them.  These forms materialise the
 * candidate list by the definition of the order: every candidate (the
 * weight-w vectors, or all 2^n vectors) sorted with the order's comparator.
 * n = 64 needs a weight (2^64 candidates do not fit a count).  orth = 1 adds
 * the Section 4.4 constraint (even weight, even inner product with every
 * earlier codeword). */
static uint64_t pascal64[65][65];
static int pascal64_ready = 0;
static uint64_t binom64c(int n, int k) {
    if (!pascal64_ready) {
        for (int p = 0; p <= 64; ++p)
            for (int q = 0; q <= 64; ++q)
                pascal64[p][q] = (q == 0) ? 1 : (p == 0 ? 0 : pascal64[p - 1][q - 1] + pascal64[p - 1][q]);
        pascal64_ready = 1;
    }
    if (n < 0 || k < 0 || k > n || n > 64) return 0;
    return pascal64[n][k];
}

static int valid_args64(int n, int ord, int w) {
    if (n < 1 || n > 64) return 0;
    if (ord < ORC_LEX || ord > ORC_GREVLEX) return 0;
    if (w < -1 || w > n) return 0;
    if (n == 64 && w < 0) return 0;
    return 1;
}

uint64_t orc64_candidate_count(int n, int w) {
    if (n < 1 || n > 64 || w < -1 || w > n || (n == 64 && w < 0)) return 0;
    return w < 0 ? (1ull << n) : binom64c(n, w);
}

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

static uint64_t gray_rank64(uint64_t g) { /* r with r ^ (r >> 1) == g */
    uint64_t r = 0;
    for (uint64_t s = g; s; s >>= 1) r ^= s;
    return r;
}
static int cmp64_lex(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}
static int cmp64_gray(const void *a, const void *b) {
    uint64_t x = gray_rank64(*(const uint64_t *)a), y = gray_rank64(*(const uint64_t *)b);
    return (x > y) - (x < y);
}
static int cmp64_grlex(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    int wx = popc64(x), wy = popc64(y);
    if (wx != wy) return wx - wy;
    return (x > y) - (x < y);
}
static int cmp64_grevlex(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    int wx = popc64(x), wy = popc64(y);
    if (wx != wy) return wx - wy;
    if (x == y) return 0;
    /* the last coordinate where they differ is the lowest differing bit; the
     * vector holding the 1 there comes first */
    for (int i = 0; i < 64; ++i) {
        uint64_t m = 1ull << i;
        if ((x ^ y) & m) return (x & m) ? -1 : 1;
    }
    return 0;
}

/* Candidates of (n, ord, w) in order, by sorting the candidate set with the
 * order's comparator.  Returns the count, or ORC_EINVAL / ORC_ENOMEM (also
 * when the count exceeds cap). */
int64_t orc64_order_list(int n, int ord, int w, uint64_t *out, int64_t cap) {
    if (!valid_args64(n, ord, w)) return ORC_EINVAL;
    uint64_t cnt = orc64_candidate_count(n, w);
    if (cnt > (uint64_t)cap) return ORC_ENOMEM;
    int64_t k = 0;
    if (w < 0) {
        for (uint64_t v = 0; v < cnt; ++v) out[k++] = v;
    } else if (w == 0) {
        out[k++] = 0;
    } else {
        /* every weight-w pattern once: Gosper's rule from the smallest */
        uint64_t y = (w == 64) ? ~0ull : ((1ull << w) - 1);
        for (uint64_t i = 0; i < cnt; ++i) {
            out[k++] = y;
            if (i + 1 < cnt) {
                uint64_t c = y & (~y + 1), r = y + c;
                y = (((r ^ y) >> 2) / c) | r;
            }
        }
    }
    int (*cmp)(const void *, const void *) =
        ord == ORC_LEX ? cmp64_lex : ord == ORC_GRAY ? cmp64_gray
        : ord == ORC_GRLEX ? cmp64_grlex : cmp64_grevlex;
    qsort(out, (size_t)k, sizeof(uint64_t), cmp);
    return k;
}

/* The greedy of Section 4 (orth = 1: with the Section 4.4 constraint),
 * pairwise, over the sorted candidate list.  Writes up to cap codewords and
 * their candidate indices; returns |C|. */
int64_t orc64_greedy(int n, int d, int ord, int w, int orth, uint64_t *out, int64_t *pos,
                     int64_t cap) {
    if (!valid_args64(n, ord, w) || d < 0) return ORC_EINVAL;
    uint64_t cnt = orc64_candidate_count(n, w);
    if (cnt > (1ull << 28)) return ORC_ENOMEM;
    uint64_t *cand = (uint64_t *)malloc((cnt ? cnt : 1) * sizeof(uint64_t));
    uint64_t *C = (uint64_t *)malloc((cnt ? cnt : 1) * sizeof(uint64_t));
    if (!cand || !C) { free(cand); free(C); return ORC_ENOMEM; }
    int64_t m = orc64_order_list(n, ord, w, cand, (int64_t)cnt);
    if (m < 0) { free(cand); free(C); return m; }
    int64_t size = 0;
    for (int64_t idx = 0; idx < m; ++idx) {
        uint64_t x = cand[idx];
        int ok = !orth || (popc64(x) % 2) == 0;
        for (int64_t j = 0; ok && j < size; ++j) {
            if (popc64(x ^ C[j]) < d) ok = 0;
            if (orth && (popc64(x & C[j]) % 2) != 0) ok = 0;
        }
        if (ok) {
            if (size < cap) { out[size] = x; if (pos) pos[size] = idx; }
            C[size++] = x;
        }
    }
    free(cand);
    free(C);
    return size;
}

/* O3 for up to 64 coordinates (no constraint): 0 iff L[0..len) is exactly
 * the greedy output; the codes are those of orc_verify. */
int orc64_verify(int n, int d, int ord, int w, const uint64_t *L, int64_t len) {
    if (!valid_args64(n, ord, w)) return 1;
    for (int64_t i = 0; i < len; ++i)
        for (int64_t j = 0; j < i; ++j)
            if (popc64(L[i] ^ L[j]) < d) return 2;
    uint64_t cnt = orc64_candidate_count(n, w);
    if (cnt > (1ull << 28)) return 4;
    uint64_t *cand = (uint64_t *)malloc((cnt ? cnt : 1) * sizeof(uint64_t));
    if (!cand) return 4;
    int64_t m = orc64_order_list(n, ord, w, cand, (int64_t)cnt);
    int64_t i = 0;
    int rc = 0;
    for (int64_t q = 0; q < m && rc == 0; ++q) {
        uint64_t x = cand[q];
        if (i < len && L[i] == x) { ++i; continue; }
        int covered = 0;
        for (int64_t j = 0; j < i; ++j)
            if (popc64(x ^ L[j]) <= d - 1) { covered = 1; break; }
        if (!covered) rc = 3;
    }
    free(cand);
    if (rc) return rc;
    return i == len ? 0 : 1;
}

/* ---- Cartesian product of two codes (Section 5, "Recursion in Self
 * orthogonal codes") ------------------------------------------------------- */
/* Every codeword of A followed by every codeword of B: out[i * nb + j] =
 * (A[i] << len_b) | B[j], A's words outermost.  Returns na * nb, or
 * ORC_EINVAL when the words would not fit 64 bits. */
int64_t orc64_product(const uint64_t *A, int64_t na, const uint64_t *B, int64_t nb, int len_a,
                      int len_b, uint64_t *out, int64_t cap) {
    if (len_a < 0 || len_b < 0 || len_a + len_b > 64 || len_a + len_b < 1) return ORC_EINVAL;
    int64_t k = 0;
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j) {
            uint64_t hi = (len_b == 64) ? 0 : (A[i] << len_b);
            if (k < cap) out[k] = hi | B[j];
            ++k;
        }
    return k;
}
