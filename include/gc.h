/*
 * gc.h -- C ABI of libgc, a GB300 (sm_103a) library for the ordered greedy
 * construction of binary codes.
 *
 * The method (Section 4, "Greedy Algorithms and Different Orderings"): order
 * the vectors of F_2^n, optionally only those of weight w; walk the order from
 * its first vector (the zero vector when no weight is given) and append a
 * vector to the code C iff its Hamming distance to every codeword already in C
 * is at least d.  Hamming distance is popcount(x XOR c) (Section 5.2).  The
 * four orderings are those Section 4.2 names.
 *
 * Conventions shared by every entry point:
 *  - A length-n vector is the low n bits of a uint32_t, coordinate 1 in the
 *    most significant of those bits ("011" is 3).  1 <= n <= 32, except for
 *    the wide entry points (gc_*64), whose vectors are the low n bits of a
 *    uint64_t with 1 <= n <= 64.
 *  - Orderings (the paper names them but defines none; these are the readings):
 *      GC_ORDER_LEX      ascending integer (Example 1 of Section 4.1).
 *      GC_ORDER_GRAY     binary-reflected Gray code: rank r -> r ^ (r >> 1).
 *      GC_ORDER_GRLEX    weight ascending, then ascending integer.
 *      GC_ORDER_GREVLEX  weight ascending; within a weight, a precedes b iff
 *                        a has the 1 at the lowest bit where a and b differ
 *                        (textbook graded reverse lexicographic order).
 *  - Constant weight: weight_or_none in [0, n] keeps only weight-w vectors, in
 *    the same relative order; GC_NO_WEIGHT (-1) keeps all 2^n vectors.
 *  - "Rank space" of a problem: 2^n ranks when no weight is given or the
 *    order is BASIS (B-ordering ranks of the wrong weight are skipped);
 *    C(n, w) ranks for LEX, GRAY, GRLEX and GREVLEX with a weight: rank i is
 *    the i-th weight-w vector of the order, found in closed form (LEX and
 *    GRLEX restricted to one weight are the same sequence).
 *  - Return value: GC_OK (0) or a positive GC_ERR_* code; no exception or
 *    abort crosses the ABI.  gc_strerror() names the code; gc_last_error()
 *    returns a one-line message about the most recent failure on the calling
 *    thread.
 *  - Pointers marked "device" must be device memory of the current CUDA
 *    device (or managed memory); "host" pointers are ordinary host memory.
 *    Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes.
 *  - Asynchronous entry points take a cudaStream_t as void*; NULL is the
 *    legacy default stream.  They return after launching; errors detected on
 *    the device (a bounded wait that expired, an overflow) are reported in the
 *    gc_stats block they fill, readable once the stream has completed.
 */
#ifndef GC_H_
#define GC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GC_ORDER_LEX = 0,
    GC_ORDER_GRAY = 1,
    GC_ORDER_GRLEX = 2,
    GC_ORDER_GREVLEX = 3,
    /* Section 4.3: the B-ordering of an ordered basis b_1..b_n of F_2^n --
     * rank r is the XOR of the b_j over the set bits j-1 of r (0, b_1, b_2,
     * b_2+b_1, b_3, ...).  Needs gc_problem.basis; 2^n ranks. */
    GC_ORDER_BASIS = 4
} gc_ordering;

#define GC_NO_WEIGHT (-1)

enum {
    GC_OK = 0,
    GC_ERR_INVALID = 1,     /* argument out of range */
    GC_ERR_CAPACITY = 2,    /* output buffer too small; nothing was written
                               past the capacity, *inout_count = required */
    GC_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    GC_ERR_OOM = 4,         /* device or host allocation failed */
    GC_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    GC_ERR_UNSUPPORTED = 6, /* valid request the library does not handle */
    GC_ERR_INTERNAL = 7     /* an internal consistency check failed */
};

/* Sweep strategy.  AUTO lets gc_plan() choose. */
typedef enum {
    GC_STRATEGY_AUTO = 0,
    GC_STRATEGY_DISTANCE = 1, /* test each candidate against the code */
    GC_STRATEGY_BITMAP = 2,   /* exclusion bitmap of radius-(d-1) balls */
    /* The same exclusion bitmap, with every SM taking part in every window
     * of the one code (lockstep windows separated by grid-wide barriers;
     * no resolver pipeline).  gc_plan() picks it for bitmap problems of at
     * least 2^GC_GRID_MIN_LOG2 candidates; a batch or a server runs such a
     * job as GC_STRATEGY_BITMAP.  n <= 32, no orthogonality constraint. */
    GC_STRATEGY_BITMAP_GRID = 3
} gc_strategy;

/* Smallest rank space (log2) for which gc_plan() runs a bitmap problem with
 * GC_STRATEGY_BITMAP_GRID. */
#define GC_GRID_MIN_LOG2 24

/* Extra constraints on the greedy. */
enum {
    GC_CONSTRAINT_NONE = 0,
    /* Section 4.4: self-orthogonal greedy codes -- a candidate must also
     * have even weight (be orthogonal to itself) and be orthogonal to every
     * codeword so far (popcount(x AND c) even).  Distance strategy only. */
    GC_CONSTRAINT_SELF_ORTHOGONAL = 1
};

/* One problem instance. */
typedef struct {
    int n;              /* code length, 1..32 (1..64 for the gc_*64 entries) */
    int d;              /* minimum distance, >= 0 (d <= 1 accepts all) */
    int ordering;       /* gc_ordering */
    int weight;         /* GC_NO_WEIGHT or 0..n */
    int constraint;     /* GC_CONSTRAINT_* (0 when the struct is zeroed) */
    const uint32_t *basis; /* GC_ORDER_BASIS: host array of n linearly
                              independent vectors, basis[j-1] = b_j (read
                              during the call); NULL otherwise */
} gc_problem;

/* Launch plan chosen by gc_plan() (or given by the caller). */
typedef struct {
    int strategy;          /* gc_strategy, never AUTO after gc_plan() */
    int grid;              /* CTAs of the persistent sweep (0 = all SMs) */
    int block;             /* threads per CTA (multiple of 32, <= 1024) */
    uint32_t window_min;   /* smallest window of ranks tested per step */
    uint32_t window_max;   /* largest window */
    uint32_t survivor_target; /* window sizing aims at this many survivors
                                 (gc_plan: 512 distance, 1024 bitmap; 4096
                                 lex/Gray and 2048 graded for bitmap sweeps
                                 of >= 2^28 candidates; 8800 for the grid
                                 strategy, whose windows end after 8192 and
                                 aim lower where survivors conflict densely) */
} gc_plan_t;

/* Counters filled by the sweep (device-side writes, read after sync). */
typedef struct {
    uint64_t codewords;        /* |C| (the true size even past capacity) */
    uint64_t candidates;       /* candidates swept (rank-space size) */
    uint64_t dense_tests;      /* sum over candidates of |C before it|
                                  (0 when ranks are skipped: BASIS with a
                                  weight, self-orthogonal problems) */
    uint64_t executed_tests;   /* distance tests the kernels executed */
    uint64_t marks;            /* bitmap words OR-ed by ball marking */
    uint64_t windows;          /* sequential window steps */
    uint64_t survivors;        /* candidates that reached the resolver */
    int32_t status;            /* GC_OK or GC_ERR_TIMEOUT / _INTERNAL */
    int32_t strategy;          /* strategy that ran */
    /* Diagnostic: SM cycles the first CTA of the job's group (or CTA
     * GC_TIMING_CTA of it) spent, summed over windows, in [0] ball marking,
     * [1] candidate generation and bitmap lookup, [2] the newest-codeword
     * test and compaction, [3] the split test against older codewords,
     * [4] publishing and waiting for the group, [5] gathering survivors,
     * [6] resolving (a pipelined job's generator CTAs: searching the window's
     * conflicting pairs), [7] committing; within [6]: [8] conflict matrix or
     * bucketed search, [9] resolution rounds, [10] appending and the kill
     * step; [11] counts resolution rounds (not cycles).  The grid bitmap
     * sweep (GC_STRATEGY_BITMAP_GRID) uses them as: [0] output of the
     * previous window's accepts, [1] generation and bitmap probes, [2] ball
     * marks, [3] row probes, [4] grid barriers, [5] gather, [6] pair tests,
     * [7] publishing kills and pairs, [8] deciding windows without pairs,
     * [9] with pair rounds, [10] with conflict matrices; [11] rounds. */
    uint64_t phase_cycles[12];
    /* Pipelined bitmap jobs in large groups: windows decided from the list
     * of their conflicting pairs that the group's generator CTAs found, and
     * windows where that list overflowed, so the conflict matrices decided
     * them. */
    uint64_t pair_windows;
    uint64_t pair_fallbacks;
} gc_stats;

/* ---- information ------------------------------------------------------ */

/* Static string naming an error code. */
const char *gc_strerror(int err);

/* One-line description of the last failure on this thread ("" if none). */
const char *gc_last_error(void);

/* Rank-space size of a problem (see "Rank space" above), n <= 64; 0 if
 * invalid or not representable (2^64 ranks at n = 64). */
uint64_t gc_candidate_count(int n, int weight_or_none, int ordering);

/* An upper bound on |C| that is always safe as an output capacity:
 * min(number of weight-admissible candidates, sphere-packing bound
 * floor(2^n / V(n, floor((d-1)/2)))) -- the radius-floor((d-1)/2) balls
 * around codewords are disjoint.  (A self-orthogonal code also has at most
 * 2^floor(n/2) words: its span is a self-orthogonal linear code; the
 * problem-struct entry points use that too.)  n <= 64.  Returns 0 for
 * invalid arguments. */
uint64_t gc_capacity_bound(int n, int d, int weight_or_none);

/* Choose a strategy and launch shape for a problem on the current device.
 * The cost model compares the estimated number of distance tests of the
 * distance strategy with the number of bitmap words the ball marking of the
 * bitmap strategy would OR (the paper's own observation, Section 6, is that
 * the best parallel form depends on how d compares with n).  Returns GC_OK
 * or GC_ERR_INVALID. */
int gc_plan(const gc_problem *prob, gc_plan_t *out_plan);

/* Measured choice: runs the candidate plans (distance or bitmap strategy,
 * survivor targets 256/512/1024/2048, all / a quarter / an eighth of the
 * SMs) for this problem (n <= 32) on the current device, returns the
 * fastest in *best and its time in *best_ms (may be NULL), and appends it
 * to the tuning cache if one is installed.  Synchronous; allocates its own
 * scratch.  GC_ORDER_BASIS problems are tuned but not cached (the basis is
 * not part of the key). */
int gc_autotune(const gc_problem *prob, gc_plan_t *best, double *best_ms);

/* Installs a plain-text tuning cache file (NULL or "" removes it; default:
 * the GC_TUNE_CACHE environment variable).  While installed, gc_plan() and
 * every entry point that plans by itself use the cached plan of a problem
 * (key: n, d, ordering, weight, constraint, device name; last entry wins). */
int gc_set_tune_cache(const char *path);

/* ---- the whole sweep ---------------------------------------------------- */

/* Device bytes of scratch gc_generate_async() needs for this problem and
 * plan (plan NULL = gc_plan()'s choice).  0 on invalid arguments. */
size_t gc_workspace_size(const gc_problem *prob, const gc_plan_t *plan);

/* Generate the greedy code (Section 4) on the current device, synchronously.
 *   out_codewords  host or device buffer of *inout_count uint32_t words;
 *                  receives the code in acceptance (= rank) order.
 *   inout_count    in: capacity in words; out: |C|.
 * Returns GC_ERR_CAPACITY (with *inout_count = |C| and the first capacity
 * words written) if the buffer is too small.  Allocates its scratch with
 * cudaMallocAsync on an internal stream and frees it before returning. */
int gc_generate(int n, int d, int ordering, int weight_or_none,
                uint32_t *out_codewords, uint64_t *inout_count);

/* Stream-ordered form.  All pointers are device pointers:
 *   d_out        capacity words for the code (acceptance order);
 *   d_stats      one gc_stats block, overwritten;
 *   workspace    >= gc_workspace_size() bytes, 256-byte aligned, owned by
 *                the caller and not touched after the stream passes this
 *                call;
 *   plan         NULL = gc_plan()'s choice.
 * The code size is d_stats->codewords; words past capacity are not written.
 * Returns GC_OK after a successful launch. */
int gc_generate_async(const gc_problem *prob, const gc_plan_t *plan,
                      uint32_t *d_out, uint64_t capacity, gc_stats *d_stats,
                      void *workspace, size_t workspace_bytes, void *stream);

/* ---- wide vectors: 1 <= n <= 64, uint64_t words ------------------------- */
/* The same sweep for codes longer than 32 (Section 7 builds constant-weight
 * codes up to length 35).  Vectors are the low n bits of a uint64_t,
 * coordinate 1 the most significant of them.  Orders LEX, GRAY, GRLEX and
 * GREVLEX, with or without a weight, and the self-orthogonal constraint;
 * GC_ORDER_BASIS is not supported here (GC_ERR_INVALID).  n = 64 needs a
 * weight (the rank space must fit a uint64).  The
 * distance strategy only: an explicit GC_STRATEGY_BITMAP plan gives
 * GC_ERR_UNSUPPORTED (0 from gc_workspace_size64), AUTO takes DISTANCE.
 * Problems with n <= 32 are accepted too and give the same code as the
 * narrow entries, zero-extended.  Arguments, ownership and errors are those
 * of the narrow forms, with words of 8 bytes. */
size_t gc_workspace_size64(const gc_problem *prob, const gc_plan_t *plan);
int gc_generate64(int n, int d, int ordering, int weight_or_none,
                  uint64_t *out_codewords, uint64_t *inout_count);
int gc_generate64_async(const gc_problem *prob, const gc_plan_t *plan,
                        uint64_t *d_out, uint64_t capacity, gc_stats *d_stats,
                        void *workspace, size_t workspace_bytes, void *stream);

/* ---- batches: many codes in one launch --------------------------------- */

/* One code of a batch. */
typedef struct {
    gc_problem prob;
    int strategy;          /* gc_strategy; AUTO = gc_plan()'s choice */
    uint32_t *d_out;       /* device, capacity words, acceptance order */
    uint64_t capacity;
    gc_stats *d_stats;     /* device, one block per job */
} gc_job;

/* Device bytes of scratch gc_batch_generate_async() needs (0 if invalid).
 * ngroups as for gc_batch_generate_async. */
size_t gc_batch_workspace_size(const gc_job *jobs, int njobs, int ngroups);

/* Generates every job's code (Section 4) in ONE persistent cooperative
 * launch.  The SMs are split into ngroups groups (ngroups <= 0: one group per
 * job, sized by an estimate of its work, for batches of up to a quarter as
 * many jobs as SMs; groups of four SMs otherwise).  With one job per group
 * every job runs at once on its own SMs; with more jobs than groups the
 * groups are of equal size and each claims the next job, longest first, as
 * it becomes free (GC_BATCH_DYNAMIC=0: a fixed longest-first assignment), so
 * independent codes run concurrently on disjoint SMs.
 * Each job's result equals what gc_generate_async gives for it alone.
 * workspace: device, >= gc_batch_workspace_size() bytes, 256-byte aligned,
 * owned by the caller.  Per-job status is in its gc_stats. */
int gc_batch_generate_async(const gc_job *jobs, int njobs, int ngroups,
                            void *workspace, size_t workspace_bytes,
                            void *stream);

/* Batches launched many times (and CUDA graphs).  gc_batch_create does the
 * host work of gc_batch_generate_async once: it checks and plans the jobs,
 * lays out the workspace and fills it on `stream` (job and group
 * descriptors, ball tables), and returns a handle.  The workspace (>=
 * gc_batch_workspace_size bytes, 256-byte aligned) and the jobs' d_out and
 * d_stats buffers stay owned by the caller and must outlive the handle.
 * gc_batch_launch then runs the batch on `stream`: it resets the per-launch
 * state in the workspace (memsets of the error word and of each group's
 * flags) and launches the persistent sweep,
 * nothing else -- only stream operations, so it can be captured into a CUDA
 * graph (stream capture) and the graph replayed.  Each run overwrites the
 * outputs and stats with the same codes.  Runs of one handle must not
 * overlap (they share the workspace).  gc_batch_destroy frees the host
 * handle only.  Errors as for gc_batch_generate_async. */
typedef struct gc_batch gc_batch;
int gc_batch_create(const gc_job *jobs, int njobs, int ngroups, void *workspace,
                    size_t workspace_bytes, void *stream, gc_batch **out);
int gc_batch_launch(gc_batch *b, void *stream);
int gc_batch_destroy(gc_batch *b);

/* Measured per-instance plans for a batch (Section 6 observes that the best
 * parallel form depends on how d compares with n; here it is measured per
 * code, where it will run).  The jobs are laid out as gc_batch_create would
 * lay them out with ngroups groups; then, for up to max_jobs (< 0: all)
 * distinct problems, costliest first by the planner's cost model, every
 * candidate plan -- distance or pipelined bitmap strategy (where each
 * applies) x survivor target 256 / 512 / 1024 / 2048, which sets the window
 * of B candidates per step -- runs once warm and once timed on as many CTAs
 * as the batch gives the job, and the fastest is appended to the installed
 * tuning cache with grid 0 (a cached grid would shrink a batch's launch).
 * gc_batch_create, gc_batch_generate_async and gc_plan then use those plans.
 * Reads only jobs[j].prob (the output and statistics pointers may be NULL).
 * Needs a tuning cache (GC_ERR_INVALID otherwise); B-orderings are skipped
 * (their basis is not part of the key).  Synchronous; allocates its own
 * scratch.  *tuned receives how many problems were tuned. */
int gc_batch_autotune(const gc_job *jobs, int njobs, int ngroups, int max_jobs, int *tuned);

/* ---- serving: requests admitted while others run ------------------------ */

/* Server settings (zero fields take the defaults in brackets). */
typedef struct {
    int max_n;              /* largest n accepted [28] */
    int ngroups;            /* SM groups running requests concurrently
                               [SMs / 8] */
    size_t pool_bytes;      /* device pool for request outputs [4 GiB] */
    int queue_capacity;     /* requests in flight at most [1024] */
    uint64_t store_words;   /* per-group code store of the distance
                               strategy [2^22 words] */
    double idle_seconds;    /* the device loop leaves after this long
                               without work and is restarted by the next
                               submit [30] */
} gc_server_config;

typedef struct gc_server gc_server;

/* Starts a server on the current device: allocates its pool and scratch and
 * launches one persistent cooperative kernel (on its own stream) that keeps
 * taking requests until gc_server_destroy.  While it runs it holds every SM;
 * other work on the device waits for it. */
int gc_server_create(const gc_server_config *cfg, gc_server **out);

/* Admits one request (Section 4 problem) if a ring slot is free and its
 * output -- gc_capacity_bound words -- fits in the pool (first fit);
 * otherwise returns GC_ERR_CAPACITY and the caller retries after releasing
 * finished requests.  strategy: gc_strategy.  Non-blocking. */
int gc_server_submit(gc_server *s, const gc_problem *prob, int strategy,
                     uint64_t *request_id);

/* Reports up to max_ids requests that finished since the last poll. */
int gc_server_poll(gc_server *s, uint64_t *done_ids, int max_ids, int *ndone);

/* Copies a finished request's code (acceptance order) and statistics to
 * host memory; *inout_count: capacity in, |C| out (GC_ERR_CAPACITY if it did
 * not fit; the first capacity words are written).  host_out/host_stats may
 * be NULL. */
int gc_server_fetch(gc_server *s, uint64_t request_id, uint32_t *host_out,
                    uint64_t *inout_count, gc_stats *host_stats);

/* Returns a finished request's pool space and ring slot. */
int gc_server_release(gc_server *s, uint64_t request_id);

/* Stops the device loop (after the requests in flight), frees everything. */
int gc_server_destroy(gc_server *s);

/* Allocation-free form of gc_generate_async (the paper has no counterpart;
 * this is a service for callers).  Some callers cannot call cudaMalloc when
 * they need a code: runtimes without a device allocator of their own,
 * processes whose device memory is all handed to another framework's pool
 * up front, or latency-critical paths that cannot take an allocation's
 * synchronisation.  This entry point allocates nothing: the caller passes
 * only the output (d_out, capacity words) and d_stats, and the sweep's
 * scratch lives in one static device array of gc_noalloc_scratch_bytes()
 * bytes (32 MiB) inside the library, which every GPU that loads the library
 * holds until the process exits.
 *  - Errors: GC_ERR_INVALID for a bad problem, plan or pointer;
 *    GC_ERR_UNSUPPORTED for a valid problem whose scratch
 *    (gc_workspace_size) exceeds that size -- the message names both sizes
 *    -- or that the sweep's layout refuses (the message gives the reason).
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    stream capture.
 *  - Every call shares the one array and it keeps the last call's contents
 *    (the parts that must start at zero are cleared by each call): calls
 *    whose work overlaps on the GPU, on any streams or threads, race.
 *  - Results are identical to gc_generate_async for the same problem/plan. */
int gc_generate_noalloc(const gc_problem *prob, const gc_plan_t *plan,
                        uint32_t *d_out, uint64_t capacity, gc_stats *d_stats,
                        void *stream);

/* Size in bytes of gc_generate_noalloc's static scratch array. */
size_t gc_noalloc_scratch_bytes(void);

/* ---- Cartesian product of codes (Section 5, "Recursion in Self
 *      orthogonal codes") --------------------------------------------------- */
/* d_out[i * nb + j] = (d_a[i] << len_b) | d_b[j] for i < na, j < nb: every
 * codeword of A (length len_a) followed by every codeword of B (length
 * len_b), A's words outermost.  The product of two self-orthogonal codes is
 * self-orthogonal and its distance is the smaller of the two; Section 5
 * builds Code[n, d] from the greedy Code[n - k, d] and Code[k, d] this way
 * (its example: the self-orthogonal [8, 4] code with Code[4, 4] gives a
 * length-12 code of distance 4).  Device pointers, stream-ordered.
 * Errors: GC_ERR_INVALID unless 1 <= len_a, 1 <= len_b and len_a + len_b <=
 * 32 (gc_product) or 64 (gc_product64), or on a null pointer with a nonzero
 * count; GC_ERR_CAPACITY (nothing written) if capacity < na * nb. */
int gc_product(const uint32_t *d_a, uint64_t na, int len_a, const uint32_t *d_b,
               uint64_t nb, int len_b, uint32_t *d_out, uint64_t capacity, void *stream);
int gc_product64(const uint64_t *d_a, uint64_t na, int len_a, const uint64_t *d_b,
                 uint64_t nb, int len_b, uint64_t *d_out, uint64_t capacity, void *stream);

/* ---- the steps of the sweep, callable one at a time (for tests and for
 *      callers composing their own pipeline) ------------------------------ */

/* Step 1, ordering (Section 4.2): d_vectors[i] = the candidate of rank
 * rank0 + i, for i < count, in the problem's rank space (with a weight: the
 * weight-w vectors in order).  Device pointer; rank0 + count must not exceed
 * the rank-space size (GC_ERR_INVALID otherwise). */
int gc_unrank(int n, int ordering, int weight_or_none, uint64_t rank0,
              uint64_t count, uint32_t *d_vectors, void *stream);

/* Inverse of gc_unrank without a weight: d_ranks[i] = rank of d_vectors[i]
 * in the full 2^n order (uint64 because 2^32 ranks exist at n = 32). */
int gc_rank(int n, int ordering, const uint32_t *d_vectors, uint64_t count,
            uint64_t *d_ranks, void *stream);

/* Step 2, block distance test (Sections 4.1, 5.2): d_alive[i] = 1 iff
 * popcount(cand[i] ^ code[j]) >= d for every j < ncode, else 0.  Candidates
 * are tested in tiles against the code staged through shared memory, most
 * recent codeword first, with warp-wide early exit.  Device pointers. */
int gc_block_test(int d, const uint32_t *d_cand, uint64_t ncand,
                  const uint32_t *d_code, uint64_t ncode, uint8_t *d_alive,
                  void *stream);

/* Step 3, in-order resolve (Section 4 restricted to a list): given
 * candidates already known to clear every earlier codeword, accept them in
 * list order exactly as the serial sweep would: d_accepted[k] = list index of
 * the k-th accepted candidate, *d_count = number accepted.  ncand <= 4096
 * (GC_ERR_INVALID above).  Lists with few conflicts go through the bucketed
 * resolver, the rest through conflict matrices; both give the serial result
 * (GC_SPARSE=0 in the environment forces the matrices).  Device pointers. */
int gc_resolve(int d, const uint32_t *d_cand, uint32_t ncand,
               uint32_t *d_accepted, uint32_t *d_count, void *stream);

/* Step 4, exclusion-ball marking: for every codeword c and every e of weight
 * <= d-1, set bit (c ^ e) of the vector-indexed bitmap d_bitmap (2^n bits,
 * word i holds vectors 32i..32i+31, bit b = vector 32i+b).  Device pointers;
 * the bitmap is OR-ed into, not cleared. */
int gc_bitmap_mark(int n, int d, const uint32_t *d_code, uint64_t ncode,
                   uint32_t *d_bitmap, void *stream);

/* Step 5, find-unmarked scan: walk ranks [rank0, rank0 + count) of the
 * problem's rank space in order and write, in rank order, the vectors whose
 * bitmap bit is clear to d_out (capacity words); *d_found = how many were
 * clear (may exceed capacity; only capacity are written).  Device pointers. */
int gc_bitmap_scan(int n, int ordering, int weight_or_none,
                   const uint32_t *d_bitmap, uint64_t rank0, uint64_t count,
                   uint32_t *d_out, uint64_t capacity, uint64_t *d_found,
                   void *stream);

/* ---- diagnostics ------------------------------------------------------ */

/* Measures, on the current device, how many candidate-codeword distance
 * tests per second the SMs sustain when operands sit in registers (XOR,
 * popcount, compare): the arithmetic ceiling of the distance test (Section
 * 5.2 reduces each test to one XOR and one population count).  Runs two
 * short kernels and synchronises.  *sm_clock_hz_hint receives the device's
 * reported SM clock (may be NULL). */
int gc_probe_test_rate(double *tests_per_second, double *sm_clock_hz_hint);

/* Measures, on the current device, how many bitmap word ORs per second the
 * memory system sustains when every one goes to a pseudo-random word of a
 * region of region_bytes (a power of two from 1 MiB to 1 GiB; 0 = 64 MiB,
 * which stays in L2): the operation of the bitmap strategy's ball marking,
 * so the ceiling of its marks.  Allocates and frees its region; runs two
 * short kernels and synchronises.  GC_ERR_INVALID for a bad size. */
int gc_probe_mark_rate(double *ors_per_second, size_t region_bytes);

#ifdef __cplusplus
}
#endif

#endif /* GC_H_ */
