// gc_steps.cu -- the steps of the sweep as stand-alone launches (ordering,
// block distance test, in-order resolve, ball marking, find-unmarked scan).
// They share the device primitives of the persistent sweep (gc_block.cuh),
// so a test of a step exercises the code the sweep runs.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "gc_block.cuh"
#include "gc_internal.h"

namespace gc {

constexpr int kStepChunk = 4096;

__device__ void load_binom(uint32_t (*C)[kMaxN + 1]) {
    for (int q = threadIdx.x; q < (kMaxN + 1) * (kMaxN + 1); q += blockDim.x) {
        const int p = q / (kMaxN + 1), k = q % (kMaxN + 1);
        uint64_t r = (k <= p) ? 1u : 0u;
        for (int i = 1; i <= k && k <= p; ++i) r = r * (uint64_t)(p - k + i) / (uint64_t)i;
        C[p][k] = (uint32_t)r;
    }
    __syncthreads();
}

static Order make_order(const HostProblem& p, bool filter) { return order_of(p, filter, false); }

static int grid_for(uint64_t items, int per_block) {
    uint64_t g = (items + per_block - 1) / per_block;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(g, 65535ull * 8));
}

static int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return GC_OK;
}

// ---------------------------------------------------------------- ordering
__global__ void unrank_kernel(const __grid_constant__ Order o, uint64_t rank0, uint64_t count,
                              uint32_t* out) {
    __shared__ uint32_t C[kMaxN + 1][kMaxN + 1];
    load_binom(C);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x;
        unrank(o, C, rank0 + i, x);
        out[i] = x;
    }
}

int launch_unrank(const HostProblem& p, uint64_t rank0, uint64_t count, uint32_t* d_vec,
                  cudaStream_t s) {
    if (count == 0) return GC_OK;
    Order o = make_order(p, false);
    unrank_kernel<<<grid_for(count, 256 * 16), 256, 0, s>>>(o, rank0, count, d_vec);
    return check_launch("unrank");
}

__global__ void rank_kernel(const __grid_constant__ Order o, const uint32_t* vec, uint64_t count,
                            uint64_t* out) {
    __shared__ uint32_t C[kMaxN + 1][kMaxN + 1];
    load_binom(C);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = rank_of(o, C, vec[i]);
}

int launch_rank(int n, int ord, const uint32_t* d_vec, uint64_t count, uint64_t* d_rank,
                cudaStream_t s) {
    if (count == 0) return GC_OK;
    HostProblem p{};
    std::string why;
    if (!make_problem(n, 2, ord, -1, &p, &why)) return fail(GC_ERR_INVALID, why);
    Order o = make_order(p, false);
    rank_kernel<<<grid_for(count, 256 * 16), 256, 0, s>>>(o, d_vec, count, d_rank);
    return check_launch("rank");
}

// ---------------------------------------------------------------- block test
struct StepSmem {
    __align__(16) uint32_t x[kStepChunk];
    __align__(16) uint32_t off[kStepChunk];
    __align__(16) uint32_t acc[kStepChunk];
    __align__(16) uint32_t tile[kStepChunk * 4];
    uint32_t M[kResolveWords][kResolveBlock];
    uint8_t dead[kStepChunk];
    BlockScratch bs;
};

// Each CTA takes kStepChunk candidates and filters them against the code,
// staged through shared memory in tiles, newest tile first.
__global__ void __launch_bounds__(kBlock, 1)
    block_test_kernel(int d, const uint32_t* cand, uint64_t ncand, const uint32_t* code,
                      uint64_t ncode, uint8_t* alive) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    StepSmem& s = *reinterpret_cast<StepSmem*>(smem_raw);
    const uint64_t c0 = (uint64_t)blockIdx.x * kStepChunk;
    if (c0 >= ncand) return;
    const uint32_t nc = (uint32_t)min((uint64_t)kStepChunk, ncand - c0);
    for (uint32_t i = threadIdx.x; i < nc; i += kBlock) {
        s.x[i] = cand[c0 + i];
        s.off[i] = i;
    }
    __syncthreads();
    uint32_t na = nc;
    uint64_t nt = 0;
    const uint32_t T = kStepChunk * 4;
    for (uint64_t top = ncode; top > 0 && na > 0;) {
        const uint64_t lo = top > T ? top - T : 0;
        const uint32_t len = (uint32_t)(top - lo);
        for (uint32_t i = threadIdx.x; i < len; i += kBlock) s.tile[i] = code[lo + i];
        __syncthreads();
        na = block_filter<false>(s.bs, s.x, s.off, s.dead, na, s.tile, 0, len, d, nt);
        top = lo;
    }
    for (uint32_t i = threadIdx.x; i < nc; i += kBlock) alive[c0 + i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < na; i += kBlock) alive[c0 + s.off[i]] = 1;
}

int launch_block_test(int d, const uint32_t* d_cand, uint64_t ncand, const uint32_t* d_code,
                      uint64_t ncode, uint8_t* d_alive, cudaStream_t st) {
    if (ncand == 0) return GC_OK;
    const size_t smem = sizeof(StepSmem);
    cudaError_t e = cudaFuncSetAttribute(block_test_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    const uint64_t blocks = (ncand + kStepChunk - 1) / kStepChunk;
    if (blocks > 0x7fffffffull) return fail(GC_ERR_INVALID, "too many candidates");
    block_test_kernel<<<(unsigned)blocks, kBlock, smem, st>>>(d, d_cand, ncand, d_code, ncode,
                                                              d_alive);
    return check_launch("block_test");
}

// ---------------------------------------------------------------- resolve
__global__ void __launch_bounds__(kBlock, 1)
    resolve_kernel(int d, const uint32_t* cand, uint32_t ncand, uint32_t* acc_idx,
                   uint32_t* count, int sparse) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    StepSmem& s = *reinterpret_cast<StepSmem*>(smem_raw);
    for (uint32_t i = threadIdx.x; i < ncand; i += kBlock) {
        s.x[i] = cand[i];
        s.off[i] = i;
    }
    __syncthreads();
    uint64_t nt = 0;
    // the bucketed resolver first (it gives up on lists with many
    // conflicts), then the conflict-matrix resolver
    uint32_t na = 0;
    const bool done = sparse && sparse_resolve(s.bs, s.x, s.off, s.dead, ncand, d, s.acc, s.tile,
                                               &s.M[0][0], (ncand * ncand) >> 3, nt, &na);
    if (!done) na = block_resolve(s.bs, s.x, s.off, s.dead, ncand, d, s.acc, s.tile, s.M, nt);
    for (uint32_t i = threadIdx.x; i < na; i += kBlock) acc_idx[i] = s.tile[i];
    if (threadIdx.x == 0) *count = na;
}

int launch_resolve(int d, const uint32_t* d_cand, uint32_t ncand, uint32_t* d_acc,
                   uint32_t* d_count, cudaStream_t st) {
    if (ncand > (uint32_t)kStepChunk) return fail(GC_ERR_INVALID, "gc_resolve: ncand > 4096");
    const size_t smem = sizeof(StepSmem);
    cudaError_t e = cudaFuncSetAttribute(resolve_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(GC_ERR_CUDA, cudaGetErrorString(e));
    const char* env = std::getenv("GC_SPARSE");
    const int sparse = (env && std::strcmp(env, "0") == 0) ? 0 : 1;
    resolve_kernel<<<1, kBlock, smem, st>>>(d, d_cand, ncand, d_acc, d_count, sparse);
    return check_launch("resolve");
}

// ---------------------------------------------------------------- marking
__global__ void bitmap_mark_kernel(int n, const uint32_t* code, uint64_t ncode,
                                   const uint32_t* hball, uint32_t hlen, uint32_t* bitmap) {
    __shared__ uint32_t lowball[8][32];
    const int nl = n < 5 ? n : 5;
    for (int q = threadIdx.x; q < 8 * 32; q += blockDim.x) {
        const int r = q / 32, c = q % 32;
        uint32_t m = 0;
        for (int y = 0; y < (1 << nl); ++y)
            if (__popc((unsigned)(y ^ c)) <= r) m |= 1u << y;
        lowball[r][c] = m;
    }
    __syncthreads();
    const uint64_t total = ncode * hlen;
    const uint32_t vmask = n >= 32 ? kFull : ((1u << n) - 1u);  // keep words inside the map
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / hlen;
        const uint32_t j = (uint32_t)(q - i * hlen);
        const uint32_t c = code[i] & vmask;
        const uint32_t e = hball[j];
        atomicOr(bitmap + ((c >> 5) ^ (e >> 3)), lowball[e & 7u][c & 31u]);
    }
}

int launch_bitmap_mark(int n, int d, const uint32_t* d_code, uint64_t ncode, uint32_t* d_bitmap,
                       uint32_t* d_hball, cudaStream_t st) {
    if (ncode == 0 || d <= 0) return GC_OK;
    const uint64_t hlen = high_ball_len(n, d);
    const int nh = n > 5 ? n - 5 : 0;
    int rc = launch_high_ball(nh, d - 1, d_hball, (uint32_t)hlen, st);
    if (rc) return rc;
    bitmap_mark_kernel<<<grid_for(ncode * hlen, 256 * 8), 256, 0, st>>>(n, d_code, ncode, d_hball,
                                                                       (uint32_t)hlen, d_bitmap);
    return check_launch("bitmap_mark");
}

// ---------------------------------------------------------------- scan
// Pass 1: clear-bit count of each CTA's contiguous range of ranks.
// Pass 2: one CTA turns the counts into exclusive offsets (in place).
// Pass 3: each CTA writes its clear candidates, in rank order, at its offset.
__global__ void __launch_bounds__(kBlock)
    scan_pass(const __grid_constant__ Order o, const uint32_t* bitmap, uint64_t rank0,
              uint64_t count, uint64_t per_block, uint64_t* counts, uint32_t* out,
              uint64_t capacity, int write) {
    __shared__ uint32_t C[kMaxN + 1][kMaxN + 1];
    __shared__ BlockScratch bs;
    __shared__ uint32_t xs[kBlock];
    load_binom(C);
    const uint64_t b0 = rank0 + (uint64_t)blockIdx.x * per_block;
    const uint64_t b1 = min(b0 + per_block, rank0 + count);
    uint64_t base = write ? counts[blockIdx.x] : 0;
    uint64_t found = 0;
    for (uint64_t t0 = b0; t0 < b1; t0 += kBlock) {
        const uint64_t r = t0 + threadIdx.x;
        uint32_t x = 0;
        bool keep = false;
        if (r < b1) {
            keep = unrank(o, C, r, x);
            if (keep) keep = !((bitmap[x >> 5] >> (x & 31u)) & 1u);
        }
        const uint32_t got = block_append(bs, keep, x, 0, xs, nullptr, 0);
        if (write)
            for (uint32_t i = threadIdx.x; i < got; i += kBlock)
                if (base + found + i < capacity) out[base + found + i] = xs[i];
        found += got;
        __syncthreads();
    }
    if (!write && threadIdx.x == 0) counts[blockIdx.x] = found;
}

__global__ void scan_offsets(uint64_t* counts, int nblocks, uint64_t* total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint64_t acc = 0;
        for (int i = 0; i < nblocks; ++i) {
            const uint64_t c = counts[i];
            counts[i] = acc;
            acc += c;
        }
        *total = acc;
    }
}

int launch_bitmap_scan(const HostProblem& p, const uint32_t* d_bitmap, uint64_t rank0,
                       uint64_t count, uint32_t* d_out, uint64_t capacity, uint64_t* d_found,
                       uint64_t* d_counts, cudaStream_t st) {
    if (count == 0) {
        cudaError_t e = cudaMemsetAsync(d_found, 0, sizeof(uint64_t), st);
        return e == cudaSuccess ? GC_OK : fail(GC_ERR_CUDA, cudaGetErrorString(e));
    }
    const int blocks = (int)std::min<uint64_t>(kScanMaxBlocks, (count + kBlock - 1) / kBlock);
    const uint64_t per = (count + blocks - 1) / blocks;
    Order o = make_order(p, p.filter);
    uint64_t* counts = d_counts;  // kScanMaxBlocks entries
    scan_pass<<<blocks, kBlock, 0, st>>>(o, d_bitmap, rank0, count, per, counts, d_out, capacity, 0);
    int rc = check_launch("scan count");
    if (rc) return rc;
    scan_offsets<<<1, 32, 0, st>>>(counts, blocks, d_found);
    if ((rc = check_launch("scan offsets"))) return rc;
    scan_pass<<<blocks, kBlock, 0, st>>>(o, d_bitmap, rank0, count, per, counts, d_out, capacity, 1);
    return check_launch("scan write");
}

// ---------------------------------------------------------------- product
// Cartesian product of two codes (Section 5): out[i * nb + j] =
// (a[i] << len_b) | b[j].  Grid-stride over the na * nb outputs.
template <typename W>
__global__ void product_kernel(const W* a, uint64_t na, const W* b, uint64_t nb, int len_b,
                               W* out) {
    const uint64_t total = na * nb;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / nb, j = q - i * nb;
        out[q] = (W)((a[i] << len_b) | b[j]);
    }
}

template <typename W>
int launch_product(const W* d_a, uint64_t na, int len_a, const W* d_b, uint64_t nb, int len_b,
                   W* d_out, uint64_t capacity, cudaStream_t s) {
    const int bits = (int)(8 * sizeof(W));
    if (len_a < 1 || len_b < 1 || len_a + len_b > bits)
        return fail(GC_ERR_INVALID, "product: need 1 <= len_a, len_b and len_a + len_b <= " +
                                        std::to_string(bits));
    if ((na && !d_a) || (nb && !d_b)) return fail(GC_ERR_INVALID, "null pointer");
    if (na && nb > UINT64_MAX / na) return fail(GC_ERR_INVALID, "product too large");
    const uint64_t total = na * nb;
    if (total > capacity) return fail(GC_ERR_CAPACITY, "product: output capacity too small");
    if (total == 0) return GC_OK;
    if (!d_out) return fail(GC_ERR_INVALID, "null pointer");
    product_kernel<W><<<grid_for(total, 256 * 8), 256, 0, s>>>(d_a, na, d_b, nb, len_b, d_out);
    return check_launch("product");
}

}  // namespace gc

using namespace gc;

extern "C" int gc_product(const uint32_t* d_a, uint64_t na, int len_a, const uint32_t* d_b,
                          uint64_t nb, int len_b, uint32_t* d_out, uint64_t capacity,
                          void* stream) {
    return launch_product<uint32_t>(d_a, na, len_a, d_b, nb, len_b, d_out, capacity,
                                    (cudaStream_t)stream);
}

extern "C" int gc_product64(const uint64_t* d_a, uint64_t na, int len_a, const uint64_t* d_b,
                            uint64_t nb, int len_b, uint64_t* d_out, uint64_t capacity,
                            void* stream) {
    return launch_product<uint64_t>(d_a, na, len_a, d_b, nb, len_b, d_out, capacity,
                                    (cudaStream_t)stream);
}
