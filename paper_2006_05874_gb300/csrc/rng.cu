// Seeded draws of the SRHT (App. C.2): Rademacher signs and the uniformly
// random m-subset of [0, n_pad) rows, sampled without replacement.
//
// Row subset: the m indices with the smallest 64-bit Philox keys (ties broken by
// index).  The m-th smallest key K* is found by an exact radix select (four
// passes over 16-bit digits, most significant first, histograms in global
// memory); then a stable two-category compaction (key < K*, key == K*) writes
// the chosen indices in ascending order.  Keys are recomputed from Philox on
// every pass instead of being stored.
#include "common.cuh"

namespace {

__global__ void k_signs(int64_t n_pad, uint32_t level, uint32_t k0, uint32_t k1, int8_t* eps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        eps[i] = srht_sign_bit((uint64_t)i, level, k0, k1) ? (int8_t)-1 : (int8_t)1;
}

// sel[0] = prefix of K* found so far, sel[1] = rank still needed (1-based).
// hist[0..65536) per-digit counts, hist[65536..65600) per-1024-digit sums.
__global__ void k_hist16(int64_t n_pad, uint32_t level, uint32_t k0, uint32_t k1, int pass,
                         const unsigned long long* __restrict__ sel, unsigned* __restrict__ hist) {
    const int shift = 48 - 16 * pass;
    const unsigned long long prefix = sel[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = srht_row_key((uint64_t)i, level, k0, k1);
        const bool match = (pass == 0) || ((key >> (shift + 16)) == (prefix >> (shift + 16)));
        if (match) {
            const unsigned digit = (unsigned)((key >> shift) & 0xFFFFu);
            atomicAdd(&hist[digit], 1u);
            atomicAdd(&hist[65536 + (digit >> 10)], 1u);
        }
    }
}

// One CTA of 1024 threads: choose the digit holding the needed rank (first the
// 1024-digit bucket from the 64 coarse sums, then the digit inside it), extend
// the prefix, reduce the rank, clear the histogram for the next pass.
__global__ void __launch_bounds__(1024) k_pick16(int pass, unsigned long long* __restrict__ sel,
                                                 unsigned* __restrict__ hist) {
    __shared__ unsigned long long fine[1024];
    __shared__ int bucket;
    __shared__ unsigned long long before_bucket;
    const int tid = threadIdx.x;
    const int shift = 48 - 16 * pass;
    const unsigned long long need = sel[1];
    if (tid == 0) {
        unsigned long long acc = 0;
        int b = 63;
        for (int i = 0; i < 64; ++i) {
            const unsigned long long h = hist[65536 + i];
            if (acc + h >= need) {
                b = i;
                break;
            }
            acc += h;
        }
        bucket = b;
        before_bucket = acc;
    }
    __syncthreads();
    const int b = bucket;
    fine[tid] = hist[b * 1024 + tid];
    __syncthreads();
    // inclusive scan of the bucket's 1024 digits (Hillis-Steele, fixed order)
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long v = tid >= off ? fine[tid - off] : 0ull;
        __syncthreads();
        fine[tid] += v;
        __syncthreads();
    }
    const unsigned long long incl = before_bucket + fine[tid];
    const unsigned long long excl = before_bucket + (tid ? fine[tid - 1] : 0ull);
    __syncthreads();
    if (excl < need && need <= incl) {
        sel[0] |= (unsigned long long)(b * 1024 + tid) << shift;
        sel[1] = need - excl;
    }
    for (int k = tid; k < 65536 + 64; k += 1024) hist[k] = 0u;
}

constexpr int kCompactBlock = 1024;

__device__ __forceinline__ int key_category(uint64_t key, unsigned long long kstar) {
    return key < kstar ? 1 : (key == kstar ? 2 : 0);
}

// Per-block counts of category 1 (key < K*) and 2 (key == K*).
__global__ void __launch_bounds__(kCompactBlock) k_compact_count(int64_t n_pad, uint32_t level, uint32_t k0,
                                                                 uint32_t k1, const unsigned long long* sel,
                                                                 uint2* __restrict__ counts) {
    __shared__ unsigned c1s[32], c2s[32];
    const int64_t i = blockIdx.x * (int64_t)kCompactBlock + threadIdx.x;
    int cat = 0;
    if (i < n_pad) cat = key_category(srht_row_key((uint64_t)i, level, k0, k1), sel[0]);
    const unsigned b1 = __ballot_sync(0xffffffffu, cat == 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, cat == 2);
    if ((threadIdx.x & 31) == 0) {
        c1s[threadIdx.x >> 5] = __popc(b1);
        c2s[threadIdx.x >> 5] = __popc(b2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0, b = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) {
            a += c1s[w];
            b += c2s[w];
        }
        counts[blockIdx.x] = make_uint2(a, b);
    }
}

// Exclusive scan of the block counts (single CTA, sequential chunks).
__global__ void __launch_bounds__(1024) k_compact_scan(int64_t nblocks, const uint2* __restrict__ counts,
                                                       uint2* __restrict__ offsets) {
    __shared__ unsigned long long s1[1024], s2[1024];
    const int tid = threadIdx.x;
    const int64_t per = (nblocks + 1023) / 1024;
    unsigned long long a = 0, b = 0;
    for (int64_t k = tid * per; k < min(nblocks, (tid + 1) * per); ++k) {
        a += counts[k].x;
        b += counts[k].y;
    }
    s1[tid] = a;
    s2[tid] = b;
    __syncthreads();
    if (tid == 0) {
        unsigned long long x1 = 0, x2 = 0;
        for (int t = 0; t < 1024; ++t) {
            const unsigned long long v1 = s1[t], v2 = s2[t];
            s1[t] = x1;
            s2[t] = x2;
            x1 += v1;
            x2 += v2;
        }
    }
    __syncthreads();
    unsigned long long x1 = s1[tid], x2 = s2[tid];
    for (int64_t k = tid * per; k < min(nblocks, (tid + 1) * per); ++k) {
        offsets[k] = make_uint2((unsigned)x1, (unsigned)x2);
        x1 += counts[k].x;
        x2 += counts[k].y;
    }
}

__global__ void __launch_bounds__(kCompactBlock) k_compact_write(int64_t n_pad, uint32_t level, uint32_t k0,
                                                                 uint32_t k1, const unsigned long long* sel,
                                                                 const uint2* __restrict__ offsets,
                                                                 int32_t* __restrict__ rows) {
    __shared__ unsigned w1[32], w2[32];
    const int64_t i = blockIdx.x * (int64_t)kCompactBlock + threadIdx.x;
    const unsigned long long need_eq = sel[1];
    int cat = 0;
    if (i < n_pad) cat = key_category(srht_row_key((uint64_t)i, level, k0, k1), sel[0]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned b1 = __ballot_sync(0xffffffffu, cat == 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, cat == 2);
    const unsigned lanemask = (1u << lane) - 1u;
    if (lane == 0) {
        w1[warp] = __popc(b1);
        w2[warp] = __popc(b2);
    }
    __syncthreads();
    unsigned before1 = 0, before2 = 0;
    for (int w = 0; w < warp; ++w) {
        before1 += w1[w];
        before2 += w2[w];
    }
    const uint2 off = offsets[blockIdx.x];
    const unsigned long long p1 = (unsigned long long)off.x + before1 + __popc(b1 & lanemask);
    const unsigned long long p2 = (unsigned long long)off.y + before2 + __popc(b2 & lanemask);
    const bool take = cat == 1 || (cat == 2 && p2 < need_eq);
    if (take) {
        const unsigned long long pos = p1 + (p2 < need_eq ? p2 : need_eq);
        rows[pos] = (int32_t)i;
    }
}

__global__ void k_select_init(unsigned long long* sel, int64_t m) {
    sel[0] = 0ull;
    sel[1] = (unsigned long long)m;
}

}  // namespace

int ihs_rows_enqueue(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint64_t seed, int32_t level, int32_t* rows) {
    if (n_pad < 1 || m < 1 || m > n_pad || n_pad > ((int64_t)1 << 31) || level < 0) return IHS_EINVAL;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t nblocks = ceil_div64(n_pad, kCompactBlock);
    void* ws = nullptr;
    const size_t hist_bytes = (65536 + 64) * sizeof(unsigned);
    const size_t cnt_bytes = (size_t)nblocks * sizeof(uint2);
    IHS_TRY(ihs_scratch(ctx, SLOT_SELECT, hist_bytes + 2 * cnt_bytes + 64, &ws));
    unsigned* hist = static_cast<unsigned*>(ws);
    uint2* counts = reinterpret_cast<uint2*>(static_cast<char*>(ws) + hist_bytes);
    uint2* offsets = counts + nblocks;
    unsigned long long* sel = reinterpret_cast<unsigned long long*>(offsets + nblocks);
    IHS_CUDA_TRY(cudaMemsetAsync(hist, 0, hist_bytes, ctx->stream));
    k_select_init<<<1, 1, 0, ctx->stream>>>(sel, m);
    IHS_LAUNCH_CHECK();
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div64(n_pad, 256), 8 * (int64_t)ctx->sm_count);
    for (int pass = 0; pass < 4; ++pass) {
        k_hist16<<<grid, 256, 0, ctx->stream>>>(n_pad, (uint32_t)level, k0, k1, pass, sel, hist);
        IHS_LAUNCH_CHECK();
        k_pick16<<<1, 1024, 0, ctx->stream>>>(pass, sel, hist);
        IHS_LAUNCH_CHECK();
    }
    k_compact_count<<<(unsigned)nblocks, kCompactBlock, 0, ctx->stream>>>(n_pad, (uint32_t)level, k0, k1, sel,
                                                                          counts);
    IHS_LAUNCH_CHECK();
    k_compact_scan<<<1, 1024, 0, ctx->stream>>>(nblocks, counts, offsets);
    IHS_LAUNCH_CHECK();
    k_compact_write<<<(unsigned)nblocks, kCompactBlock, 0, ctx->stream>>>(n_pad, (uint32_t)level, k0, k1, sel,
                                                                          offsets, rows);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

extern "C" int ihs_srht_signs(ihs_ctx* ctx, int64_t n_pad, uint64_t seed, int32_t level, int8_t* eps) {
    if (!ctx || !eps || n_pad < 1 || level < 0) return IHS_EINVAL;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div64(n_pad, 256), 8 * (int64_t)ctx->sm_count);
    k_signs<<<grid, 256, 0, ctx->stream>>>(n_pad, (uint32_t)level, (uint32_t)seed, (uint32_t)(seed >> 32), eps);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

extern "C" int ihs_srht_rows(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint64_t seed, int32_t level,
                             int32_t* rows) {
    if (!ctx || !rows) return IHS_EINVAL;
    return ihs_rows_enqueue(ctx, n_pad, m, seed, level, rows);
}
