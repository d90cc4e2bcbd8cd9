// Seeded draws of the SRHT (App. C.2): Rademacher signs and the uniformly
// random m-subset of [0, n_pad) rows, sampled without replacement.
//
// Row subset: the m indices with the smallest 64-bit Philox keys (ties broken by
// index), written in ascending order.  For m <= 6144: a threshold pass collects
// the few rows whose key can be among the m smallest and one CTA selects among
// them (two launches).  Larger m: the m-th smallest key K* is found by an exact
// radix select (four passes over 16-bit digits, most significant first,
// histograms in global memory); then a stable two-category compaction (key <
// K*, key == K*) writes the chosen indices.  Keys are recomputed from Philox
// on every pass instead of being stored.
#include <cmath>
#include <cstdlib>

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

// ---------------------------------------------------------------------------
// Two-launch selection for m <= kSelMaxM.  Every row whose key lies below a
// threshold T (chosen so that the candidate count ~ Binomial(n_pad, T / 2^64)
// has mean m + 10 sqrt(m) + 20) is a candidate; each CTA appends the
// candidates of its contiguous row range in index order to its own segment.
// One CTA then holds all candidates in shared memory, finds the m smallest
// (key, index) pairs by an MSB-first radix select over 8-bit digits and writes
// their indices in ascending order.  When the candidates do not contain the m
// smallest keys or do not fit (probability below 1e-20 with this margin), the
// same CTA finds K* by bisection over all n_pad keys and compacts directly:
// the result never depends on T.
constexpr int kSelCap = 8192;    // candidates held in shared memory
constexpr int kSelMaxM = 6144;
constexpr int kSelThreads = 1024;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* wsum, unsigned& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned t = wsum[lane];
        unsigned u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        wsum[lane] = u - t;          // exclusive warp offsets
        if (lane == 31) wsum[32] = u;
    }
    __syncthreads();
    const unsigned r = wsum[warp] + x - v;
    total = wsum[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kSelThreads) k_sel_cand(int64_t n_pad, int64_t R, unsigned long long T, int all,
                                                         uint32_t level, uint32_t k0, uint32_t k1, int segcap,
                                                         unsigned long long* __restrict__ ckey,
                                                         int32_t* __restrict__ cidx, unsigned* __restrict__ counts) {
    __shared__ unsigned wsum[33];
    const int64_t r0 = blockIdx.x * R, r1 = min(n_pad, r0 + R);
    const size_t seg = (size_t)blockIdx.x * segcap;
    unsigned total = 0;
    for (int64_t c0 = r0; c0 < r1; c0 += kSelThreads) {
        const int64_t i = c0 + threadIdx.x;
        uint64_t key = 0;
        bool take = false;
        if (i < r1) {
            key = srht_row_key((uint64_t)i, level, k0, k1);
            take = all || key < T;
        }
        unsigned chunk = 0;
        const unsigned before = block_excl_scan(take ? 1u : 0u, wsum, chunk);
        if (take) {
            const unsigned pos = total + before;
            if (pos < (unsigned)segcap) {
                ckey[seg + pos] = key;
                cidx[seg + pos] = (int32_t)i;
            }
        }
        total += chunk;
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Rows of [0, n_pad) with key < kstar, then the first need_eq with key == kstar,
// in ascending index order (one CTA, index-ordered chunks).
__device__ void sel_compact_all(int64_t n_pad, uint32_t level, uint32_t k0, uint32_t k1, uint64_t kstar,
                                unsigned long long need_eq, unsigned* wsum, int32_t* rows) {
    unsigned long long taken = 0, eq_seen = 0;
    for (int64_t c0 = 0; c0 < n_pad; c0 += kSelThreads) {
        const int64_t i = c0 + threadIdx.x;
        int cat = 0;
        if (i < n_pad) {
            const uint64_t key = srht_row_key((uint64_t)i, level, k0, k1);
            cat = key < kstar ? 1 : (key == kstar ? 2 : 0);
        }
        unsigned neq = 0;
        const unsigned eq_before = block_excl_scan(cat == 2 ? 1u : 0u, wsum, neq);
        const bool take = cat == 1 || (cat == 2 && eq_seen + eq_before < need_eq);
        unsigned ntake = 0;
        const unsigned before = block_excl_scan(take ? 1u : 0u, wsum, ntake);
        if (take) rows[taken + before] = (int32_t)i;
        taken += ntake;
        eq_seen += neq;
    }
}

// Number of rows of [0, n_pad) with key < t (one CTA).
__device__ unsigned long long sel_count_lt(int64_t n_pad, uint32_t level, uint32_t k0, uint32_t k1, uint64_t t,
                                           unsigned* wsum) {
    unsigned long long c = 0;
    for (int64_t c0 = 0; c0 < n_pad; c0 += kSelThreads) {
        const int64_t i = c0 + threadIdx.x;
        const bool lt = i < n_pad && srht_row_key((uint64_t)i, level, k0, k1) < t;
        unsigned tot = 0;
        block_excl_scan(lt ? 1u : 0u, wsum, tot);
        c += tot;
    }
    return c;
}

struct SelShared {
    unsigned long long key[kSelCap];
    int32_t idx[kSelCap];
    unsigned off[kSelThreads + 1];
    unsigned hist[256];
    unsigned wsum[33];
    unsigned long long bcast[4];
};

__global__ void __launch_bounds__(kSelThreads) k_sel_resolve(int64_t n_pad, int64_t m, int G, int segcap,
                                                            uint32_t level, uint32_t k0, uint32_t k1,
                                                            const unsigned long long* __restrict__ ckey,
                                                            const int32_t* __restrict__ cidx,
                                                            const unsigned* __restrict__ counts,
                                                            int force_fallback, int32_t* __restrict__ rows) {
    extern __shared__ __align__(16) unsigned char selraw[];
    SelShared& S = *reinterpret_cast<SelShared*>(selraw);
    const int tid = threadIdx.x;
    // segment offsets (G <= kSelThreads)
    unsigned cnt = tid < G ? counts[tid] : 0u;
    const bool over = tid < G && cnt > (unsigned)segcap;
    const int any_over = __syncthreads_or(over);
    unsigned total = 0;
    const unsigned myoff = block_excl_scan(cnt, S.wsum, total);
    if (tid < G) S.off[tid] = myoff;
    if (tid == 0) S.off[G] = total;
    __syncthreads();
    if (force_fallback || any_over || total < (unsigned)m || total > (unsigned)kSelCap) {
        // K* = the m-th smallest key: the largest t with count(key < t) < m
        uint64_t lo = 0, hi = ~0ull;   // count(< lo) < m; answer in [lo, hi]
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2 + 1;
            const unsigned long long c = sel_count_lt(n_pad, level, k0, k1, mid, S.wsum);
            if (c < (unsigned long long)m) lo = mid;
            else hi = mid - 1;
        }
        const unsigned long long below = sel_count_lt(n_pad, level, k0, k1, lo, S.wsum);
        sel_compact_all(n_pad, level, k0, k1, lo, (unsigned long long)m - below, S.wsum, rows);
        return;
    }
    // gather the segments in index order
    for (unsigned e = tid; e < total; e += kSelThreads) {
        int a = 0, b = G - 1;   // last segment with off <= e
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (S.off[mid] <= e) a = mid;
            else b = mid - 1;
        }
        const size_t src = (size_t)a * segcap + (e - S.off[a]);
        S.key[e] = ckey[src];
        S.idx[e] = cidx[src];
    }
    // highest set bit over all candidate keys
    unsigned long long orv = 0;
    for (unsigned e = tid; e < total; e += kSelThreads) orv |= S.key[e];
    if (tid == 0) S.bcast[0] = 0ull;
    __syncthreads();
    atomicOr(&S.bcast[0], orv);
    __syncthreads();
    const unsigned long long allor = S.bcast[0];
    int shift = allor ? ((63 - __clzll((long long)allor)) / 8) * 8 : 0;
    // radix select: after each pass P holds the digits of K* above `shift`
    unsigned long long P = 0, need = (unsigned long long)m;
    bool whole = false;   // every key with top digits == P is selected
    for (;;) {
        for (int h = tid; h < 256; h += kSelThreads) S.hist[h] = 0u;
        __syncthreads();
        for (unsigned e = tid; e < total; e += kSelThreads) {
            const unsigned long long k = S.key[e];
            const bool match = shift + 8 >= 64 || (k >> (shift + 8)) == P;
            if (match) atomicAdd(&S.hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        // the first digit b whose inclusive prefix count reaches `need`
        // (digit 255 with the whole count when none does): a shuffle scan in
        // each of eight warps over the 256 bins, then one test per bin
        unsigned hv = 0, incl = 0;
        if (tid < 256) {
            hv = S.hist[tid];
            incl = hv;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
                if ((tid & 31) >= off) incl += y;
            }
            if ((tid & 31) == 31) S.wsum[tid >> 5] = incl;
        }
        __syncthreads();
        if (tid < 256) {
            unsigned long long inc = incl;
            for (int w = 0; w < (tid >> 5); ++w) inc += S.wsum[w];
            const unsigned long long exc = inc - hv;
            if ((exc < need && inc >= need) || (tid == 255 && inc < need)) {
                const unsigned long long acc = inc >= need ? exc : inc;
                S.bcast[1] = (P << 8) | (unsigned long long)tid;
                S.bcast[2] = need - acc;
                S.bcast[3] = (unsigned long long)hv;
            }
        }
        __syncthreads();
        P = S.bcast[1];
        need = S.bcast[2];
        const unsigned long long inb = S.bcast[3];
        __syncthreads();
        if (inb == need) {
            whole = true;
            break;
        }
        if (shift == 0) break;   // ties on the full key: the first `need` by index
        shift -= 8;
    }
    // selected: top digits < P, or == P (all when whole, else the first `need`
    // of them in index order); each thread owns 8 consecutive candidates
    const unsigned e0 = (unsigned)tid * (kSelCap / kSelThreads);
    unsigned eqc = 0;
#pragma unroll
    for (int q = 0; q < kSelCap / kSelThreads; ++q) {
        const unsigned e = e0 + q;
        if (e < total && (S.key[e] >> shift) == P) ++eqc;
    }
    unsigned eqtot = 0;
    unsigned eqb = block_excl_scan(eqc, S.wsum, eqtot);
    unsigned tc = 0;
    bool takes[kSelCap / kSelThreads];
#pragma unroll
    for (int q = 0; q < kSelCap / kSelThreads; ++q) {
        const unsigned e = e0 + q;
        bool t = false;
        if (e < total) {
            const unsigned long long top = S.key[e] >> shift;
            if (top < P) t = true;
            else if (top == P) {
                t = whole || eqb < need;
                ++eqb;
            }
        }
        takes[q] = t;
        tc += t ? 1u : 0u;
    }
    unsigned ttot = 0;
    const unsigned pos0 = block_excl_scan(tc, S.wsum, ttot);
    unsigned pos = pos0;
#pragma unroll
    for (int q = 0; q < kSelCap / kSelThreads; ++q) {
        if (takes[q]) rows[pos++] = S.idx[e0 + q];
    }
}

}  // namespace

static int rows_enqueue_radix(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint32_t level, uint32_t k0, uint32_t k1,
                              int32_t* rows) {
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
        k_hist16<<<grid, 256, 0, ctx->stream>>>(n_pad, level, k0, k1, pass, sel, hist);
        IHS_LAUNCH_CHECK();
        k_pick16<<<1, 1024, 0, ctx->stream>>>(pass, sel, hist);
        IHS_LAUNCH_CHECK();
    }
    k_compact_count<<<(unsigned)nblocks, kCompactBlock, 0, ctx->stream>>>(n_pad, level, k0, k1, sel, counts);
    IHS_LAUNCH_CHECK();
    k_compact_scan<<<1, 1024, 0, ctx->stream>>>(nblocks, counts, offsets);
    IHS_LAUNCH_CHECK();
    k_compact_write<<<(unsigned)nblocks, kCompactBlock, 0, ctx->stream>>>(n_pad, level, k0, k1, sel, offsets,
                                                                          rows);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

int ihs_rows_enqueue(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint64_t seed, int32_t level, int32_t* rows) {
    if (n_pad < 1 || m < 1 || m > n_pad || n_pad > ((int64_t)1 << 31) || level < 0) return IHS_EINVAL;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    if (m > kSelMaxM) return rows_enqueue_radix(ctx, n_pad, m, (uint32_t)level, k0, k1, rows);
    // candidate threshold: mean count m + 10 sqrt(m) + 20 (all rows when that
    // reaches n_pad).  IHS_SELECT_FORCE_FALLBACK=1 makes the resolving CTA
    // take its exact fallback (a test hook; the result is the same).
    const double want = (double)m + 10.0 * std::sqrt((double)m) + 20.0;
    int all = 0;
    unsigned long long T = 0;
    if (want >= (double)n_pad) all = 1;
    else T = (unsigned long long)std::ldexp(want / (double)n_pad, 64);
    const char* ff = std::getenv("IHS_SELECT_FORCE_FALLBACK");
    const int force = (ff && ff[0] == '1') ? 1 : 0;
    const int64_t chunks = ceil_div64(n_pad, kSelThreads);
    const int G = (int)std::min<int64_t>(chunks, std::min<int64_t>(2 * (int64_t)ctx->sm_count, kSelThreads));
    const int64_t R = ceil_div64(chunks, G) * kSelThreads;
    const int Gr = (int)ceil_div64(n_pad, R);
    const double per = all ? (double)R : want * (double)R / (double)n_pad;
    int segcap = (int)std::ceil(per + 10.0 * std::sqrt(per) + 32.0);
    segcap = (int)std::min<int64_t>((segcap + 31) / 32 * 32, R);
    const size_t key_bytes = (size_t)Gr * segcap * sizeof(unsigned long long);
    const size_t idx_bytes = (size_t)Gr * segcap * sizeof(int32_t);
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_SELECT, key_bytes + idx_bytes + (size_t)Gr * sizeof(unsigned) + 256, &ws));
    unsigned long long* ckey = static_cast<unsigned long long*>(ws);
    int32_t* cidx = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + key_bytes);
    unsigned* counts = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + key_bytes + idx_bytes);
    k_sel_cand<<<(unsigned)Gr, kSelThreads, 0, ctx->stream>>>(n_pad, R, T, all, (uint32_t)level, k0, k1, segcap,
                                                             ckey, cidx, counts);
    IHS_LAUNCH_CHECK();
    const size_t smem = sizeof(SelShared);
    IHS_CUDA_TRY(ihs_allow_smem(k_sel_resolve, smem));
    k_sel_resolve<<<1, kSelThreads, smem, ctx->stream>>>(n_pad, m, Gr, segcap, (uint32_t)level, k0, k1, ckey, cidx,
                                                        counts, force, rows);
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
