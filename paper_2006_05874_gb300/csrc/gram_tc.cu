// The Gram matrix of the sketched Hessian on the 5th-generation tensor cores:
// K = X X^T + nu^2 I with X = SA (Woodbury form, m x d, K = nu^2 I_m + SA SA^T)
// or X = (SA)^T (direct form, d x m, K = SA^T SA + nu^2 I_d), App. B.4.
//
// Every FP32 entry x of X splits exactly into three BF16 pieces,
// x = p1 + p2 + p3 (p1 = bf16(x), p2 = bf16(x - p1), p3 = x - p1 - p2; each
// residual keeps at most 8 significant bits fewer than the one before, so the
// last piece is exact).  A product of two pieces is exact in FP32, and
// x_a x_b = sum over the nine piece pairs.  The tensor core forms, for every
// 32-wide stretch of the inner dimension (two MMA slices of 16), the nine
// piece-pair products of a 128 x 128 output tile in one FP32 accumulator in
// tensor memory; the CTA's warps read each accumulator back (tcgen05.ld) and
// add it into double-float (hi, lo) accumulators in registers.  The only
// roundings are the FP32 sum of one stretch's 32 x 9 exact products and the
// compensated additions, so K comes out about as accurate as with
// compensated FP32 FMA chains on the CUDA cores.
//
// Layout: one CTA per output tile (and split of the inner dimension), 512
// threads (16 warps) and all 512 tensor-memory columns: two pairs of 128-column
// accumulators, a 64-wide chunk's two stretches in one pair, so that the MMAs
// of the next chunk (in the other pair) run while the warps drain this one.
// The chunk's pieces (3 for the tile's rows, 3 for its columns; 128 rows x
// 128 bytes each, K-major without swizzle: core matrices of 8 rows x 16 bytes)
// sit in one of two shared-memory stages, so that the warps split the next
// chunk while the tensor core works on this one.  Warp w drains TMEM lanes
// 32 (w % 4) ... and 32 columns starting at 32 (w / 4).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int GT = 128;                        // output tile (M = N = 128)
constexpr int GKE = 64;                        // inner entries per chunk
constexpr int GTHREADS = 512;
constexpr uint32_t GRB = GKE * 2;              // bytes of one row of a piece per chunk
constexpr uint32_t GPIECE = GT * GRB;          // 16 KiB per piece
constexpr uint32_t GSTAGE = 6 * GPIECE;        // three pieces of the rows, three of the columns
constexpr size_t gram_tc_smem() { return 2 * (size_t)GSTAGE + 64; }

__device__ __forceinline__ uint64_t gdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t desc = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    desc |= (uint64_t)(lbo >> 4) << 16;
    desc |= (uint64_t)(sbo >> 4) << 32;
    desc |= 1ull << 46;   // descriptor version of the sm_100 family; no swizzle
    return desc;
}

// byte offset of (row r, byte kb along K) in a K-major no-swizzle piece of
// GRB bytes per row
__device__ __forceinline__ uint32_t gkmaj(int r, int kb) {
    return (uint32_t)((r >> 3) * (GRB / 16) * 128 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

__device__ __forceinline__ void g_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void g_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// x = p1 + p2 + p3 exactly (BF16 pieces, round to nearest at each step), for
// two entries at once as packed BF16 pairs (first entry in the low half): one
// conversion instruction per piece for both entries, the widening back to
// binary32 by shifts and masks, the residuals by f32x2 subtraction.
__device__ __forceinline__ f2 bf2_widen(uint32_t u) {
    return f2_pack(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}
__device__ __forceinline__ uint32_t bf2_round(f2 x) {
    float a, b;
    f2_unpack(x, a, b);
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void split3x2(float a, float b, uint32_t& p1, uint32_t& p2, uint32_t& p3) {
    const f2 x = f2_pack(a, b);
    p1 = bf2_round(x);
    const f2 r1 = f2_sub(x, bf2_widen(p1));
    p2 = bf2_round(r1);
    const f2 r2 = f2_sub(r1, bf2_widen(p2));
    p3 = bf2_round(r2);
}

}  // namespace

namespace {

// Tile (I, J), J <= I, of K (linear index blockIdx.x = I (I + 1) / 2 + J) over
// the inner entries [y kchunk, (y + 1) kchunk) of split y = blockIdx.y.  With
// more than one split the tile's (hi, lo) pairs go to `part` (one 128 x 128
// tile of float2 per (split, tile)), else K (lower part, nu^2 on the
// diagonal) goes to G as double-float pairs (out_df) or FP64.
__global__ void __launch_bounds__(GTHREADS, 1)
k_gram_tc(const float* __restrict__ SA, int64_t d, int woodbury, int64_t kdim, int64_t K, int64_t kchunk,
          float2 nu2df, double nu2, int out_df, double* __restrict__ G, float2* __restrict__ part,
          unsigned* status) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char* stage = gsm;                                        // 2 x GSTAGE
    uint64_t* bar = reinterpret_cast<uint64_t*>(gsm + 2 * GSTAGE);      // one per accumulator
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const bool diag = I == J;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    const int64_t nch = kend > kbeg ? ceil_div64(kend - kbeg, GKE) : 0;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    g_fence_before();
    __syncthreads();
    g_fence_after();
    const uint32_t taddr = *tslot;

    // chunk c split into stage s: pieces 0-2 of the tile's rows, and off the
    // diagonal pieces 3-5 of its columns; thread = 8 consecutive inner entries
    // of one row (one 16-byte store per piece)
    auto split_chunk = [&](int64_t c, int s) {
        unsigned char* st = stage + (size_t)s * GSTAGE;
        const int64_t k0 = kbeg + c * GKE;
        for (int op = 0; op < (diag ? 1 : 2); ++op) {
            const int64_t rbase = (op == 0 ? I : J) * GT;
            unsigned char* pc = st + (size_t)op * 3 * GPIECE;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int e8 = tid + GTHREADS * i;
                const int r = woodbury ? (e8 >> 3) : (e8 & (GT - 1));
                const int kq = woodbury ? (e8 & 7) * 8 : (e8 >> 7) * 8;
                const int64_t row = rbase + r;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t kk = k0 + kq + j;
                    v[j] = (row < kdim && kk < kend) ? (woodbury ? __ldg(SA + row * d + kk) : __ldg(SA + kk * d + row))
                                                     : 0.f;
                }
                uint32_t p[3][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) split3x2(v[2 * j], v[2 * j + 1], p[0][j], p[1][j], p[2][j]);
                const uint32_t off = gkmaj(r, kq * 2);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    *reinterpret_cast<uint4*>(pc + (size_t)q * GPIECE + off) = make_uint4(p[q][0], p[q][1], p[q][2], p[q][3]);
            }
        }
    };
    // F32 accumulator, BF16 A and B, both K-major, N = M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GT >> 3) << 17) |
                           ((uint32_t)(GT >> 4) << 24);
    // the nine piece-pair MMAs of the chunk's four 16-wide slices: slices 2h
    // and 2h + 1 into accumulator 2 pr + h of pair pr (one commit each)
    auto issue = [&](int s, int pr) {
        const uint32_t abase = smem_u32(stage + (size_t)s * GSTAGE);
        const uint32_t bbase = diag ? abase : abase + 3 * GPIECE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t tacc = taddr + (uint32_t)((2 * pr + h) * GT);
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
                const int ks = 2 * h + sl;
#pragma unroll
                for (int pq = 0; pq < 9; ++pq) {
                    const int p = pq / 3, q = pq % 3;
                    const uint64_t ad = gdesc(abase + (uint32_t)p * GPIECE + ks * 256, 128, (GRB / 16) * 128);
                    const uint64_t bd = gdesc(bbase + (uint32_t)q * GPIECE + ks * 256, 128, (GRB / 16) * 128);
                    const uint32_t accum = (sl > 0 || pq > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tacc),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[2 * pr + h]))
                         : "memory");
        }
    };

    const int quad = warp & 3, cpart = warp >> 2;   // TMEM lanes 32 quad .., columns 32 cpart ..
    // the 32 entries' (hi, lo) sums as packed pairs of adjacent columns: each
    // TwoSum step is one f32x2 instruction for two entries (the same
    // operations per entry as Acc2::add)
    Acc2x2 acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j].hi.v = acc[j].lo.v = 0ull;
    bool ok = true;
    int64_t issued = -1;   // last chunk whose MMAs were issued
    // pipeline: the MMAs of chunk c + 1 (accumulator pair (c + 1) & 1) run
    // while the warps drain chunk c; the split of chunk c + 1 runs while the
    // MMAs of chunk c do.  Barrier 2 pr + h completes once every two chunks.
    if (nch > 0) split_chunk(0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    g_fence_before();
    __syncthreads();
    g_fence_after();
    if (nch > 0 && tid == 0) issue(0, 0);
    issued = nch > 0 ? 0 : -1;
    for (int64_t c = 0; c < nch && ok; ++c) {
        const int pr = (int)(c & 1);
        if (c + 1 < nch) {
            // stage (c + 1) & 1 was read by the MMAs of chunk c - 1, drained
            // in the previous iteration; so was accumulator pair (c + 1) & 1
            split_chunk(c + 1, (int)((c + 1) & 1));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            g_fence_before();
            __syncthreads();
            g_fence_after();
            if (tid == 0) issue((int)((c + 1) & 1), pr ^ 1);
            issued = c + 1;
        }
        // drain chunk c's two accumulators into the double-float sums
        for (int h = 0; h < 2; ++h) {
            const bool w = mbar_wait_bounded(&bar[2 * pr + h], (uint32_t)((c >> 1) & 1), status);
            if (__syncthreads_or(!w)) {
                ok = false;
                break;
            }
            g_fence_after();
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {   // two loads of 16 columns each
                uint32_t v[16];
                const uint32_t a = taddr + ((uint32_t)(32 * quad) << 16) +
                                   (uint32_t)((2 * pr + h) * GT + 32 * cpart + 16 * hh);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[8 * hh + j].add(f2_pack(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])));
            }
        }
        // accumulator pair pr read: chunk c + 2 may be issued into it
        g_fence_before();
        __syncthreads();
        g_fence_after();
    }
    if (!ok) {
        // a wait gave up: let the last issued MMAs finish before the TMEM is freed
        if (tid == 0 && issued >= 0)
            mbar_wait_bounded(&bar[2 * (int)(issued & 1) + 1], (uint32_t)((issued >> 1) & 1), status);
        g_fence_before();
        __syncthreads();
        g_fence_after();
    }
    if (ok) {
        // through a 32 x 33 shared tile per warp (the stages are idle now), so
        // that each store writes 32 consecutive entries of one row
        float2* tile = reinterpret_cast<float2*>(stage) + (size_t)warp * (32 * 33);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float h0, h1, l0, l1;
            f2_unpack(acc[j].hi, h0, h1);
            f2_unpack(acc[j].lo, l0, l1);
            tile[lane * 33 + 2 * j] = make_float2(h0, l0);
            tile[lane * 33 + 2 * j + 1] = make_float2(h1, l1);
        }
        __syncwarp();
        const int64_t col = J * GT + 32 * cpart + lane;
        if (gridDim.y > 1) {
            float2* pt = part + ((size_t)blockIdx.y * gridDim.x + t) * GT * GT;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) pt[(32 * quad + rr) * GT + 32 * cpart + lane] = tile[rr * 33 + lane];
        } else {
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int64_t row = I * GT + 32 * quad + rr;
                if (row >= kdim || col >= kdim || col > row) continue;
                const float2 hl = tile[rr * 33 + lane];
                if (out_df) {
                    float sh, se;
                    two_sum(hl.x, hl.y, sh, se);
                    float2 v = make_float2(sh, se);
                    if (row == col) {
                        float s2, e2;
                        two_sum(v.x, nu2df.x, s2, e2);
                        const float l2 = __fadd_rn(e2, __fadd_rn(v.y, nu2df.y));
                        const float s3 = __fadd_rn(s2, l2);
                        v = make_float2(s3, __fsub_rn(l2, __fsub_rn(s3, s2)));
                    }
                    reinterpret_cast<float2*>(G)[row * kdim + col] = v;
                } else {
                    G[row * kdim + col] = (double)hl.x + (double)hl.y + (row == col ? nu2 : 0.0);
                }
            }
        }
    }
    g_fence_before();
    __syncthreads();
    g_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(512));
}

// K tile t = sum over the KS splits of the (hi, lo) pairs (fixed order,
// compensated binary32, eight loads in flight), + nu^2 on the diagonal;
// grid (tiles, GT * GT / 256), one entry per thread.
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const float2* __restrict__ part, int KS, int64_t ntiles,
                                                        int64_t kdim, float2 nu2df, double nu2, int out_df,
                                                        double* __restrict__ G) {
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const int e = blockIdx.y * 256 + threadIdx.x;
    const int64_t r = I * GT + e / GT, c = J * GT + e % GT;
    if (r >= kdim || c >= kdim || c > r) return;
    Acc2 acc{0.f, 0.f};
    for (int y0 = 0; y0 < KS; y0 += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (y0 + u < KS) v[u] = part[((size_t)(y0 + u) * ntiles + t) * GT * GT + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (y0 + u >= KS) break;
            acc.add_pair(v[u].x, v[u].y);
        }
    }
    if (out_df) {
        if (r == c) acc.add_pair(nu2df.x, nu2df.y);
        const float hi = __fadd_rn(acc.hi, acc.lo);
        reinterpret_cast<float2*>(G)[r * kdim + c] = make_float2(hi, __fsub_rn(acc.lo, __fsub_rn(hi, acc.hi)));
    } else {
        G[r * kdim + c] = (double)acc.hi + (double)acc.lo + (r == c ? nu2 : 0.0);
    }
}

}  // namespace

int ihs_gram_tc_enqueue(ihs_ctx* ctx, const float* SA, int64_t d, int woodbury, int64_t kdim, int64_t K, double nu2,
                        int out_df, double* G, cudaStream_t s) {
    if (kdim < 1 || K < 1) return IHS_EINVAL;
    const int64_t T = ceil_div64(kdim, GT);
    const int64_t ntiles = T * (T + 1) / 2;
    const int64_t nchunks = ceil_div64(K, GKE);
    // splits of the inner dimension so that the tiles x splits fill the SMs
    // (one CTA per SM: each holds the whole tensor memory)
    int64_t KS = std::max<int64_t>(1, ctx->sm_count / ntiles);
    KS = std::min<int64_t>(KS, nchunks);
    const int64_t kchunk = ceil_div64(nchunks, KS) * GKE;
    KS = ceil_div64(K, kchunk);
    float2* part = nullptr;
    if (KS > 1) {
        void* ws = nullptr;
        IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)KS * ntiles * GT * GT * sizeof(float2), &ws));
        part = static_cast<float2*>(ws);
    }
    const float nh = (float)nu2;
    const float2 nu2df = make_float2(nh, (float)(nu2 - (double)nh));
    IHS_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem()));
    k_gram_tc<<<dim3((unsigned)ntiles, (unsigned)KS), GTHREADS, gram_tc_smem(), s>>>(
        SA, d, woodbury, kdim, K, kchunk, nu2df, nu2, out_df, G, part, ctx->d_status);
    IHS_LAUNCH_CHECK();
    if (KS > 1) {
        k_gram_tc_reduce<<<dim3((unsigned)ntiles, GT * GT / 256), 256, 0, s>>>(part, (int)KS, ntiles, kdim, nu2df,
                                                                                 nu2, out_df, G);
        IHS_LAUNCH_CHECK();
    }
    return IHS_OK;
}
