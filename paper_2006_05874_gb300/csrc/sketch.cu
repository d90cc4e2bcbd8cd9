// Sketch SA = S A (Sec. 1, Eq. 3) for the two embeddings of the paper.
//
// SRHT (App. C.2): S = sqrt(n_pad/m) R H_norm diag(eps) on A zero-padded to
// n_pad rows.  With n_pad = P Q and i = p Q + q, the Hadamard entry factors as
// (-1)^popcount(r & i) = (-1)^popcount(r_hi & p) (-1)^popcount(r_lo & q), so
//   SA_j = m^-1/2 sum_p (-1)^popcount(r_hi_j & p) Y_p[r_lo_j],
//   Y_p  = H_Q diag(eps_p) A_p   (length-Q FWHT of the sign-flipped block p).
// A CTA owns a tile of C columns and a range of blocks p: it transforms each
// Q x C block in shared memory and accumulates the m selected rows; block
// ranges are combined by a fixed-order reduction.  A is read once.
//
// Gaussian (Sec. 1, App. C.1): S_ji = z_ji / sqrt(m), z drawn in-kernel from
// Philox (never stored); split over n with a fixed-order reduction.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kSrhtQmax = 1024;
constexpr int kSrhtC = 16;
constexpr int kSrhtThreads = 512;

__global__ void __launch_bounds__(kSrhtThreads)
k_srht_fwht(const float* __restrict__ A, int64_t n, int d, int64_t m, int Q, int logQ, int64_t P, int PG,
            const int32_t* __restrict__ rows, uint32_t level, uint32_t k0, uint32_t k1, int acc_in_smem,
            float* __restrict__ out /* PG x m x d partials */) {
    extern __shared__ __align__(16) float sm[];
    const int CP = kSrhtC + 1;   // padded row stride
    float* X = sm;               // Q x CP
    float* sg = X + (size_t)Q * CP;          // Q signs (+-1)
    float* acc = sg + Q;                     // m x C (when in shared memory)
    const int tid = threadIdx.x;
    const int col0 = blockIdx.x * kSrhtC;
    const int ncol = min(kSrhtC, d - col0);
    const int pg = blockIdx.y;
    const int64_t p0 = (int64_t)pg * P / PG, p1 = (int64_t)(pg + 1) * P / PG;
    float* outp = out + (size_t)pg * m * d;

    if (acc_in_smem) {
        for (int64_t e = tid; e < m * kSrhtC; e += kSrhtThreads) acc[e] = 0.f;
    } else {
        for (int64_t e = tid; e < m * kSrhtC; e += kSrhtThreads) {
            const int64_t j = e / kSrhtC;
            const int c = (int)(e % kSrhtC);
            if (c < ncol) outp[j * d + col0 + c] = 0.f;
        }
    }
    for (int64_t p = p0; p < p1; ++p) {
        __syncthreads();
        for (int q = tid; q < Q; q += kSrhtThreads) {
            const uint64_t i = (uint64_t)(p * Q + q);
            sg[q] = srht_sign_bit(i, level, k0, k1) ? -1.f : 1.f;
        }
        __syncthreads();
        for (int e = tid; e < Q * kSrhtC; e += kSrhtThreads) {
            const int q = e / kSrhtC, c = e % kSrhtC;
            const int64_t i = p * Q + q;
            float v = 0.f;
            if (i < n && c < ncol) v = A[i * d + col0 + c];
            X[q * CP + c] = sg[q] * v;
        }
        __syncthreads();
        // radix-2 butterflies along q
        for (int h = 1; h < Q; h <<= 1) {
            for (int e = tid; e < (Q / 2) * kSrhtC; e += kSrhtThreads) {
                const int bfly = e / kSrhtC, c = e % kSrhtC;
                const int q0 = (bfly / h) * 2 * h + (bfly % h);
                const float a = X[q0 * CP + c], b = X[(q0 + h) * CP + c];
                X[q0 * CP + c] = a + b;
                X[(q0 + h) * CP + c] = a - b;
            }
            __syncthreads();
        }
        // accumulate the selected rows of this block
        for (int64_t e = tid; e < m * kSrhtC; e += kSrhtThreads) {
            const int64_t j = e / kSrhtC;
            const int c = (int)(e % kSrhtC);
            const uint32_t r = (uint32_t)rows[j];
            const uint32_t lo = r & (uint32_t)(Q - 1);
            const uint64_t hi = (uint64_t)(r >> logQ);
            const float v = X[lo * CP + c];
            const float sv = (__popcll(hi & (uint64_t)p) & 1) ? -v : v;
            if (acc_in_smem) {
                acc[e] += sv;
            } else if (c < ncol) {
                outp[j * d + col0 + c] += sv;
            }
        }
    }
    if (acc_in_smem) {
        __syncthreads();
        for (int64_t e = tid; e < m * kSrhtC; e += kSrhtThreads) {
            const int64_t j = e / kSrhtC;
            const int c = (int)(e % kSrhtC);
            if (c < ncol) outp[j * d + col0 + c] = acc[e];
        }
    }
}

// Radix-32 register FWHT for blocks of Q = 1024 rows (n_pad >= 1024).
// CTA = 512 threads = 16 columns x 32 "lanes" ql; thread (c, ql) holds rows
// 32k + ql (k = 0..31) of its column in registers: a 32-point WHT over k, a
// padded shared-memory transpose, a 32-point WHT over ql (H_1024 = H_32 (x)
// H_32), then the selected rows are accumulated with the sign of their high
// index bits against the block index p.
constexpr int kR32C = 16, kR32T = 512, kR32Stride = 528;   // 528 = 33 x 16: conflict-free transposes

__device__ __forceinline__ void wht32(float (&v)[32]) {
#pragma unroll
    for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if ((i & h) == 0) {
                const float a = v[i], b = v[i + h];
                v[i] = __fadd_rn(a, b);
                v[i + h] = __fsub_rn(a, b);
            }
        }
    }
}

// Shared memory of k_srht_r32: two TMA stages of 1024 x 16 floats, the padded
// transpose buffer, sign words, two mbarriers, per-row offsets.
constexpr size_t kR32Stage = 1024 * kR32C * sizeof(float);   // 64 KiB
__host__ __device__ inline size_t r32_smem_bytes(int64_t mrows) {
    return 2 * kR32Stage + (size_t)32 * kR32Stride * sizeof(float) + 32 * sizeof(uint32_t) + 2 * sizeof(uint64_t) +
           2 * (size_t)mrows * sizeof(int32_t);
}

// MA accumulators per thread: this launch handles m <= 32 MA selected rows;
// thread (c, ql) accumulates rows ql + 32 i (i < MA) of column c in registers.
// Blocks of 1024 x 16 arrive by TMA (four 256-row boxes) into a two-stage
// ring; rows >= n and columns >= d read as zero.
template <int MA>
__global__ void __launch_bounds__(kR32T, 1)
k_srht_r32(const __grid_constant__ CUtensorMap amap, int d, int64_t m, int64_t m_total, int64_t row_off, int64_t P,
           int PG, const int32_t* __restrict__ rows, uint32_t level, uint32_t k0, uint32_t k1, unsigned* status,
           float* __restrict__ out /* PG x m_total x d partials; this launch writes rows [row_off, row_off + m) */) {
    extern __shared__ __align__(128) unsigned char smraw[];
    float* stage = reinterpret_cast<float*>(smraw);                                   // 2 x 1024 x 16
    float* T = reinterpret_cast<float*>(smraw + 2 * kR32Stage);                      // 32 x 528
    uint32_t* sbits = reinterpret_cast<uint32_t*>(T + 32 * kR32Stride);              // 32 sign words
    uint64_t* full = reinterpret_cast<uint64_t*>(sbits + 32);                        // 2 mbarriers
    int32_t* toff = reinterpret_cast<int32_t*>(full + 2);                            // T offset per selected row
    uint32_t* rhi = reinterpret_cast<uint32_t*>(toff + m);                           // its block-index bits
    const int tid = threadIdx.x;
    const int c = tid & 15, ql = tid >> 4;
    const int col0 = blockIdx.x * kR32C;
    const int col = col0 + c;
    const int pg = blockIdx.y;
    const int64_t p0 = (int64_t)pg * P / PG, p1 = (int64_t)(pg + 1) * P / PG;
    const int64_t nblk = p1 - p0;

    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_mbar_init();
    }
    for (int64_t j = tid; j < m; j += kR32T) {
        const uint32_t r = (uint32_t)rows[j];
        const uint32_t lo = r & 1023u;
        toff[j] = (int32_t)((lo >> 5) * kR32Stride + (lo & 31u) * 16);
        rhi[j] = r >> 10;
    }
    __syncthreads();
    auto issue = [&](int64_t b) {   // block p0 + b into stage b & 1
        float* dst = stage + (size_t)(b & 1) * (1024 * kR32C);
        uint64_t* bar = &full[b & 1];
        mbar_arrive_expect_tx(bar, (uint32_t)kR32Stage);
        const int y0 = (int)((p0 + b) * 1024);
#pragma unroll
        for (int q = 0; q < 4; ++q) tma_load_2d(dst + q * 256 * kR32C, &amap, col0, y0 + 256 * q, bar);
    };
    if (tid == 0) {
        issue(0);
        if (nblk > 1) issue(1);
    }
    float acc[MA];
#pragma unroll
    for (int i = 0; i < MA; ++i) acc[i] = 0.f;
    int64_t b = 0;
    for (; b < nblk; ++b) {
        const int64_t p = p0 + b;
        if (tid < 8) {
            const uint4 w = srht_sign_words((uint64_t)p * 8 + tid, level, k0, k1);
            sbits[4 * tid + 0] = w.x;
            sbits[4 * tid + 1] = w.y;
            sbits[4 * tid + 2] = w.z;
            sbits[4 * tid + 3] = w.w;
        }
        const bool ok = mbar_wait_bounded(&full[b & 1], (uint32_t)((b >> 1) & 1), status);
        if (__syncthreads_or(!ok)) break;   // also: sign words ready, previous gather done with T
        const float* st = stage + (size_t)(b & 1) * (1024 * kR32C);
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = st[(ql + 32 * k) * kR32C + c];
        // row 32 k + ql of the block takes bit k of word ql: flip the float's sign bit
        const uint32_t word = sbits[ql];
#pragma unroll
        for (int k = 0; k < 32; ++k)
            v[k] = __int_as_float(__float_as_int(v[k]) ^ (int)((word << (31 - k)) & 0x80000000u));
        wht32(v);   // over k (high five index bits)
#pragma unroll
        for (int k = 0; k < 32; ++k) T[k * kR32Stride + ql * 16 + c] = v[k];
        __syncthreads();   // stage b & 1 fully read: refill it with block b + 2
        if (tid == 0 && b + 2 < nblk) issue(b + 2);
#pragma unroll
        for (int l = 0; l < 32; ++l) v[l] = T[ql * kR32Stride + l * 16 + c];
        wht32(v);   // over the low five index bits; thread now holds Y[32 ql + l]
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 32; ++l) T[ql * kR32Stride + l * 16 + c] = v[l];
        __syncthreads();
        const uint32_t pb = (uint32_t)p;
#pragma unroll
        for (int i = 0; i < MA; ++i) {
            const int64_t j = ql + 32 * i;
            if (j < m) {
                const float val = T[toff[j] + c];
                acc[i] += (__popc(rhi[j] & pb) & 1) ? -val : val;
            }
        }
    }
    if (b < nblk) {
        // a wait gave up: let the copies in flight land before exiting
        if (tid == 0) {
            for (int64_t q = b; q < nblk && q < b + 2; ++q)
                mbar_wait_bounded(&full[q & 1], (uint32_t)((q >> 1) & 1), status);
        }
        __syncthreads();
        return;
    }
    if (col < d) {
        float* outp = out + ((size_t)pg * m_total + row_off) * d + col;
#pragma unroll
        for (int i = 0; i < MA; ++i) {
            const int64_t j = ql + 32 * i;
            if (j < m) outp[j * d] = acc[i];
        }
    }
}

template <int MA>
int launch_r32(ihs_ctx* ctx, const CUtensorMap& amap, int d, int64_t mc, int64_t m, int64_t c0, int64_t P, int PG,
               const int32_t* rows, int32_t level, uint64_t seed, float* part) {
    const size_t smem = r32_smem_bytes(mc);
    auto kern = k_srht_r32<MA>;
    IHS_CUDA_TRY(ihs_allow_smem(kern, smem));
    dim3 grid((unsigned)ceil_div64(d, kR32C), (unsigned)PG);
    kern<<<grid, kR32T, smem, ctx->stream>>>(amap, d, mc, m, c0, P, PG, rows, (uint32_t)level, (uint32_t)seed,
                                            (uint32_t)(seed >> 32), ctx->d_status, part);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

// out[e] = scale * sum_k part[k][e] in a fixed order (FP64).
__global__ void k_reduce_parts(const float* __restrict__ part, int K, int64_t count, double scale,
                               float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (double)part[(size_t)k * count + e];
        out[e] = (float)(s * scale);
    }
}

__global__ void k_reduce_parts2(const float2* __restrict__ part, int K, int64_t count, double scale,
                                float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const float2 v = part[(size_t)k * count + e];
            s += (double)v.x + (double)v.y;
        }
        out[e] = (float)(s * scale);
    }
}

// Gaussian sketch, FP32 SIMT: tile BM x BN of SA over a K range of rows of A;
// z tile generated in shared memory from Philox, compensated accumulation per
// BK-chunk.
constexpr int kGBM = 64, kGBN = 64, kGBK = 32, kGThreads = 256;

__global__ void __launch_bounds__(kGThreads)
k_gauss_simt(const float* __restrict__ A, int64_t n, int d, int64_t m, int64_t rows_per_split, uint32_t level,
             uint32_t k0, uint32_t k1, float2* __restrict__ part /* KS x m x d */) {
    __shared__ float zs[kGBK][kGBM + 4];
    __shared__ float as[kGBK][kGBN + 4];
    const int tid = threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.x * kGBM;
    const int c0 = blockIdx.y * kGBN;
    const int64_t i_begin = (int64_t)blockIdx.z * rows_per_split;
    const int64_t i_end = min(n, i_begin + rows_per_split);
    const int ty = tid / 16, tx = tid % 16;   // 16 x 16 threads, 4 x 4 outputs each
    Acc2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = Acc2{0.f, 0.f};
    for (int64_t i0 = i_begin; i0 < i_end; i0 += kGBK) {
        __syncthreads();
        // z tile: kGBK columns i x kGBM rows j; one Philox call gives 4 rows.
        for (int e = tid; e < kGBK * (kGBM / 4); e += kGThreads) {
            const int ii = e / (kGBM / 4), qq = e % (kGBM / 4);
            const int64_t i = i0 + ii;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < i_end) z = gauss4((uint32_t)i, (uint32_t)((j0 >> 2) + qq), level, k0, k1);
            zs[ii][qq * 4 + 0] = z.x;
            zs[ii][qq * 4 + 1] = z.y;
            zs[ii][qq * 4 + 2] = z.z;
            zs[ii][qq * 4 + 3] = z.w;
        }
        for (int e = tid; e < kGBK * kGBN; e += kGThreads) {
            const int ii = e / kGBN, cc = e % kGBN;
            const int64_t i = i0 + ii;
            as[ii][cc] = (i < i_end && c0 + cc < d) ? A[i * d + c0 + cc] : 0.f;
        }
        __syncthreads();
        float cacc[4][4] = {};
#pragma unroll 8
        for (int kk = 0; kk < kGBK; ++kk) {
            float zr[4], ar[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) zr[a] = zs[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) ar[b] = as[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cacc[a][b] = __fmaf_rn(zr[a], ar[b], cacc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b].add(cacc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t j = j0 + ty * 4 + a;
        if (j >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + tx * 4 + b;
            if (c < d) part[((size_t)blockIdx.z * m + j) * d + c] = make_float2(acc[a][b].hi, acc[a][b].lo);
        }
    }
}

int srht_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                 float* SA) {
    const int64_t n_pad = next_pow2_64(n);
    if (m > n_pad) return IHS_EINVAL;
    const int Q = (int)std::min<int64_t>(n_pad, kSrhtQmax);
    int logQ = 0;
    while ((1 << logQ) < Q) ++logQ;
    const int64_t P = n_pad / Q;
    const int64_t CT = ceil_div64(d, kSrhtC);
    int64_t PG = std::max<int64_t>(1, ceil_div64(2 * (int64_t)ctx->sm_count, CT));
    PG = std::min<int64_t>(PG, P);
    // rows + partial buffer
    void* rws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_ROWS, (size_t)m * sizeof(int32_t), &rws));
    int32_t* rows = static_cast<int32_t*>(rws);
    IHS_TRY(ihs_rows_enqueue(ctx, n_pad, m, seed, level, rows));
    void* pws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)PG * m * d * sizeof(float), &pws));
    float* part = static_cast<float*>(pws);
    CUtensorMap amap;
    const bool tma = Q == 1024 && ihs_tensor_map_f32(&amap, A, n, d, d, kR32C, 256) == IHS_OK;
    if (tma) {
        // Selected rows go in chunks of at most 1024 (32 register accumulators
        // per thread); each chunk re-reads A.
        const int64_t chunk = std::min<int64_t>(m, 1024);
        const int64_t CT32 = ceil_div64(d, kR32C);
        // one CTA per SM: a grid of CT32 x PG32 CTAs in whole waves when the
        // block ranges allow it (PG32 = SMs / gcd(CT32, SMs)), else >= 1 wave
        int64_t g = CT32, h = ctx->sm_count;
        while (h) {
            const int64_t t = g % h;
            g = h;
            h = t;
        }
        int64_t PG32 = ctx->sm_count / g;
        if (PG32 > P || PG32 * m * d * 4 > ((int64_t)1 << 30)) PG32 = std::max<int64_t>(1, ceil_div64((int64_t)ctx->sm_count, CT32));
        PG32 = std::min<int64_t>(PG32, P);
        if (PG32 > PG) {
            IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)PG32 * m * d * sizeof(float), &pws));
            part = static_cast<float*>(pws);
        }
        PG = PG32;
        for (int64_t c0 = 0; c0 < m; c0 += chunk) {
            const int64_t mc = std::min<int64_t>(chunk, m - c0);
            int st;
            if (mc <= 32 * 4) st = launch_r32<4>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, part);
            else if (mc <= 32 * 16) st = launch_r32<16>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, part);
            else st = launch_r32<32>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, part);
            IHS_TRY(st);
        }
    } else {
        const size_t base = ((size_t)Q * (kSrhtC + 1) + Q) * sizeof(float);
        const size_t acc_bytes = (size_t)m * kSrhtC * sizeof(float);
        const int acc_in_smem = (base + acc_bytes <= 200 * 1024) ? 1 : 0;
        const size_t smem = base + (acc_in_smem ? acc_bytes : 0);
        IHS_CUDA_TRY(ihs_allow_smem(k_srht_fwht, smem));
        dim3 grid((unsigned)CT, (unsigned)PG);
        k_srht_fwht<<<grid, kSrhtThreads, smem, ctx->stream>>>(A, n, (int)d, m, Q, logQ, P, (int)PG, rows,
                                                              (uint32_t)level, (uint32_t)seed,
                                                              (uint32_t)(seed >> 32), acc_in_smem, part);
        IHS_LAUNCH_CHECK();
    }
    const int64_t count = m * d;
    const unsigned rgrid = (unsigned)std::min<int64_t>(ceil_div64(count, 256), 8 * (int64_t)ctx->sm_count);
    k_reduce_parts<<<rgrid, 256, 0, ctx->stream>>>(part, (int)PG, count, 1.0 / sqrt((double)m), SA);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

int gauss_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                  float* SA) {
    const int64_t MT = ceil_div64(m, kGBM), NT = ceil_div64(d, kGBN);
    int64_t KS = std::max<int64_t>(1, ceil_div64(4 * (int64_t)ctx->sm_count, MT * NT));
    KS = std::min<int64_t>(KS, ceil_div64(n, 4 * kGBK));
    KS = std::min<int64_t>(KS, 256);
    const int64_t rows_per_split = ceil_div64(ceil_div64(n, KS), kGBK) * kGBK;
    KS = ceil_div64(n, rows_per_split);
    void* pws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)KS * m * d * sizeof(float2), &pws));
    float2* part = static_cast<float2*>(pws);
    dim3 grid((unsigned)MT, (unsigned)NT, (unsigned)KS);
    k_gauss_simt<<<grid, kGThreads, 0, ctx->stream>>>(A, n, (int)d, m, rows_per_split, (uint32_t)level,
                                                     (uint32_t)seed, (uint32_t)(seed >> 32), part);
    IHS_LAUNCH_CHECK();
    const int64_t count = m * d;
    const unsigned rgrid = (unsigned)std::min<int64_t>(ceil_div64(count, 256), 8 * (int64_t)ctx->sm_count);
    k_reduce_parts2<<<rgrid, 256, 0, ctx->stream>>>(part, (int)KS, count, 1.0 / sqrt((double)m), SA);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

}  // namespace

int ihs_gauss_fp32_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                           int32_t level, float* SA) {
    if (n < 1 || d < 1 || m < 1 || level < 0) return IHS_EINVAL;
    return gauss_enqueue(ctx, A, n, d, m, seed, level, SA);
}

int ihs_sketch_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, int32_t kind,
                       uint64_t seed, int32_t level, float* SA) {
    if (n < 1 || d < 1 || m < 1 || level < 0 || m > ((int64_t)1 << 31)) return IHS_EINVAL;
    if (kind == IHS_SKETCH_SRHT) return srht_enqueue(ctx, A, n, d, m, seed, level, SA);
    if (kind == IHS_SKETCH_GAUSS) {
        if (ctx->p.precision == IHS_PREC_BF16) return ihs_gauss_tc_enqueue(ctx, A, n, d, m, seed, level, SA, 0);
        if (ctx->p.precision == IHS_PREC_FP8) return ihs_gauss_tc_enqueue(ctx, A, n, d, m, seed, level, SA, 1);
        return gauss_enqueue(ctx, A, n, d, m, seed, level, SA);
    }
    return IHS_EINVAL;
}

extern "C" int ihs_sketch(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, int32_t kind,
                          uint64_t seed, int32_t level, float* SA) {
    if (!ctx || !A || !SA) return IHS_EINVAL;
    IHS_TRY(ihs_sketch_enqueue(ctx, A, n, d, m, kind, seed, level, SA));
    return IHS_OK;
}
