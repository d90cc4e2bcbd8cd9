// Gaussian sketch SA = S A on the 5th-generation tensor cores (tcgen05).
//
// S_ji = z_ji / sqrt(m) (Sec. 1, App. C.1) is generated in-kernel from Philox
// and Box-Muller and never stored.  One CTA (one per SM: it holds all 512
// tensor-memory columns) computes a 128 x 512 tile of Z A over a range of
// rows of A (split-K), in chunks of 32 rows:
//   * the FP32 rows of A arrive by TMA (two 256-column boxes) in one of two
//     staging buffers, two chunks ahead;
//   * all threads generate the 128 x 32 Z tile and convert the staged A tile,
//     rounding both to BF16 (or E4M3) while writing them to shared memory in
//     the K-major, no-swizzle canonical layout of the tensor core (core
//     matrices of 8 rows x 16 bytes; 128 B apart along K, RB / 16 * 128 B apart
//     along M/N, RB = bytes of one row per chunk);
//   * one thread issues the MMAs (M = 128, N = 256 for each half of the tile,
//     FP32 accumulation in tensor memory) and commits them to the operand
//     stage's mbarrier, so the next chunk is produced while the tensor core
//     consumes this one.
// The epilogue reads the accumulators with tcgen05.ld and writes FP32
// partials, which a fixed-order reduction sums and scales by 1/sqrt(m).
//
// FP8 (E4M3) variant: the same pipeline with tcgen05.mma kind::f8f6f4 (K = 32),
// Z rounded to E4M3, and A quantised per column: s_j = fl32(amax_j / 448),
// r_j = fl32(1 / s_j), q_ij = E4M3(fl32(a_ij r_j)); the reduction multiplies
// column j by s_j.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace {

constexpr int TC_M = 128, TC_N = 512, TC_THREADS = 512;
constexpr int TC_KE = 32;                                     // rows of A per chunk
constexpr uint32_t TC_STG = TC_KE * TC_N * 4;                 // FP32 staging buffer: 64 KiB
// operand stage of format FMT (bytes per element EB): Z 128 x RB, A 512 x RB
__host__ __device__ constexpr uint32_t tc_rb(int fmt) { return TC_KE * (fmt == 0 ? 2 : 1); }
__host__ __device__ constexpr uint32_t tc_stage(int fmt) { return (TC_M + TC_N) * tc_rb(fmt); }
__host__ __device__ constexpr uint32_t tc_smem(int fmt) { return 2 * TC_STG + 2 * tc_stage(fmt) + 64; }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t desc = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    desc |= (uint64_t)(lbo >> 4) << 16;
    desc |= (uint64_t)(sbo >> 4) << 32;
    desc |= 1ull << 46;   // descriptor version of the sm_100 family; no swizzle
    return desc;
}

// byte offset of (row r, byte kb along K) in a K-major no-swizzle tile whose
// rows hold RB bytes: core matrices of 8 rows x 16 bytes
template <int RB>
__device__ __forceinline__ uint32_t kmaj(int r, int kb) {
    return (uint32_t)((r >> 3) * (RB / 16) * 128 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// four E4M3 bytes, first value in the lowest byte
__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float e) {
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, e), __NV_SATFINITE, __NV_E4M3);
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// FMT 0: BF16 operands (MMA K 16); FMT 1: E4M3 (MMA K 32).  TMA false: A
// cannot be described by a tensor map (d % 4 != 0 or misaligned); the
// threads then read the chunk's A values from global memory directly.
template <int FMT, bool TMA>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_gauss_tc(const __grid_constant__ CUtensorMap amap, const float* __restrict__ A, int64_t n, int d, int64_t m,
           int64_t rows_per_split,
           uint32_t level, uint32_t k0, uint32_t k1, uint32_t zq0 /* first z row / 4 */,
           uint32_t ibase /* global row of A's row 0 */, const float* __restrict__ col_recip, unsigned* status,
           float* __restrict__ part /* KS x m x d */) {
    constexpr int RB = (int)tc_rb(FMT);                 // operand bytes per row per chunk
    constexpr uint32_t ZB = TC_M * RB, STAGE = tc_stage(FMT);
    constexpr int KSTEPS = RB / 32;                      // MMAs along K per chunk and half
    extern __shared__ __align__(1024) unsigned char sm[];
    float* stg = reinterpret_cast<float*>(sm);                                   // 2 x [32][512] FP32
    unsigned char* ops = sm + 2 * TC_STG;                                        // 2 operand stages
    uint64_t* bar = reinterpret_cast<uint64_t*>(ops + 2 * STAGE);                // mma_done[2], tma_full[2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t j0 = (int64_t)blockIdx.x * TC_M;
    const int c0 = blockIdx.y * TC_N;
    const int64_t i_begin = (int64_t)blockIdx.z * rows_per_split;
    const int64_t i_end = min(n, i_begin + rows_per_split);
    const int64_t nchunks = i_end > i_begin ? ceil_div64(i_end - i_begin, TC_KE) : 0;
    const int mrows = (int)min((int64_t)TC_M, m - j0);
    const int nq = (mrows + 3) >> 2;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    int64_t issued = 0;   // chunks whose staging load thread 0 has issued
    auto issue_tma = [&](int64_t c) {
        issued = c + 1;
        const int b = (int)(c & 1);
        mbar_arrive_expect_tx(&bar[2 + b], TC_STG);
        const int y = (int)(i_begin + c * TC_KE);
        tma_load_2d(stg + (size_t)b * TC_KE * TC_N, &amap, c0, y, &bar[2 + b]);
        tma_load_2d(stg + (size_t)b * TC_KE * TC_N + TC_KE * 256, &amap, c0 + 256, y, &bar[2 + b]);
    };
    if (TMA && tid == 0) {
        for (int64_t c = 0; c < min((int64_t)2, nchunks); ++c) issue_tma(c);
    }
    // F32 accumulator; A/B formats: BF16 = 1 (kind::f16), E4M3 = 0 (kind::f8f6f4); both K-major; N = 256
    const uint32_t fmtbits = FMT == 0 ? ((1u << 7) | (1u << 10)) : 0u;
    const uint32_t idesc = (1u << 4) | fmtbits | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    // this thread's column of A (FP8 scale)
    const int nc = tid;
    const float crec0 = (FMT == 1 && c0 + nc < d) ? col_recip[c0 + nc] : 1.f;
    bool ok = true;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int s = (int)(c & 1);
        unsigned char* zt = ops + s * STAGE;
        unsigned char* at = zt + ZB;
        if (c >= 2) {
            // the MMAs of chunk c-2 must be done reading this operand stage
            const bool w = mbar_wait_bounded(&bar[s], (uint32_t)(((c - 2) >> 1) & 1), status);
            if (__syncthreads_or(!w)) {
                ok = false;
                break;
            }
        }
        const int64_t i0 = i_begin + c * TC_KE;
        // Z tile: thread = (quad q of four sketch rows, two consecutive columns of Z)
        {
            const int q = tid >> 4, ig = tid & 15;
            float zv[4][2];
            if (q < nq) {
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const float4 z = gauss4_fast(ibase + (uint32_t)(i0 + 2 * ig + t), zq0 + (uint32_t)((j0 >> 2) + q), level, k0, k1);
                    zv[0][t] = z.x;
                    zv[1][t] = z.y;
                    zv[2][t] = z.z;
                    zv[3][t] = z.w;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) zv[r][0] = zv[r][1] = 0.f;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (FMT == 0) {
                    *reinterpret_cast<uint32_t*>(zt + kmaj<RB>(4 * q + r, 4 * ig)) = pack_bf16(zv[r][0], zv[r][1]);
                } else {
                    *reinterpret_cast<uint16_t*>(zt + kmaj<RB>(4 * q + r, 2 * ig)) =
                        (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(zv[r][0], zv[r][1]), __NV_SATFINITE, __NV_E4M3);
                }
            }
        }
        // A tile from the staging buffer: thread = one column, all 32 rows
        {
            if (TMA) {
                const bool w = mbar_wait_bounded(&bar[2 + s], (uint32_t)((c >> 1) & 1), status);
                if (__syncthreads_or(!w)) {
                    ok = false;
                    break;
                }
            }
            const float* sb = stg + (size_t)s * TC_KE * TC_N;
            const int rvalid = (int)min((int64_t)TC_KE, i_end - i0);   // rows of the split in this chunk
            constexpr int G = FMT == 0 ? 8 : 16;                        // rows per 16-byte group
#pragma unroll
            for (int g = 0; g < TC_KE / G; ++g) {
                float v0[G];
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int r = G * g + t;
                    const bool rv = r < rvalid;
                    float a;
                    if (TMA) {
                        const int half = nc >= 256;
                        a = sb[half * TC_KE * 256 + r * 256 + (nc & 255)];
                    } else {
                        a = (rv && c0 + nc < d) ? __ldg(A + (i0 + r) * (int64_t)d + c0 + nc) : 0.f;
                    }
                    v0[t] = rv ? (FMT == 1 ? __fmul_rn(a, crec0) : a) : 0.f;
                }
                uint4 p0;
                if (FMT == 0) {
                    p0 = make_uint4(pack_bf16(v0[0], v0[1]), pack_bf16(v0[2], v0[3]), pack_bf16(v0[4], v0[5]),
                                    pack_bf16(v0[6], v0[7]));
                } else {
                    p0 = make_uint4(pack_e4m3(v0[0], v0[1], v0[2 % G], v0[3 % G]),
                                    pack_e4m3(v0[4 % G], v0[5 % G], v0[6 % G], v0[7 % G]),
                                    pack_e4m3(v0[8 % G], v0[9 % G], v0[10 % G], v0[11 % G]),
                                    pack_e4m3(v0[12 % G], v0[13 % G], v0[14 % G], v0[15 % G]));
                }
                *reinterpret_cast<uint4*>(at + kmaj<RB>(nc, 16 * g)) = p0;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            // the staging buffer of chunk c is free again: fetch chunk c + 2 into it
            if (TMA && c + 2 < nchunks) issue_tma(c + 2);
            const uint32_t za = smem_u32(zt), aa = smem_u32(at);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int ks = 0; ks < KSTEPS; ++ks) {   // MMAs of 32 bytes along K
                    const uint64_t ad = umma_desc(za + ks * 256, 128, (RB / 16) * 128);
                    const uint64_t bd = umma_desc(aa + (uint32_t)h * (256 / 8) * (RB / 16) * 128 + ks * 256, 128,
                                                  (RB / 16) * 128);
                    const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
                    const uint32_t tacc = taddr + (uint32_t)(h * 256);
                    if (FMT == 0) {
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tacc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    } else {
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tacc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[s]))
                         : "memory");
        }
    }
    if (nchunks > 0) {
        // the last commit tracks every MMA issued before it; TMA loads issued
        // for chunks never consumed (only after a failed wait) land first
        const int64_t last = nchunks - 1;
        if (tid == 0) {
            if (!mbar_wait_bounded(&bar[last & 1], (uint32_t)((last >> 1) & 1), status)) ok = false;
        }
    }
    ok = !__syncthreads_or(!ok);
    if (!ok && tid == 0) {
        // let the (at most two) staging loads still in flight land
        for (int64_t cc = max((int64_t)0, issued - 2); cc < issued; ++cc)
            mbar_wait_bounded(&bar[2 + (cc & 1)], (uint32_t)((cc >> 1) & 1), status);
    }
    tc_fence_after();
    if (ok) {
        const int quad = warp & 3, cpart = warp >> 2;   // TMEM lane quadrant, quarter of the columns
        float* tile = stg + warp * (32 * 33);            // the staging buffers are idle now
#pragma unroll 1
        for (int cc = 0; cc < TC_N / 4; cc += 32) {
            const int colb = cpart * (TC_N / 4) + cc;
            uint32_t v[32];
            const uint32_t a = taddr + ((uint32_t)(32 * quad) << 16) + (uint32_t)colb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(a));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // transpose through this warp's 32 x 33 shared tile so that each
            // store writes 32 consecutive floats of one row
#pragma unroll
            for (int t = 0; t < 32; ++t) tile[lane * 33 + t] = nchunks > 0 ? __uint_as_float(v[t]) : 0.f;
            __syncwarp();
            const int cidx = c0 + colb + lane;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int grow = 32 * quad + rr;
                if (grow < mrows && cidx < d)
                    part[((size_t)blockIdx.z * m + j0 + grow) * d + cidx] = tile[rr * 33 + lane];
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_N));
}

// Column maxima of |A| (as ordered uint bits of non-negative floats).
__global__ void k_col_amax(const float* __restrict__ A, int64_t n, int d, int64_t rows_per_block,
                           unsigned* __restrict__ amax) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= d) return;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_block;
    const int64_t i1 = min(n, i0 + rows_per_block);
    float mx = 0.f;
    for (int64_t i = i0; i < i1; ++i) mx = fmaxf(mx, fabsf(A[i * d + col]));
    atomicMax(&amax[col], __float_as_uint(mx));
}

// s_j = fl32(amax_j / 448) (1 when the column is zero), r_j = fl32(1 / s_j).
__global__ void k_col_scales(const unsigned* __restrict__ amax, int d, float* __restrict__ scale,
                             float* __restrict__ recip) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= d) return;
    const float a = __uint_as_float(amax[col]);
    const float sc = a > 0.f ? __fdiv_rn(a, 448.f) : 1.f;
    scale[col] = sc;
    recip[col] = __frcp_rn(sc);
}

}  // namespace

int ihs_gauss_tc_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                         float* SA, int fp8, int64_t zrow0, int64_t m_scale, int64_t grow0) {
    if (m_scale <= 0) m_scale = m;
    CUtensorMap amap;
    memset(&amap, 0, sizeof(amap));
    const bool tma = ihs_tensor_map_f32(&amap, A, n, d, d, 256, TC_KE) == IHS_OK;
    const int64_t MT = ceil_div64(m, TC_M), NT = ceil_div64(d, TC_N);
    // split-K so that the CTAs (one per SM) fill whole waves: the wave count w
    // in 1..4 whose split count KS = floor(w SMs / (MT NT)) wastes the least
    const int64_t sms = ctx->sm_count, tiles = MT * NT;
    const int64_t kmax = std::max<int64_t>(1, n / (4 * TC_KE));
    int64_t KS = 1;
    double best = -1.0;
    for (int64_t w = 1; w <= 4; ++w) {
        const int64_t ks = std::min<int64_t>(kmax, std::max<int64_t>(1, (w * sms) / tiles));
        const double eff = (double)(tiles * ks) / (double)(ceil_div64(tiles * ks, sms) * sms);
        if (eff > best + 1e-9) {
            best = eff;
            KS = ks;
        }
    }
    const int64_t rows_per_split = ceil_div64(ceil_div64(n, KS), TC_KE) * TC_KE;
    KS = ceil_div64(n, rows_per_split);
    void* pws = nullptr;
    const size_t part_bytes = ((size_t)KS * m * d * sizeof(float) + 255) & ~(size_t)255;
    IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, part_bytes + 3 * (size_t)d * sizeof(float) + 256, &pws));
    float* part = static_cast<float*>(pws);
    unsigned* amax = reinterpret_cast<unsigned*>(static_cast<char*>(pws) + part_bytes);
    float* cscale = reinterpret_cast<float*>(amax + d);
    float* crecip = cscale + d;
    if (fp8) {
        IHS_CUDA_TRY(cudaMemsetAsync(amax, 0, (size_t)d * sizeof(unsigned), ctx->stream));
        const int64_t rpb = std::max<int64_t>(256, ceil_div64(n, 4 * (int64_t)ctx->sm_count / std::max<int64_t>(1, ceil_div64(d, 256))));
        dim3 g((unsigned)ceil_div64(d, 256), (unsigned)ceil_div64(n, rpb));
        k_col_amax<<<g, 256, 0, ctx->stream>>>(A, n, (int)d, rpb, amax);
        IHS_LAUNCH_CHECK();
        k_col_scales<<<(unsigned)ceil_div64(d, 256), 256, 0, ctx->stream>>>(amax, (int)d, cscale, crecip);
        IHS_LAUNCH_CHECK();
    }
    dim3 grid((unsigned)MT, (unsigned)NT, (unsigned)KS);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    auto launch = [&](auto kern, int fmt, const float* crec) -> int {
        IHS_CUDA_TRY(ihs_allow_smem(kern, tc_smem(fmt)));
        kern<<<grid, TC_THREADS, tc_smem(fmt), ctx->stream>>>(amap, A, n, (int)d, m, rows_per_split, (uint32_t)level,
                                                              k0, k1, (uint32_t)(zrow0 >> 2), (uint32_t)grow0, crec,
                                                              ctx->d_status, part);
        return IHS_OK;
    };
    if (fp8) IHS_TRY(tma ? launch(k_gauss_tc<1, true>, 1, crecip) : launch(k_gauss_tc<1, false>, 1, crecip));
    else IHS_TRY(tma ? launch(k_gauss_tc<0, true>, 0, nullptr) : launch(k_gauss_tc<0, false>, 0, nullptr));
    IHS_LAUNCH_CHECK();
    return ihs_reduce_parts_enqueue(ctx, part, false, (int)KS, m * d, d, 1.0 / sqrt((double)m_scale),
                                    fp8 ? cscale : nullptr, SA);
}
