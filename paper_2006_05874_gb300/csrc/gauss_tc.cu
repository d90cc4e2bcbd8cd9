// Gaussian sketch SA = S A on the 5th-generation tensor cores (tcgen05).
//
// S_ji = z_ji / sqrt(m) (Sec. 1, App. C.1) is generated in-kernel from Philox
// and Box-Muller and never stored; A (FP32 in HBM) and the generated Z tile are
// rounded to BF16 while being written to shared memory in the K-major,
// no-swizzle canonical layout of the tensor core (core matrices of 8 rows x 16
// bytes; 128 B apart along K, (K/8) 128 B apart along M/N).  One CTA computes a
// 128 x 256 tile of Z A over a range of rows of A (split-K): per 64-row chunk,
// all threads produce the operand tiles into one of two shared stages, one
// thread issues four tcgen05.mma (M=128, N=256, K=16, FP32 accumulation in
// tensor memory) and commits them to the stage's mbarrier, so the next chunk
// is produced while the tensor core consumes this one.  The epilogue reads the
// accumulator with tcgen05.ld and writes FP32 partials, which a fixed-order
// reduction sums and scales by 1/sqrt(m).
//
// FP8 (E4M3) variant: the same pipeline with 128-element K chunks (still 128
// bytes per row), tcgen05.mma kind::f8f6f4 with K = 32, Z rounded to E4M3, and
// A quantised per column: s_j = fl32(amax_j / 448), r_j = fl32(1 / s_j),
// q_ij = E4M3(fl32(a_ij r_j)); the reduction multiplies column j by s_j.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int TC_M = 128, TC_N = 256, TC_THREADS = 256;
constexpr int TC_RB = 128;                                   // bytes of one row per K chunk
constexpr uint32_t TC_ZBYTES = TC_M * TC_RB;                 // 16 KiB
constexpr uint32_t TC_ABYTES = TC_N * TC_RB;                 // 32 KiB
constexpr uint32_t TC_STAGE = TC_ZBYTES + TC_ABYTES;         // 48 KiB
constexpr uint32_t TC_SMEM = 2 * TC_STAGE + 64;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t desc = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    desc |= (uint64_t)(lbo >> 4) << 16;
    desc |= (uint64_t)(sbo >> 4) << 32;
    desc |= 1ull << 46;   // descriptor version of the sm_100 family; no swizzle
    return desc;
}

// byte offset of (row r, byte kb along K) in a K-major no-swizzle tile whose
// rows hold TC_RB bytes: core matrices of 8 rows x 16 bytes
__device__ __forceinline__ uint32_t kmaj(int r, int kb) {
    return (uint32_t)((r >> 3) * (TC_RB / 16) * 128 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
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

// FMT 0: BF16 operands (K chunk 64, MMA K 16); FMT 1: E4M3 (K chunk 128, MMA K 32).
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_gauss_tc(const float* __restrict__ A, int64_t n, int d, int64_t m, int64_t rows_per_split, uint32_t level,
           uint32_t k0, uint32_t k1, const float* __restrict__ col_recip, unsigned* status,
           float* __restrict__ part /* KS x m x d */) {
    constexpr int EB = FMT == 0 ? 2 : 1;     // bytes per element
    constexpr int KE = TC_RB / EB;           // K elements per chunk
    constexpr int CW = 16 / EB;              // elements per 16-byte vector
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * TC_STAGE);   // 2 mbarriers
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t j0 = (int64_t)blockIdx.x * TC_M;
    const int c0 = blockIdx.y * TC_N;
    const int64_t i_begin = (int64_t)blockIdx.z * rows_per_split;
    const int64_t i_end = min(n, i_begin + rows_per_split);
    const int64_t nchunks = i_end > i_begin ? ceil_div64(i_end - i_begin, KE) : 0;
    const int mrows = (int)min((int64_t)TC_M, m - j0);
    const int nq = (mrows + 3) >> 2;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
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
    // F32 accumulator; A/B formats: BF16 = 1 (kind::f16), E4M3 = 0 (kind::f8f6f4); both K-major
    const uint32_t fmtbits = FMT == 0 ? ((1u << 7) | (1u << 10)) : 0u;
    const uint32_t idesc = (1u << 4) | fmtbits | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    const int col = c0 + tid;
    const bool colok = col < d;
    const float crec = (FMT == 1 && colok) ? col_recip[col] : 1.f;
    bool ok = true;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int s = (int)(c & 1);
        unsigned char* zt = sm + s * TC_STAGE;
        unsigned char* at = zt + TC_ZBYTES;
        if (c >= 2) {
            // the MMAs of chunk c-2 must be done reading this stage
            const bool w = mbar_wait_bounded(&bar[s], (uint32_t)(((c - 2) >> 1) & 1), status);
            if (__syncthreads_or(!w)) {
                ok = false;
                break;
            }
        }
        const int64_t i0 = i_begin + c * KE;
        // Z tile: thread = (quad q of four sketch rows, group of CW columns of Z)
        {
            const int q = tid >> 3, ig = tid & 7;
            uint32_t pk[4][4];
            if (q < nq) {
                float zv[4][CW];
#pragma unroll
                for (int t = 0; t < CW; ++t) {
                    const float4 z = gauss4_fast((uint32_t)(i0 + CW * ig + t), (uint32_t)((j0 >> 2) + q), level, k0, k1);
                    zv[0][t] = z.x;
                    zv[1][t] = z.y;
                    zv[2][t] = z.z;
                    zv[3][t] = z.w;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        pk[r][t] = FMT == 0 ? pack_bf16(zv[r][2 * t], zv[r][2 * t + 1])
                                            : pack_e4m3(zv[r][4 * t], zv[r][4 * t + 1], zv[r][(4 * t + 2) % CW],
                                                        zv[r][(4 * t + 3) % CW]);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int t = 0; t < 4; ++t) pk[r][t] = 0u;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                *reinterpret_cast<uint4*>(zt + kmaj(4 * q + r, 16 * ig)) = make_uint4(pk[r][0], pk[r][1], pk[r][2], pk[r][3]);
        }
        // A tile: thread = one column of A, KE/CW groups of CW consecutive rows
        {
#pragma unroll 2
            for (int kg = 0; kg < KE / CW; ++kg) {
                float v[CW];
#pragma unroll
                for (int t = 0; t < CW; ++t) {
                    const int64_t row = i0 + CW * kg + t;
                    const float a = (colok && row < i_end) ? __ldg(A + row * d + col) : 0.f;
                    v[t] = FMT == 1 ? __fmul_rn(a, crec) : a;
                }
                uint4 pk;
                if (FMT == 0) {
                    pk = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                    pack_bf16(v[6], v[7]));
                } else {
                    pk = make_uint4(pack_e4m3(v[0], v[1], v[2 % CW], v[3 % CW]), pack_e4m3(v[4 % CW], v[5 % CW], v[6 % CW], v[7 % CW]),
                                    pack_e4m3(v[8 % CW], v[9 % CW], v[10 % CW], v[11 % CW]),
                                    pack_e4m3(v[12 % CW], v[13 % CW], v[14 % CW], v[15 % CW]));
                }
                *reinterpret_cast<uint4*>(at + kmaj(tid, 16 * kg)) = pk;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t za = smem_u32(zt), aa = smem_u32(at);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {   // four MMAs of 32 bytes along K
                const uint64_t ad = umma_desc(za + ks * 256, 128, (TC_RB / 16) * 128);
                const uint64_t bd = umma_desc(aa + ks * 256, 128, (TC_RB / 16) * 128);
                const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
                if (FMT == 0) {
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                } else {
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[s]))
                         : "memory");
        }
    }
    if (nchunks > 0) {
        // the last commit tracks every MMA issued before it
        const int64_t last = nchunks - 1;
        const bool w = mbar_wait_bounded(&bar[last & 1], (uint32_t)((last >> 1) & 1), status);
        if (!w) ok = false;
    }
    ok = !__syncthreads_or(!ok);
    tc_fence_after();
    if (ok) {
        const int quad = warp & 3, half = warp >> 2;
        const int row = 32 * quad + lane;
        float* dst = part + ((size_t)blockIdx.z * m + j0 + row) * d;
#pragma unroll 1
        for (int cc = 0; cc < TC_N / 2; cc += 32) {
            const int colb = half * (TC_N / 2) + cc;
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
            if (row < mrows) {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int cidx = c0 + colb + t;
                    if (cidx < d) dst[cidx] = nchunks > 0 ? __uint_as_float(v[t]) : 0.f;
                }
            }
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

// out[e] = colscale[e % d] * scale * sum_k part[k][e]  (fixed order, FP64)
__global__ void k_reduce_parts_colscale(const float* __restrict__ part, int K, int64_t count, int d, double scale,
                                        const float* __restrict__ colscale, float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (double)part[(size_t)k * count + e];
        out[e] = (float)(s * scale * (double)colscale[e % d]);
    }
}

__global__ void k_reduce_parts_tc(const float* __restrict__ part, int K, int64_t count, double scale,
                                  float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (double)part[(size_t)k * count + e];
        out[e] = (float)(s * scale);
    }
}

}  // namespace

int ihs_gauss_tc_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                         float* SA, int fp8) {
    const int KE = fp8 ? 128 : 64;
    const int64_t MT = ceil_div64(m, TC_M), NT = ceil_div64(d, TC_N);
    int64_t KS = std::max<int64_t>(1, ceil_div64(2 * (int64_t)ctx->sm_count, MT * NT));
    KS = std::min<int64_t>(KS, std::max<int64_t>(1, n / (4 * KE)));
    const int64_t rows_per_split = ceil_div64(ceil_div64(n, KS), KE) * KE;
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
    if (fp8) {
        IHS_CUDA_TRY(cudaFuncSetAttribute(k_gauss_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        k_gauss_tc<1><<<grid, TC_THREADS, TC_SMEM, ctx->stream>>>(A, n, (int)d, m, rows_per_split, (uint32_t)level,
                                                                 (uint32_t)seed, (uint32_t)(seed >> 32), crecip,
                                                                 ctx->d_status, part);
    } else {
        IHS_CUDA_TRY(cudaFuncSetAttribute(k_gauss_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        k_gauss_tc<0><<<grid, TC_THREADS, TC_SMEM, ctx->stream>>>(A, n, (int)d, m, rows_per_split, (uint32_t)level,
                                                                 (uint32_t)seed, (uint32_t)(seed >> 32), nullptr,
                                                                 ctx->d_status, part);
    }
    IHS_LAUNCH_CHECK();
    const int64_t count = m * d;
    const unsigned rgrid = (unsigned)std::min<int64_t>(ceil_div64(count, 256), 8 * (int64_t)ctx->sm_count);
    if (fp8) {
        k_reduce_parts_colscale<<<rgrid, 256, 0, ctx->stream>>>(part, (int)KS, count, (int)d, 1.0 / sqrt((double)m),
                                                               cscale, SA);
    } else {
        k_reduce_parts_tc<<<rgrid, 256, 0, ctx->stream>>>(part, (int)KS, count, 1.0 / sqrt((double)m), SA);
    }
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}
