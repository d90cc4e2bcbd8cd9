// Fused gradient pass g = A^T (A x - b) + nu^2 x (gradient of Eq. 1; the
// per-iteration O(nd) cost of App. B.4), one read of A.
//
// Fast path (d % 4 == 0, 16-byte aligned A): a persistent grid, one CTA per
// SM, streams contiguous row tiles of A through a ring of shared-memory
// stages filled by 1-D bulk copies (cp.async.bulk, completion on mbarriers).
// Each thread owns CPT float4 column chunks of a row; per row it forms a
// compensated (Dot2) partial of a_i . x, the partials of a row are combined by
// warp shuffles and, across warps, in shared memory in a fixed order; then
// r_i = a_i . x - b_i is broadcast and every thread accumulates r_i a_i into
// compensated per-column accumulators held in registers.  Each CTA writes its
// d partial sums (hi, lo); a second kernel adds the partials in a fixed order
// in FP64, adds nu^2 x and rounds to FP32.  The result is bitwise reproducible
// for a given GPU.
//
// Generic path (any d, any alignment): r = A x - b (one warp per row), then
// A^T r with one thread per column, then the same reduction.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Dynamic shared-memory layout of k_grad_fast: [stages][R*d floats] | mbarriers
// | per-warp row partials | row residuals | FP64 block-reduction slots.
struct FastLayout {
    size_t full, red, rbuf, dred, total;
    __host__ __device__ FastLayout(int stages, int R, int W, int d) {
        full = (size_t)stages * R * d * sizeof(float);
        red = align16(full + 8 * (size_t)stages);
        rbuf = align16(red + sizeof(Acc2) * (size_t)R * W);
        dred = align16(rbuf + sizeof(float) * (size_t)R);
        total = dred + sizeof(double) * kThreads;
    }
};

// Butterfly reduce-scatter of RT per-row compensated partials across the 32
// lanes of a warp: at each of the first log2(RT) steps a lane keeps half of
// its rows and sends the other half to its partner (xor 16, 8, ...); the
// remaining steps are a full butterfly on the one value left.  Lane l ends
// with the warp's sum for row `row_of_lane(l)`; all lanes sharing that row
// hold the same value.
template <int RT>
__device__ __forceinline__ Acc2 warp_reduce_scatter(Acc2 (&v)[RT], int lane, int& row) {
    int count = RT;
    row = 0;
#pragma unroll
    for (int mask = 16; mask >= 1; mask >>= 1) {
        if (count > 1) {
            const int half = count / 2;
            const bool up = (lane & mask) != 0;
#pragma unroll
            for (int i = 0; i < RT / 2; ++i) {
                if (i < half) {
                    const Acc2 keep = up ? v[half + i] : v[i];
                    const Acc2 send = up ? v[i] : v[half + i];
                    const Acc2 got = acc2_shfl_xor(send, mask);
                    v[i] = keep;
                    v[i].add_pair(got.hi, got.lo);
                }
            }
            if (up) row += half;
            count = half;
        } else {
            const Acc2 got = acc2_shfl_xor(v[0], mask);
            v[0].add_pair(got.hi, got.lo);
        }
    }
    return v[0];
}

template <int TPR, int CPT, int RT, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
k_grad_fast(const float* __restrict__ A, const float* __restrict__ b, const float* __restrict__ x,
            int64_t n, int d, int64_t ntiles, int stages, float2* __restrict__ part,
            double* __restrict__ part_ax2, unsigned* status) {
    constexpr int RP = kThreads / TPR;  // rows handled in parallel
    constexpr int R = RT * RP;          // rows per stage
    constexpr int W = TPR / 32;         // warps per row
    extern __shared__ __align__(128) unsigned char smem[];
    const int stage_floats = R * d;
    const FastLayout lay(stages, R, W, d);
    float* stage_base = reinterpret_cast<float*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.full);
    Acc2* red = reinterpret_cast<Acc2*>(smem + lay.red);      // R * W
    float* rbuf = reinterpret_cast<float*>(smem + lay.rbuf);  // R
    double* dred = reinterpret_cast<double*>(smem + lay.dred);

    const int tid = threadIdx.x;
    const int grp = tid / TPR;
    const int t = tid % TPR;
    const int wir = t / 32;   // warp index within the row's warps
    const int lane = tid & 31;
    const int chunks = d >> 2;

    const int64_t t0 = (int64_t)blockIdx.x * ntiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * ntiles / gridDim.x;
    const int64_t my_tiles = t1 - t0;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    float4 xr[CPT];
    bool cvalid[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = t + TPR * k;
        cvalid[k] = c < chunks;
        xr[k] = cvalid[k] ? reinterpret_cast<const float4*>(x)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    Acc2 gacc[CPT][4];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) gacc[k][q] = Acc2{0.f, 0.f};
    double ax2 = 0.0;

    auto issue = [&](int64_t local) {
        const int s = (int)(local % stages);
        const int64_t row0 = (t0 + local) * R;
        const int64_t rows = min((int64_t)R, n - row0);
        const uint32_t bytes = (uint32_t)(rows * d * sizeof(float));
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_g2s(stage_base + (size_t)s * stage_floats, A + row0 * d, bytes, &full[s]);
    };

    int64_t issued = 0;
    if (tid == 0) {
        for (; issued < min((int64_t)(stages - 1), my_tiles); ++issued) issue(issued);
    }
    int64_t consumed = 0;
    int s = 0;
    uint32_t ph = 0;
    for (int64_t l = 0; l < my_tiles; ++l, s = (s + 1 == stages ? 0 : s + 1), ph ^= (s == 0 ? 1u : 0u)) {
        if (tid == 0 && l + stages - 1 < my_tiles) {
            issue(l + stages - 1);
            issued = l + stages;
        }
        const bool ok = mbar_wait_bounded(&full[s], ph, status);
        if (__syncthreads_or(!ok)) break;
        consumed = l + 1;

        const float* st = stage_base + (size_t)s * stage_floats;
        const int64_t row0 = (t0 + l) * R;
        const int rows = (int)min((int64_t)R, n - row0);

        float4 a[RT][CPT];
        Acc2 dot[RT];
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const int rr = grp + j * RP;
            dot[j] = Acc2{0.f, 0.f};
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int c = t + TPR * k;
                a[j][k] = (cvalid[k] && rr < rows) ? reinterpret_cast<const float4*>(st + (size_t)rr * d)[c]
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                dot[j].add_prod(a[j][k].x, xr[k].x);
                dot[j].add_prod(a[j][k].y, xr[k].y);
                dot[j].add_prod(a[j][k].z, xr[k].z);
                dot[j].add_prod(a[j][k].w, xr[k].w);
            }
        }
        int myrow = 0;   // row (0..RT-1 within this thread's rows) whose warp sum this lane holds
        const Acc2 wsum = warp_reduce_scatter<RT>(dot, lane, myrow);
        // lanes holding row j: a contiguous group of 32/RT lanes starting at j*(32/RT)
        const bool leader = (lane & (32 / RT - 1)) == 0;
        float rv[RT];
        if (W == 1) {
            // the warp owns whole rows: lanes form r and broadcast it with shuffles
            __syncthreads();   // every thread is done with stage s
            const int rr = grp + myrow * RP;
            float r = 0.f;
            if (rr < rows) {
                r = __fadd_rn(__fsub_rn(wsum.hi, b[row0 + rr]), wsum.lo);
                if (leader) {
                    const double v = (double)wsum.hi + (double)wsum.lo;
                    ax2 += v * v;
                }
            }
#pragma unroll
            for (int j = 0; j < RT; ++j) rv[j] = __shfl_sync(0xffffffffu, r, j * (32 / RT));
        } else {
            if (leader) red[(grp + myrow * RP) * W + wir] = wsum;
            __syncthreads();   // stage s consumed, per-warp partials visible
            if (tid < R) {
                const int rr = tid;
                Acc2 s2 = red[rr * W];
#pragma unroll
                for (int w = 1; w < W; ++w) s2.add_pair(red[rr * W + w].hi, red[rr * W + w].lo);
                float r = 0.f;
                if (rr < rows) {
                    r = __fadd_rn(__fsub_rn(s2.hi, b[row0 + rr]), s2.lo);
                    const double v = (double)s2.hi + (double)s2.lo;
                    ax2 += v * v;
                }
                rbuf[rr] = r;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < RT; ++j) rv[j] = rbuf[grp + j * RP];
        }
        // g += sum_rows r_i a_i : an FMA chain over the RT rows, then one
        // compensated add per column.
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                s0 = __fmaf_rn(rv[j], a[j][k].x, s0);
                s1 = __fmaf_rn(rv[j], a[j][k].y, s1);
                s2 = __fmaf_rn(rv[j], a[j][k].z, s2);
                s3 = __fmaf_rn(rv[j], a[j][k].w, s3);
            }
            gacc[k][0].add(s0);
            gacc[k][1].add(s1);
            gacc[k][2].add(s2);
            gacc[k][3].add(s3);
        }
    }
    if (consumed < my_tiles) {
        // A wait gave up: let the copies already issued land before exiting.
        if (tid == 0) {
            for (int64_t l = consumed; l < issued; ++l)
                mbar_wait_bounded(&full[l % stages], (uint32_t)((l / stages) & 1), status);
        }
        __syncthreads();
        return;
    }
    __syncthreads();
    // Combine the RP row groups (same columns) in a fixed order.
    Acc2* comb = reinterpret_cast<Acc2*>(smem);   // RP x d, stages are idle now
    if (RP > 1) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = t + TPR * k;
            if (cvalid[k]) {
#pragma unroll
                for (int q = 0; q < 4; ++q) comb[(size_t)grp * d + 4 * c + q] = gacc[k][q];
            }
        }
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int c = t + TPR * k;
                if (cvalid[k]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        for (int g2 = 1; g2 < RP; ++g2) {
                            const Acc2 o = comb[(size_t)g2 * d + 4 * c + q];
                            gacc[k][q].add_pair(o.hi, o.lo);
                        }
                    }
                }
            }
        }
    }
    if (grp == 0) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = t + TPR * k;
            if (cvalid[k]) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    part[(size_t)blockIdx.x * d + 4 * c + q] = make_float2(gacc[k][q].hi, gacc[k][q].lo);
            }
        }
    }
    // ||A x||^2 partial of this CTA, fixed-order block reduction.
    __syncthreads();
    dred[tid] = ax2;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads; ++i) s += dred[i];
        part_ax2[blockIdx.x] = s;
    }
}

// Wide-row fast path (1024 <= d <= 8192): warp-specialised, two-phase, with
// packed FP32x2 arithmetic.
//
// Tiles of R rows (32 KB) stream through S shared-memory stages: a producer
// thread issues one 1-D bulk copy for the rows and 4-byte cp.async copies for
// their b entries, both completing on the stage's `full` mbarrier.  Sixteen
// consumer warps split every row into NSEG column segments of 128 float4
// chunks (warp w: row w / NSEG, segment w % NSEG) and run per tile:
//   phase 1: per lane a compensated Dot2 partial of a_i . x over its 16
//            columns (two at a time in packed FP32x2 registers), stored to
//            shared memory;
//   phase 2: for the previous tile, every consumer thread adds r_i a_i over
//            the tile's rows into compensated accumulators for the CPT float4
//            column chunks it owns.
// A finaliser warp adds the 512 lane partials of a tile in a fixed tree (16
// per lane, then a butterfly over the lanes of a row), forms
// r_i = (hi - b_i) + lo and the FP64 ||A x||^2 terms, and publishes r.  All
// hand-offs (tile landed, partials ready, r ready, stage free) are mbarriers
// with bounded waits; no CTA-wide barrier sits on the streaming path.  The
// partial layout and the final reduction are those of the path above.
constexpr int kV3Consumers = 16;
constexpr int kV3Threads = (kV3Consumers + 2) * 32;   // + finaliser + producer

struct V3Layout {
    size_t pdot, bsh, rsh, bars, total;
    // np: lane partials per tile (consumer lanes x rows per lane)
    __host__ __device__ V3Layout(int S, int R, int d, int np) {
        pdot = align16((size_t)S * R * d * sizeof(float));
        bsh = pdot + (size_t)S * np * sizeof(Acc2);
        rsh = align16(bsh + (size_t)S * R * sizeof(float));
        bars = align16(rsh + (size_t)S * R * 2 * sizeof(float));
        total = bars + 4 * (size_t)S * sizeof(uint64_t);
    }
};

__device__ __forceinline__ void lds_f2x2(uint32_t addr, f2& a, f2& b) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a.v), "=l"(b.v) : "r"(addr));
}
__device__ __forceinline__ f2 lds_f2(uint32_t addr) {
    f2 a;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(a.v) : "r"(addr));
    return a;
}

template <int NSEG, int CPT, bool FULL, int RPW>
__global__ void __launch_bounds__(kV3Threads, 1)
k_grad_v3(const float* __restrict__ A, const float* __restrict__ b, const float* __restrict__ x, int64_t n,
          int d, int64_t ntiles, int S, float2* __restrict__ part, double* __restrict__ part_ax2,
          unsigned* status) {
    constexpr int G16 = kV3Consumers / NSEG;   // row groups of NSEG warps
    constexpr int R = G16 * RPW;               // rows per tile (RPW per row group)
    constexpr int XC = 4;                      // float4 chunks per lane per row
    constexpr int LPR = 32 / R;                // finaliser lanes per row
    constexpr int NP = kV3Consumers * 32 * RPW;   // lane partials per tile
    static_assert(R <= 32, "one finaliser lane per row at least");
    extern __shared__ __align__(128) unsigned char smem[];
    const V3Layout lay(S, R, d, NP);
    float* stage_base = reinterpret_cast<float*>(smem);
    Acc2* pdot = reinterpret_cast<Acc2*>(smem + lay.pdot);   // [S][R][NP / R]
    float* bsh = reinterpret_cast<float*>(smem + lay.bsh);   // [S][R]
    f2* rsh = reinterpret_cast<f2*>(smem + lay.rsh);         // [S][R], (r_i, r_i)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint64_t* rready = full + S;
    uint64_t* rfinal = rready + S;
    uint64_t* empty = rfinal + S;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunks = d >> 2;
    const int64_t t0 = (int64_t)blockIdx.x * ntiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * ntiles / gridDim.x;
    const int64_t my_tiles = t1 - t0;
    const size_t stage_floats = (size_t)R * d;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 2);   // bulk copy of the rows + cp.async of their b
            mbar_init(&rready[s], kV3Consumers);
            mbar_init(&rfinal[s], 1);
            mbar_init(&empty[s], kV3Consumers);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kV3Consumers + 1) {
        // ---- producer ----
        if (lane == 0) {
            int64_t issued = 0;
            bool ok = true;
            int s = 0;
            uint32_t ph = 0;   // parity of the stage's current use
            for (int64_t l = 0; l < my_tiles; ++l) {
                if (l >= S) {
                    ok = mbar_wait_bounded(&empty[s], ph ^ 1u, status);
                    if (!ok) break;
                }
                const int64_t row0 = (t0 + l) * R;
                const int64_t rows = min((int64_t)R, n - row0);
                const uint32_t bytes = (uint32_t)(rows * d * sizeof(float));
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(stage_base + (size_t)s * stage_floats, A + row0 * d, bytes, &full[s]);
                for (int i = 0; i < (int)rows; ++i) cp_async_4(&bsh[s * R + i], b + row0 + i);
                cp_async_mbar_arrive_noinc(&full[s]);
                issued = l + 1;
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) {
                // let the copies still in flight land before the CTA exits
                for (int64_t l = max((int64_t)0, issued - S); l < issued; ++l)
                    mbar_wait_bounded(&full[l % S], (uint32_t)((l / S) & 1), status);
            }
        }
        return;
    }

    if (warp == kV3Consumers) {
        // ---- finaliser: r_i and ||A x||^2 ----
        // lane = row * LPR + q sums partials q, q + LPR, ... of its row, then
        // the LPR lanes of the row combine by a butterfly.
        const int frow = lane / LPR, q = lane % LPR;
        double ax2 = 0.0;
        bool ok = true;
        int s = 0;
        uint32_t ph = 0;
        for (int64_t l = 0; l < my_tiles; ++l) {
            const int rows = (int)min((int64_t)R, n - (t0 + l) * R);
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(&rready[s], ph, status));
            if (!ok) break;
            const Acc2* pr = pdot + ((size_t)s * R + frow) * (NP / R);
            Acc2 acc = pr[q];
#pragma unroll
            for (int t = 1; t < NP / R / LPR; ++t) {
                const Acc2 o = pr[t * LPR + q];
                acc.add_pair(o.hi, o.lo);
            }
#pragma unroll
            for (int off = LPR / 2; off >= 1; off >>= 1) {
                const Acc2 o = acc2_shfl_xor(acc, off);
                acc.add_pair(o.hi, o.lo);
            }
            if (q == 0) {
                float r = 0.f;
                if (frow < rows) {
                    r = __fadd_rn(__fsub_rn(acc.hi, bsh[s * R + frow]), acc.lo);
                    const double v = (double)acc.hi + (double)acc.lo;
                    ax2 += v * v;
                }
                rsh[s * R + frow] = f2_pack(r, r);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&rfinal[s]);
            if (++s == S) {
                s = 0;
                ph ^= 1u;
            }
        }
        // fixed-order fold of the R row-lane sums
        double tot = 0.0;
        for (int i = 0; i < R; ++i) tot += __shfl_sync(0xffffffffu, ax2, i * LPR);
        if (lane == 0) part_ax2[blockIdx.x] = ok ? tot : 0.0;
        return;
    }

    // ---- consumers ----
    const int seg = warp % NSEG, prow = warp / NSEG;
    f2 xa[XC], xb[XC], xan[XC], xbn[XC];   // x chunk as (x, y) and (z, w), and negated
    bool cv[XC];
#pragma unroll
    for (int k = 0; k < XC; ++k) {
        const int c = seg * 32 + lane + NSEG * 32 * k;
        cv[k] = FULL || c < chunks;
        const float4 v = cv[k] ? reinterpret_cast<const float4*>(x)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        xa[k] = f2_pack(v.x, v.y);
        xb[k] = f2_pack(v.z, v.w);
        xan[k] = f2_pack(-v.x, -v.y);
        xbn[k] = f2_pack(-v.z, -v.w);
    }
    // FULL: d = 512 NSEG is a compile-time constant, and so is every shared-memory
    // offset below (no per-tile integer arithmetic beyond the stage step)
    const int dd = FULL ? 512 * NSEG : d;
    constexpr bool ALLP = FULL && NSEG >= 4;   // every consumer thread owns CPT full chunks
    bool pv[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) pv[k] = ALLP || tid + kV3Consumers * 32 * k < chunks;
    // shared-memory byte addresses: stage 0, this lane's phase-1 chunk 0 of its
    // row, this thread's phase-2 chunk 0 of row 0, its pdot slot
    const uint32_t sm0 = smem_u32(smem);
    const uint32_t sbytes = (uint32_t)(R * dd * 4);
    const uint32_t p1_off = (uint32_t)(prow * dd + (seg * 32 + lane) * 4) * 4u;
    const uint32_t p2_off = (uint32_t)tid * 16u;
    const uint32_t row_bytes = (uint32_t)dd * 4u;
    const uint32_t pd0 = smem_u32(pdot) + (uint32_t)((prow * (NP / R) + seg * 32 + lane) * sizeof(Acc2));
    const uint32_t pd_stage = (uint32_t)(R * (NP / R) * sizeof(Acc2));
    const uint32_t rs0 = smem_u32(rsh);
    Acc2x2 gacc[CPT][2];
    const f2 zero2 = f2_pack(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int q = 0; q < 2; ++q) gacc[k][q] = Acc2x2{zero2, zero2};
    bool ok = true;
    int s1 = 0, s2 = 0;          // stages of phase 1 (tile l) and phase 2 (tile l - 1)
    uint32_t ph1 = 0, ph2 = 0;   // their parities
    int64_t row0 = t0 * R;   // first row of tile l
    for (int64_t l = 0; l <= my_tiles; ++l, row0 += R) {
        if (l < my_tiles) {
            const int rows = (int)min((int64_t)R, n - row0);
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s1], ph1, status));
            if (!ok) break;
#pragma unroll
            for (int u = 0; u < RPW; ++u) {
                const int row = prow + G16 * u;
                Acc2x2 pa{zero2, zero2}, pb{zero2, zero2};
                if (row < rows) {
                    const uint32_t base = sm0 + (uint32_t)s1 * sbytes + p1_off + (uint32_t)(u * G16) * row_bytes;
#pragma unroll
                    for (int k = 0; k < XC; ++k) {
                        if (cv[k]) {
                            f2 a01, a23;
                            lds_f2x2(base + (uint32_t)(k * NSEG * 32 * 16), a01, a23);
                            pa.add_prod(a01, xa[k], xan[k]);
                            pb.add_prod(a23, xb[k], xbn[k]);
                        }
                    }
                }
                pa.add_pair(pb.hi, pb.lo);
                float h0, h1, l0, l1;
                f2_unpack(pa.hi, h0, h1);
                f2_unpack(pa.lo, l0, l1);
                Acc2 a0{h0, l0};
                a0.add_pair(h1, l1);
                asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(pd0 + (uint32_t)s1 * pd_stage +
                                                                     (uint32_t)(u * G16 * (NP / R) * sizeof(Acc2))),
                             "f"(a0.hi), "f"(a0.lo)
                             : "memory");
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&rready[s1]);
            if (++s1 == S) {
                s1 = 0;
                ph1 ^= 1u;
            }
        }
        if (l >= 1) {
            const int rows = (int)min((int64_t)R, n - (row0 - R));
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(&rfinal[s2], ph2, status));
            if (!ok) break;
            const uint32_t base = sm0 + (uint32_t)s2 * sbytes + p2_off;
            f2 rr[R];
#pragma unroll
            for (int i = 0; i < R; ++i) rr[i] = lds_f2(rs0 + (uint32_t)((s2 * R + i) * 8));
            if (rows == R) {
                // full tile: no per-row predicates
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    if (pv[k]) {
                        f2 s01 = zero2, s23 = zero2;
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            f2 a01, a23;
                            lds_f2x2(base + (uint32_t)i * row_bytes + (uint32_t)(k * kV3Consumers * 32 * 16), a01,
                                     a23);
                            s01 = f2_fma(rr[i], a01, s01);
                            s23 = f2_fma(rr[i], a23, s23);
                        }
                        gacc[k][0].add(s01);
                        gacc[k][1].add(s23);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    if (pv[k]) {
                        f2 s01 = zero2, s23 = zero2;
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            if (i < rows) {
                                f2 a01, a23;
                                lds_f2x2(base + (uint32_t)i * row_bytes + (uint32_t)(k * kV3Consumers * 32 * 16),
                                         a01, a23);
                                s01 = f2_fma(rr[i], a01, s01);
                                s23 = f2_fma(rr[i], a23, s23);
                            }
                        }
                        gacc[k][0].add(s01);
                        gacc[k][1].add(s23);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s2]);
            if (++s2 == S) {
                s2 = 0;
                ph2 ^= 1u;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = tid + kV3Consumers * 32 * k;
        if (pv[k]) {
            float h0, h1, h2, h3, l0, l1, l2, l3;
            f2_unpack(gacc[k][0].hi, h0, h1);
            f2_unpack(gacc[k][0].lo, l0, l1);
            f2_unpack(gacc[k][1].hi, h2, h3);
            f2_unpack(gacc[k][1].lo, l2, l3);
            float2* o = part + (size_t)blockIdx.x * d + 4 * c;
            o[0] = make_float2(h0, l0);
            o[1] = make_float2(h1, l1);
            o[2] = make_float2(h2, l2);
            o[3] = make_float2(h3, l3);
        }
    }
    (void)ok;
}

// Row group sy's share of column col of the G partials (rows sy, sy + 8, ...),
// summed in order as a compensated pair; the loads go in batches of eight
// ahead of the dependent additions.
__device__ __forceinline__ Acc2 grad_column_sum(const float2* __restrict__ part, int G, int d, int col, int sy) {
    Acc2 a{0.f, 0.f};
    if (col >= d) return a;
    for (int g0 = sy; g0 < G; g0 += 64) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (g0 + 8 * u < G) v[u] = part[(size_t)(g0 + 8 * u) * d + col];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (g0 + 8 * u >= G) break;
            a.add_pair(v[u].x, v[u].y);
        }
    }
    return a;
}

// g[c] = fl32(sum_g (hi + lo) + nu^2 x[c]) over G partials in a fixed order,
// as a compensated binary32 pair (TwoSum): FP64 runs at a small fraction of
// the FP32 rate on this GPU.  ||A x||^2: the G FP64 partials summed by one
// warp in a fixed order (lane strides, then a butterfly).  A non-zero *status
// (status may be NULL) marks a gradient pass whose bounded wait gave up: the
// results are then NaN.
__global__ void __launch_bounds__(256) k_grad_reduce(const float2* __restrict__ part,
                                                     const double* __restrict__ part_ax2, int G, int d, float nu2h,
                                                     float nu2l, const float* __restrict__ x, float* __restrict__ g,
                                                     double* __restrict__ axnorm2, const unsigned* __restrict__ status) {
    __shared__ float2 sm[8][33];
    const bool failed = status != nullptr && *status != 0u;
    const int cx = threadIdx.x & 31, sy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + cx;
    Acc2 a = grad_column_sum(part, G, d, col, sy);
    sm[sy][cx] = make_float2(a.hi, a.lo);
    __syncthreads();
    if (sy == 0 && col < d) {
        for (int k = 1; k < 8; ++k) a.add_pair(sm[k][cx].x, sm[k][cx].y);
        const float2 q = df_mul(x[col], 0.f, nu2h, nu2l);
        a.add_pair(q.x, q.y);
        g[col] = failed ? __int_as_float(0x7fc00000) : __fadd_rn(a.hi, a.lo);
    }
    if (blockIdx.x == 0 && sy == 1 && axnorm2 != nullptr) {
        double t = 0.0;
        for (int gi = cx; gi < G; gi += 32) t += part_ax2[gi];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (cx == 0) *axnorm2 = failed ? __longlong_as_double(0x7ff8000000000000ll) : t;
    }
}

// Generic path, step 1: r_i = a_i . x - b_i (Dot2), one warp per row; per-block
// FP64 partial of ||A x||^2.
__global__ void k_resid_generic(const float* __restrict__ A, const float* __restrict__ b,
                                const float* __restrict__ x, int64_t n, int d, float* __restrict__ r,
                                double* __restrict__ part_ax2) {
    __shared__ double sm[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rows_per_block = 8 * 16;
    const int64_t row_begin = (int64_t)blockIdx.x * rows_per_block;
    double ax2 = 0.0;
    for (int64_t i = row_begin + warp; i < min(n, row_begin + rows_per_block); i += 8) {
        Acc2 acc{0.f, 0.f};
        const float* ai = A + i * d;
        for (int c = lane; c < d; c += 32) acc.add_prod(ai[c], x[c]);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const Acc2 o = acc2_shfl_xor(acc, off);
            acc.add_pair(o.hi, o.lo);
        }
        if (lane == 0) {
            r[i] = __fadd_rn(__fsub_rn(acc.hi, b[i]), acc.lo);
            const double v = (double)acc.hi + (double)acc.lo;
            ax2 += v * v;
        }
    }
    if (lane == 0) sm[warp] = ax2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sm[w];
        part_ax2[blockIdx.x] = s;
    }
}

// Generic path, step 2: per row-group partials of A^T r, one thread per column.
__global__ void k_atr_generic(const float* __restrict__ A, const float* __restrict__ r, int64_t n, int d,
                              int64_t rows_per_group, float2* __restrict__ part) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_group;
    const int64_t i1 = min(n, i0 + rows_per_group);
    if (col >= d) return;
    Acc2 acc{0.f, 0.f};
    for (int64_t i = i0; i < i1; ++i) acc.add(__fmul_rn(r[i], A[i * d + col]));
    part[(size_t)blockIdx.y * d + col] = make_float2(acc.hi, acc.lo);
}

// Sum src[0..count) in order into dst[0] and zero dst[1..G).
__global__ void k_fold_doubles(const double* src, int64_t count, double* dst, int G) {
    double s = 0.0;
    for (int64_t i = 0; i < count; ++i) s += src[i];
    for (int i = 1; i < G; ++i) dst[i] = 0.0;
    dst[0] = s;
}

struct FastCfg {
    int tpr, cpt, rt;
};

FastCfg pick_fast(int d) {
    const int chunks = d / 4;
    if (chunks <= 32) return {32, 1, 8};
    if (chunks <= 64) return {64, 1, 8};
    if (chunks <= 128) return {128, 1, 8};
    if (chunks <= 256) return {256, 1, 8};
    if (chunks <= 512) return {256, 2, 4};
    if (chunks <= 1024) return {256, 4, 2};
    return {256, 8, 1};
}

// Where a gradient launch goes: stream, SM count (grid size) and the status
// word its bounded waits report to.
struct GradTarget {
    cudaStream_t stream;
    int sm_count;
    unsigned* status;
};

template <int TPR, int CPT, int RT, int MINB>
int launch_fast(const GradTarget& tg, const float* A, const float* b, const float* x, int64_t n, int d, float2* part,
                double* part_ax2, int* G_out) {
    constexpr int RP = kThreads / TPR;
    constexpr int R = RT * RP;
    constexpr int W = TPR / 32;
    const size_t stage_bytes = (size_t)R * d * sizeof(float);
    const size_t budget = MINB >= 2 ? 104 * 1024 : 200 * 1024;
    int stages = 8;
    while (stages > 2 && FastLayout(stages, R, W, d).total > budget) --stages;
    size_t smem = FastLayout(stages, R, W, d).total;
    if (smem > budget || stage_bytes * stages > budget) return IHS_EINVAL;
    const size_t comb = (size_t)RP * d * sizeof(Acc2);
    if (smem < comb) smem = comb;
    const int64_t ntiles = ceil_div64(n, R);
    int64_t G = (int64_t)MINB * tg.sm_count;
    if (G > ntiles) G = ntiles;
    auto kern = k_grad_fast<TPR, CPT, RT, MINB>;
    IHS_CUDA_TRY(ihs_allow_smem(kern, smem));
    kern<<<(unsigned)G, kThreads, smem, tg.stream>>>(A, b, x, n, d, ntiles, stages, part, part_ax2, tg.status);
    IHS_LAUNCH_CHECK();
    *G_out = (int)G;
    return IHS_OK;
}

template <int NSEG, int CPT, bool FULL>
int launch_v3(const GradTarget& tg, const float* A, const float* b, const float* x, int64_t n, int d, float2* part,
              double* part_ax2, int* G_out) {
    // two rows per row group: a tile is 64 KB at d = 1024 ... 8192, so the
    // per-tile hand-offs are spread over twice the elements
    constexpr int RPW = 2;
    constexpr int R = RPW * kV3Consumers / NSEG;
    const size_t stage_bytes = (size_t)R * d * sizeof(float);
    int S = (int)std::min<size_t>(8, (192 * 1024) / stage_bytes);
    if (S < 3) return IHS_EINVAL;
    const size_t smem = V3Layout(S, R, d, kV3Consumers * 32 * RPW).total;
    const int64_t ntiles = ceil_div64(n, R);
    int64_t G = tg.sm_count;
    if (G > ntiles) G = ntiles;
    auto kern = k_grad_v3<NSEG, CPT, FULL, RPW>;
    IHS_CUDA_TRY(ihs_allow_smem(kern, smem));
    kern<<<(unsigned)G, kV3Threads, smem, tg.stream>>>(A, b, x, n, d, ntiles, S, part, part_ax2, tg.status);
    IHS_LAUNCH_CHECK();
    *G_out = (int)G;
    return IHS_OK;
}

// Segments per row of the wide-row path for this d: the smallest power of two
// NSEG >= 2 with d / 4 <= 128 NSEG (0: the path does not apply).
int pick_v3(int64_t d) {
    if (d < 1024 || d > 8192 || d % 4) return 0;
    const int64_t chunks = d / 4;
    int nseg = 2;
    while (128 * nseg < chunks) nseg *= 2;
    return nseg;
}

// The fused pass for 16-byte aligned A and x, d % 4 == 0, d <= 8192: the
// wide-row pipeline for 1024 <= d <= 8192, the register reduce-scatter kernel
// (two CTAs per SM) below; partials of G CTAs into part / part_ax2.
int grad_pass_fast(const GradTarget& tg, const float* A, const float* b, const float* x, int64_t n, int64_t d,
                   float2* part, double* part_ax2, int* G_out) {
    int& G = *G_out;
    const int wpr = pick_v3(d);
    if (wpr) {
        int st;
        const bool full = (d % (wpr * 512)) == 0;
        if (wpr == 2) st = full ? launch_v3<2, 1, true>(tg, A, b, x, n, (int)d, part, part_ax2, &G)
                                : launch_v3<2, 1, false>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
        else if (wpr == 4) st = full ? launch_v3<4, 1, true>(tg, A, b, x, n, (int)d, part, part_ax2, &G)
                                     : launch_v3<4, 1, false>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
        else if (wpr == 8) st = full ? launch_v3<8, 2, true>(tg, A, b, x, n, (int)d, part, part_ax2, &G)
                                     : launch_v3<8, 2, false>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
        else st = full ? launch_v3<16, 4, true>(tg, A, b, x, n, (int)d, part, part_ax2, &G)
                       : launch_v3<16, 4, false>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
        return st;
    }
    const FastCfg c = pick_fast((int)d);
    if (c.tpr == 32) return launch_fast<32, 1, 8, 2>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    if (c.tpr == 64) return launch_fast<64, 1, 8, 2>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    if (c.tpr == 128) return launch_fast<128, 1, 8, 2>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    if (c.cpt == 1) return launch_fast<256, 1, 8, 2>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    if (c.cpt == 2) return launch_fast<256, 2, 4, 2>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    if (c.cpt == 4) return launch_fast<256, 4, 2, 1>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
    return launch_fast<256, 8, 1, 1>(tg, A, b, x, n, (int)d, part, part_ax2, &G);
}

}  // namespace

// The per-CTA (or per-row-group) partial sums of A^T (A x - b) and ||A x||^2:
// G partials of d float2 pairs at *part, G doubles at *part_ax2.
static int grad_partials(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, const float* x,
                         float2** part_out, double** part_ax2_out, int* G_out) {
    if (n < 1 || d < 1 || d > (1 << 20)) return IHS_EINVAL;
    const bool aligned = ((uintptr_t)A % 16 == 0) && ((uintptr_t)x % 16 == 0) && (d % 4 == 0) && d <= 8192;
    const int64_t Gmax = 4 * (int64_t)ctx->sm_count + 1024;
    void* ws = nullptr;
    const size_t part_bytes = (size_t)Gmax * d * sizeof(float2);
    IHS_TRY(ihs_scratch(ctx, SLOT_GRAD_PART, part_bytes + Gmax * sizeof(double) + 256, &ws));
    float2* part = static_cast<float2*>(ws);
    double* part_ax2 = reinterpret_cast<double*>(static_cast<char*>(ws) + part_bytes);
    int G = 0;
    const GradTarget tg{ctx->stream, ctx->sm_count, ctx->d_status};
    if (aligned) {
        IHS_TRY(grad_pass_fast(tg, A, b, x, n, d, part, part_ax2, &G));
    } else {
        const int64_t rblocks = ceil_div64(n, 128);
        void* rws = nullptr;
        const size_t rbytes = ((size_t)n * sizeof(float) + 15) & ~(size_t)15;
        IHS_TRY(ihs_scratch(ctx, SLOT_GRAD_R, rbytes + (size_t)rblocks * sizeof(double), &rws));
        float* r = static_cast<float*>(rws);
        double* rpart = reinterpret_cast<double*>(static_cast<char*>(rws) + rbytes);
        const int64_t groups =
            std::min<int64_t>(Gmax, std::max<int64_t>(1, 2 * (int64_t)ctx->sm_count / ceil_div64(d, 256)));
        const int64_t rows_per_group = ceil_div64(n, groups);
        const int64_t ngroups = ceil_div64(n, rows_per_group);
        k_resid_generic<<<(unsigned)rblocks, 256, 0, ctx->stream>>>(A, b, x, n, (int)d, r, rpart);
        IHS_LAUNCH_CHECK();
        dim3 grid((unsigned)ceil_div64(d, 256), (unsigned)ngroups);
        k_atr_generic<<<grid, 256, 0, ctx->stream>>>(A, r, n, (int)d, rows_per_group, part);
        IHS_LAUNCH_CHECK();
        G = (int)ngroups;
        k_fold_doubles<<<1, 1, 0, ctx->stream>>>(rpart, rblocks, part_ax2, G);
        IHS_LAUNCH_CHECK();
    }
    *part_out = part;
    *part_ax2_out = part_ax2;
    *G_out = G;
    return IHS_OK;
}

int ihs_grad_enqueue(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu,
                     const float* x, float* g, double* d_axnorm2) {
    float2* part = nullptr;
    double* part_ax2 = nullptr;
    int G = 0;
    IHS_TRY(grad_partials(ctx, A, b, n, d, x, &part, &part_ax2, &G));
    const DfConst nu2 = df_const(nu * nu);
    k_grad_reduce<<<(unsigned)ceil_div64(d, 32), 256, 0, ctx->stream>>>(part, part_ax2, G, (int)d, nu2.hi, nu2.lo, x,
                                                                        g, d_axnorm2, nullptr);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

namespace {

// gp[c] = sum of the partials of column c, gp[d] = sum of the ||A x||^2
// partials: the fixed-order sums of k_grad_reduce, left unrounded (the
// compensated pair widened to FP64) and without nu^2 x, for a row shard whose
// sums other shards add to.
__global__ void __launch_bounds__(256) k_grad_reduce_f64(const float2* __restrict__ part,
                                                         const double* __restrict__ part_ax2, int G, int d,
                                                         double* __restrict__ gp) {
    __shared__ float2 sm[8][33];
    const int cx = threadIdx.x & 31, sy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + cx;
    Acc2 a = grad_column_sum(part, G, d, col, sy);
    sm[sy][cx] = make_float2(a.hi, a.lo);
    __syncthreads();
    if (sy == 0 && col < d) {
        for (int k = 1; k < 8; ++k) a.add_pair(sm[k][cx].x, sm[k][cx].y);
        gp[col] = (double)a.hi + (double)a.lo;
    }
    if (blockIdx.x == 0 && sy == 1) {
        double t = 0.0;
        for (int gi = cx; gi < G; gi += 32) t += part_ax2[gi];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (cx == 0) gp[d] = t;
    }
}

// g = fl32(gp + nu^2 x) and ||A x||^2 = gp[d] from the summed shard partials.
__global__ void k_grad_finish(const double* __restrict__ gp, int d, double nu2, const float* __restrict__ x,
                              float* __restrict__ g, double* __restrict__ axnorm2) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < d) g[c] = (float)(gp[c] + nu2 * (double)x[c]);
    if (c == 0 && axnorm2) *axnorm2 = gp[d];
}

}  // namespace

int ihs_grad_partial_enqueue(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, const float* x,
                             double* gp) {
    float2* part = nullptr;
    double* part_ax2 = nullptr;
    int G = 0;
    IHS_TRY(grad_partials(ctx, A, b, n, d, x, &part, &part_ax2, &G));
    k_grad_reduce_f64<<<(unsigned)ceil_div64(d, 32), 256, 0, ctx->stream>>>(part, part_ax2, G, (int)d, gp);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

int ihs_grad_finish_enqueue(ihs_ctx* ctx, const double* gp, int64_t d, double nu, const float* x, float* g,
                            double* d_axnorm2) {
    k_grad_finish<<<(unsigned)ceil_div64(d, 256), 256, 0, ctx->stream>>>(gp, (int)d, nu * nu, x, g, d_axnorm2);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

extern "C" int ihs_grad_shard(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, const float* x,
                              double* gp) {
    IhsRange range("ihs_grad_shard");
    if (!ctx || !A || !b || !x || !gp) return IHS_EINVAL;
    IHS_TRY(ihs_grad_partial_enqueue(ctx, A, b, n, d, x, gp));
    return IHS_OK;
}


extern "C" int ihs_grad(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu,
                        const float* x, float* g, double* axnorm2_h) {
    IhsRange range("ihs_grad");
    if (!ctx || !A || !b || !x || !g) return IHS_EINVAL;
    if (!(nu >= 0.0) || n < 1 || d < 1) return IHS_EINVAL;
    double* d_ax = nullptr;
    if (axnorm2_h) {
        void* ws = nullptr;
        IHS_TRY(ihs_scratch(ctx, SLOT_MISC, 4096, &ws));
        d_ax = static_cast<double*>(ws) + 256;
    }
    IHS_TRY(ihs_grad_enqueue(ctx, A, b, n, d, nu, x, g, d_ax));
    if (axnorm2_h) {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, d_ax, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *axnorm2_h = ctx->pinned[0];
    }
    return ihs_check_status(ctx);
}

// ---------------------------------------------------------------------------
// Allocation-free gradient pass (ihs_grad_noalloc).
//
// Some callers cannot let a library call cudaMalloc or cudaFree: code whose
// device memory is owned by another allocator (a framework's caching pool or
// a fixed arena sized up front, where a hidden allocation breaks the memory
// budget), and latency-critical loops that must not block in cudaMalloc /
// cudaFree, which synchronise the device.  This variant of the gradient pass
// needs no context and allocates nothing: its scratch (the per-CTA partial
// sums and a status word) lives in a file-scope __device__ array of fixed
// size, which every GPU that loads the library holds until the process exits.
// It launches the same kernels with the same grid as ihs_grad (for 16-byte
// aligned A and x and d % 4 == 0), so on a GPU with at most 160 SMs the two
// return the same bits.
#include <mutex>

#define IHS_NOALLOC_MAX_SMS 160
#define IHS_NOALLOC_MAX_D 8192

namespace {

// Partials: G CTAs x d columns of float2, G = SMs (d >= 1024) or 2 x SMs
// (d < 1024), so G x d <= 160 x 8192 in both cases.
constexpr size_t kNoallocPartBytes = (size_t)IHS_NOALLOC_MAX_SMS * IHS_NOALLOC_MAX_D * sizeof(float2);
constexpr size_t kNoallocAx2Bytes = (size_t)2 * IHS_NOALLOC_MAX_SMS * sizeof(double);
constexpr size_t kNoallocBytes = kNoallocPartBytes + kNoallocAx2Bytes + 256;   // + status word

// ~10 MiB: 160 x 8192 float2 partials, 320 double partials, a status word.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocDevice {
    unsigned char* scratch;   // device address of g_noalloc_scratch on this device
    int sm_count;
    bool ready;
};
NoallocDevice g_noalloc_dev[128];
std::mutex g_noalloc_mu;

// The device address of the scratch array on the current device (the
// host-side symbol is only a stand-in) and the SM count.  The address is
// looked up again on every call made outside stream capture (cheap, and
// correct after the module was reloaded, e.g. following cudaDeviceReset); a
// call on a capturing stream uses the address cached by an earlier call on the
// same device, and fails with IHS_EINVAL if there was none.
int noalloc_setup(cudaStream_t stream, NoallocDevice** out) {
    int dev = 0;
    IHS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return IHS_EINVAL;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    IHS_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice& nd = g_noalloc_dev[dev];
    if (cap != cudaStreamCaptureStatusNone) {
        if (!nd.ready) return IHS_EINVAL;
        *out = &nd;
        return IHS_OK;
    }
    void* ptr = nullptr;
    IHS_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (!nd.ready) {
        int sms = 0;
        IHS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        nd.sm_count = sms;
    }
    nd.scratch = static_cast<unsigned char*>(ptr);
    nd.ready = true;
    *out = &nd;
    return IHS_OK;
}

}  // namespace

extern "C" int ihs_grad_noalloc(void* stream_v, const float* A, const float* b, int64_t n, int64_t d, double nu,
                                const float* x, float* g, double* axnorm2) {
    if (!A || !b || !x || !g) return IHS_EINVAL;
    if (n < 1 || d < 4 || d > IHS_NOALLOC_MAX_D || d % 4 != 0) return IHS_EINVAL;
    if (!(nu >= 0.0) || !isfinite(nu)) return IHS_EINVAL;
    if ((uintptr_t)A % 16 != 0 || (uintptr_t)x % 16 != 0) return IHS_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    NoallocDevice* nd = nullptr;
    IHS_TRY(noalloc_setup(stream, &nd));
    float2* part = reinterpret_cast<float2*>(nd->scratch);
    double* part_ax2 = reinterpret_cast<double*>(nd->scratch + kNoallocPartBytes);
    unsigned* status = reinterpret_cast<unsigned*>(nd->scratch + kNoallocPartBytes + kNoallocAx2Bytes);
    // The status word must start at zero; the partials are fully rewritten.
    IHS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), stream));
    const GradTarget tg{stream, std::min(nd->sm_count, IHS_NOALLOC_MAX_SMS), status};
    int G = 0;
    IHS_TRY(grad_pass_fast(tg, A, b, x, n, d, part, part_ax2, &G));
    // the reduction of the regular entry point, NaN where the pass gave up
    const DfConst nu2 = df_const(nu * nu);
    k_grad_reduce<<<(unsigned)ceil_div64(d, 32), 256, 0, stream>>>(part, part_ax2, G, (int)d, nu2.hi, nu2.lo, x, g,
                                                                   axnorm2, status);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}
