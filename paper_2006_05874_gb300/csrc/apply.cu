// Fused apply of the sketched Hessian inverse: gt = H_S^{-1} g and the
// sketched Newton decrement r = 1/2 g^T gt (Lemma 4.1), in one cooperative
// launch instead of a chain of dependent kernels.
//
// H_S = (SA)^T SA + nu^2 I (Eq. 3).  With X = L^{-1} (FP32, from the FP64
// Cholesky K = L L^T of factor.cu) every application is a sequence of
// matrix-vector products, with one step of iterative refinement whose
// residual applies the exact operator K from the FP32 sketch in double-float:
//   Woodbury form (m < d, App. B.4), K = nu^2 I_m + SA SA^T:
//     t = SA g, u0 = X^T X t, res = t - (nu^2 u0 + SA (SA^T u0)),
//     u1 = u0 + X^T X res, gt = nu^-2 (g - SA^T u1)
//   direct form (m >= d), K = SA^T SA + nu^2 I_d:
//     u0 = X^T X g, res = g - (nu^2 u0 + SA^T (SA u0)), gt = u1 = u0 + X^T X res.
// SA^T is kept as an FP32 copy made with the factor, so that every stage is a
// row-parallel product: a warp takes one (row, segment) item at a time, a
// segment being 1024 entries (eight 16-byte loads per lane); the segment sums
// go to partial vectors that the next stage adds up in a fixed order while it
// copies its input vector into shared memory.
// The stages are separated by grid barriers on a monotonic 64-bit arrival
// counter (bounded waits: a wait that exceeds one second sets IHS_DEV_TIMEOUT
// and the CTAs leave); each warp loads the matrix rows of its first two items
// of the next stage before it waits, so the barrier overlaps the loads.  The
// decrement's per-CTA FP64 partials are added in CTA order by the last CTA to
// finish.  Arithmetic and results match the multi-launch apply of factor.cu to
// rounding: double-float vectors, exact products, compensated sums.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kApplyThreads = 512;
constexpr int kApplyWarps = kApplyThreads / 32;
constexpr int kSlots = 8;                      // 16-byte loads per lane per item
constexpr int kSegFloats = 32 * 4 * kSlots;    // 1024 floats per segment
constexpr int kPrefetch = 2;                   // items loaded before a barrier
constexpr int kLocalK = 128;                   // Woodbury k up to which each CTA forms X^T X v itself

__device__ __forceinline__ float2 df_norm(float hi, float lo) {   // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, make_float2(-b.x, -b.y)); }

// acc += m (x.hi + x.lo): the product m x.hi exactly (TwoProduct), m x.lo
// rounded once, the sum compensated.
__device__ __forceinline__ void acc_mul(Acc2& acc, float m, float2 x) {
    float p, e, s, es;
    two_prod(m, x.x, p, e);
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fmaf_rn(m, x.y, e), es));
}

// acc += (a.x + a.y)(b.x + b.y): the high product exactly, the cross terms
// rounded once, a.y b.y dropped (2^-48 relative).
__device__ __forceinline__ void acc_dfdf(Acc2& acc, float2 a, float2 b) {
    float p, e, s, es;
    two_prod(a.x, b.x, p, e);
    const float cross = __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x));
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fadd_rn(e, cross), es));
}

__device__ __forceinline__ Acc2 warp_sum(Acc2 a) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const Acc2 o = acc2_shfl_xor(a, off);
        a.add_pair(o.hi, o.lo);
    }
    return a;
}

// A row-major matrix read by rows.  Entries are FP32 (dbl = 0) or double-float
// pairs (dbl = 1); a row holds cols entries, i.e. cols (or 2 cols) floats, a
// multiple of 4.  tri: 0 full, 1 lower (entries right of the diagonal are
// stored zeros), 2 upper (entries left of it are stored zeros).  A row splits
// into segments of kSegFloats floats; item (s, i) = segment s of row i, listed
// segment-major, it = s rows + i, and only the segments that can hold a
// non-zero entry are items.
struct Mat {
    const float* p;
    int64_t rows, cols;
    int tri, dbl;
    __device__ __forceinline__ int64_t row_floats() const { return dbl ? 2 * cols : cols; }
    __device__ __forceinline__ int64_t seg_entries() const { return dbl ? kSegFloats / 2 : kSegFloats; }
    __device__ __forceinline__ int64_t nseg() const { return (row_floats() + kSegFloats - 1) / kSegFloats; }
    __device__ __forceinline__ int64_t items() const { return nseg() * rows; }
    __device__ __forceinline__ bool valid(int64_t it) const {
        if (tri == 0) return true;
        const int64_t s = it / rows, i = it - s * rows;
        const int64_t si = i / seg_entries();   // segment holding the diagonal entry (i, i)
        return tri == 1 ? s <= si : s >= si;
    }
};

// The next item of warp gw at or after `it` (stride W), or -1.
__device__ __forceinline__ int64_t next_item(const Mat& M, int64_t it, int64_t W) {
    const int64_t total = M.items();
    for (; it < total; it += W)
        if (M.valid(it)) return it;
    return -1;
}

// The lane's eight 16-byte pieces of item `it` (zeros past the row's end).
__device__ __forceinline__ void load_item(const Mat& M, int64_t it, float4 (&buf)[kSlots]) {
    const int lane = threadIdx.x & 31;
    const int64_t s = it / M.rows, i = it - s * M.rows;
    const int64_t rf = M.row_floats();
    const float* row = M.p + i * rf;
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
        const int64_t f = s * kSegFloats + (int64_t)(q * 32 + lane) * 4;
        buf[q] = f < rf ? __ldcg(reinterpret_cast<const float4*>(row + f)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The warp's dot product of item `it` with the shared-memory vector: vf (FP32
// entries) or vd (double-float entries); lane 0 stores the segment's sum at
// y[it] as a normalised pair.
__device__ __forceinline__ void dot_item(const Mat& M, int64_t it, const float4 (&buf)[kSlots],
                                         const float* vf, const float2* vd, float2* y) {
    const int lane = threadIdx.x & 31;
    const int64_t s = it / M.rows;
    const int64_t rf = M.row_floats();
    Acc2 acc{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
        const int64_t f = s * kSegFloats + (int64_t)(q * 32 + lane) * 4;
        if (f >= rf) break;
        const float4 a = buf[q];
        if (M.dbl) {
            const int64_t c = f / 2;   // two double-float entries
            acc_dfdf(acc, make_float2(a.x, a.y), vd[c]);
            acc_dfdf(acc, make_float2(a.z, a.w), vd[c + 1]);
        } else if (vd) {
            acc_mul(acc, a.x, vd[f]);
            acc_mul(acc, a.y, vd[f + 1]);
            acc_mul(acc, a.z, vd[f + 2]);
            acc_mul(acc, a.w, vd[f + 3]);
        } else {
            acc.add_prod(a.x, vf[f]);
            acc.add_prod(a.y, vf[f + 1]);
            acc.add_prod(a.z, vf[f + 2]);
            acc.add_prod(a.w, vf[f + 3]);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) y[it] = df_norm(acc.hi, acc.lo);
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `nbar` (1, 2, ...) of this launch: passed when the
// counter reaches base + nbar * gridDim.x.  Returns false (and sets
// IHS_DEV_TIMEOUT) if the wait exceeds one second.
__device__ __forceinline__ bool apply_grid_sync(unsigned long long* cnt, unsigned long long base, int nbar,
                                                unsigned* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned long long target = base + (unsigned long long)nbar * gridDim.x;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
        if (ld_acquire_u64(cnt) < target) {
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_u64(cnt) < target) {
                if (global_timer_ns() - t0 > 1000000000ull) {
                    atomicOr(status, IHS_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// Items a warp loads before the barrier that precedes their stage.
struct Pref {
    int64_t it[kPrefetch];
    float4 buf[kPrefetch][kSlots];
};

__device__ __forceinline__ void prefetch(const Mat& M, int64_t gw, int64_t W, Pref& P) {
    int64_t it = next_item(M, gw, W);
#pragma unroll
    for (int j = 0; j < kPrefetch; ++j) {
        P.it[j] = it;
        if (it >= 0) {
            load_item(M, it, P.buf[j]);
            it = next_item(M, it + W, W);
        }
    }
}

// Every item of warp gw: the prefetched ones first, then the rest one by one.
__device__ __forceinline__ void run_stage(const Mat& M, int64_t gw, int64_t W, const Pref& P, const float* vf,
                                          const float2* vd, float2* y) {
#pragma unroll
    for (int j = 0; j < kPrefetch; ++j)
        if (P.it[j] >= 0) dot_item(M, P.it[j], P.buf[j], vf, vd, y);
    int64_t it = P.it[kPrefetch - 1] >= 0 ? next_item(M, P.it[kPrefetch - 1] + W, W) : -1;
    float4 buf[kSlots];
    while (it >= 0) {
        load_item(M, it, buf);
        dot_item(M, it, buf, vf, vd, y);
        it = next_item(M, it + W, W);
    }
}

// y = M v for a matrix of at most kSegFloats columns, every row in this CTA
// (warp w takes rows w, w + 16, ...): the same per-row arithmetic as a stage's
// item, so y[i] equals the item's single segment sum bit for bit.  v and y
// may be shared-memory vectors.
__device__ __forceinline__ void local_matvec(const Mat& M, const float2* v, float2* y) {
    float4 buf[kSlots];
    for (int64_t i = threadIdx.x >> 5; i < M.rows; i += kApplyWarps) {
        load_item(M, i, buf);
        dot_item(M, i, buf, nullptr, v, y);
    }
}

// Entry i of a product whose segment sums are in Y (rows entries per
// segment): the sum over segments [s0, s1) in increasing order.
__device__ __forceinline__ float2 sum_parts(const float2* Y, int64_t rows, int64_t i, int64_t s0, int64_t s1) {
    float2 v = __ldcg(Y + s0 * rows + i);
    for (int64_t s = s0 + 1; s < s1; ++s) v = df_add(v, __ldcg(Y + s * rows + i));
    return v;
}

struct ApplyArgs {
    const float* SA;     // m x d
    const float* SAT;    // d x m (Woodbury form)
    const float* X;      // k x k lower, L^{-1}
    const float* XT;     // k x k upper, its transpose
    const float* g;      // d
    float* gt;           // d
    double* r_out;       // device scalar or NULL
    float2* Y0;
    float2* Y1;
    float2* Y2;
    float2* Y3;
    double* rpart;       // one FP64 partial of g . gt per CTA
    int64_t m, d, k;
    int woodbury;
    double inv_nu2;
    double nu2;
    unsigned long long* bar;
    unsigned long long base;
    unsigned* done;      // last-CTA ticket of the decrement (left at 0)
    unsigned* status;
};

// The decrement's last step: this CTA's FP64 partial of g . gt (threads' terms
// `prod` added in a fixed tree), then the last CTA to finish adds the CTA
// partials in CTA order: r = 1/2 sum.
__device__ __forceinline__ void finish_decrement(const ApplyArgs& a, double prod) {
    __shared__ double red[kApplyThreads];
    __shared__ bool last;
    red[threadIdx.x] = prod;
    __syncthreads();
    for (int w = kApplyThreads / 2; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.rpart[blockIdx.x] = red[0];
        __threadfence();
        const unsigned ticket = atomicAdd(a.done, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned c = 0; c < gridDim.x; ++c) s += __ldcg(a.rpart + c);
        if (a.r_out) *a.r_out = 0.5 * s;
        atomicExch(a.done, 0u);
    }
}

// A barrier that gave up ends the launch; the decrement reads NaN, so that a
// controller reading it stops, and the status word holds IHS_DEV_TIMEOUT.
#define IHS_APPLY_SYNC()                                                              \
    do {                                                                              \
        if (!apply_grid_sync(a.bar, a.base, ++nb, a.status)) {                        \
            if (threadIdx.x == 0 && a.r_out) *a.r_out = __longlong_as_double(0x7ff8000000000000ll); \
            return;                                                                   \
        }                                                                             \
    } while (0)

// res = t - (nu^2 u + w) in double-float, nu^2 split into a binary32 pair.
__device__ __forceinline__ float2 df_residual(float2 t, float2 u, double nu2, float2 w) {
    const float sh = (float)nu2, sl = (float)(nu2 - (double)sh);
    float p, e;
    two_prod(u.x, sh, p, e);
    const float2 nu2u = df_norm(p, __fadd_rn(e, __fmaf_rn(u.x, sl, __fmul_rn(u.y, sh))));
    return df_sub(t, df_add(nu2u, w));
}

__global__ void __launch_bounds__(kApplyThreads, 1) k_apply_fused(const ApplyArgs a) {
    extern __shared__ float4 apply_smem[];
    float2* vd = reinterpret_cast<float2*>(apply_smem);   // stage input, double-float
    float* vf = reinterpret_cast<float*>(apply_smem);     // or FP32 (g in the first Woodbury stage)
    const int tid = threadIdx.x;
    const int64_t W = (int64_t)gridDim.x * kApplyWarps;
    const int64_t gw = (int64_t)blockIdx.x * kApplyWarps + (tid >> 5);
    const int64_t k = a.k, m = a.m, d = a.d;
    const Mat mX{a.X, k, k, 1, 0};
    const Mat mXT{a.XT, k, k, 2, 0};
    const Mat mSA{a.SA, m, d, 0, 0};
    const Mat mSAT{a.SAT, d, m, 0, 0};
    const int64_t segX = kSegFloats, PX = (k + segX - 1) / segX;   // segments of X / X^T rows
    const int64_t PSA = (d + kSegFloats - 1) / kSegFloats;          // of SA rows
    const int64_t PSAT = (m + kSegFloats - 1) / kSegFloats;         // of SA^T rows
    Pref P;
    int nb = 0;
    if (a.woodbury && k <= kLocalK) {
        // Small k: every CTA forms u0 = X^T X t and the refinement X^T X res
        // itself (the vectors are identical to the distributed stages'), four
        // grid barriers instead of eight.
        __shared__ float2 loc_u0[kLocalK], loc_a[kLocalK], loc_b[kLocalK];
        // 1: t = SA g
        prefetch(mSA, gw, W, P);
        for (int64_t e = tid; e < d; e += kApplyThreads) vf[e] = __ldg(a.g + e);
        __syncthreads();
        run_stage(mSA, gw, W, P, vf, nullptr, a.Y0);
        prefetch(mSAT, gw, W, P);
        IHS_APPLY_SYNC();
        // u0 = X^T (X t)
        for (int64_t i = tid; i < m; i += kApplyThreads) vd[i] = sum_parts(a.Y0, m, i, 0, PSA);
        __syncthreads();
        local_matvec(mX, vd, loc_a);
        __syncthreads();
        local_matvec(mXT, loc_a, loc_u0);
        __syncthreads();
        // 4: w = SA^T u0
        run_stage(mSAT, gw, W, P, nullptr, loc_u0, a.Y3);
        prefetch(mSA, gw, W, P);
        IHS_APPLY_SYNC();
        // 5: w2 = SA w
        for (int64_t c = tid; c < d; c += kApplyThreads) vd[c] = sum_parts(a.Y3, d, c, 0, PSAT);
        __syncthreads();
        run_stage(mSA, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mSAT, gw, W, P);
        IHS_APPLY_SYNC();
        // res = t - (nu^2 u0 + w2), u1 = u0 + X^T (X res)
        for (int64_t i = tid; i < k; i += kApplyThreads)
            loc_a[i] = df_residual(sum_parts(a.Y0, m, i, 0, PSA), loc_u0[i], a.nu2, sum_parts(a.Y1, m, i, 0, PSA));
        __syncthreads();
        local_matvec(mX, loc_a, loc_b);
        __syncthreads();
        local_matvec(mXT, loc_b, loc_a);
        __syncthreads();
        for (int64_t i = tid; i < k; i += kApplyThreads) loc_b[i] = df_add(loc_u0[i], loc_a[i]);
        __syncthreads();
        // 8: w = SA^T u1
        run_stage(mSAT, gw, W, P, nullptr, loc_b, a.Y3);
        IHS_APPLY_SYNC();
        // gt = (g - w) / nu^2 and the decrement
        double prod = 0.0;
        for (int64_t c = (int64_t)blockIdx.x * kApplyThreads + tid; c < d; c += (int64_t)gridDim.x * kApplyThreads) {
            const float2 w = sum_parts(a.Y3, d, c, 0, PSAT);
            const double gc = (double)__ldg(a.g + c);
            const double v = (gc - ((double)w.x + (double)w.y)) * a.inv_nu2;
            a.gt[c] = (float)v;
            prod += gc * v;
        }
        finish_decrement(a, prod);
    } else if (a.woodbury) {
        // 1: t = SA g
        prefetch(mSA, gw, W, P);
        for (int64_t e = tid; e < d; e += kApplyThreads) vf[e] = __ldg(a.g + e);
        __syncthreads();
        run_stage(mSA, gw, W, P, vf, nullptr, a.Y0);
        prefetch(mX, gw, W, P);
        IHS_APPLY_SYNC();
        // 2: v = X t
        for (int64_t i = tid; i < m; i += kApplyThreads) vd[i] = sum_parts(a.Y0, m, i, 0, PSA);
        __syncthreads();
        run_stage(mX, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mXT, gw, W, P);
        IHS_APPLY_SYNC();
        // 3: u0 = X^T v
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y1, k, i, 0, i / segX + 1);
        __syncthreads();
        run_stage(mXT, gw, W, P, nullptr, vd, a.Y2);
        prefetch(mSAT, gw, W, P);
        IHS_APPLY_SYNC();
        // 4: w = SA^T u0
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y2, k, i, i / segX, PX);
        __syncthreads();
        run_stage(mSAT, gw, W, P, nullptr, vd, a.Y3);
        prefetch(mSA, gw, W, P);
        IHS_APPLY_SYNC();
        // 5: w2 = SA w
        for (int64_t c = tid; c < d; c += kApplyThreads) vd[c] = sum_parts(a.Y3, d, c, 0, PSAT);
        __syncthreads();
        run_stage(mSA, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mX, gw, W, P);
        IHS_APPLY_SYNC();
        // 6: v = X res, res = t - K u0 = t - (nu^2 u0 + w2)
        for (int64_t i = tid; i < k; i += kApplyThreads)
            vd[i] = df_residual(sum_parts(a.Y0, m, i, 0, PSA), sum_parts(a.Y2, k, i, i / segX, PX), a.nu2,
                                sum_parts(a.Y1, m, i, 0, PSA));
        __syncthreads();
        run_stage(mX, gw, W, P, nullptr, vd, a.Y3);
        prefetch(mXT, gw, W, P);
        IHS_APPLY_SYNC();
        // 7: X^T v
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y3, k, i, 0, i / segX + 1);
        __syncthreads();
        run_stage(mXT, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mSAT, gw, W, P);
        IHS_APPLY_SYNC();
        // 8: w = SA^T u1, u1 = u0 + X^T v
        for (int64_t i = tid; i < k; i += kApplyThreads)
            vd[i] = df_add(sum_parts(a.Y2, k, i, i / segX, PX), sum_parts(a.Y1, k, i, i / segX, PX));
        __syncthreads();
        run_stage(mSAT, gw, W, P, nullptr, vd, a.Y3);
        IHS_APPLY_SYNC();
        // gt = (g - w) / nu^2 and the decrement
        double prod = 0.0;
        for (int64_t c = (int64_t)blockIdx.x * kApplyThreads + tid; c < d; c += (int64_t)gridDim.x * kApplyThreads) {
            const float2 w = sum_parts(a.Y3, d, c, 0, PSAT);
            const double gc = (double)__ldg(a.g + c);
            const double v = (gc - ((double)w.x + (double)w.y)) * a.inv_nu2;
            a.gt[c] = (float)v;
            prod += gc * v;
        }
        finish_decrement(a, prod);
    } else {
        // 1: v = X g
        prefetch(mX, gw, W, P);
        for (int64_t e = tid; e < k; e += kApplyThreads) vd[e] = make_float2(__ldg(a.g + e), 0.f);
        __syncthreads();
        run_stage(mX, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mXT, gw, W, P);
        IHS_APPLY_SYNC();
        // 2: u0 = X^T v
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y1, k, i, 0, i / segX + 1);
        __syncthreads();
        run_stage(mXT, gw, W, P, nullptr, vd, a.Y2);
        prefetch(mSA, gw, W, P);
        IHS_APPLY_SYNC();
        // 3: w = SA u0
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y2, k, i, i / segX, PX);
        __syncthreads();
        run_stage(mSA, gw, W, P, nullptr, vd, a.Y0);
        prefetch(mSAT, gw, W, P);
        IHS_APPLY_SYNC();
        // 4: w2 = SA^T w
        for (int64_t j = tid; j < m; j += kApplyThreads) vd[j] = sum_parts(a.Y0, m, j, 0, PSA);
        __syncthreads();
        run_stage(mSAT, gw, W, P, nullptr, vd, a.Y3);
        prefetch(mX, gw, W, P);
        IHS_APPLY_SYNC();
        // 5: v = X res, res = g - K u0 = g - (nu^2 u0 + w2)
        for (int64_t i = tid; i < k; i += kApplyThreads)
            vd[i] = df_residual(make_float2(__ldg(a.g + i), 0.f), sum_parts(a.Y2, k, i, i / segX, PX), a.nu2,
                                sum_parts(a.Y3, d, i, 0, PSAT));
        __syncthreads();
        run_stage(mX, gw, W, P, nullptr, vd, a.Y1);
        prefetch(mXT, gw, W, P);
        IHS_APPLY_SYNC();
        // 6: X^T v
        for (int64_t i = tid; i < k; i += kApplyThreads) vd[i] = sum_parts(a.Y1, k, i, 0, i / segX + 1);
        __syncthreads();
        run_stage(mXT, gw, W, P, nullptr, vd, a.Y3);
        IHS_APPLY_SYNC();
        // gt = u1 = u0 + X^T v and the decrement
        double prod = 0.0;
        for (int64_t c = (int64_t)blockIdx.x * kApplyThreads + tid; c < d; c += (int64_t)gridDim.x * kApplyThreads) {
            const float2 u1 = df_add(sum_parts(a.Y2, k, c, c / segX, PX), sum_parts(a.Y3, k, c, c / segX, PX));
            const double v = (double)u1.x + (double)u1.y;
            a.gt[c] = (float)v;
            prod += (double)__ldg(a.g + c) * v;
        }
        finish_decrement(a, prod);
    }
}

// Barriers per launch of k_apply_fused.
constexpr int kBarriersWoodburyLocal = 4;
constexpr int kBarriersWoodbury = 8;
constexpr int kBarriersDirect = 6;

// SAT = SA^T (SA: m x d row-major), 32 x 32 tiles.
__global__ void __launch_bounds__(256) k_sat(const float* __restrict__ SA, int64_t m, int64_t d,
                                             float* __restrict__ SAT) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = r0 + r, gc = c0 + tx;
        tile[r][tx] = (gr < m && gc < d) ? SA[gr * d + gc] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = c0 + r, gc = r0 + tx;
        if (gr < d && gc < m) SAT[gr * m + gc] = tile[tx][r];
    }
}

size_t fused_smem_bytes(int64_t m, int64_t d) {
    // the largest stage vector: max(m, d) double-float entries
    return (size_t)std::max(m, d) * sizeof(float2);
}

}  // namespace

// The fused apply needs 16-byte rows (k, m and d multiples of 4) and its
// stage vectors in shared memory (at most 16384 double-float entries, 128 KB).
bool ihs_apply_fused_ok(int64_t k, int64_t m, int64_t d) {
    if (k < 4 || k % 4 || d % 4 || m % 4) return false;
    return fused_smem_bytes(m, d) <= 128 * 1024;
}

size_t ihs_apply_partials(int64_t k, int64_t m, int64_t d) {
    auto seg = [](int64_t floats) { return (floats + kSegFloats - 1) / kSegFloats; };
    size_t n = (size_t)(seg(k) * k);                       // X, X^T rows
    n = std::max(n, (size_t)(seg(d) * m));                 // SA rows
    n = std::max(n, (size_t)(seg(m) * d));                 // SA^T rows
    return n;
}

int ihs_apply_prepare(ihs_ctx* ctx, ihs_factor_t* F) {
    if (!F->fused) return IHS_OK;
    dim3 grid((unsigned)ceil_div64(F->d, 32), (unsigned)ceil_div64(F->m, 32));
    k_sat<<<grid, 256, 0, ctx->stream>>>(F->SA, F->m, F->d, F->SAT);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

int ihs_apply_fused(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* d_r) {
    const size_t smem = fused_smem_bytes(F->m, F->d);
    // one fixed limit for every launch (the kernel also holds 4 KB of static
    // shared memory, so the device's whole opt-in maximum cannot be granted)
    IHS_CUDA_TRY(cudaFuncSetAttribute(k_apply_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
    int per_sm = 0;
    IHS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_fused, kApplyThreads, smem));
    if (per_sm < 1) return IHS_EINVAL;
    // one CTA per SM, all resident (cooperative launch), unless set lower
    const int G = (ctx->apply_ctas >= 1 && ctx->apply_ctas < ctx->sm_count) ? ctx->apply_ctas : ctx->sm_count;
    const size_t np = ihs_apply_partials(F->k, F->m, F->d);
    ApplyArgs a;
    a.SA = F->SA;
    a.SAT = F->SAT;
    a.X = F->X;
    a.XT = F->XT;
    a.g = g;
    a.gt = gt;
    a.r_out = d_r;
    a.Y0 = F->Y;
    a.Y1 = F->Y + np;
    a.Y2 = F->Y + 2 * np;
    a.Y3 = F->Y + 3 * np;
    a.rpart = reinterpret_cast<double*>(F->Y + 4 * np);
    a.m = F->m;
    a.d = F->d;
    a.k = F->k;
    a.woodbury = F->woodbury;
    a.inv_nu2 = 1.0 / (F->nu * F->nu);
    a.nu2 = F->nu * F->nu;
    a.bar = reinterpret_cast<unsigned long long*>(ctx->d_status + 32);
    a.base = ctx->apply_epoch;
    a.done = ctx->d_status + 40;
    a.status = ctx->d_status;
    void* args[] = {&a};
    IHS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_apply_fused, dim3((unsigned)G), dim3(kApplyThreads),
                                             args, smem, ctx->stream));
    ihs_count_launch();
    const int nbar = F->woodbury ? (F->k <= kLocalK ? kBarriersWoodburyLocal : kBarriersWoodbury) : kBarriersDirect;
    ctx->apply_epoch += (uint64_t)nbar * (uint64_t)G;
    return IHS_OK;
}
