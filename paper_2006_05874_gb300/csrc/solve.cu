// Adaptive IHS controller: Algorithm 1 (Polyak candidate first, then the
// gradient-IHS candidate, else m <- 2m and a new sketch) and its gradient-only
// variant (Sec. 5).  Every step of the path runs in the library's kernels; the
// host reads back three FP64 scalars per candidate (the sketched Newton
// decrement r of Lemma 4.1, ||A x||^2 and ||x||^2) to take the accept /
// double / stop decisions in FP64.
//
// Readings of points the paper leaves open (they match the CPU reference):
//  * sketches are keyed by (seed, level), level = log2 m;
//  * after a doubling both gt_t and r_t are recomputed; r_1 keeps its value;
//  * m is capped at n_pad (SRHT) or n (Gaussian); at the cap a rejected
//    gradient step is accepted and report flag bit 0 is set;
//  * stop before an iteration once sqrt(2 Lambda r_t) <= tol ||Abar x_t||
//    (delta_t <= gamma_1 r_t <= Lambda r_t, proofs of Thm 4.1 / 4.2);
//  * optional floor guard: a rejected step with r_t <= floor^2 r_1 stops.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace {

struct Params {
    double lam, Lam, mu_gd, c_gd, mu_p, beta_p, c_p;
};

// Thm 2.1 / 2.2 step sizes and rates at the bounds of Def 3.1 / Def 3.2.
Params make_params(int kind, double rho, double eta) {
    double lo, hi;
    if (kind == IHS_SKETCH_GAUSS) {
        const double c_eta = (1.0 + 3.0 * sqrt(eta)) * (1.0 + 3.0 * sqrt(eta));
        const double s = sqrt(c_eta * rho);
        lo = (1.0 - s) * (1.0 - s);
        hi = (1.0 + s) * (1.0 + s);
    } else {
        lo = 1.0 - sqrt(rho);
        hi = 1.0 + sqrt(rho);
    }
    Params p;
    p.lam = lo;
    p.Lam = hi;
    p.mu_gd = 2.0 / (1.0 / lo + 1.0 / hi);
    p.c_gd = ((hi - lo) / (hi + lo)) * ((hi - lo) / (hi + lo));
    const double a = 1.0 / sqrt(lo) + 1.0 / sqrt(hi);
    p.mu_p = 4.0 / (a * a);
    const double q = (sqrt(hi) - sqrt(lo)) / (sqrt(hi) + sqrt(lo));
    p.beta_p = q * q;
    p.c_p = p.beta_p;
    return p;
}

// One block of kSolveThreads threads walks a d-vector (d is small next to the
// n x d passes) and sums one double per thread in a fixed order: a butterfly
// in each warp, then the warp sums by warp 0; the result is valid in warp 0.
// (A block of partials folded by one serial thread, and a second launch to
// fold the blocks, cost more than the vector work.)
constexpr int kSolveThreads = 1024;
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kSolveThreads / 32];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = ws[lane];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    }
    return t;
}

// xc = x - mu gt + beta (x - xp); *xx = ||xc||^2 (FP64).
__global__ void __launch_bounds__(kSolveThreads) k_candidate(const float* __restrict__ x, const float* __restrict__ gt,
                                                             const float* __restrict__ xp, int64_t d, float mu,
                                                             float beta, float* __restrict__ xc,
                                                             double* __restrict__ xx) {
    double sq = 0.0;
    for (int64_t i = threadIdx.x; i < d; i += kSolveThreads) {
        float v = __fmaf_rn(-mu, gt[i], x[i]);
        if (beta != 0.f) v = __fmaf_rn(beta, __fsub_rn(x[i], xp[i]), v);
        xc[i] = v;
        sq += (double)v * (double)v;
    }
    sq = block_sum(sq);
    if (threadIdx.x == 0) *xx = sq;
}

// *xx = ||x||^2 (FP64).
__global__ void __launch_bounds__(kSolveThreads) k_sumsq(const float* __restrict__ x, int64_t d,
                                                         double* __restrict__ xx) {
    double sq = 0.0;
    for (int64_t i = threadIdx.x; i < d; i += kSolveThreads) {
        const double v = (double)x[i];
        sq += v * v;
    }
    sq = block_sum(sq);
    if (threadIdx.x == 0) *xx = sq;
}

// AT = A^T for row-major A (rows x cols), 32 x 32 tiles through shared memory.
__global__ void k_transpose_rect(const float* __restrict__ A, int64_t rows, int64_t cols, float* __restrict__ AT) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = r0 + r, gc = c0 + tx;
        tile[r][tx] = (gr < rows && gc < cols) ? A[gr * cols + gc] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = c0 + r, gc = r0 + tx;   // row of AT = column of A
        if (gr < cols && gc < rows) AT[gr * rows + gc] = tile[tx][r];
    }
}

// ---- the underdetermined case (App. A.2) ----------------------------------
// The dual iterate z is kept as a double-float pair (z + zlo): its gradient
// A A^T z - b + nu^2 z cancels to a small vector against b, which the FP32
// iterate of the primal path would not resolve once sigma_1^2 / nu^2 is large.
// With M = A^T (rows = d, cols = n): r = M (z + zlo) in double-float, then
// g = M^T r + nu^2 (z + zlo) - b with exact products and FP64 sums.

__device__ __forceinline__ float2 df_two_sum_norm(float a, float b) {   // a + b as a normalised pair
    float s, e;
    two_sum(a, b, s, e);
    return make_float2(s, e);
}

// r_i = M_i . (z + zlo) (Dot2 on z, FMA on zlo), one warp per row, eight warps
// per block of 128 rows; block partials of ||r||^2 (FP64).
__global__ void k_dual_resid(const float* __restrict__ M, int64_t rows, int cols, const float* __restrict__ z,
                             const float* __restrict__ zlo, float2* __restrict__ r, double* __restrict__ part) {
    __shared__ double sm[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row_begin = (int64_t)blockIdx.x * 128;
    double ax2 = 0.0;
    for (int64_t i = row_begin + warp; i < min(rows, row_begin + 128); i += 8) {
        Acc2 acc{0.f, 0.f};
        float l2 = 0.f;
        const float* mi = M + i * cols;
        for (int c = lane; c < cols; c += 32) {
            const float a = mi[c];
            acc.add_prod(a, z[c]);
            l2 = __fmaf_rn(a, zlo[c], l2);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const Acc2 o = acc2_shfl_xor(acc, off);
            acc.add_pair(o.hi, o.lo);
            l2 = __fadd_rn(l2, __shfl_xor_sync(0xffffffffu, l2, off));
        }
        if (lane == 0) {
            const float2 v = df_two_sum_norm(acc.hi, __fadd_rn(acc.lo, l2));
            r[i] = v;
            const double dv = (double)v.x + (double)v.y;
            ax2 += dv * dv;
        }
    }
    if (lane == 0) sm[warp] = ax2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        part[blockIdx.x] = t;
    }
}

// part[y][c] = sum over the rows of group y of (r_i + r_lo_i) M_ic: exact
// products of the high parts (TwoProduct), the low parts by FMA.
__global__ void k_dual_atr(const float* __restrict__ M, int64_t rows, int cols, const float2* __restrict__ r,
                           int64_t rows_per_group, float2* __restrict__ part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_group;
    const int64_t i1 = min(rows, i0 + rows_per_group);
    if (c >= cols) return;
    Acc2 acc{0.f, 0.f};
    for (int64_t i = i0; i < i1; ++i) {
        const float a = M[i * cols + c];
        const float2 ri = r[i];
        acc.add_prod(ri.x, a);
        acc.lo = __fmaf_rn(ri.y, a, acc.lo);
    }
    part[(size_t)blockIdx.y * cols + c] = make_float2(acc.hi, acc.lo);
}

// g_c = sum of the partials + nu^2 (z_c + zlo_c) - b_c in FP64, one rounding;
// block 0 also folds the ||r||^2 partials.
__global__ void k_dual_reduce(const float2* __restrict__ part, int G, int cols, double nu2,
                              const float* __restrict__ z, const float* __restrict__ zlo,
                              const float* __restrict__ b, float* __restrict__ g, const double* __restrict__ rpart,
                              int nrb, double* __restrict__ ax2) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cols) {
        double t = 0.0;
        for (int y = 0; y < G; ++y) {
            const float2 v = part[(size_t)y * cols + c];
            t += (double)v.x + (double)v.y;
        }
        t += nu2 * ((double)z[c] + (double)zlo[c]);
        g[c] = (float)(t - (double)b[c]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && ax2) {
        double t = 0.0;
        for (int k = 0; k < nrb; ++k) t += rpart[k];
        *ax2 = t;
    }
}

// xc = (x + xlo) - mu gt + beta ((x + xlo) - (xp + xplo)) as a double-float pair;
// *xx = ||xc||^2 (FP64).
__global__ void __launch_bounds__(kSolveThreads)
k_candidate_df(const float* __restrict__ x, const float* __restrict__ xlo, const float* __restrict__ gt,
               const float* __restrict__ xp, const float* __restrict__ xplo, int64_t d, float mu, float beta,
               float* __restrict__ xc, float* __restrict__ xclo, double* __restrict__ xx) {
    double sq = 0.0;
    for (int64_t i = threadIdx.x; i < d; i += kSolveThreads) {
        float p, e, s, es;
        two_prod(-mu, gt[i], p, e);                 // -mu gt exactly
        two_sum(x[i], p, s, es);
        float lo = __fadd_rn(xlo[i], __fadd_rn(e, es));
        if (beta != 0.f) {
            float dh, de;
            two_sum(x[i], -xp[i], dh, de);          // x - xp
            de = __fadd_rn(de, __fsub_rn(xlo[i], xplo[i]));
            float q, qe, s2, e2;
            two_prod(beta, dh, q, qe);
            two_sum(s, q, s2, e2);
            s = s2;
            lo = __fadd_rn(lo, __fadd_rn(e2, __fmaf_rn(beta, de, qe)));
        }
        const float2 v = df_two_sum_norm(s, lo);
        xc[i] = v.x;
        xclo[i] = v.y;
        const double w = (double)v.x + (double)v.y;
        sq += w * w;
    }
    sq = block_sum(sq);
    if (threadIdx.x == 0) *xx = sq;
}

// x = M (z + zlo) for row-major M (rows x cols): one warp per row, Dot2 on z,
// FMA on zlo, the fixed-order butterfly over the lanes.
__global__ void k_rows_dot(const float* __restrict__ M, int64_t rows, int64_t cols, const float* __restrict__ z,
                           const float* __restrict__ zlo, float* __restrict__ x) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= rows) return;
    const float* row = M + i * cols;
    Acc2 acc{0.f, 0.f};
    float l2 = 0.f;
    for (int64_t l = lane; l < cols; l += 32) {
        acc.add_prod(row[l], z[l]);
        l2 = __fmaf_rn(row[l], zlo[l], l2);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const Acc2 o = acc2_shfl_xor(acc, off);
        acc.add_pair(o.hi, o.lo);
        l2 = __fadd_rn(l2, __shfl_xor_sync(0xffffffffu, l2, off));
    }
    if (lane == 0) x[i] = __fadd_rn(acc.hi, __fadd_rn(acc.lo, l2));
}

// Scratch of the dual gradient.
struct DualScratch {
    float2* r;        // rows
    double* rpart;    // ceil(rows / 128)
    float2* part;     // G x cols
    int G;
    int64_t rows_per_group;
};

struct Solver {
    ihs_ctx* ctx;
    const float* A;
    const float* b;
    const float* bsub;    // dual mode: the right-hand side b of App. A.2
    float* vlo[7];        // dual mode: low parts of the double-float iterates
    DualScratch ds;
    int64_t n, d;
    double nu;
    float* vec[7];        // x, x_prev, g, gt, xc, gc, gtc
    double* dsc;          // device scalars: [0] r, [1] ax2, [2] xx, [8..] partials
    ihs_factor_t* F;      // points at Fs once a level is factored
    ihs_factor_t Fs;      // scratch-backed factor of the current level
    float* SA;
    int sa_slot;          // scratch slot holding SA (nested mode alternates two)
    int64_t m;
    int level;
    float ms_sketch, ms_iter, ms_grad;
    // row-sharded solve: A holds rows [row0, row0 + n) of n_total; the sketch
    // and the gradient's partial sums are summed over ranks by `ar`
    int64_t row0, n_total;
    ihs_allreduce_fn ar;
    void* ar_user;
    double* gp;           // d + 1 FP64 gradient partials (sharded solves)
    bool sketch_pending;  // a level's sketch + factor awaits its status check and timing
};

// Enqueue the copy of the device status word next to the scalars a caller is
// about to read back (the factor of a new level is checked there instead of
// with a synchronisation of its own).
int status_copy(Solver& S) {
    unsigned* hs = reinterpret_cast<unsigned*>(S.ctx->pinned + 16);
    IHS_CUDA_TRY(cudaMemcpyAsync(hs, S.ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, S.ctx->stream));
    return IHS_OK;
}

// After the synchronisation: the pending level's timing, and any device error
// (a non-positive pivot, a wait that gave up) as its status code.
int status_after_sync(Solver& S) {
    if (S.sketch_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S.ctx->ev[4], S.ctx->ev[5]);
        S.ms_sketch += ms;
        S.sketch_pending = false;
    }
    const unsigned hs = *reinterpret_cast<const unsigned*>(S.ctx->pinned + 16);
    if (hs != 0u) return ihs_check_status(S.ctx);
    return IHS_OK;
}

// Sum a device buffer over the ranks of a sharded solve, in place.
int shard_sum(Solver& S, void* buf, int64_t count, int32_t dtype) {
    const int st = S.ar(S.ar_user, buf, count, dtype, (void*)S.ctx->stream);
    if (st != 0) {
        ihs_set_error("the all-reduce callback of a sharded solve failed");
        return IHS_ECUDA;
    }
    return IHS_OK;
}

// old rows of a nested Gaussian sketch: dst = src * scale
__global__ void k_scale_copy(const float* __restrict__ src, int64_t count, float scale, float* __restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = __fmul_rn(src[e], scale);
}

int sketch_level(Solver& S, int64_t m, int level) {
    ihs_ctx* ctx = S.ctx;
    const bool nested = ctx->p.nested != 0;
    const int draw = nested ? 0 : level;   // nested: every size drawn with the key of level 0
    // nested Gaussian doubling: S_m A = [S_{m/2} A / sqrt 2; the new rows], the
    // previous SA read from the slot it lives in, the new one formed in the other
    const bool reuse = nested && ctx->p.kind == IHS_SKETCH_GAUSS && S.SA && S.m >= 4 && m > S.m && S.m % 4 == 0;
    const int slot = reuse ? (S.sa_slot == SLOT_SOLVE_SA ? SLOT_SOLVE_SA2 : SLOT_SOLVE_SA) : SLOT_SOLVE_SA;
    const float* old_SA = S.SA;
    const int64_t old_m = S.m;
    S.F = nullptr;
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, slot, (size_t)m * S.d * sizeof(float), &ws));
    S.SA = static_cast<float*>(ws);
    S.sa_slot = slot;
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[4], ctx->stream));
    if (S.ar) {
        IHS_TRY(ihs_sketch_shard_enqueue(ctx, S.A, S.n, S.d, S.row0, S.n_total, m, ctx->p.kind, ctx->p.seed, draw,
                                         S.SA));
        IHS_TRY(shard_sum(S, S.SA, m * S.d, IHS_DTYPE_F32));
    } else if (reuse) {
        const int64_t count = old_m * S.d;
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div64(count, 256), 8 * (int64_t)ctx->sm_count);
        k_scale_copy<<<grid, 256, 0, ctx->stream>>>(old_SA, count, (float)sqrt((double)old_m / (double)m), S.SA);
        IHS_LAUNCH_CHECK();
        IHS_TRY(ihs_sketch_rows_enqueue(ctx, S.A, S.n, S.d, m, ctx->p.seed, draw, old_m, m - old_m,
                                        S.SA + (size_t)old_m * S.d));
    } else {
        IHS_TRY(ihs_sketch_enqueue(ctx, S.A, S.n, S.d, m, ctx->p.kind, ctx->p.seed, draw, S.SA));
    }
    // enqueue only: the pivot check (status word) and the interval's timing are
    // read after the next synchronisation, in evaluate() or reapply()
    IHS_TRY(ihs_factor_scratch(ctx, S.SA, m, S.d, S.nu, &S.Fs, false));
    S.F = &S.Fs;
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[5], ctx->stream));
    S.sketch_pending = true;
    S.m = m;
    S.level = level;
    return IHS_OK;
}

// g, gt, r, ax2, xx at point `x` (vector indices into S.vec); reads back scalars.
int evaluate(Solver& S, int ix, int ig, int igt, double* r, double* ax2, double* xx, bool need_xx) {
    ihs_ctx* ctx = S.ctx;
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[2], ctx->stream));
    if (S.bsub) {
        const unsigned nrb = (unsigned)ceil_div64(S.n, 128);
        k_dual_resid<<<nrb, 256, 0, ctx->stream>>>(S.A, S.n, (int)S.d, S.vec[ix], S.vlo[ix], S.ds.r, S.ds.rpart);
        IHS_LAUNCH_CHECK();
        dim3 grid((unsigned)ceil_div64(S.d, 256), (unsigned)S.ds.G);
        k_dual_atr<<<grid, 256, 0, ctx->stream>>>(S.A, S.n, (int)S.d, S.ds.r, S.ds.rows_per_group, S.ds.part);
        IHS_LAUNCH_CHECK();
        k_dual_reduce<<<(unsigned)ceil_div64(S.d, 256), 256, 0, ctx->stream>>>(
            S.ds.part, S.ds.G, (int)S.d, S.nu * S.nu, S.vec[ix], S.vlo[ix], S.bsub, S.vec[ig], S.ds.rpart, (int)nrb,
            S.dsc + 1);
        IHS_LAUNCH_CHECK();
    } else if (S.ar) {
        IHS_TRY(ihs_grad_partial_enqueue(ctx, S.A, S.b, S.n, S.d, S.vec[ix], S.gp));
        IHS_TRY(shard_sum(S, S.gp, S.d + 1, IHS_DTYPE_F64));
        IHS_TRY(ihs_grad_finish_enqueue(ctx, S.gp, S.d, S.nu, S.vec[ix], S.vec[ig], S.dsc + 1));
    } else {
        IHS_TRY(ihs_grad_enqueue(ctx, S.A, S.b, S.n, S.d, S.nu, S.vec[ix], S.vec[ig], S.dsc + 1));
    }
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[0], ctx->stream));
    IHS_TRY(ihs_apply_enqueue(ctx, S.F, S.vec[ig], S.vec[igt], S.dsc + 0));
    if (need_xx) {
        k_sumsq<<<1, kSolveThreads, 0, ctx->stream>>>(S.vec[ix], S.d, S.dsc + 2);
        IHS_LAUNCH_CHECK();
    }
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[3], ctx->stream));
    IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, S.dsc, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    IHS_TRY(status_copy(S));
    IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    IHS_TRY(status_after_sync(S));
    float ms = 0.f, msg = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&msg, ctx->ev[2], ctx->ev[0]);
    S.ms_iter += ms;
    S.ms_grad += msg;
    *r = ctx->pinned[0];
    *ax2 = ctx->pinned[1];
    if (need_xx) *xx = ctx->pinned[2];
    return IHS_OK;
}

// Re-apply the (new) factor to the current gradient: gt_t and r_t.
int reapply(Solver& S, int ig, int igt, double* r) {
    ihs_ctx* ctx = S.ctx;
    IHS_TRY(ihs_apply_enqueue(ctx, S.F, S.vec[ig], S.vec[igt], S.dsc + 0));
    IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, S.dsc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    IHS_TRY(status_copy(S));
    IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    IHS_TRY(status_after_sync(S));
    *r = ctx->pinned[0];
    return IHS_OK;
}

int make_candidate(Solver& S, int ix, int igt, int ixp, double mu, double beta, int ixc, double* xx) {
    ihs_ctx* ctx = S.ctx;
    if (S.bsub) {
        k_candidate_df<<<1, kSolveThreads, 0, ctx->stream>>>(S.vec[ix], S.vlo[ix], S.vec[igt], S.vec[ixp], S.vlo[ixp],
                                                            S.d, (float)mu, (float)beta, S.vec[ixc], S.vlo[ixc],
                                                            S.dsc + 2);
    } else {
        k_candidate<<<1, kSolveThreads, 0, ctx->stream>>>(S.vec[ix], S.vec[igt], S.vec[ixp], S.d, (float)mu,
                                                         (float)beta, S.vec[ixc], S.dsc + 2);
    }
    IHS_LAUNCH_CHECK();
    (void)xx;
    return IHS_OK;
}

// st (may be NULL): st->t > 0 continues a run at (t, level, r1) from x_t in
// vec[X] and x_{t-1} in `x_prev_in`; on return *st holds the state at exit and
// x_{T-1} is copied to `x_prev_out` (both may be NULL).
int solve_impl(Solver& S, double tol, ihs_report* rep, ihs_state* st = nullptr, const float* x_prev_in = nullptr,
               float* x_prev_out = nullptr) {
    ihs_ctx* ctx = S.ctx;
    const ihs_params& p = ctx->p;
    const Params prm = make_params(p.kind, p.rho, p.eta);
    const int64_t n_all = S.n_total > 0 ? S.n_total : S.n;   // rows of the whole matrix
    const int64_t m_cap = p.kind == IHS_SKETCH_SRHT ? next_pow2_64(n_all) : n_all;
    const bool resume = st && st->t > 0;
    int64_t m = resume ? st->m : std::min<int64_t>(p.m_init, m_cap);
    int level = 0;
    if (resume) {
        level = st->level;
    } else {
        while (((int64_t)1 << level) < m) ++level;
    }
    ihs_trace_reset(ctx);
    enum { X = 0, XP = 1, G = 2, GT = 3, XC = 4, GC = 5, GTC = 6 };
    int ix = X, ixp = XP, ig = G, igt = GT, ixc = XC, igc = GC, igtc = GTC;
    const size_t vbytes = (size_t)S.d * sizeof(float);
    const float* xp_src = (resume && x_prev_in) ? x_prev_in : S.vec[X];
    IHS_CUDA_TRY(cudaMemcpyAsync(S.vec[XP], xp_src, vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (S.bsub) IHS_CUDA_TRY(cudaMemcpyAsync(S.vlo[XP], S.vlo[X], vbytes, cudaMemcpyDeviceToDevice, ctx->stream));

    IHS_TRY(sketch_level(S, m, level));
    rep->m_levels[0] = m;
    rep->n_levels = 1;
    double r, ax2, xx;
    IHS_TRY(evaluate(S, ix, ig, igt, &r, &ax2, &xx, true));
    rep->grad_passes = 1;
    const double r1 = resume ? st->r1 : r;
    rep->r1 = r1;
    int t = resume ? st->t : 1;
    int status = IHS_EMAXITER;
    while (true) {
        if (!isfinite(r) || !isfinite(ax2)) {
            status = IHS_ENONFINITE;
            break;
        }
        const double scale = tol * sqrt(ax2 + S.nu * S.nu * xx);
        if (r <= 0.0 || sqrt(2.0 * prm.Lam * r) <= scale) {
            ihs_trace_add(ctx, IHS_EV_STOP, t, S.m, r, scale > 0.0 ? sqrt(2.0 * prm.Lam * fmax(r, 0.0)) / scale : 0.0);
            status = IHS_OK;
            break;
        }
        if (t >= p.max_iter) break;
        bool accepted = false;
        if (p.variant == IHS_VARIANT_POLYAK) {
            double rc, ax2c, xxc;
            IHS_TRY(make_candidate(S, ix, igt, ixp, prm.mu_p, prm.beta_p, ixc, nullptr));
            IHS_TRY(evaluate(S, ixc, igc, igtc, &rc, &ax2c, &xxc, false));
            xxc = ctx->pinned[2];
            rep->grad_passes++;
            const double ratio = rc > 0.0 ? pow(rc / r1, 1.0 / t) : 0.0;
            ihs_trace_add(ctx, (isfinite(rc) && ratio <= prm.c_p) ? IHS_EV_POLYAK : IHS_EV_POLYAK_REJECT, t, S.m, r,
                          ratio);
            if (isfinite(rc) && ratio <= prm.c_p) {
                std::swap(ixp, ix);
                std::swap(ix, ixc);   // x_prev <- x, x <- xc, xc <- old x_prev
                std::swap(ig, igc);
                std::swap(igt, igtc);
                r = rc;
                ax2 = ax2c;
                xx = xxc;
                rep->accepted_polyak++;
                accepted = true;
            }
        }
        if (!accepted) {
            double rc, ax2c, xxc;
            IHS_TRY(make_candidate(S, ix, igt, ixp, prm.mu_gd, 0.0, ixc, nullptr));
            IHS_TRY(evaluate(S, ixc, igc, igtc, &rc, &ax2c, &xxc, false));
            xxc = ctx->pinned[2];
            rep->grad_passes++;
            if (!isfinite(rc)) {
                status = IHS_ENONFINITE;
                break;
            }
            const double ratio = rc / r;
            if (ratio <= prm.c_gd || S.m >= m_cap) {
                ihs_trace_add(ctx, ratio <= prm.c_gd ? IHS_EV_GD : IHS_EV_GD_AT_CAP, t, S.m, r, ratio);
                if (!(ratio <= prm.c_gd)) rep->flags |= 1;
                std::swap(ixp, ix);
                std::swap(ix, ixc);
                std::swap(ig, igc);
                std::swap(igt, igtc);
                r = rc;
                ax2 = ax2c;
                xx = xxc;
                rep->accepted_gd++;
                accepted = true;
            } else if (p.floor > 0.0 && r <= p.floor * p.floor * r1) {
                ihs_trace_add(ctx, IHS_EV_FLOOR, t, S.m, r, ratio);
                rep->flags |= 2;
                status = IHS_OK;
                break;
            } else {
                ihs_trace_add(ctx, IHS_EV_DOUBLE, t, S.m, r, ratio);
                rep->rejected++;
                const int64_t m_new = std::min<int64_t>(2 * S.m, m_cap);
                IHS_TRY(sketch_level(S, m_new, S.level + 1));
                if (rep->n_levels < IHS_REPORT_MAX_LEVELS) rep->m_levels[rep->n_levels] = m_new;
                rep->n_levels++;
                IHS_TRY(reapply(S, ig, igt, &r));
                continue;
            }
        }
        ++t;
    }
    if (x_prev_out)
        IHS_CUDA_TRY(cudaMemcpyAsync(x_prev_out, S.vec[ixp], vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ix != X) {
        IHS_CUDA_TRY(cudaMemcpyAsync(S.vec[X], S.vec[ix], vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        if (S.bsub) IHS_CUDA_TRY(cudaMemcpyAsync(S.vlo[X], S.vlo[ix], vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (st) {
        st->grad_passes = (resume ? st->grad_passes : 0) + rep->grad_passes;
        st->n_levels = (resume ? st->n_levels : 0) + rep->n_levels;
        st->t = t;
        st->level = S.level;
        st->m = S.m;
        st->r1 = r1;
    }
    rep->status = status;
    rep->iterations = t;
    rep->m_final = S.m;
    rep->r_final = r;
    rep->axnorm_final = sqrt(ax2 + S.nu * S.nu * xx);
    rep->ms_sketch = S.ms_sketch;
    rep->ms_iterate = S.ms_iter;
    rep->ms_grad = S.ms_grad;
    return status;
}

}  // namespace

extern "C" int ihs_solve(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu, double tol,
                         float* x, ihs_report* rep_h) {
    if (!ctx || !A || !b || !x) return IHS_EINVAL;
    if (n < 1 || d < 1 || n < d || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    if (!(tol > 0.0)) tol = ctx->p.tol;
    IhsRange range("ihs_solve");
    ihs_report rep;
    memset(&rep, 0, sizeof(rep));
    Solver S;
    memset(&S, 0, sizeof(S));
    S.ctx = ctx;
    S.A = A;
    S.b = b;
    S.n = n;
    S.d = d;
    S.nu = nu;
    void* ws = nullptr;
    const size_t vb = ((size_t)d * sizeof(float) + 255) & ~(size_t)255;
    IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE, 7 * vb + 8192 * sizeof(double), &ws));
    char* base = static_cast<char*>(ws);
    S.vec[0] = x;
    for (int i = 1; i < 7; ++i) S.vec[i] = reinterpret_cast<float*>(base + i * vb);
    S.dsc = reinterpret_cast<double*>(base + 7 * vb);
    const int st = solve_impl(S, tol, &rep);
    if (rep_h) *rep_h = rep;
    if (st == IHS_OK || st == IHS_EMAXITER || st == IHS_ENONFINITE) {
        // a device wait that gave up poisons r (non-finite): report the cause
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return st;
}

extern "C" int ihs_solve_host(ihs_ctx* ctx, const float* A_h, const float* b_h, int64_t n, int64_t d, double nu,
                              double tol, float* x_h, ihs_report* rep_h) {
    if (!ctx || !A_h || !b_h || !x_h) return IHS_EINVAL;
    if (n < 1 || d < 1 || n < d || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    IhsRange range("ihs_solve_host");
    // A, b, x in one context-owned block (each piece 256-byte aligned)
    const size_t bA = ((size_t)n * d * sizeof(float) + 255) & ~(size_t)255;
    const size_t bb = ((size_t)n * sizeof(float) + 255) & ~(size_t)255;
    const size_t bx = ((size_t)d * sizeof(float) + 255) & ~(size_t)255;
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_HOST_IN, bA + bb + bx, &ws));
    char* base = static_cast<char*>(ws);
    float* A = reinterpret_cast<float*>(base);
    float* b = reinterpret_cast<float*>(base + bA);
    float* x = reinterpret_cast<float*>(base + bA + bb);
    // one copy per piece, A in 256 MiB pieces so that the first ones can start
    // the DMA engine while the next are issued (copies spread over several
    // streams measured no faster: the host link sets the rate)
    const size_t total = (size_t)n * d * sizeof(float), piece = (size_t)256 << 20;
    for (size_t o = 0; o < total; o += piece) {
        const size_t len = total - o < piece ? total - o : piece;
        IHS_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(A) + o, reinterpret_cast<const char*>(A_h) + o, len,
                                     cudaMemcpyHostToDevice, ctx->stream));
    }
    IHS_CUDA_TRY(cudaMemcpyAsync(b, b_h, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    IHS_CUDA_TRY(cudaMemcpyAsync(x, x_h, (size_t)d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    const int st = ihs_solve(ctx, A, b, n, d, nu, tol, x, rep_h);
    if (st == IHS_OK || st == IHS_EMAXITER) {
        IHS_CUDA_TRY(cudaMemcpyAsync(x_h, x, (size_t)d * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return st;
}

extern "C" int ihs_solve_resume(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu,
                                double tol, float* x, float* x_prev, ihs_state* st_h, ihs_report* rep_h) {
    if (!ctx || !A || !b || !x || !x_prev || !st_h) return IHS_EINVAL;
    if (n < 1 || d < 1 || n < d || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    if (st_h->t < 0) return IHS_EINVAL;
    if (st_h->t > 0) {
        const int64_t m_cap = ctx->p.kind == IHS_SKETCH_SRHT ? next_pow2_64(n) : n;
        if (st_h->level < 0 || st_h->level > 62 || st_h->m < 1 || st_h->m > m_cap || !(st_h->r1 > 0.0) ||
            (st_h->m != ((int64_t)1 << st_h->level) && st_h->m != m_cap))
            return IHS_EINVAL;
    }
    if (!(tol > 0.0)) tol = ctx->p.tol;
    IhsRange range("ihs_solve_resume");
    ihs_report rep;
    memset(&rep, 0, sizeof(rep));
    Solver S;
    memset(&S, 0, sizeof(S));
    S.ctx = ctx;
    S.A = A;
    S.b = b;
    S.n = n;
    S.d = d;
    S.nu = nu;
    void* ws = nullptr;
    const size_t vb = ((size_t)d * sizeof(float) + 255) & ~(size_t)255;
    IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE, 7 * vb + 8192 * sizeof(double), &ws));
    char* base = static_cast<char*>(ws);
    S.vec[0] = x;
    for (int i = 1; i < 7; ++i) S.vec[i] = reinterpret_cast<float*>(base + i * vb);
    S.dsc = reinterpret_cast<double*>(base + 7 * vb);
    const int st = solve_impl(S, tol, &rep, st_h, x_prev, x_prev);
    if (rep_h) *rep_h = rep;
    if (st == IHS_OK || st == IHS_EMAXITER || st == IHS_ENONFINITE) {
        // a device wait that gave up poisons r (non-finite): report the cause
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return st;
}

extern "C" int ihs_solve_sharded(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, int64_t row0,
                                 int64_t n_total, double nu, double tol, float* x, ihs_report* rep_h,
                                 ihs_allreduce_fn allreduce, void* user) {
    if (!ctx || !A || !b || !x || !allreduce) return IHS_EINVAL;
    if (n < 1 || d < 1 || row0 < 0 || n_total < row0 + n || n_total < d || !(nu > 0.0) || !isfinite(nu))
        return IHS_EINVAL;
    if (ctx->p.nested) return IHS_EINVAL;
    if (ctx->p.kind == IHS_SKETCH_SRHT && (row0 % 1024 || (n % 1024 && row0 + n != n_total))) return IHS_EINVAL;
    if (!(tol > 0.0)) tol = ctx->p.tol;
    IhsRange range("ihs_solve_sharded");
    ihs_report rep;
    memset(&rep, 0, sizeof(rep));
    Solver S;
    memset(&S, 0, sizeof(S));
    S.ctx = ctx;
    S.A = A;
    S.b = b;
    S.n = n;
    S.d = d;
    S.nu = nu;
    S.row0 = row0;
    S.n_total = n_total;
    S.ar = allreduce;
    S.ar_user = user;
    void* ws = nullptr;
    const size_t vb = ((size_t)d * sizeof(float) + 255) & ~(size_t)255;
    const size_t gb = ((size_t)(d + 1) * sizeof(double) + 255) & ~(size_t)255;
    IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE, 7 * vb + gb + 8192 * sizeof(double), &ws));
    char* base = static_cast<char*>(ws);
    S.vec[0] = x;
    for (int i = 1; i < 7; ++i) S.vec[i] = reinterpret_cast<float*>(base + i * vb);
    S.gp = reinterpret_cast<double*>(base + 7 * vb);
    S.dsc = reinterpret_cast<double*>(base + 7 * vb + gb);
    const int st = solve_impl(S, tol, &rep);
    if (rep_h) *rep_h = rep;
    if (st == IHS_OK || st == IHS_EMAXITER || st == IHS_ENONFINITE) {
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return st;
}

// Underdetermined case (App. A.2): the controller runs on the dual
// z* = argmin 1/2 ||A^T z||^2 + nu^2/2 ||z||^2 - b^T z, an overdetermined
// problem with data matrix A^T (d x n) and gradient A A^T z - b + nu^2 z
// (double-float iterate and residual, see k_dual_resid); sketches are drawn
// over the d rows of A^T.  x = A^T z at the end.
extern "C" int ihs_solve_dual(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu,
                              double tol, float* x, ihs_report* rep_h) {
    IhsRange range("ihs_solve_dual");
    if (!ctx || !A || !b || !x) return IHS_EINVAL;
    if (n < 1 || d < 1 || n > d || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    if (!(tol > 0.0)) tol = ctx->p.tol;
    ihs_report rep;
    memset(&rep, 0, sizeof(rep));
    // A^T (d x n), then the dual gradient's scratch: r (d pairs), its ||r||^2
    // partials, and G x n column partials
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(256, (2 * (int64_t)ctx->sm_count * 256) / n));
    const size_t at_bytes = ((size_t)n * d * sizeof(float) + 255) & ~(size_t)255;
    const size_t r_bytes = ((size_t)d * sizeof(float2) + 255) & ~(size_t)255;
    const size_t rp_bytes = (((size_t)ceil_div64(d, 128)) * sizeof(double) + 255) & ~(size_t)255;
    const size_t part_bytes = (size_t)G * n * sizeof(float2);
    void* dws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_DUAL, at_bytes + r_bytes + rp_bytes + part_bytes, &dws));
    char* dp = static_cast<char*>(dws);
    float* AT = reinterpret_cast<float*>(dp);
    dim3 tg((unsigned)ceil_div64(d, 32), (unsigned)ceil_div64(n, 32));
    k_transpose_rect<<<tg, 256, 0, ctx->stream>>>(A, n, d, AT);
    IHS_LAUNCH_CHECK();
    Solver S;
    memset(&S, 0, sizeof(S));
    S.ctx = ctx;
    S.A = AT;
    S.b = nullptr;
    S.bsub = b;
    S.n = d;
    S.d = n;
    S.nu = nu;
    S.ds.r = reinterpret_cast<float2*>(dp + at_bytes);
    S.ds.rpart = reinterpret_cast<double*>(dp + at_bytes + r_bytes);
    S.ds.part = reinterpret_cast<float2*>(dp + at_bytes + r_bytes + rp_bytes);
    S.ds.G = (int)G;
    S.ds.rows_per_group = ceil_div64(d, G);
    void* ws = nullptr;
    const size_t vb = ((size_t)n * sizeof(float) + 255) & ~(size_t)255;
    IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE, 14 * vb + 8192 * sizeof(double), &ws));
    char* base = static_cast<char*>(ws);
    for (int i = 0; i < 7; ++i) {
        S.vec[i] = reinterpret_cast<float*>(base + i * vb);   // vec[0] = z
        S.vlo[i] = reinterpret_cast<float*>(base + (7 + i) * vb);
    }
    S.dsc = reinterpret_cast<double*>(base + 14 * vb);
    IHS_CUDA_TRY(cudaMemsetAsync(base, 0, 14 * vb, ctx->stream));   // z_0 = 0 (both parts)
    const int st = solve_impl(S, tol, &rep);
    if (rep_h) *rep_h = rep;
    if (st == IHS_OK || st == IHS_EMAXITER) {
        k_rows_dot<<<(unsigned)ceil_div64(d * 32, 256), 256, 0, ctx->stream>>>(AT, d, n, S.vec[0], S.vlo[0], x);
        IHS_LAUNCH_CHECK();
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return st;
}
