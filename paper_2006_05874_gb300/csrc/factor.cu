// Factor and apply of the sketched Hessian H_S = (SA)^T SA + nu^2 I (Eq. 3).
//
// m < d : Woodbury form (App. B.4)
//         H_S^{-1} g = nu^-2 (g - (SA)^T K^{-1} SA g),  K = nu^2 I_m + SA (SA)^T,
// m >= d: K = H_S itself (d x d) and H_S^{-1} g = K^{-1} g.
// K is formed in FP64 from the FP32 sketch (products exact, FP64 sums),
// factored K = L L^T by a blocked FP64 Cholesky (non-positive or non-finite
// pivots set IHS_DEV_NOTPD), and L is inverted once (blocked triangular
// inverse) so that every apply is a chain of parallel matrix-vector products:
//   t = SA g, v = L^-1 t, u = L^-T v, gt = nu^-2 (g - SA^T u)   (Woodbury)
//   v = L^-1 g, gt = L^-T v                                     (direct)
// and r = 1/2 g^T gt (Lemma 4.1) in FP64.
#include <algorithm>
#include <new>

#include "common.cuh"

namespace {

constexpr int NB = 32;   // block size of the factorisations

// K = X X^T (+ nu^2 I) on lower tiles, X(r, k) = woodbury ? SA[r][k] : SA[k][r].
__global__ void __launch_bounds__(256) k_gram64(const float* __restrict__ SA, int64_t m, int64_t d,
                                                int woodbury, int64_t kdim, int64_t K, double nu2,
                                                double* __restrict__ G) {
    __shared__ double xa[32][33];
    __shared__ double xb[32][33];
    // lower-tile index -> (I, J), I >= J
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        __syncthreads();
        if (woodbury) {
            // X(r, k) = SA[r][k]: rows of SA, coalesced along k
            for (int e = threadIdx.x; e < 32 * 32; e += 256) {
                const int rr = e / 32, kk = e % 32;
                const int64_t ra = I * 32 + rr, rb = J * 32 + rr, k = k0 + kk;
                xa[rr][kk] = (ra < kdim && k < K) ? (double)SA[ra * d + k] : 0.0;
                xb[rr][kk] = (rb < kdim && k < K) ? (double)SA[rb * d + k] : 0.0;
            }
        } else {
            // X(r, k) = SA[k][r]: rows of SA, coalesced along r
            for (int e = threadIdx.x; e < 32 * 32; e += 256) {
                const int kk = e / 32, rr = e % 32;
                const int64_t ra = I * 32 + rr, rb = J * 32 + rr, k = k0 + kk;
                xa[rr][kk] = (ra < kdim && k < K) ? (double)SA[k * d + ra] : 0.0;
                xb[rr][kk] = (rb < kdim && k < K) ? (double)SA[k * d + rb] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const double a0 = xa[ty * 2][kk], a1 = xa[ty * 2 + 1][kk];
            const double b0 = xb[tx * 2][kk], b1 = xb[tx * 2 + 1][kk];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t r = I * 32 + ty * 2 + a, c = J * 32 + tx * 2 + b;
            if (r < kdim && c < kdim && c <= r) G[r * kdim + c] = acc[a][b] + (r == c ? nu2 : 0.0);
        }
}

// Unblocked Cholesky of the diagonal block [j0, j0+nb) in place (lower).
__global__ void __launch_bounds__(NB * NB) k_potrf_diag(double* __restrict__ K, int64_t k, int64_t j0, int nb,
                                                        unsigned* status) {
    __shared__ double a[NB][NB + 1];
    __shared__ int bad;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    if (threadIdx.x == 0) bad = 0;
    if (r < nb && c < nb && c <= r) a[r][c] = K[(j0 + r) * k + j0 + c];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double p = a[j][j];
            if (!(p > 0.0) || !isfinite(p)) {
                bad = 1;
                a[j][j] = 1.0;
            } else {
                a[j][j] = sqrt(p);
            }
        }
        __syncthreads();
        if (c == j && r > j && r < nb) a[r][j] /= a[j][j];
        __syncthreads();
        if (r > j && c > j && c <= r && r < nb) a[r][c] -= a[r][j] * a[c][j];
        __syncthreads();
    }
    if (r < nb && c < nb && c <= r) K[(j0 + r) * k + j0 + c] = a[r][c];
    if (threadIdx.x == 0 && bad) atomicOr(status, IHS_DEV_NOTPD);
}

// Panel: rows i >= j0 + nb solve x L_jj^T = K[i][j0:j0+nb] (forward substitution).
__global__ void k_trsm_panel(double* __restrict__ K, int64_t k, int64_t j0, int nb) {
    __shared__ double l[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e / nb, c = e % nb;
        l[r][c] = c <= r ? K[(j0 + r) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    const int64_t i = j0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c < nb) {
            double s = K[i * k + j0 + c];
            for (int c2 = 0; c2 < c; ++c2) s -= x[c2] * l[c][c2];
            x[c] = s / l[c][c];
            K[i * k + j0 + c] = x[c];
        }
    }
}

// Trailing update K[j1:, j1:] -= P P^T on lower tiles, P = K[j1:, j0:j1].
__global__ void __launch_bounds__(256) k_syrk_update(double* __restrict__ K, int64_t k, int64_t j0, int nb) {
    __shared__ double pa[32][NB + 1];
    __shared__ double pb[32][NB + 1];
    const int64_t j1 = j0 + nb;
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < 32 * nb; e += 256) {
        const int rr = e / nb, kk = e % nb;
        const int64_t ra = j1 + I * 32 + rr, rb = j1 + J * 32 + rr;
        pa[rr][kk] = ra < k ? K[ra * k + j0 + kk] : 0.0;
        pb[rr][kk] = rb < k ? K[rb * k + j0 + kk] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int kk = 0; kk < nb; ++kk) {
        const double a0 = pa[ty * 2][kk], a1 = pa[ty * 2 + 1][kk];
        const double b0 = pb[tx * 2][kk], b1 = pb[tx * 2 + 1][kk];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t r = j1 + I * 32 + ty * 2 + a, c = j1 + J * 32 + tx * 2 + b;
            if (r < k && c <= r) K[r * k + c] -= acc[a][b];
        }
}

// Inverse of each diagonal NB x NB block of L (one CTA per block, thread = column).
__global__ void k_trtri_diag(const double* __restrict__ L, int64_t k, double* __restrict__ X) {
    __shared__ double l[NB][NB + 1];
    const int64_t b0 = (int64_t)blockIdx.x * NB;
    const int nb = (int)(k - b0 < NB ? k - b0 : NB);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        l[r][c] = (r < nb && c < nb && c <= r) ? L[(b0 + r) * k + b0 + c] : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c >= nb) return;
    double x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (r < nb) {
            if (r < c) {
                x[r] = 0.0;
            } else {
                double s = (r == c) ? 1.0 : 0.0;
                for (int l2 = c; l2 < r; ++l2) s -= l[r][l2] * x[l2];
                x[r] = s / l[r][r];
            }
            X[(b0 + r) * k + b0 + c] = x[r];
        }
    }
}

// Off-diagonal blocks at distance `dist`: X_IJ = -X_II sum_{K=J}^{I-1} L_IK X_KJ.
__global__ void __launch_bounds__(256) k_trtri_off(const double* __restrict__ L, int64_t k, int64_t T, int64_t dist,
                                                   double* __restrict__ X) {
    __shared__ double la[NB][NB + 1];
    __shared__ double xb[NB][NB + 1];
    __shared__ double tm[NB][NB + 1];
    const int64_t J = blockIdx.x, I = J + dist;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t Kb = J; Kb < I; ++Kb) {
        __syncthreads();
        for (int e = threadIdx.x; e < NB * NB; e += 256) {
            const int r = e / NB, c = e % NB;
            const int64_t gi = I * NB + r, gk = Kb * NB + c;
            la[r][c] = (gi < k && gk < k) ? L[gi * k + gk] : 0.0;
            const int64_t gk2 = Kb * NB + r, gj = J * NB + c;
            xb[r][c] = (gk2 < k && gj < k) ? X[gk2 * k + gj] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < NB; ++kk) {
            const double a0 = la[ty * 2][kk], a1 = la[ty * 2 + 1][kk];
            const double b0 = xb[kk][tx * 2], b1 = xb[kk][tx * 2 + 1];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
    }
    __syncthreads();
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) tm[ty * 2 + a][tx * 2 + b] = acc[a][b];
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
        const int r = e / NB, c = e % NB;
        const int64_t gi = I * NB + r, gc = I * NB + c;
        la[r][c] = (gi < k && gc < k) ? X[gi * k + gc] : 0.0;   // X_II
    }
    __syncthreads();
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int r = ty * 2 + a, c = tx * 2 + b;
            double s = 0.0;
            for (int kk = 0; kk < NB; ++kk) s = fma(la[r][kk], tm[kk][c], s);
            const int64_t gi = I * NB + r, gj = J * NB + c;
            if (gi < k && gj < k) X[gi * k + gj] = -s;
        }
}

// XT = X^T on the lower triangle (XT upper), zero elsewhere.
__global__ void k_transpose_lower(const double* __restrict__ X, int64_t k, double* __restrict__ XT) {
    __shared__ double tile[32][33];
    const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = by + r, gc = bx + tx;
        tile[r][tx] = (gr < k && gc < k && gc <= gr) ? X[gr * k + gc] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = bx + r, gc = by + tx;
        if (gr < k && gc < k) XT[gr * k + gc] = tile[tx][r];
    }
}

// y[i] = sum_l M[i][l] v[l], l in [lo(i), hi(i)) with tri = 0 full row, 1 lower
// (l <= i), 2 upper (l >= i).  One warp per row; FP64.  v_f (float) or v_d (double).
__global__ void k_gemv64(const double* __restrict__ M, int64_t rows, int64_t cols, int tri,
                         const double* __restrict__ v_d, double* __restrict__ y) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const int64_t i = warp;
    const int64_t lo = tri == 2 ? i : 0, hi = tri == 1 ? i + 1 : cols;
    double s = 0.0;
    for (int64_t l = lo + lane; l < hi; l += 32) s = fma(M[i * cols + l], v_d[l], s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) y[i] = s;
}

// t[j] = sum_l SA[j][l] g[l] in FP64 (products exact), one warp per row.
__global__ void k_sa_g(const float* __restrict__ SA, int64_t m, int64_t d, const float* __restrict__ g,
                       double* __restrict__ t) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= m) return;
    double s = 0.0;
    for (int64_t l = lane; l < d; l += 32) s = fma((double)SA[warp * d + l], (double)g[l], s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) t[warp] = s;
}

// Partial column sums of SA^T u over row chunks: part[chunk][c] (FP64).
__global__ void k_sat_u(const float* __restrict__ SA, int64_t m, int64_t d, const double* __restrict__ u,
                        int64_t rows_per_chunk, double* __restrict__ part) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t j1 = m < j0 + rows_per_chunk ? m : j0 + rows_per_chunk;
    if (c >= d) return;
    double s = 0.0;
    for (int64_t j = j0; j < j1; ++j) s = fma((double)SA[j * d + c], u[j], s);
    part[blockIdx.y * d + c] = s;
}

// gt = scale (g - sum_chunks part) (woodbury) or gt = u (direct); per-block
// partials of g . gt for r.
__global__ void k_apply_final(const float* __restrict__ g, const double* __restrict__ part, int chunks,
                              const double* __restrict__ u_direct, int64_t d, double inv_nu2,
                              float* __restrict__ gt, double* __restrict__ rpart) {
    __shared__ double sm[256];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double prod = 0.0;
    if (c < d) {
        double v;
        if (u_direct) {
            v = u_direct[c];
        } else {
            double s = 0.0;
            for (int k = 0; k < chunks; ++k) s += part[k * d + c];
            v = ((double)g[c] - s) * inv_nu2;
        }
        gt[c] = (float)v;
        prod = (double)g[c] * v;
    }
    sm[threadIdx.x] = prod;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 256; ++i) s += sm[i];
        rpart[blockIdx.x] = s;
    }
}

__global__ void k_sum_half(const double* __restrict__ rpart, int count, double* __restrict__ r) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += rpart[i];
    *r = 0.5 * s;
}

__global__ void k_to_double(const float* __restrict__ a, int64_t n, double* __restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

}  // namespace

int ihs_factor_build(ihs_ctx* ctx, ihs_factor_t* F) {
    const int64_t k = F->k;
    cudaStream_t s = ctx->stream;
    const int64_t T = ceil_div64(k, NB);
    // K = X X^T + nu^2 I on lower tiles
    const int64_t ntiles = T * (T + 1) / 2;
    const int64_t K = F->woodbury ? F->d : F->m;
    k_gram64<<<(unsigned)ntiles, 256, 0, s>>>(F->SA, F->m, F->d, F->woodbury, k, K, F->nu * F->nu, F->L);
    IHS_LAUNCH_CHECK();
    for (int64_t j0 = 0; j0 < k; j0 += NB) {
        const int nb = (int)std::min<int64_t>(NB, k - j0);
        k_potrf_diag<<<1, NB * NB, 0, s>>>(F->L, k, j0, nb, ctx->d_status);
        IHS_LAUNCH_CHECK();
        const int64_t rest = k - j0 - nb;
        if (rest > 0) {
            k_trsm_panel<<<(unsigned)ceil_div64(rest, 128), 128, 0, s>>>(F->L, k, j0, nb);
            IHS_LAUNCH_CHECK();
            const int64_t Tr = ceil_div64(rest, 32);
            k_syrk_update<<<(unsigned)(Tr * (Tr + 1) / 2), 256, 0, s>>>(F->L, k, j0, nb);
            IHS_LAUNCH_CHECK();
        }
    }
    // Linv (stored in F->Linv, lower), then its transpose in F->work area? keep
    // LinvT in the upper part of a separate buffer: reuse L's storage for L^-T.
    IHS_CUDA_TRY(cudaMemsetAsync(F->Linv, 0, (size_t)k * k * sizeof(double), s));
    k_trtri_diag<<<(unsigned)T, NB, 0, s>>>(F->L, k, F->Linv);
    IHS_LAUNCH_CHECK();
    for (int64_t dist = 1; dist < T; ++dist) {
        k_trtri_off<<<(unsigned)(T - dist), 256, 0, s>>>(F->L, k, T, dist, F->Linv);
        IHS_LAUNCH_CHECK();
    }
    // L is no longer needed: overwrite it with Linv^T (full row-major, upper).
    dim3 tg((unsigned)ceil_div64(k, 32), (unsigned)ceil_div64(k, 32));
    k_transpose_lower<<<tg, 256, 0, s>>>(F->Linv, k, F->L);
    IHS_LAUNCH_CHECK();
    return ihs_check_status(ctx);
}

int ihs_apply_enqueue(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* d_r) {
    cudaStream_t s = ctx->stream;
    const int64_t k = F->k, d = F->d, m = F->m;
    double* t = F->work;            // k
    double* v = t + k;              // k
    double* u = v + k;              // k
    double* rpart = u + k;          // up to 4096
    double* part = rpart + 4096;    // chunks x d
    const double* LinvT = F->L;     // after factor_build
    const unsigned wblocks = (unsigned)ceil_div64(k * 32, 256);
    if (F->woodbury) {
        k_sa_g<<<wblocks, 256, 0, s>>>(F->SA, m, d, g, t);
        IHS_LAUNCH_CHECK();
    } else {
        k_to_double<<<(unsigned)ceil_div64(d, 256), 256, 0, s>>>(g, d, t);
        IHS_LAUNCH_CHECK();
    }
    k_gemv64<<<wblocks, 256, 0, s>>>(F->Linv, k, k, 1, t, v);
    IHS_LAUNCH_CHECK();
    k_gemv64<<<wblocks, 256, 0, s>>>(LinvT, k, k, 2, v, u);
    IHS_LAUNCH_CHECK();
    const unsigned fblocks = (unsigned)ceil_div64(d, 256);
    if (F->woodbury) {
        const int64_t chunks = std::min<int64_t>(32, std::max<int64_t>(1, m / 32));
        const int64_t rpc = ceil_div64(m, chunks);
        const int64_t nch = ceil_div64(m, rpc);
        dim3 grid(fblocks, (unsigned)nch);
        k_sat_u<<<grid, 256, 0, s>>>(F->SA, m, d, u, rpc, part);
        IHS_LAUNCH_CHECK();
        k_apply_final<<<fblocks, 256, 0, s>>>(g, part, (int)nch, nullptr, d, 1.0 / (F->nu * F->nu), gt, rpart);
    } else {
        k_apply_final<<<fblocks, 256, 0, s>>>(g, nullptr, 0, u, d, 0.0, gt, rpart);
    }
    IHS_LAUNCH_CHECK();
    if (d_r) {
        k_sum_half<<<1, 1, 0, s>>>(rpart, (int)fblocks, d_r);
        IHS_LAUNCH_CHECK();
    }
    return IHS_OK;
}

extern "C" int ihs_factor(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** out) {
    if (!ctx || !SA || !out || m < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    *out = nullptr;
    ihs_factor_t* F = new (std::nothrow) ihs_factor_t;
    if (!F) return IHS_ENOMEM;
    F->ctx = ctx;
    F->SA = SA;
    F->m = m;
    F->d = d;
    F->nu = nu;
    F->woodbury = m < d ? 1 : 0;
    F->k = F->woodbury ? m : d;
    F->L = F->Linv = F->work = nullptr;
    const size_t kk = (size_t)F->k * F->k * sizeof(double);
    const size_t work = (3 * (size_t)F->k + 4096 + 32 * (size_t)d + 64) * sizeof(double);
    if (cudaMalloc(&F->L, kk) != cudaSuccess || cudaMalloc(&F->Linv, kk) != cudaSuccess ||
        cudaMalloc(&F->work, work) != cudaSuccess) {
        cudaGetLastError();
        ihs_factor_destroy(F);
        return IHS_ENOMEM;
    }
    const int st = ihs_factor_build(ctx, F);
    if (st != IHS_OK) {
        ihs_factor_destroy(F);
        return st;
    }
    *out = F;
    return IHS_OK;
}

extern "C" int ihs_factor_destroy(ihs_factor_t* F) {
    if (!F) return IHS_OK;
    if (F->ctx) cudaStreamSynchronize(F->ctx->stream);
    if (F->L) cudaFree(F->L);
    if (F->Linv) cudaFree(F->Linv);
    if (F->work) cudaFree(F->work);
    delete F;
    return IHS_OK;
}

extern "C" int ihs_apply_hinv(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* r_h) {
    if (!ctx || !F || !g || !gt) return IHS_EINVAL;
    double* d_r = F->work + 3 * F->k + 4096 + 32 * F->d;
    IHS_TRY(ihs_apply_enqueue(ctx, F, g, gt, d_r));
    if (r_h) {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, d_r, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *r_h = ctx->pinned[0];
    }
    return IHS_OK;
}
