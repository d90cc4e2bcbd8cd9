// Factor and apply of the sketched Hessian H_S = (SA)^T SA + nu^2 I (Eq. 3).
//
// m < d : Woodbury form (App. B.4)
//         H_S^{-1} g = nu^-2 (g - (SA)^T K^{-1} SA g),  K = nu^2 I_m + SA (SA)^T,
// m >= d: K = H_S itself (d x d) and H_S^{-1} g = K^{-1} g.
// K is formed from the FP32 sketch with compensated FP32 accumulation and
// stored in FP64; K = L L^T by a blocked FP64 Cholesky (64-wide blocks; the
// diagonal block also yields its inverse, the panel is a GEMM with it, the
// trailing update is an FP64 SYRK on 64 x 64 tiles; non-positive or non-finite
// pivots set IHS_DEV_NOTPD).  X = L^{-1} is formed once in FP32 by recursive
// doubling ([L11 0; L21 L22]^{-1} has lower-left block -X22 L21 X11), so every
// apply is a chain of parallel matrix-vector products, followed by one step of
// iterative refinement against the exact operator in FP64 accumulation:
//   u0 = X^T X t, u1 = u0 + X^T X (t - K u0)
// with t = SA g, gt = nu^-2 (g - SA^T u1) (Woodbury) or t = g, gt = u1
// (direct); r = 1/2 g^T gt (Lemma 4.1) in FP64.
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"

namespace {

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

__global__ void k_sum_half(const double* __restrict__ rpart, int count, double* __restrict__ r) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += rpart[i];
    *r = 0.5 * s;
}

__global__ void k_to_double(const float* __restrict__ a, int64_t n, double* __restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}


// ---------------------------------------------------------------------------
// Factor v2 building blocks.

constexpr int FB = 64;   // block size of the FP64 Cholesky and of the inverse

// K = X X^T + nu^2 I on lower 64x64 tiles from the FP32 sketch with
// compensated FP32 accumulation: FMA chains over 4 terms, each chain added to
// a (hi, lo) pair by TwoSum; K stored in FP64.  X(r, k) = SA[r][k] (Woodbury)
// or SA[k][r] (direct).
__global__ void __launch_bounds__(256) k_gram_c32(const float* __restrict__ SA, int64_t d, int woodbury,
                                                  int64_t kdim, int64_t K, double nu2, double* __restrict__ G) {
    __shared__ float xa[32][FB + 4];
    __shared__ float xb[32][FB + 4];
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        __syncthreads();
        if (woodbury) {
            for (int e = threadIdx.x; e < 32 * FB; e += 256) {
                const int rr = e / 32, kk = e % 32;
                const int64_t ra = I * FB + rr, rb = J * FB + rr, k = k0 + kk;
                xa[kk][rr] = (ra < kdim && k < K) ? SA[ra * d + k] : 0.f;
                xb[kk][rr] = (rb < kdim && k < K) ? SA[rb * d + k] : 0.f;
            }
        } else {
            for (int e = threadIdx.x; e < 32 * FB; e += 256) {
                const int kk = e / FB, rr = e % FB;
                const int64_t ra = I * FB + rr, rb = J * FB + rr, k = k0 + kk;
                xa[kk][rr] = (ra < kdim && k < K) ? SA[k * d + ra] : 0.f;
                xb[kk][rr] = (rb < kdim && k < K) ? SA[k * d + rb] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < 32; kc += 4) {
            float av[4][4], bv[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    av[q][a] = xa[kc + q][ty + 16 * a];
                    bv[q][a] = xb[kc + q][tx + 16 * a];
                }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float c4 = __fmul_rn(av[0][a], bv[0][b]);
                    c4 = __fmaf_rn(av[1][a], bv[1][b], c4);
                    c4 = __fmaf_rn(av[2][a], bv[2][b], c4);
                    c4 = __fmaf_rn(av[3][a], bv[3][b], c4);
                    float s, e;
                    two_sum(hi[a][b], c4, s, e);
                    hi[a][b] = s;
                    lo[a][b] = __fadd_rn(lo[a][b], e);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t r = I * FB + ty + 16 * a, c = J * FB + tx + 16 * b;
            if (r < kdim && c < kdim && c <= r)
                G[r * kdim + c] = (double)hi[a][b] + (double)lo[a][b] + (r == c ? nu2 : 0.0);
        }
}

// Diagonal block [j0, j0+nb) of the FP64 Cholesky: L_jj in place and
// W = L_jj^{-1} (lower, nb x nb, stored FB x FB at Wd).  Non-positive or
// non-finite pivots set IHS_DEV_NOTPD (the pivot is replaced by 1 so that the
// kernel finishes).
__global__ void __launch_bounds__(256) k_potrf64(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                                                 double* __restrict__ Wd, unsigned* status) {
    __shared__ double a[FB][FB + 1];
    __shared__ double w[FB][FB + 1];
    __shared__ double inv_piv;
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < FB * FB; e += 256) {
        const int r = e / FB, c = e % FB;
        a[r][c] = (r < nb && c < nb && c <= r) ? Kmat[(j0 + r) * k + j0 + c] : (r == c ? 1.0 : 0.0);
        w[r][c] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            double p = a[j][j];
            if (!(p > 0.0) || !isfinite(p)) {
                bad = 1;
                p = 1.0;
            }
            const double dj = sqrt(p);
            a[j][j] = dj;
            inv_piv = 1.0 / dj;
        }
        __syncthreads();
        const double ip = inv_piv;
        for (int r = j + 1 + tid; r < nb; r += 256) a[r][j] *= ip;
        __syncthreads();
        const int rem = nb - j - 1;
        for (int e = tid; e < rem * rem; e += 256) {
            const int r = j + 1 + e / rem, c = j + 1 + e % rem;
            if (c <= r) a[r][c] = fma(-a[r][j], a[c][j], a[r][c]);
        }
        __syncthreads();
    }
    // W = L^{-1}: thread c solves column c by forward substitution.
    if (tid < nb) {
        const int c = tid;
        for (int r = c; r < nb; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int l = c; l < r; ++l) s = fma(-a[r][l], w[l][c], s);
            w[r][c] = s / a[r][r];
        }
    }
    __syncthreads();
    for (int e = tid; e < FB * FB; e += 256) {
        const int r = e / FB, c = e % FB;
        if (r < nb && c < nb && c <= r) Kmat[(j0 + r) * k + j0 + c] = a[r][c];
        Wd[e] = (r < nb && c < nb && c <= r) ? w[r][c] : 0.0;
    }
    if (tid == 0 && bad) atomicOr(status, IHS_DEV_NOTPD);
}

// Panel: rows i in [j0+nb, k): L[i][j0:j0+nb] = K[i][j0:j0+nb] W^T (64 rows per CTA).
__global__ void __launch_bounds__(256) k_panel64(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                                                 const double* __restrict__ Wd) {
    __shared__ double pr[FB][FB + 1];
    __shared__ double wt[FB][FB + 1];
    const int64_t r0 = j0 + nb + (int64_t)blockIdx.x * FB;
    for (int e = threadIdx.x; e < FB * FB; e += 256) {
        const int r = e / FB, c = e % FB;
        pr[r][c] = (r0 + r < k && c < nb) ? Kmat[(r0 + r) * k + j0 + c] : 0.0;
        wt[c][r] = Wd[e];   // wt[c][r] = W[r][c]
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int q = 0; q < nb; ++q) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = pr[ty + 16 * a][q];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = wt[q][tx + 16 * b];   // W[tx+16b][q]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t r = r0 + ty + 16 * a;
            const int c = tx + 16 * b;
            if (r < k && c < nb) Kmat[r * k + j0 + c] = acc[a][b];
        }
}

// Trailing update K[j1:, j1:] -= P P^T on lower 64x64 tiles, P = L[j1:, j0:j0+nb].
__global__ void __launch_bounds__(256) k_syrk64(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb) {
    __shared__ double pa[FB][FB + 1];
    __shared__ double pb[FB][FB + 1];
    const int64_t j1 = j0 + nb;
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < FB * FB; e += 256) {
        const int rr = e / FB, q = e % FB;
        const int64_t ra = j1 + I * FB + rr, rb = j1 + J * FB + rr;
        pa[rr][q] = (ra < k && q < nb) ? Kmat[ra * k + j0 + q] : 0.0;
        pb[rr][q] = (rb < k && q < nb) ? Kmat[rb * k + j0 + q] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int q = 0; q < nb; ++q) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = pa[ty + 16 * a][q];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = pb[tx + 16 * b][q];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t r = j1 + I * FB + ty + 16 * a, c = j1 + J * FB + tx + 16 * b;
            if (r < k && c <= r) Kmat[r * k + c] -= acc[a][b];
        }
}

// X (FP32, k x k, lower) <- diagonal blocks W of L^{-1} from k_potrf64; zero elsewhere.
__global__ void k_inv_init(const double* __restrict__ Wall, int64_t k, float* __restrict__ X) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int64_t r = idx / k, c = idx % k;
    float v = 0.f;
    if (r / FB == c / FB && c <= r) {
        const int64_t b = r / FB;
        v = (float)Wall[b * FB * FB + (r % FB) * FB + (c % FB)];
    }
    X[idx] = v;
}

// Batched FP32 GEMM for the recursive-doubling inverse: for pair p,
// C_p = alpha * A_p B_p, with A_p, B_p, C_p sub-blocks of row-major k x k
// matrices addressed by (row, col) offsets that depend on p:
//   A_p at (ra + p*pstride, ca + p*pstride), B_p at (rb + p*pstride, cb + p*pstride), ...
// Size s x s x s.  A is float (X) or double (L) by `a_is_l`.
__global__ void __launch_bounds__(256) k_pair_gemm(const float* __restrict__ Xf, const double* __restrict__ Ld,
                                                   int a_is_l, int64_t k, int64_t s, int64_t pstride,
                                                   int64_t ra, int64_t ca, int64_t rb, int64_t cb, const float* Bsrc,
                                                   float* __restrict__ C, int64_t rc, int64_t cc, float alpha) {
    __shared__ float as[32][FB + 4];
    __shared__ float bs[32][FB + 4];
    const int64_t pair = blockIdx.z;
    const int64_t off = pair * pstride;
    const int64_t tr = (int64_t)blockIdx.y * FB, tc = (int64_t)blockIdx.x * FB;   // tile within the s x s block
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int64_t q0 = 0; q0 < s; q0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * FB; e += 256) {
            const int rr = e / 32, qq = e % 32;
            const int64_t gr = ra + off + tr + rr, gq = ca + off + q0 + qq;
            float v = 0.f;
            if (tr + rr < s && q0 + qq < s && gr < k && gq < k)
                v = a_is_l ? (float)Ld[gr * k + gq] : Xf[gr * k + gq];
            as[qq][rr] = v;
            const int qq2 = e / FB, cc2 = e % FB;
            const int64_t br = rb + off + q0 + qq2, bc = cb + off + tc + cc2;
            bs[qq2][cc2] = (q0 + qq2 < s && tc + cc2 < s && br < k && bc < k) ? Bsrc[br * k + bc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = as[q][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = bs[q][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = __fmaf_rn(av[a], bv[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t r = tr + ty + 16 * a, c = tc + tx + 16 * b;
            const int64_t gr = rc + off + r, gc = cc + off + c;
            if (r < s && c < s && gr < k && gc < k) C[gr * k + gc] = alpha * acc[a][b];
        }
}

// XT = X^T for FP32 lower-triangular X.
__global__ void k_transpose_f32(const float* __restrict__ X, int64_t k, float* __restrict__ XT) {
    __shared__ float tile[32][33];
    const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = by + r, gc = bx + tx;
        tile[r][tx] = (gr < k && gc < k) ? X[gr * k + gc] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t gr = bx + r, gc = by + tx;
        if (gr < k && gc < k) XT[gr * k + gc] = tile[tx][r];
    }
}

// y = M v (FP32 matrix, FP64 vector and accumulation), rows restricted to the
// triangle: tri = 1 lower (l <= i), 2 upper (l >= i).  One warp per row.
__global__ void k_trmv32(const float* __restrict__ M, int64_t k, int tri, const double* __restrict__ v,
                         double* __restrict__ y) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= k) return;
    const int64_t lo = tri == 2 ? warp : 0, hi = tri == 1 ? warp + 1 : k;
    double s = 0.0;
    for (int64_t l = lo + lane; l < hi; l += 32) s = fma((double)M[warp * k + l], v[l], s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) y[warp] = s;
}

// y[j] = sum_l SA[j][l] v[l] (FP64 vector), one warp per row.
__global__ void k_sa_v64(const float* __restrict__ SA, int64_t rows, int64_t d, const double* __restrict__ v,
                         double* __restrict__ y) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= rows) return;
    double s = 0.0;
    for (int64_t l = lane; l < d; l += 32) s = fma((double)SA[warp * d + l], v[l], s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) y[warp] = s;
}

// out[c] = sum_chunks part[chunk][c] (fixed order)
__global__ void k_sum_chunks(const double* __restrict__ part, int chunks, int64_t d, double* __restrict__ out) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (int q = 0; q < chunks; ++q) s += part[q * d + c];
    out[c] = s;
}

// res = t - (alpha * u + w), elementwise FP64; also u1 bookkeeping done by caller.
__global__ void k_residual(const double* __restrict__ t, const double* __restrict__ u, double alpha,
                           const double* __restrict__ w, int64_t n, double* __restrict__ res) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) res[i] = t[i] - (alpha * u[i] + w[i]);
}

__global__ void k_axpy64(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

// gt = (g - w) * inv_nu2 (woodbury) or gt = u (direct) in FP64 -> FP32, and
// per-block partials of g . gt.
__global__ void k_apply_out(const float* __restrict__ g, const double* __restrict__ w, const double* __restrict__ u,
                            int64_t d, double inv_nu2, float* __restrict__ gt, double* __restrict__ rpart) {
    __shared__ double sm[256];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double prod = 0.0;
    if (c < d) {
        const double v = u ? u[c] : ((double)g[c] - w[c]) * inv_nu2;
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

}  // namespace

int ihs_factor_build(ihs_ctx* ctx, ihs_factor_t* F) {
    const int64_t k = F->k;
    cudaStream_t s = ctx->stream;
    const int64_t T = ceil_div64(k, FB);
    double* Kmat = F->L;
    double* Wall = F->W;
    const int64_t K = F->woodbury ? F->d : F->m;
    k_gram_c32<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(F->SA, F->d, F->woodbury, k, K, F->nu * F->nu, Kmat);
    IHS_LAUNCH_CHECK();
    for (int64_t jb = 0; jb < T; ++jb) {
        const int64_t j0 = jb * FB;
        const int nb = (int)std::min<int64_t>(FB, k - j0);
        k_potrf64<<<1, 256, 0, s>>>(Kmat, k, j0, nb, Wall + jb * FB * FB, ctx->d_status);
        IHS_LAUNCH_CHECK();
        const int64_t rest = k - j0 - nb;
        if (rest > 0) {
            k_panel64<<<(unsigned)ceil_div64(rest, FB), 256, 0, s>>>(Kmat, k, j0, nb, Wall + jb * FB * FB);
            IHS_LAUNCH_CHECK();
            const int64_t Tr = ceil_div64(rest, FB);
            k_syrk64<<<(unsigned)(Tr * (Tr + 1) / 2), 256, 0, s>>>(Kmat, k, j0, nb);
            IHS_LAUNCH_CHECK();
        }
    }
    // X = L^{-1} in FP32 by recursive doubling: diagonal blocks come from the
    // FP64 factorisation; for block size sz = 64, 128, ... the lower-left
    // block of each pair is X21 = -X22 (L21 X11).
    float* X = F->X;
    float* tmp = F->XT;   // scratch for L21 X11 (overwritten by X^T at the end)
    k_inv_init<<<(unsigned)ceil_div64(k * k, 256), 256, 0, s>>>(Wall, k, X);
    IHS_LAUNCH_CHECK();
    for (int64_t sz = FB; sz < k; sz *= 2) {
        const int64_t pairs = ceil_div64(k, 2 * sz);
        const int64_t tiles = ceil_div64(sz, FB);
        dim3 grid((unsigned)tiles, (unsigned)tiles, (unsigned)pairs);
        // tmp21 = L21 X11   (L21 at rows [sz, 2sz), cols [0, sz) of the pair)
        k_pair_gemm<<<grid, 256, 0, s>>>(X, F->L, 1, k, sz, 2 * sz, sz, 0, 0, 0, X, tmp, sz, 0, 1.0f);
        IHS_LAUNCH_CHECK();
        // X21 = -X22 tmp21
        k_pair_gemm<<<grid, 256, 0, s>>>(X, nullptr, 0, k, sz, 2 * sz, sz, sz, sz, 0, tmp, X, sz, 0, -1.0f);
        IHS_LAUNCH_CHECK();
    }
    dim3 tg((unsigned)ceil_div64(k, 32), (unsigned)ceil_div64(k, 32));
    k_transpose_f32<<<tg, 256, 0, s>>>(X, k, F->XT);
    IHS_LAUNCH_CHECK();
    return ihs_check_status(ctx);
}

// H_S^{-1} g with one step of iterative refinement: the FP32 inverse factor X
// gives u0 = X^T X t; the residual t - K u0 uses the exact operator
// (K u = nu^2 u + SA (SA^T u), or SA^T (SA u) + nu^2 u) in FP64 accumulation.
int ihs_apply_enqueue(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* d_r) {
    cudaStream_t s = ctx->stream;
    const int64_t k = F->k, d = F->d, m = F->m;
    double* t = F->work;       // k
    double* v = t + k;         // k
    double* u = v + k;         // k (u0, then u1)
    double* res = u + k;       // k
    double* w = res + k;       // max(m, d)
    double* w2 = w + std::max(m, d);   // max(m, d)
    double* rpart = w2 + std::max(m, d);   // 4096
    double* part = rpart + 4096;            // 32 x d
    const unsigned kb = (unsigned)ceil_div64(k * 32, 256);
    const unsigned db = (unsigned)ceil_div64(d, 256);
    const unsigned mb = (unsigned)ceil_div64(m * 32, 256);
    const int64_t chunks = std::min<int64_t>(32, std::max<int64_t>(1, m / 32));
    const int64_t rpc = ceil_div64(m, chunks);
    const int64_t nch = ceil_div64(m, rpc);
    auto sat = [&](const double* uu, double* out) -> int {   // out = SA^T uu (d)
        dim3 grid(db, (unsigned)nch);
        k_sat_u<<<grid, 256, 0, s>>>(F->SA, m, d, uu, rpc, part);
        IHS_LAUNCH_CHECK();
        k_sum_chunks<<<db, 256, 0, s>>>(part, (int)nch, d, out);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    auto minv = [&](const double* in, double* out) -> int {   // out = X^T X in
        k_trmv32<<<kb, 256, 0, s>>>(F->X, k, 1, in, v);
        IHS_LAUNCH_CHECK();
        k_trmv32<<<kb, 256, 0, s>>>(F->XT, k, 2, v, out);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    const unsigned kvb = (unsigned)ceil_div64(k, 256);
    if (F->woodbury) {
        k_sa_g<<<(unsigned)ceil_div64(m * 32, 256), 256, 0, s>>>(F->SA, m, d, g, t);
        IHS_LAUNCH_CHECK();
    } else {
        k_to_double<<<db, 256, 0, s>>>(g, d, t);
        IHS_LAUNCH_CHECK();
    }
    IHS_TRY(minv(t, u));
    // K u0
    if (F->woodbury) {
        IHS_TRY(sat(u, w));                                        // w = SA^T u0 (d)
        k_sa_v64<<<mb, 256, 0, s>>>(F->SA, m, d, w, w2);             // w2 = SA w (m)
        IHS_LAUNCH_CHECK();
    } else {
        k_sa_v64<<<mb, 256, 0, s>>>(F->SA, m, d, u, w);              // w = SA u0 (m)
        IHS_LAUNCH_CHECK();
        IHS_TRY(sat(w, w2));                                       // w2 = SA^T w (d)
    }
    k_residual<<<kvb, 256, 0, s>>>(t, u, F->nu * F->nu, w2, k, res);
    IHS_LAUNCH_CHECK();
    IHS_TRY(minv(res, w2));
    k_axpy64<<<kvb, 256, 0, s>>>(u, w2, k);                         // u1 = u0 + X^T X res
    IHS_LAUNCH_CHECK();
    if (F->woodbury) {
        IHS_TRY(sat(u, w));                                        // w = SA^T u1
        k_apply_out<<<db, 256, 0, s>>>(g, w, nullptr, d, 1.0 / (F->nu * F->nu), gt, rpart);
    } else {
        k_apply_out<<<db, 256, 0, s>>>(g, nullptr, u, d, 0.0, gt, rpart);
    }
    IHS_LAUNCH_CHECK();
    if (d_r) {
        k_sum_half<<<1, 1, 0, s>>>(rpart, (int)db, d_r);
        IHS_LAUNCH_CHECK();
    }
    return IHS_OK;
}

static size_t factor_work_doubles(int64_t k, int64_t m, int64_t d) {
    return 4 * (size_t)k + 2 * (size_t)std::max(m, d) + 4096 + 32 * (size_t)d + 64;
}

extern "C" int ihs_factor(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** out) {
    if (!ctx || !SA || !out || m < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    *out = nullptr;
    ihs_factor_t* F = new (std::nothrow) ihs_factor_t;
    if (!F) return IHS_ENOMEM;
    memset(F, 0, sizeof(*F));
    F->ctx = ctx;
    F->SA = SA;
    F->m = m;
    F->d = d;
    F->nu = nu;
    F->woodbury = m < d ? 1 : 0;
    F->k = F->woodbury ? m : d;
    const int64_t k = F->k;
    const int64_t T = ceil_div64(k, FB);
    const size_t kk = (size_t)k * k;
    if (cudaMalloc(&F->L, kk * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F->W, (size_t)T * FB * FB * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F->X, kk * sizeof(float)) != cudaSuccess || cudaMalloc(&F->XT, kk * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&F->work, factor_work_doubles(k, m, d) * sizeof(double)) != cudaSuccess) {
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
    if (F->W) cudaFree(F->W);
    if (F->X) cudaFree(F->X);
    if (F->XT) cudaFree(F->XT);
    if (F->work) cudaFree(F->work);
    delete F;
    return IHS_OK;
}

extern "C" int ihs_apply_hinv(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* r_h) {
    if (!ctx || !F || !g || !gt) return IHS_EINVAL;
    double* d_r = F->work + factor_work_doubles(F->k, F->m, F->d) - 8;
    IHS_TRY(ihs_apply_enqueue(ctx, F, g, gt, d_r));
    if (r_h) {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, d_r, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *r_h = ctx->pinned[0];
    }
    return IHS_OK;
}
