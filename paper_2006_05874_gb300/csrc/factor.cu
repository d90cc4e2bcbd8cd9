// Factor and apply of the sketched Hessian H_S = (SA)^T SA + nu^2 I (Eq. 3).
//
// m < d : Woodbury form (App. B.4)
//         H_S^{-1} g = nu^-2 (g - (SA)^T K^{-1} SA g),  K = nu^2 I_m + SA (SA)^T,
// m >= d: K = H_S itself (d x d) and H_S^{-1} g = K^{-1} g.
// K is formed from the FP32 sketch with compensated FP32 accumulation and
// stored in FP64; K = L L^T by a blocked, right-looking FP64 Cholesky with one
// step of look-ahead (64-wide blocks; an rsqrt per pivot, a row-parallel
// substitution for the panel, FP64 SYRK tiles for the trailing update;
// non-positive or non-finite pivots set IHS_DEV_NOTPD).  X = L^{-1} is formed
// once in FP32 by recursive doubling ([L11 0; L21 L22]^{-1} has lower-left
// block -X22 L21 X11), so every apply is a chain of parallel matrix-vector
// products, followed by one step of iterative refinement against the exact
// operator, with double-float (binary32 pair) vectors and dot products:
//   u0 = X^T X t, u1 = u0 + X^T X (t - K u0)
// with t = SA g, gt = nu^-2 (g - SA^T u1) (Woodbury) or t = g, gt = u1
// (direct); r = 1/2 g^T gt (Lemma 4.1) in FP64.
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"

namespace {

__global__ void k_sum_half(const double* __restrict__ rpart, int count, double* __restrict__ r) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += rpart[i];
    *r = 0.5 * s;
}

constexpr int FB = 64;   // block size of the FP64 Cholesky and of the inverse

// K = X X^T + nu^2 I on lower 64x64 tiles from the FP32 sketch with
// compensated FP32 accumulation: FMA chains over 4 terms, each chain added to
// a (hi, lo) pair by TwoSum; K stored in FP64.  X(r, k) = SA[r][k] (Woodbury)
// or SA[k][r] (direct).
// Split-K: blockIdx.y takes rows [y * kchunk, (y + 1) * kchunk) of the inner
// dimension; with gridDim.y > 1 the (hi, lo) pairs go to `part` (one 64 x 64
// tile of float2 per (split, tile)) for k_gram_reduce, else straight to G.
// Thread (ty, tx) holds rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3 of the
// tile as packed FP32x2 pairs of adjacent columns, so that every multiply,
// FMA and TwoSum step does two entries' work in one instruction (the same
// operations per entry as the scalar form, hence the same K bit for bit).
// The inner dimension goes in chunks of 32 rows through two shared-memory
// buffers, the next chunk loaded into registers while the current one is
// used.
__global__ void __launch_bounds__(256, 2) k_gram_c32(const float* __restrict__ SA, int64_t d, int woodbury,
                                                  int64_t kdim, int64_t K, int64_t kchunk, double nu2,
                                                  float2 nu2df, int out_df, double* __restrict__ G,
                                                  float2* __restrict__ part) {
    __shared__ __align__(16) float xa[2][32][FB + 4];
    __shared__ __align__(16) float xb[2][32][FB + 4];
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    // staging: 8 entries of each operand per thread and chunk
    float la[8], lb[8];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + 256 * i;
            int rr, kk;
            if (woodbury) {
                rr = e / 32;
                kk = e % 32;
            } else {
                kk = e / FB;
                rr = e % FB;
            }
            const int64_t ra = I * FB + rr, rb = J * FB + rr, kq = k0 + kk;
            const bool kin = kq < kend;
            la[i] = (ra < kdim && kin) ? (woodbury ? SA[ra * d + kq] : SA[kq * d + ra]) : 0.f;
            lb[i] = (rb < kdim && kin) ? (woodbury ? SA[rb * d + kq] : SA[kq * d + rb]) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + 256 * i;
            const int rr = woodbury ? e / 32 : e % FB, kk = woodbury ? e % 32 : e / FB;
            xa[buf][kk][rr] = la[i];
            xb[buf][kk][rr] = lb[i];
        }
    };
    f2 hi[4][2], lo[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int p = 0; p < 2; ++p) hi[a][p].v = lo[a][p].v = 0ull;
    int buf = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    for (int64_t k0 = kbeg; k0 < kend; k0 += 32) {
        const bool more = k0 + 32 < kend;
        if (more) load(k0 + 32);
#pragma unroll
        for (int kc = 0; kc < 32; kc += 4) {
            f2 c4[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 a4 = *reinterpret_cast<const float4*>(&xa[buf][kc + q][ty * 4]);
                const float4 b4 = *reinterpret_cast<const float4*>(&xb[buf][kc + q][tx * 4]);
                const f2 b01 = f2_pack(b4.x, b4.y), b23 = f2_pack(b4.z, b4.w);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const f2 aa = f2_pack(av[a], av[a]);
                    if (q == 0) {
                        c4[a][0] = f2_mul(aa, b01);
                        c4[a][1] = f2_mul(aa, b23);
                    } else {
                        c4[a][0] = f2_fma(aa, b01, c4[a][0]);
                        c4[a][1] = f2_fma(aa, b23, c4[a][1]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    Acc2x2 acc{hi[a][p], lo[a][p]};
                    acc.add(c4[a][p]);
                    hi[a][p] = acc.hi;
                    lo[a][p] = acc.lo;
                }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    // entry (a, b) of this thread: row 4 ty + a, column 4 tx + b
    auto entry = [&](int a, int b, float& h, float& l) {
        float h0, h1, l0, l1;
        f2_unpack(hi[a][b >> 1], h0, h1);
        f2_unpack(lo[a][b >> 1], l0, l1);
        h = (b & 1) ? h1 : h0;
        l = (b & 1) ? l1 : l0;
    };
    if (gridDim.y > 1) {
        float2* pt = part + ((size_t)blockIdx.y * gridDim.x + t) * FB * FB;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float h, l;
                entry(a, b, h, l);
                pt[(ty * 4 + a) * FB + tx * 4 + b] = make_float2(h, l);
            }
        return;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t r = I * FB + ty * 4 + a, c = J * FB + tx * 4 + b;
            if (r < kdim && c < kdim && c <= r) {
                float h, l;
                entry(a, b, h, l);
                if (out_df) {   // double-float pairs, the FP32 pipes only
                    float s, e;
                    two_sum(h, l, s, e);
                    float2 v = make_float2(s, e);
                    if (r == c) {
                        float s2, e2;
                        two_sum(v.x, nu2df.x, s2, e2);
                        const float l2 = __fadd_rn(e2, __fadd_rn(v.y, nu2df.y));
                        const float s3 = __fadd_rn(s2, l2);
                        v = make_float2(s3, __fsub_rn(l2, __fsub_rn(s3, s2)));
                    }
                    reinterpret_cast<float2*>(G)[r * kdim + c] = v;
                } else {
                    G[r * kdim + c] = (double)h + (double)l + (r == c ? nu2 : 0.0);
                }
            }
        }
}

// G tile t = sum over the KS splits of hi + lo, + nu^2 I: the pairs summed in
// a fixed order as a compensated binary32 pair (FP64 runs at a small fraction
// of the FP32 rate), then stored as a normalised pair (out_df) or widened to
// FP64.  Grid (tiles, FB * FB / 256): one entry per thread, its KS loads in
// batches of eight ahead of the dependent additions.
__global__ void __launch_bounds__(256) k_gram_reduce(const float2* __restrict__ part, int KS, int64_t ntiles,
                                                     int64_t kdim, float2 nu2df, int out_df, double* __restrict__ G) {
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;
    const int e = blockIdx.y * 256 + threadIdx.x;
    const int rr = e / FB, cc = e % FB;
    const int64_t r = I * FB + rr, c = J * FB + cc;
    if (r >= kdim || c >= kdim || c > r) return;
    Acc2 acc{0.f, 0.f};
    for (int y0 = 0; y0 < KS; y0 += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (y0 + u < KS) v[u] = part[((size_t)(y0 + u) * ntiles + t) * FB * FB + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (y0 + u >= KS) break;
            acc.add_pair(v[u].x, v[u].y);
        }
    }
    if (r == c) acc.add_pair(nu2df.x, nu2df.y);
    if (out_df) {
        const float hi = __fadd_rn(acc.hi, acc.lo);
        reinterpret_cast<float2*>(G)[r * kdim + c] = make_float2(hi, __fsub_rn(acc.lo, __fsub_rn(hi, acc.hi)));
    } else {
        G[r * kdim + c] = (double)acc.hi + (double)acc.lo;
    }
}

// The FP64 Cholesky runs on CB x CB blocks (CB = 32): with FP64 at a small
// fraction of the FP32 rate, the diagonal-block factorisation on one SM sits
// on the critical path, and its cost grows as CB^3 per block step.
constexpr int CB = 32;

// Diagonal block [j0, j0+nb) of the FP64 Cholesky, in place, and (WANT_W) its
// inverse W = L_jj^{-1} (CB x CB, lower, at Wd) for the panel; one CTA of 256
// threads.
// The pivots form a dependent chain of CB reciprocal square roots (a long
// FP64 latency each), so thread 0 runs that chain alone: at step j it applies
// column j to the next pivot itself, p_{j+1} = a_{j+1,j+1} - (a_{j+1,j} / sqrt(p_j))^2,
// and starts its rsqrt at once, while warps 1..7 apply column j to the rest
// of the trailing triangle (entries packed by descending column, so that the
// warps with no entries left skip the step).  Columns stay unscaled (a_rc with
// the pivot p_c on the diagonal) until one final pass forms L_rc = a_rc / sqrt(p_c).
// With WANT_W, W = L^{-1} follows by forward substitution row by row, one
// trailing entry per thread per row; without it the reciprocal diagonal
// 1 / L_cc goes to Wd[0..CB) for a panel formed by substitution.  Rows and columns >= nb are padded with the identity.
// Non-positive or non-finite pivots set IHS_DEV_NOTPD (the pivot is replaced
// by 1 so that the kernel finishes).
struct CholSmem {
    double a[CB][CB + 1];
    double w[CB][CB + 1];
    double dinv[CB];
    int bad;
};

template <bool WANT_W>
__device__ void chol_potrf(CholSmem& S, double* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                           double* __restrict__ Wd, unsigned* status) {
    static_assert(CB == 32, "the packed entry mapping assumes CB = 32 and 256 threads");
    const int tid = threadIdx.x;
    if (tid == 0) S.bad = 0;
    for (int e = tid; e < CB * CB; e += 256) {
        const int r = e / CB, c = e % CB;
        double v = 0.0;
        if (c <= r) v = (r < nb) ? (c < nb ? __ldcg(Kmat + (j0 + r) * k + j0 + c) : 0.0) : (r == c ? 1.0 : 0.0);
        S.a[r][c] = v;
        S.w[r][c] = 0.0;
    }
    // this thread's trailing entries (bulk threads 32..255): lower-triangle
    // entries ordered by descending column, e -> group g = 31 - c of g + 1 rows
    int er[3], ec[3], ei[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = tid - 32 + 224 * q;
        ei[q] = e;
        int g = 0;
        if (e >= 0 && e < CB * (CB + 1) / 2) {
            g = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
            while (g * (g + 1) / 2 > e) --g;
            while ((g + 1) * (g + 2) / 2 <= e) ++g;
        } else {
            ei[q] = 1 << 20;   // never active
        }
        ec[q] = CB - 1 - g;
        er[q] = ec[q] + (e - g * (g + 1) / 2);
    }
    __syncthreads();
    double ri = 0.0;   // thread 0: 1 / sqrt(p_j) of the current step
    if (tid == 0) {
        double p = S.a[0][0];
        if (!(p > 0.0) || !isfinite(p)) {
            S.bad = 1;
            p = 1.0;
            S.a[0][0] = p;
        }
        ri = rsqrt(p);
        S.dinv[0] = ri;
    }
    __syncthreads();
    for (int j = 0; j < CB - 1; ++j) {
        if (tid == 0) {
            const double l = S.a[j + 1][j] * ri;
            double p = fma(-l, l, S.a[j + 1][j + 1]);
            if (!(p > 0.0) || !isfinite(p)) {
                S.bad = 1;
                p = 1.0;
            }
            S.a[j + 1][j + 1] = p;
            ri = rsqrt(p);
            S.dinv[j + 1] = ri;
        } else if (tid >= 32) {
            // entries with column > j lead the order: e < (31 - j)(32 - j) / 2
            const int active = (CB - 1 - j) * (CB - j) / 2;
            const int diag_next = (CB - 2 - j) * (CB - 1 - j) / 2;   // entry (j+1, j+1): thread 0's
            if (tid - 32 < active) {
                const double rj = S.dinv[j];
                const double ip2 = rj * rj;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (ei[q] < active && ei[q] != diag_next) {
                        const int r = er[q], c = ec[q];
                        S.a[r][c] = fma(-S.a[r][j] * ip2, S.a[c][j], S.a[r][c]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // L_rc = a_rc / sqrt(p_c) (on the diagonal p_c / sqrt(p_c))
    for (int e = tid; e < CB * CB; e += 256) {
        const int r = e / CB, c = e % CB;
        if (c <= r) S.a[r][c] *= S.dinv[c];
    }
    if (WANT_W) {
        if (tid == 0) S.w[0][0] = S.dinv[0];
        __syncthreads();
        // W = L^{-1}: after step l, row l + 1 is final
        for (int l = 0; l < CB - 1; ++l) {
            const int width = l + 1;
            if (tid < (CB - 1 - l) * width) {
                const int r = l + 1 + tid / width, c = tid % width;
                double v = fma(-S.a[r][l], S.w[l][c], S.w[r][c]);
                if (r == l + 1) v *= S.dinv[l + 1];
                S.w[r][c] = v;
            }
            if (tid == 0) S.w[l + 1][l + 1] = S.dinv[l + 1];
            __syncthreads();
        }
    } else {
        __syncthreads();
    }
    for (int e = tid; e < CB * CB; e += 256) {
        const int r = e / CB, c = e % CB;
        if (r < nb && c < nb && c <= r) Kmat[(j0 + r) * k + j0 + c] = S.a[r][c];
        if (WANT_W) Wd[e] = (r < nb && c < nb && c <= r) ? S.w[r][c] : 0.0;
    }
    if (!WANT_W && tid < CB) Wd[tid] = tid < nb ? S.dinv[tid] : 0.0;   // 1 / L_cc
    if (tid == 0 && S.bad) atomicOr(status, IHS_DEV_NOTPD);
}

__global__ void __launch_bounds__(256) k_potrf32(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                                                 double* __restrict__ Wd, unsigned* status) {
    __shared__ CholSmem S;
    chol_potrf<true>(S, Kmat, k, j0, nb, Wd, status);
}

// Panel: rows i in [j0+nb, k): L[i][j0:j0+nb] = K[i][j0:j0+nb] W^T with
// W = L_jj^{-1} (8 rows per CTA, thread = one entry).
constexpr int kPanelRows = 8;
__global__ void __launch_bounds__(256) k_panel32(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                                                 const double* __restrict__ Wd) {
    __shared__ double pr[kPanelRows][CB + 1];
    __shared__ double wt[CB][CB + 1];
    const int64_t r0 = j0 + nb + (int64_t)blockIdx.x * kPanelRows;
    for (int e = threadIdx.x; e < CB * CB; e += 256) wt[e % CB][e / CB] = Wd[e];   // wt[c][r] = W[r][c]
    {
        const int r = threadIdx.x / CB, c = threadIdx.x % CB;
        pr[r][c] = (r0 + r < k && c < nb) ? Kmat[(r0 + r) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % CB, ty = threadIdx.x / CB;
    double acc = 0.0;
    for (int q = 0; q < nb; ++q) acc = fma(pr[ty][q], wt[q][tx], acc);   // W[tx][q]
    const int64_t r = r0 + ty;
    if (r < k && tx < nb) Kmat[r * k + j0 + tx] = acc;
}

// Look-ahead pieces of the trailing update after block step j0 (panel P =
// L[j1:, j0:j0+nb], j1 = j0 + nb):
//  * k_syrk_next: the next block column, K[i][j1 : j1+CB] -= P_i P_{j1..}^T for
//    i >= j1 (lower part), 8 rows per CTA (short tiles keep the critical path
//    of the factorisation short);
//  * k_syrk_rest: every lower CB x CB tile of the trailing matrix from tile
//    column 1 on (a 1-D grid over the lower tiles).
__global__ void __launch_bounds__(256) k_syrk_next(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb) {
    __shared__ double pr[8][CB + 1];
    __shared__ double pc[CB][CB + 1];
    const int64_t j1 = j0 + nb;
    const int64_t r0 = j1 + (int64_t)blockIdx.x * 8;
    const int ncol = (int)min((int64_t)CB, k - j1);
    for (int e = threadIdx.x; e < CB * CB; e += 256) {
        const int c = e / CB, q = e % CB;
        pc[c][q] = (c < ncol && q < nb) ? Kmat[(j1 + c) * k + j0 + q] : 0.0;
    }
    {
        const int r = threadIdx.x / CB, q = threadIdx.x % CB;
        pr[r][q] = (r0 + r < k && q < nb) ? Kmat[(r0 + r) * k + j0 + q] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % CB, ty = threadIdx.x / CB;
    double acc = 0.0;
    for (int q = 0; q < nb; ++q) acc = fma(pr[ty][q], pc[tx][q], acc);
    const int64_t r = r0 + ty, c = j1 + tx;
    if (r < k && tx < ncol && c <= r) Kmat[r * k + c] -= acc;
}

__global__ void __launch_bounds__(256) k_syrk_rest(double* __restrict__ Kmat, int64_t k, int64_t j0, int nb) {
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int64_t J = t - I * (I + 1) / 2;   // trailing tile (I, J), J <= I
    if (J < 1) return;
    __shared__ double pa[CB][CB + 1];
    __shared__ double pb[CB][CB + 1];
    const int64_t j1 = j0 + nb;
    for (int e = threadIdx.x; e < CB * CB; e += 256) {
        const int rr = e / CB, q = e % CB;
        const int64_t ra = j1 + I * CB + rr, rb = j1 + J * CB + rr;
        pa[rr][q] = (ra < k && q < nb) ? Kmat[ra * k + j0 + q] : 0.0;
        pb[rr][q] = (rb < k && q < nb) ? Kmat[rb * k + j0 + q] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[2][2] = {};
    for (int q = 0; q < nb; ++q) {
        const double a0 = pa[ty][q], a1 = pa[ty + 16][q];
        const double b0 = pb[tx][q], b1 = pb[tx + 16][q];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t r = j1 + I * CB + ty + 16 * a, c = j1 + J * CB + tx + 16 * b;
            if (r < k && c <= r) Kmat[r * k + c] -= acc[a][b];
        }
}

// ---------------------------------------------------------------------------
// The same blocked Cholesky as one cooperative (persistent) launch: every CTA
// stays resident and the block steps are separated by grid barriers instead
// of kernel boundaries and stream events.  Step j:
//   phase P: CTA 0 factors diagonal block j (and its inverse W_j) while the
//            other CTAs apply panel j-1 to the trailing tiles of column
//            blocks >= j+1 (the look-ahead overlap of the stream version);
//   phase N: all CTAs form panel j (rows below block j) = K W_j^T;
//   phase S: all CTAs update column block j+1 with panel j, once the two CTAs
//            that formed its first 32 rows (which every row's update reads)
//            have published them on a counter: no grid barrier between N and S.
// Matrix reads go through L2 (__ldcg): other SMs wrote them since the last
// barrier.  Every barrier wait is bounded; a wait that gives up sets
// IHS_DEV_TIMEOUT and the CTAs leave.

// Grid barrier over gridDim.x CTAs on a monotonic arrival counter (zeroed
// before the launch): barrier number t (1, 2, ...) is passed when the counter
// reaches t * gridDim.x.  Arrival is a release reduction after the CTA's
// writes, the wait an acquire load; a wait that exceeds one second sets
// IHS_DEV_TIMEOUT and returns false.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync_bounded(unsigned* cnt, unsigned& nbar, unsigned* status,
                                                  unsigned extra, uint64_t limit_ns) {
    __shared__ int gs_ok;
    __syncthreads();
    ++nbar;
    if (threadIdx.x == 0) {
        gs_ok = 1;
        const unsigned target = nbar * gridDim.x + extra;
        __threadfence();   // the whole CTA's writes (ordered by the barrier above) before the arrival
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
        if (ld_acquire_gpu(cnt) < target) {
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_gpu(cnt) < target) {
                if (global_timer_ns() - t0 > limit_ns) {
                    atomicOr(status, IHS_DEV_TIMEOUT);
                    gs_ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return gs_ok != 0;
}

// Wait (bounded, like grid_sync_bounded) until the counter at `flag` reaches
// `target`: the CTAs that published what this CTA reads next have arrived.
__device__ __forceinline__ bool flag_wait_bounded(const unsigned* flag, unsigned target, unsigned* status,
                                                  uint64_t limit_ns) {
    __shared__ int fw_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        fw_ok = 1;
        if (ld_acquire_gpu(flag) < target) {
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_gpu(flag) < target) {
                if (global_timer_ns() - t0 > limit_ns) {
                    atomicOr(status, IHS_DEV_TIMEOUT);
                    fw_ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return fw_ok != 0;
}

// acc += (a.x + a.y)(b.x + b.y) for double-float operands (pairs of binary32
// whose sum carries about 48 bits): the high product exactly (TwoProduct), the
// cross terms rounded once, a.y b.y dropped (2^-48 relative), the sum
// compensated (TwoSum).  Thirteen FP32 operations in place of one FP64 FMA,
// whose rate on this part is 1/64 of FP32.
__device__ __forceinline__ void df_fma_acc(Acc2& acc, float2 a, float2 b) {
    float p, e, s, es;
    two_prod(a.x, b.x, p, e);
    const float cross = __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x));
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fadd_rn(e, cross), es));
}

// x y for double-float operands, renormalised: about 2^-47 relative
__device__ __forceinline__ float2 df_mul2(float2 x, float2 y) {
    float p, e;
    two_prod(x.x, y.x, p, e);
    e = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
    const float s = __fadd_rn(p, e);
    return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

// k - x y for double-float operands
__device__ __forceinline__ float2 df_fnms(float2 k, float2 x, float2 y) {
    const float2 q = df_mul2(x, y);
    float s, e;
    two_sum(k.x, -q.x, s, e);
    e = __fadd_rn(e, __fsub_rn(k.y, q.y));
    const float t = __fadd_rn(s, e);
    return make_float2(t, __fsub_rn(e, __fsub_rn(t, s)));
}

// Sums of double-float pairs (binary32 hi + lo): the result renormalised.
__device__ __forceinline__ float2 pair_norm(float hi, float lo) {   // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return pair_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 pair_sub(float2 a, float2 b) { return pair_add(a, make_float2(-b.x, -b.y)); }

// Lower-triangle tile (I, J), J <= I, of linear index t = I (I + 1) / 2 + J
// (binary32 square root, corrected exactly in integers).
__device__ __forceinline__ void tri_tile(int64_t t, int64_t& I, int64_t& J) {
    I = (int64_t)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    J = t - I * (I + 1) / 2;
}

// 1 / sqrt(p) for a positive double-float p: the single-precision estimate
// rsqrtf(p.hi) refined by one Newton-Raphson step for f(y) = 1/y^2 - p,
// y <- y + y (1 - p y^2) / 2, with the residual 1 - p y^2 formed in
// double-float (the step squares the estimate's relative error, about 2^-22,
// to about 2^-44 plus the rounding of the pair arithmetic).
__device__ __forceinline__ float2 df_rsqrt(float2 p) {
    float2 y = make_float2(rsqrtf(p.x), 0.f);
#pragma unroll
    for (int it = 0; it < 1; ++it) {
        const float2 q = df_mul2(p, df_mul2(y, y));   // p y^2, close to 1
        float s, e;
        two_sum(1.0f, -q.x, s, e);
        const float r = __fadd_rn(s, __fsub_rn(e, q.y));   // 1 - p y^2 (small)
        const float h = __fmul_rn(__fmul_rn(0.5f, y.x), r);
        float hi, lo;
        two_sum(y.x, h, hi, lo);
        y = make_float2(hi, __fadd_rn(lo, __fadd_rn(y.y, __fmul_rn(__fmul_rn(0.5f, y.y), r))));
    }
    return y;
}

// The diagonal block [j0, j0 + nb) of the persistent Cholesky, in place, in
// double-float arithmetic on the FP32 pipes (about 2^-46 relative; the FP64
// pipe runs at a small fraction of the FP32 rate and a dependent FP64
// reciprocal square root costs hundreds of nanoseconds, which the 32-pivot
// chain would pay 32 times per block step).  Same schedule as chol_potrf:
// thread 0 runs the pivot chain with one column of look-ahead while threads
// 32..255 apply column j to the packed trailing entries; columns stay
// unscaled until a final pass forms L_rc = a_rc / sqrt(p_c).  L goes back to
// Kmat as double-float pairs, 1 / L_cc to Wd[0..CB) in FP64.  Rows and columns >= nb are padded with
// the identity; a non-positive or non-finite pivot sets IHS_DEV_NOTPD (and is
// replaced by 1).
struct CholSmemDf {
    float2 a[CB][CB + 1];
    float2 dinv[CB];
    int bad;
};

__device__ void chol_potrf_df(CholSmemDf& S, float2* __restrict__ Kmat, int64_t k, int64_t j0, int nb,
                              double* __restrict__ Wd, unsigned* status) {
    static_assert(CB == 32, "the packed entry mapping assumes CB = 32 and 256 threads");
    const int tid = threadIdx.x;
    if (tid == 0) S.bad = 0;
    for (int e = tid; e < CB * CB; e += 256) {
        const int r = e / CB, c = e % CB;
        float2 v = make_float2(0.f, 0.f);
        if (c <= r) {
            if (r < nb) v = c < nb ? __ldcg(Kmat + (j0 + r) * k + j0 + c) : make_float2(0.f, 0.f);
            else v = make_float2(r == c ? 1.f : 0.f, 0.f);
        }
        S.a[r][c] = v;
    }
    int er[3], ec[3], ei[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = tid - 32 + 224 * q;
        ei[q] = e;
        int g = 0;
        if (e >= 0 && e < CB * (CB + 1) / 2) {
            g = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
            while (g * (g + 1) / 2 > e) --g;
            while ((g + 1) * (g + 2) / 2 <= e) ++g;
        } else {
            ei[q] = 1 << 20;   // never active
        }
        ec[q] = CB - 1 - g;
        er[q] = ec[q] + (e - g * (g + 1) / 2);
    }
    __syncthreads();
    float2 ri = make_float2(0.f, 0.f);   // thread 0: 1 / sqrt(p_j) of the current step
    if (tid == 0) {
        float2 p = S.a[0][0];
        if (!(p.x > 0.f) || !isfinite(p.x)) {
            S.bad = 1;
            p = make_float2(1.f, 0.f);
            S.a[0][0] = p;
        }
        ri = df_rsqrt(p);
        S.dinv[0] = ri;
    }
    __syncthreads();
    for (int j = 0; j < CB - 1; ++j) {
        if (tid == 0) {
            const float2 l = df_mul2(S.a[j + 1][j], ri);
            float2 p = df_fnms(S.a[j + 1][j + 1], l, l);
            if (!(p.x > 0.f) || !isfinite(p.x)) {
                S.bad = 1;
                p = make_float2(1.f, 0.f);
            }
            S.a[j + 1][j + 1] = p;
            ri = df_rsqrt(p);
            S.dinv[j + 1] = ri;
        } else if (tid >= 32) {
            const int active = (CB - 1 - j) * (CB - j) / 2;
            const int diag_next = (CB - 2 - j) * (CB - 1 - j) / 2;   // entry (j+1, j+1): thread 0's
            if (tid - 32 < active) {
                const float2 rj = S.dinv[j];
                const float2 ip2 = df_mul2(rj, rj);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (ei[q] < active && ei[q] != diag_next) {
                        const int r = er[q], c = ec[q];
                        S.a[r][c] = df_fnms(S.a[r][c], df_mul2(S.a[r][j], ip2), S.a[c][j]);
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < CB * CB; e += 256) {
        const int r = e / CB, c = e % CB;
        if (c <= r && r < nb && c < nb) Kmat[(j0 + r) * k + j0 + c] = df_mul2(S.a[r][c], S.dinv[c]);
    }
    if (tid < CB) Wd[tid] = tid < nb ? (double)S.dinv[tid].x + (double)S.dinv[tid].y : 0.0;   // 1 / L_cc
    if (tid == 0 && S.bad) atomicOr(status, IHS_DEV_NOTPD);
}

__global__ void __launch_bounds__(256) k_chol_persistent(float2* __restrict__ Kmat, int64_t k,
                                                         double* __restrict__ Wall, unsigned* bar,
                                                         unsigned* status, unsigned bar_extra,
                                                         uint64_t bar_limit_ns) {
    __shared__ CholSmemDf S;
    // operands of the panel, column and trailing products as double-float pairs
    __shared__ float2 fa[CB][CB + 1];
    __shared__ float2 fb[CB][CB + 1];
    const int tid = threadIdx.x;
    const int G = gridDim.x, cta = blockIdx.x;
    const int64_t T = ceil_div64(k, CB);
    // Wall: 1 / L_cc of every block step (T x CB), then the current panel as
    // double-float pairs, row r at Pdf + r * CB (written once per element in
    // phase N, read by phase S and by the next step's trailing tiles)
    float2* Pdf = reinterpret_cast<float2*>(Wall + T * CB);
    unsigned nbar = 0;   // grid barriers passed
    unsigned panel_target = 0;   // arrivals due so far on the panel counter (bar + 1)
    for (int64_t jb = 0; jb < T; ++jb) {
        const int64_t j0 = jb * CB;
        const int nb = (int)min((int64_t)CB, k - j0);
        // ---- phase P: diagonal block jb | rest of the update by panel jb-1
        if (cta == 0) chol_potrf_df(S, Kmat, k, j0, nb, Wall + jb * CB, status);
        if (jb > 0 && (cta > 0 || G == 1)) {
            const int64_t j1 = j0;                 // trailing region starts at block jb
            const int64_t Tr = ceil_div64(k - j1, CB);
            const int64_t ntile = Tr * (Tr + 1) / 2;
            const int workers = G > 1 ? G - 1 : 1, me = G > 1 ? cta - 1 : 0;
            // tiles of column blocks >= 1 of the trailing region: Tr (Tr - 1) / 2;
            // when they are fewer than two per worker, split each into two
            // 16-row halves so that the short last steps spread wider
            const int H = (Tr * (Tr - 1) / 2 < 2 * (int64_t)workers) ? 2 : 1;
            const int64_t total = ntile * H;
            auto tile_of = [&](int64_t it, int64_t& I, int64_t& J) { tri_tile(it / H, I, J); };
            // column block jb (J = 0) was done in phase S of step jb-1
            auto next_item = [&](int64_t it) -> int64_t {
                for (; it < total; it += workers) {
                    int64_t I, J;
                    tile_of(it, I, J);
                    if (J >= 1) return it;
                }
                return total;
            };
            // operands of the next item are loaded into registers while the
            // current one computes
            float2 va[4], vb[4];
            auto fetch = [&](int64_t it) {
                int64_t I, J;
                tile_of(it, I, J);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = tid + 256 * i;
                    const int rr = e / CB, q = e % CB;
                    const int64_t ra = j1 + I * CB + rr, rb = j1 + J * CB + rr;
                    va[i] = ra < k ? __ldcg(Pdf + ra * CB + q) : make_float2(0.f, 0.f);
                    vb[i] = rb < k ? __ldcg(Pdf + rb * CB + q) : make_float2(0.f, 0.f);
                }
            };
            int64_t it = next_item(me);
            if (it < total) fetch(it);
            const int tx = tid % 16, ty = tid / 16;
            while (it < total) {
                int64_t I, J;
                tile_of(it, I, J);
                const int hsel = (int)(it % H);
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = tid + 256 * i;
                    fa[e / CB][e % CB] = va[i];
                    fb[e / CB][e % CB] = vb[i];
                }
                __syncthreads();
                const int64_t nx = next_item(it + workers);
                if (nx < total) fetch(nx);
                // the rank-32 product and the subtraction from K in double-float
                // on the FP32 pipes
                if (H == 1) {
                    float2 kold[2][2];
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int64_t r = j1 + I * CB + ty + 16 * a, c = j1 + J * CB + tx + 16 * b;
                            kold[a][b] = (r < k && c <= r) ? __ldcg(Kmat + r * k + c) : make_float2(0.f, 0.f);
                        }
                    Acc2 acc[2][2] = {};
#pragma unroll 4
                    for (int q = 0; q < CB; ++q) {
                        const float2 a0 = fa[ty][q], a1 = fa[ty + 16][q];
                        const float2 b0 = fb[tx][q], b1 = fb[tx + 16][q];
                        df_fma_acc(acc[0][0], a0, b0);
                        df_fma_acc(acc[0][1], a0, b1);
                        df_fma_acc(acc[1][0], a1, b0);
                        df_fma_acc(acc[1][1], a1, b1);
                    }
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int64_t r = j1 + I * CB + ty + 16 * a, c = j1 + J * CB + tx + 16 * b;
                            if (r < k && c <= r)
                                Kmat[r * k + c] = pair_sub(kold[a][b], pair_norm(acc[a][b].hi, acc[a][b].lo));
                        }
                } else {
                    // rows ty + 16 hsel only
                    const int ra = ty + 16 * hsel;
                    float2 kold[2];
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int64_t r = j1 + I * CB + ra, c = j1 + J * CB + tx + 16 * b;
                        kold[b] = (r < k && c <= r) ? __ldcg(Kmat + r * k + c) : make_float2(0.f, 0.f);
                    }
                    Acc2 acc[2] = {};
#pragma unroll 4
                    for (int q = 0; q < CB; ++q) {
                        const float2 a0 = fa[ra][q];
                        df_fma_acc(acc[0], a0, fb[tx][q]);
                        df_fma_acc(acc[1], a0, fb[tx + 16][q]);
                    }
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int64_t r = j1 + I * CB + ra, c = j1 + J * CB + tx + 16 * b;
                        if (r < k && c <= r) Kmat[r * k + c] = pair_sub(kold[b], pair_norm(acc[b].hi, acc[b].lo));
                    }
                }
                it = nx;
            }
        }
        if (!grid_sync_bounded(bar, nbar, status, nbar == 0 ? bar_extra : 0u, bar_limit_ns)) return;
        const int64_t rest = k - j0 - nb;
        if (rest <= 0) break;
        // ---- phase N: panel jb = K L_jj^{-T} by forward substitution, 16 rows per
        // work item: warp w solves rows r0 + w and r0 + 8 + w side by side (two
        // independent chains), lane c holds column c
        {
            const double* dinv = Wall + jb * CB;   // 1 / L_cc
            const int64_t items = ceil_div64(rest, 16);
            const int lane = tid & 31, wq = tid >> 5;
            bool loaded = false;
            for (int64_t it = cta; it < items; it += G) {
                const int64_t r0 = j0 + nb + it * 16;
                // the item's rows of K first, so that their loads overlap those of L_jj
                const int64_t ra = r0 + wq, rb = r0 + 8 + wq;
                float2 ka = (ra < k && lane < nb) ? __ldcg(Kmat + ra * k + j0 + lane) : make_float2(0.f, 0.f);
                float2 kb = (rb < k && lane < nb) ? __ldcg(Kmat + rb * k + j0 + lane) : make_float2(0.f, 0.f);
                if (!loaded) {
                    // L_jj and 1 / L_cc as double-float pairs, once per step
                    for (int e = tid; e < CB * CB; e += 256) {
                        const int r = e / CB, c = e % CB;
                        fa[r][c] = (c <= r && r < nb) ? __ldcg(Kmat + (j0 + r) * k + j0 + c) : make_float2(0.f, 0.f);
                    }
                    if (tid < CB) fb[0][tid] = df_split(__ldcg(dinv + tid));
                    __syncthreads();
                    loaded = true;
                }
                // substitution in double-float (FP32 latencies on the dependent chains)
                float2 xa = make_float2(0.f, 0.f), xb = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const float2 kca = make_float2(__shfl_sync(0xffffffffu, ka.x, c), __shfl_sync(0xffffffffu, ka.y, c));
                    const float2 kcb = make_float2(__shfl_sync(0xffffffffu, kb.x, c), __shfl_sync(0xffffffffu, kb.y, c));
                    const float2 dc = fb[0][c];
                    const float2 xca = df_mul2(kca, dc);
                    const float2 xcb = df_mul2(kcb, dc);
                    if (lane == c) {
                        xa = xca;
                        xb = xcb;
                    } else if (lane > c) {
                        const float2 lc = fa[lane][c];
                        ka = df_fnms(ka, xca, lc);
                        kb = df_fnms(kb, xcb, lc);
                    }
                }
                if (ra < k && lane < nb) Kmat[ra * k + j0 + lane] = xa;
                if (ra < k) Pdf[ra * CB + lane] = xa;   // 0 for lanes >= nb
                if (rb < k && lane < nb) Kmat[rb * k + j0 + lane] = xb;
                if (rb < k) Pdf[rb * CB + lane] = xb;
            }
        }
        // The column update reads panel rows j1 .. j1+31 (items 0 and 1, on
        // CTAs 0 and 1 % G) and the CTA's own rows: the two producers publish
        // their items on a counter instead of a grid barrier.
        {
            const int64_t items = ceil_div64(rest, 16);
            const unsigned mine = (cta == 0 ? 1u : 0u) + ((items >= 2 && cta == 1 % G) ? 1u : 0u);
            panel_target += items >= 2 ? 2u : 1u;
            if (mine) {
                __syncthreads();   // every warp's rows of the items are written
                if (tid == 0) {
                    __threadfence();
                    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar + 1), "r"(mine) : "memory");
                }
            }
            if (!flag_wait_bounded(bar + 1, panel_target, status, bar_limit_ns)) return;
        }
        // ---- phase S: column block jb+1 updated by panel jb, 16 rows per work
        // item (thread (ty, tx) takes rows ty and ty + 8 of the item, column tx)
        {
            const int64_t j1 = j0 + nb;
            const int ncol = (int)min((int64_t)CB, k - j1);
            const int64_t items = ceil_div64(k - j1, 16);
            for (int64_t it = cta; it < items; it += G) {
                const int64_t r0 = j1 + it * 16;
                // the two K entries this thread updates, loaded ahead of the operands
                const int tx = tid % CB, ty = tid / CB;
                const int64_t c = j1 + tx;
                const int64_t ra = r0 + ty, rb = r0 + 8 + ty;
                const bool wa = ra < k && tx < ncol && c <= ra, wb = rb < k && tx < ncol && c <= rb;
                const float2 ka = wa ? __ldcg(Kmat + ra * k + c) : make_float2(0.f, 0.f);
                const float2 kb = wb ? __ldcg(Kmat + rb * k + c) : make_float2(0.f, 0.f);
                __syncthreads();
                for (int e = tid; e < CB * CB; e += 256) {
                    const int c = e / CB, q = e % CB;
                    fb[c][q] = c < ncol ? __ldcg(Pdf + (j1 + c) * CB + q) : make_float2(0.f, 0.f);
                }
                for (int e = tid; e < 16 * CB; e += 256) {
                    const int r = e / CB, q = e % CB;
                    fa[r][q] = r0 + r < k ? __ldcg(Pdf + (r0 + r) * CB + q) : make_float2(0.f, 0.f);
                }
                __syncthreads();
                Acc2 a0{0.f, 0.f}, a1{0.f, 0.f}, b0{0.f, 0.f}, b1{0.f, 0.f};
#pragma unroll
                for (int q = 0; q < CB; q += 2) {
                    const float2 f0 = fb[tx][q], f1 = fb[tx][q + 1];
                    df_fma_acc(a0, fa[ty][q], f0);
                    df_fma_acc(a1, fa[ty][q + 1], f1);
                    df_fma_acc(b0, fa[ty + 8][q], f0);
                    df_fma_acc(b1, fa[ty + 8][q + 1], f1);
                }
                if (wa) Kmat[ra * k + c] = pair_sub(ka, pair_add(pair_norm(a0.hi, a0.lo), pair_norm(a1.hi, a1.lo)));
                if (wb) Kmat[rb * k + c] = pair_sub(kb, pair_add(pair_norm(b0.hi, b0.lo), pair_norm(b1.hi, b1.lo)));
            }
        }
        if (!grid_sync_bounded(bar, nbar, status, nbar == 0 ? bar_extra : 0u, bar_limit_ns)) return;
    }
}

// X (FP32, k x k) <- zero, then each 64 x 64 diagonal block of X = the FP32
// inverse of the matching block of L (one CTA per block, thread = column,
// forward substitution); these start the recursive doubling below.
__global__ void k_zero_f32(float* __restrict__ X, int64_t count) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < count) X[idx] = 0.f;
}

// L as FP64 (l_df = 0) or as double-float pairs (l_df = 1): its value in FP32.
__device__ __forceinline__ float l_entry(const double* L, int l_df, int64_t idx) {
    if (l_df) {
        const float2 v = reinterpret_cast<const float2*>(L)[idx];
        return __fadd_rn(v.x, v.y);
    }
    return (float)L[idx];
}

// One 64 x 64 diagonal block L_b = [A 0; B C] per CTA of 256 threads, its
// inverse in two levels: A^-1 and C^-1 (32 x 32 each) by forward substitution,
// thread c of each half forming column c, w_r = (delta_rc - sum_{q<r} l_rq w_q)
// / l_rr with the column in registers (rows above the diagonal give w_q = 0,
// which adds nothing); then the lower-left block -C^-1 (B A^-1) by two 32 x 32
// products over all threads.  The serial chains are 32 rows long and the
// unrolled code stays small.  Padding rows of a short last block carry 1 on
// the diagonal.
__global__ void __launch_bounds__(256) k_blockinv32(const double* __restrict__ L, int l_df, int64_t k,
                                                    float* __restrict__ X) {
    constexpr int H = FB / 2;                      // 32
    __shared__ __align__(16) float l[FB][FB + 4];  // the block of L
    __shared__ __align__(16) float w[FB][FB + 4];  // its inverse (lower)
    __shared__ __align__(16) float t[H][H + 4];    // B A^-1
    const int tid = threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.x * FB;
    const int nb = (int)(k - b0 < FB ? k - b0 : FB);
#pragma unroll
    for (int i = 0; i < FB * FB / 256; ++i) {
        const int e = tid + 256 * i;
        const int r = e / FB, c = e % FB;
        l[r][c] = (r < nb && c < nb && c <= r) ? l_entry(L, l_df, (b0 + r) * k + b0 + c) : (r == c ? 1.f : 0.f);
    }
    __syncthreads();
    if (tid < FB) {   // A^-1 (tid < 32) and C^-1 (32 <= tid < 64)
        const int o = (tid / H) * H, c = tid % H;
        float v[H];
#pragma unroll
        for (int r = 0; r < H; ++r) {
            float sacc = (r == c) ? 1.f : 0.f;
#pragma unroll
            for (int q = 0; q < r; q += 4) {
                const float4 lv = *reinterpret_cast<const float4*>(&l[o + r][o + q]);
                sacc = __fmaf_rn(-lv.x, v[q], sacc);
                if (q + 1 < r) sacc = __fmaf_rn(-lv.y, v[q + 1], sacc);
                if (q + 2 < r) sacc = __fmaf_rn(-lv.z, v[q + 2], sacc);
                if (q + 3 < r) sacc = __fmaf_rn(-lv.w, v[q + 3], sacc);
            }
            v[r] = __fdiv_rn(sacc, l[o + r][o + r]);
        }
#pragma unroll
        for (int r = 0; r < H; ++r) w[o + r][o + c] = v[r];
    }
    __syncthreads();
    // thread: row i of the lower-left block, columns j0 .. j0 + 3
    const int i = tid >> 3, j0 = (tid & 7) * 4;
    {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);   // (B A^-1)[i][j0..]: A^-1[q][j] = 0 for q < j
#pragma unroll 8
        for (int q = 0; q < H; ++q) {
            const float bq = l[H + i][q];
            const float4 a = *reinterpret_cast<const float4*>(&w[q][j0]);
            acc.x = __fmaf_rn(bq, a.x, acc.x);
            acc.y = __fmaf_rn(bq, a.y, acc.y);
            acc.z = __fmaf_rn(bq, a.z, acc.z);
            acc.w = __fmaf_rn(bq, a.w, acc.w);
        }
        *reinterpret_cast<float4*>(&t[i][j0]) = acc;
    }
    __syncthreads();
    {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);   // (C^-1 T)[i][j0..]: C^-1[i][q] = 0 for q > i
#pragma unroll 8
        for (int q = 0; q < H; ++q) {
            const float cq = w[H + i][H + q];
            const float4 tv = *reinterpret_cast<const float4*>(&t[q][j0]);
            acc.x = __fmaf_rn(cq, tv.x, acc.x);
            acc.y = __fmaf_rn(cq, tv.y, acc.y);
            acc.z = __fmaf_rn(cq, tv.z, acc.z);
            acc.w = __fmaf_rn(cq, tv.w, acc.w);
        }
        *reinterpret_cast<float4*>(&w[H + i][j0]) = make_float4(-acc.x, -acc.y, -acc.z, -acc.w);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < FB * FB / 256; ++u) {
        const int e = tid + 256 * u;
        const int r = e / FB, c = e % FB;
        if (c <= r && r < nb) X[(b0 + r) * k + b0 + c] = w[r][c];
    }
}

// Batched FP32 GEMM for the recursive-doubling inverse: for pair p,
// C_p = alpha * A_p B_p, with A_p, B_p, C_p sub-blocks of row-major k x k
// matrices addressed by (row, col) offsets that depend on p:
//   A_p at (ra + p*pstride, ca + p*pstride), B_p at (rb + p*pstride, cb + p*pstride), ...
// Size s x s x s.  A is float (X) or double (L) by `a_is_l`.
__global__ void __launch_bounds__(256) k_pair_gemm(const float* __restrict__ Xf, const double* __restrict__ Ld,
                                                   int a_is_l, int l_df, int64_t k, int64_t s, int64_t pstride,
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
                v = a_is_l ? l_entry(Ld, l_df, gr * k + gq) : Xf[gr * k + gq];
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

// The same pair products for blocks of s a multiple of TT (TT = 128 or 64, k a
// multiple of 8): TT x TT output tiles, TT/16 x TT/16 per thread (rows and
// columns h 64 + 4 t + {0..3}), the inner dimension in double-buffered chunks
// of 16 staged through shared memory with 16-byte global loads (A from L is
// converted from its FP64 or double-float storage on the fly).  The 64 tiles
// serve the merges whose 128 tiles would leave SMs idle.  tri skips the inner
// range where a triangular operand is zero: 1 = B lower (B[q][c] = 0 for
// q < c: q starts at the tile's first column), 2 = A lower (A[r][q] = 0 for
// q > r: q ends after the tile's last row).
constexpr int PGK = 16;
template <int TT>
__global__ void __launch_bounds__(256) k_pair_sgemm(const float* __restrict__ Xf, const double* __restrict__ Ld,
                                                    int a_is_l, int l_df, int64_t k, int64_t s, int64_t pstride,
                                                    int64_t ra, int64_t ca, int64_t rb, int64_t cb, const float* Bsrc,
                                                    float* __restrict__ C, int64_t rc, int64_t cc, float alpha,
                                                    int tri) {
    static_assert(TT == 128 || TT == 64, "tile of 128 or 64");
    constexpr int RT = TT / 16;          // rows (and columns) of C per thread
    constexpr int E = TT * PGK / 256;    // A (and B) elements a thread stages per chunk: 8 or 4
    __shared__ __align__(16) float As[2][PGK][TT + 4];   // As[q][r]
    __shared__ __align__(16) float Bs[2][PGK][TT + 4];   // Bs[q][c]
    const int tid = threadIdx.x;
    const int64_t off = (int64_t)blockIdx.z * pstride;
    const int64_t tr = (int64_t)blockIdx.y * TT, tc = (int64_t)blockIdx.x * TT;
    int64_t q0 = 0, q1 = s;
    if (tri == 1) q0 = tc;
    if (tri == 2) q1 = min(s, tr + TT);
    // loaders: A row ar, inner elements [ak, ak + E); B inner row bq, columns [bc, bc + E)
    const int ar = tid / (PGK / E), ak = (tid % (PGK / E)) * E;
    const int bq = tid / (TT / E), bc = (tid % (TT / E)) * E;
    const int64_t ga_r = ra + off + tr + ar;        // global row of A
    const int64_t gb_c = cb + off + tc + bc;        // global column of B
    float la[E], lb[E];
    auto load = [&](int64_t q) {
        const int64_t ga_c = ca + off + q + ak;     // global column of A
        if (ga_r < k && ga_c < k) {
            if (a_is_l && l_df) {
                const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(Ld) + ga_r * k + ga_c);
#pragma unroll
                for (int u = 0; u < E / 2; ++u) {
                    const float4 v = src[u];   // two (hi, lo) pairs
                    la[2 * u] = __fadd_rn(v.x, v.y);
                    la[2 * u + 1] = __fadd_rn(v.z, v.w);
                }
            } else if (a_is_l) {
                const double2* src = reinterpret_cast<const double2*>(Ld + ga_r * k + ga_c);
#pragma unroll
                for (int u = 0; u < E / 2; ++u) {
                    const double2 v = src[u];
                    la[2 * u] = (float)v.x;
                    la[2 * u + 1] = (float)v.y;
                }
            } else {
                const float4* src = reinterpret_cast<const float4*>(Xf + ga_r * k + ga_c);
#pragma unroll
                for (int u = 0; u < E / 4; ++u) {
                    const float4 v = src[u];
                    la[4 * u] = v.x; la[4 * u + 1] = v.y; la[4 * u + 2] = v.z; la[4 * u + 3] = v.w;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < E; ++u) la[u] = 0.f;
        }
        const int64_t gb_r = rb + off + q + bq;     // global row of B
        if (gb_r < k && gb_c < k) {
            const float4* src = reinterpret_cast<const float4*>(Bsrc + gb_r * k + gb_c);
#pragma unroll
            for (int u = 0; u < E / 4; ++u) {
                const float4 v = src[u];
                lb[4 * u] = v.x; lb[4 * u + 1] = v.y; lb[4 * u + 2] = v.z; lb[4 * u + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < E; ++u) lb[u] = 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < E; ++u) As[buf][ak + u][ar] = la[u];
#pragma unroll
        for (int u = 0; u < E / 4; ++u)
            *reinterpret_cast<float4*>(&Bs[buf][bq][bc + 4 * u]) =
                make_float4(lb[4 * u], lb[4 * u + 1], lb[4 * u + 2], lb[4 * u + 3]);
    };
    const int ty = tid >> 4, tx = tid & 15;
    float acc[RT][RT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = 0.f;
    int buf = 0;
    if (q0 < q1) {
        load(q0);
        store(0);
    }
    __syncthreads();
    for (int64_t q = q0; q < q1; q += PGK) {
        const bool more = q + PGK < q1;
        if (more) load(q + PGK);
#pragma unroll
        for (int kk = 0; kk < PGK; ++kk) {
            float av[RT], bv[RT];
#pragma unroll
            for (int h = 0; h < RT / 4; ++h) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][64 * h + ty * 4]);
                const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 * h + tx * 4]);
                av[4 * h] = a4.x; av[4 * h + 1] = a4.y; av[4 * h + 2] = a4.z; av[4 * h + 3] = a4.w;
                bv[4 * h] = b4.x; bv[4 * h + 1] = b4.y; bv[4 * h + 2] = b4.z; bv[4 * h + 3] = b4.w;
            }
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < RT; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int64_t r = tr + 64 * (i / 4) + ty * 4 + (i % 4);
        const int64_t gr = rc + off + r;
        if (r >= s || gr >= k) continue;
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const int64_t c = tc + 64 * (j / 4) + tx * 4 + (j % 4);
            const int64_t gc = cc + off + c;
            if (c < s && gc < k) C[gr * k + gc] = alpha * acc[i][j];
        }
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

// ---------------------------------------------------------------------------
// Apply kernels: vectors are double-float pairs (hi, lo) of binary32; dot
// products use exact products (TwoProduct) and compensated sums, so every
// dependent step is an FP32 operation (FP64 has a long dependent latency).

__device__ __forceinline__ void acc_mul(Acc2& acc, float m, float2 x) {   // acc += m * (x.hi + x.lo)
    float p, e, s, es;
    two_prod(m, x.x, p, e);
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fmaf_rn(m, x.y, e), es));
}

__device__ __forceinline__ float2 df_norm(float hi, float lo) {   // fast renormalisation (|hi| >= |lo|)
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_scale(float2 a, double sc) {   // a * sc with sc a double
    const float sh = (float)sc, sl = (float)(sc - (double)sh);
    float p, e;
    two_prod(a.x, sh, p, e);
    return df_norm(p, __fadd_rn(e, __fmaf_rn(a.x, sl, __fmul_rn(a.y, sh))));
}

__device__ __forceinline__ Acc2 warp_sum_acc2(Acc2 a) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const Acc2 o = acc2_shfl_xor(a, off);
        a.add_pair(o.hi, o.lo);
    }
    return a;
}

// y[i] = (add ? add[i] : 0) + sum_l M[i][l] x[l], l in [lo(i), hi(i)):
// tri 0 = all columns, 1 = l <= i (lower), 2 = l >= i (upper).  M row-major
// FP32 with leading dimension ld; x double-float, or FP32 when xf != NULL.
// One warp per row.
__global__ void k_rowdot(const float* __restrict__ M, int64_t rows, int64_t cols, int64_t ld, int tri,
                         const float2* __restrict__ x, const float* __restrict__ xf, const float2* add,
                         float2* y) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= rows) return;
    const int64_t l0 = tri == 2 ? i : 0, l1 = tri == 1 ? i + 1 : cols;
    const float* row = M + i * ld;
    // four independent accumulators per lane (loads of four strides in flight)
    Acc2 acc{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
    int64_t l = l0 + lane;
    if (xf) {
        for (; l + 96 < l1; l += 128) {
            const float m0 = row[l], m1 = row[l + 32], m2 = row[l + 64], m3 = row[l + 96];
            const float x0 = xf[l], x1 = xf[l + 32], x2 = xf[l + 64], x3 = xf[l + 96];
            acc_mul(acc, m0, make_float2(x0, 0.f));
            acc_mul(a1, m1, make_float2(x1, 0.f));
            acc_mul(a2, m2, make_float2(x2, 0.f));
            acc_mul(a3, m3, make_float2(x3, 0.f));
        }
        for (; l < l1; l += 32) acc_mul(acc, row[l], make_float2(xf[l], 0.f));
    } else {
        for (; l + 96 < l1; l += 128) {
            const float m0 = row[l], m1 = row[l + 32], m2 = row[l + 64], m3 = row[l + 96];
            const float2 x0 = x[l], x1 = x[l + 32], x2 = x[l + 64], x3 = x[l + 96];
            acc_mul(acc, m0, x0);
            acc_mul(a1, m1, x1);
            acc_mul(a2, m2, x2);
            acc_mul(a3, m3, x3);
        }
        for (; l < l1; l += 32) acc_mul(acc, row[l], x[l]);
    }
    acc.add_pair(a1.hi, a1.lo);
    a2.add_pair(a3.hi, a3.lo);
    acc.add_pair(a2.hi, a2.lo);
    acc = warp_sum_acc2(acc);
    if (lane == 0) {
        float2 r = df_norm(acc.hi, acc.lo);
        if (add) r = df_add(r, add[i]);
        y[i] = r;
    }
}

// part[chunk][c] = sum_{j in chunk} M[j][c] x[j] (column dots of a row-major
// FP32 matrix, one thread per column, coalesced along c).
__global__ void k_coldot_part(const float* __restrict__ M, int64_t rows, int64_t cols, const float2* __restrict__ x,
                              int64_t rows_per_chunk, float2* __restrict__ part) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t j1 = rows < j0 + rows_per_chunk ? rows : j0 + rows_per_chunk;
    if (c >= cols) return;
    Acc2 acc{0.f, 0.f}, a1{0.f, 0.f};
    int64_t j = j0;
    for (; j + 1 < j1; j += 2) {
        const float m0 = M[j * cols + c], m1 = M[(j + 1) * cols + c];
        acc_mul(acc, m0, x[j]);
        acc_mul(a1, m1, x[j + 1]);
    }
    if (j < j1) acc_mul(acc, M[j * cols + c], x[j]);
    acc.add_pair(a1.hi, a1.lo);
    part[blockIdx.y * cols + c] = df_norm(acc.hi, acc.lo);
}

// Reduce the column-dot partials in a fixed order into w; if g != NULL also
// finish a Woodbury apply: gt = (g - w) / nu^2, with per-block FP64 partials
// of g . gt for the decrement.
__global__ void k_coldot_reduce(const float2* __restrict__ part, int chunks, int64_t cols, float2* __restrict__ w,
                                const float* __restrict__ g, double inv_nu2, float* __restrict__ gt,
                                double* __restrict__ rpart) {
    __shared__ double sm[256];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double prod = 0.0;
    if (c < cols) {
        float2 sum = part[c];
        for (int q = 1; q < chunks; ++q) sum = df_add(sum, part[q * cols + c]);
        if (w) w[c] = sum;
        if (g) {
            const double v = ((double)g[c] - ((double)sum.x + (double)sum.y)) * inv_nu2;
            gt[c] = (float)v;
            prod = (double)g[c] * v;
        }
    }
    if (g) {
        sm[threadIdx.x] = prod;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < 256; ++i) t += sm[i];
            rpart[blockIdx.x] = t;
        }
    }
}

// res = t - (nu^2 u + w) in double-float.
__global__ void k_res_df(const float2* __restrict__ t, const float2* __restrict__ u, double nu2,
                         const float2* __restrict__ w, int64_t n, float2* __restrict__ res) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) res[i] = df_add(t[i], df_neg(df_add(df_scale(u[i], nu2), w[i])));
}

// t = g as double-float.
__global__ void k_f2df(const float* __restrict__ g, int64_t n, float2* __restrict__ t) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) t[i] = make_float2(g[i], 0.f);
}

// gt = u (direct form) and per-block FP64 partials of g . gt.
__global__ void k_direct_out(const float* __restrict__ g, const float2* __restrict__ u, int64_t d,
                             float* __restrict__ gt, double* __restrict__ rpart) {
    __shared__ double sm[256];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double prod = 0.0;
    if (c < d) {
        const double v = (double)u[c].x + (double)u[c].y;
        gt[c] = (float)v;
        prod = (double)g[c] * v;
    }
    sm[threadIdx.x] = prod;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 256; ++i) t += sm[i];
        rpart[blockIdx.x] = t;
    }
}

}  // namespace

int ihs_factor_build(ihs_ctx* ctx, ihs_factor_t* F) {
    IHS_TRY(ihs_factor_enqueue(ctx, F));
    return ihs_check_status(ctx);
}

int ihs_factor_enqueue(ihs_ctx* ctx, ihs_factor_t* F) {
    const int64_t k = F->k;
    cudaStream_t s = ctx->stream;
    const int64_t T = ceil_div64(k, FB);
    double* Kmat = F->L;
    double* Wall = F->W;
    const int64_t K = F->woodbury ? F->d : F->m;
    // One cooperative launch of the Cholesky when the context allows it
    // (contexts that run many factorisations side by side take the stream
    // version); that path keeps K and L as double-float pairs (the FP32 pipes
    // only), the stream version in FP64.
    const int64_t TC = ceil_div64(k, CB);
    int Gcoop = 0;
    if (!ctx->no_coop && TC > 1) {
        int per_sm = 0;
        IHS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_persistent, 256, 0));
        const int64_t first_tiles = (TC - 1) * TC / 2;
        Gcoop = (int)std::min<int64_t>((int64_t)ctx->chol_per_sm * ctx->sm_count,
                                       std::max<int64_t>(1, (first_tiles + 1) / 2));
        Gcoop = std::min(Gcoop, per_sm * ctx->sm_count);
    }
    F->l_df = Gcoop >= 1 ? 1 : 0;
    const double nu2 = F->nu * F->nu;
    const float nu2_hi = (float)nu2;
    const float2 nu2df = make_float2(nu2_hi, (float)(nu2 - (double)nu2_hi));
    if (!ctx->gram_simt) {
        // tensor cores: exact three-piece BF16 split, slice sums added in double-float
        IHS_TRY(ihs_gram_tc_enqueue(ctx, F->SA, F->d, F->woodbury, k, K, nu2, F->l_df, Kmat, s));
    } else {
        // split the inner dimension so that at least two CTAs per SM work on
        // the Gram, with at least 64 inner rows per split
        const int64_t ntiles = T * (T + 1) / 2;
        int64_t KS = std::max<int64_t>(1, ceil_div64(2 * (int64_t)ctx->sm_count, ntiles));
        KS = std::min<int64_t>(KS, std::max<int64_t>(1, K / 64));
        const int64_t kchunk = ceil_div64(ceil_div64(K, KS), 32) * 32;
        KS = ceil_div64(K, kchunk);
        float2* gpart = nullptr;
        if (KS > 1) {
            void* ws = nullptr;
            IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)KS * ntiles * FB * FB * sizeof(float2), &ws));
            gpart = static_cast<float2*>(ws);
        }
        k_gram_c32<<<dim3((unsigned)ntiles, (unsigned)KS), 256, 0, s>>>(F->SA, F->d, F->woodbury, k, K, kchunk,
                                                                        nu2, nu2df, F->l_df, Kmat, gpart);
        IHS_LAUNCH_CHECK();
        if (KS > 1) {
            k_gram_reduce<<<dim3((unsigned)ntiles, FB * FB / 256), 256, 0, s>>>(gpart, (int)KS, ntiles, k, nu2df, F->l_df,
                                                                              Kmat);
            IHS_LAUNCH_CHECK();
        }
    }
    // the fused apply's copy of SA^T
    IHS_TRY(ihs_apply_prepare(ctx, F));
    // Blocked right-looking Cholesky with one step of look-ahead: on the main
    // stream, diagonal block jb, its panel and the update of block column jb+1;
    // on the auxiliary stream, the rest of the trailing update of step jb,
    // which overlaps the factorisation of block jb+1.  Events order the
    // writes: the update of column jb+1 (main) follows the previous rest
    // update (aux), and each rest update follows its panel.
    if (F->l_df) {
        const int G = Gcoop;
        {
            unsigned* bar = ctx->d_status + 16;   // grid-barrier counter, then the panel counter
            IHS_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
            int64_t kk = k;
            // test-only: the first launch of a context with the knob set gets an
            // unreachable first barrier (see ihs_ctx)
            unsigned extra = ctx->test_bar_unreachable ? 1u : 0u;
            ctx->test_bar_unreachable = 0;
            uint64_t limit = ctx->bar_limit_ns;
            float2* Kdf = reinterpret_cast<float2*>(Kmat);
            void* args[] = {&Kdf, &kk, &Wall, &bar, &ctx->d_status, &extra, &limit};
            IHS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_chol_persistent, dim3((unsigned)G), dim3(256),
                                                     args, 0, s));
            ihs_count_launch();
            goto inverse;
        }
    }
    {
    cudaStream_t aux = ctx->aux;
    IHS_CUDA_TRY(cudaEventRecord(ctx->fev[7], s));     // gram done
    IHS_CUDA_TRY(cudaStreamWaitEvent(aux, ctx->fev[7], 0));
    for (int64_t jb = 0; jb < TC; ++jb) {
        const int64_t j0 = jb * CB;
        const int nb = (int)std::min<int64_t>(CB, k - j0);
        double* Wj = Wall + jb * CB * CB;
        k_potrf32<<<1, 256, 0, s>>>(Kmat, k, j0, nb, Wj, ctx->d_status);
        IHS_LAUNCH_CHECK();
        const int64_t rest = k - j0 - nb;
        if (rest > 0) {
            k_panel32<<<(unsigned)ceil_div64(rest, kPanelRows), 256, 0, s>>>(Kmat, k, j0, nb, Wj);
            IHS_LAUNCH_CHECK();
            cudaEvent_t panel_done = ctx->fev[jb % 3];
            IHS_CUDA_TRY(cudaEventRecord(panel_done, s));
            // column jb+1 must not race with the previous step's rest update
            if (jb > 0) IHS_CUDA_TRY(cudaStreamWaitEvent(s, ctx->fev[3 + (jb - 1) % 3], 0));
            k_syrk_next<<<(unsigned)ceil_div64(rest, 8), 256, 0, s>>>(Kmat, k, j0, nb);
            IHS_LAUNCH_CHECK();
            const int64_t Tr = ceil_div64(rest, CB);
            IHS_CUDA_TRY(cudaStreamWaitEvent(aux, panel_done, 0));
            if (Tr > 1) {
                k_syrk_rest<<<(unsigned)(Tr * (Tr + 1) / 2), 256, 0, aux>>>(Kmat, k, j0, nb);
                IHS_LAUNCH_CHECK();
            }
            IHS_CUDA_TRY(cudaEventRecord(ctx->fev[3 + jb % 3], aux));
        }
    }
    IHS_CUDA_TRY(cudaEventRecord(ctx->fev[6], aux));
    IHS_CUDA_TRY(cudaStreamWaitEvent(s, ctx->fev[6], 0));
    }
inverse:
    // X = L^{-1} in FP32 by recursive doubling: diagonal 64-blocks are FP32
    // inverses of L's blocks; for block size sz = 64, 128, ... the lower-left
    // block of each pair is X21 = -X22 (L21 X11).
    float* X = F->X;
    float* tmp = F->XT;   // scratch for L21 X11 (overwritten by X^T at the end)
    k_zero_f32<<<(unsigned)ceil_div64(k * k, 256), 256, 0, s>>>(X, k * k);
    IHS_LAUNCH_CHECK();
    k_blockinv32<<<(unsigned)T, 256, 0, s>>>(F->L, F->l_df, k, X);
    IHS_LAUNCH_CHECK();
    for (int64_t sz = FB; sz < k; sz *= 2) {
        const int64_t pairs = ceil_div64(k, 2 * sz);
        const int64_t tiles = ceil_div64(sz, FB);
        dim3 grid((unsigned)tiles, (unsigned)tiles, (unsigned)pairs);
        if (sz % 64 == 0 && k % 8 == 0) {
            // 128 tiles when they fill every SM, else 64 tiles
            const int64_t t128 = sz / 128;
            const bool big = sz % 128 == 0 && t128 * t128 * pairs >= ctx->sm_count;
            const int64_t tt = big ? t128 : sz / 64;
            dim3 g2((unsigned)tt, (unsigned)tt, (unsigned)pairs);
            auto kern = big ? k_pair_sgemm<128> : k_pair_sgemm<64>;
            // tmp21 = L21 X11 (X11 lower), X21 = -X22 tmp21 (X22 lower)
            kern<<<g2, 256, 0, s>>>(X, F->L, 1, F->l_df, k, sz, 2 * sz, sz, 0, 0, 0, X, tmp, sz, 0, 1.0f, 1);
            IHS_LAUNCH_CHECK();
            kern<<<g2, 256, 0, s>>>(X, nullptr, 0, 0, k, sz, 2 * sz, sz, sz, sz, 0, tmp, X, sz, 0, -1.0f, 2);
            IHS_LAUNCH_CHECK();
            continue;
        }
        // tmp21 = L21 X11   (L21 at rows [sz, 2sz), cols [0, sz) of the pair)
        k_pair_gemm<<<grid, 256, 0, s>>>(X, F->L, 1, F->l_df, k, sz, 2 * sz, sz, 0, 0, 0, X, tmp, sz, 0, 1.0f);
        IHS_LAUNCH_CHECK();
        // X21 = -X22 tmp21 (X is both the A operand and C: X22 is read, the
        // disjoint block X21 written)
        k_pair_gemm<<<grid, 256, 0, s>>>(X, nullptr, 0, 0, k, sz, 2 * sz, sz, sz, sz, 0, tmp, X, sz, 0, -1.0f);
        IHS_LAUNCH_CHECK();
    }
    dim3 tg((unsigned)ceil_div64(k, 32), (unsigned)ceil_div64(k, 32));
    k_transpose_f32<<<tg, 256, 0, s>>>(X, k, F->XT);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

// H_S^{-1} g with one step of iterative refinement: the FP32 inverse factor X
// gives u0 = X^T X t; the residual t - K u0 uses the exact operator
// (K u = nu^2 u + SA (SA^T u), or SA^T (SA u) + nu^2 u); vectors and dot
// products are double-float (binary32 pairs with compensated sums).
int ihs_apply_enqueue(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* d_r) {
    if (F->fused) return ihs_apply_fused(ctx, F, g, gt, d_r);
    cudaStream_t s = ctx->stream;
    const int64_t k = F->k, d = F->d, m = F->m;
    const int64_t mx = std::max(m, d);
    float2* t = reinterpret_cast<float2*>(F->work);   // k
    float2* v = t + k;                                 // k
    float2* u = v + k;                                 // k
    float2* res = u + k;                               // k
    float2* w = res + k;                               // max(m, d)
    float2* w2 = w + mx;                               // max(m, d)
    float2* part = w2 + mx;                            // 32 x max(m, d)
    double* rpart = reinterpret_cast<double*>(part + 32 * mx);   // 4096
    const unsigned kw = (unsigned)ceil_div64(k * 32, 256);
    const unsigned kb = (unsigned)ceil_div64(k, 256);
    const unsigned db = (unsigned)ceil_div64(d, 256);
    const unsigned mw = (unsigned)ceil_div64(m * 32, 256);
    const int64_t chunks = std::min<int64_t>(32, std::max<int64_t>(1, m / 64));
    const int64_t rpc = ceil_div64(m, chunks);
    const int64_t nch = ceil_div64(m, rpc);
    const double nu2 = F->nu * F->nu;
    // SA^T x (d) into out; with gg != NULL the Woodbury output gt is produced instead
    auto sat = [&](const float2* x, float2* out, const float* gg) -> int {
        dim3 grid(db, (unsigned)nch);
        k_coldot_part<<<grid, 256, 0, s>>>(F->SA, m, d, x, rpc, part);
        IHS_LAUNCH_CHECK();
        k_coldot_reduce<<<db, 256, 0, s>>>(part, (int)nch, d, out, gg, 1.0 / nu2, gt, rpart);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    if (F->woodbury) {
        k_rowdot<<<mw, 256, 0, s>>>(F->SA, m, d, d, 0, nullptr, g, nullptr, t);   // t = SA g
        IHS_LAUNCH_CHECK();
        k_rowdot<<<kw, 256, 0, s>>>(F->X, k, k, k, 1, t, nullptr, nullptr, v);    // v = X t
        IHS_LAUNCH_CHECK();
    } else {
        k_f2df<<<kb, 256, 0, s>>>(g, k, t);                                        // t = g
        IHS_LAUNCH_CHECK();
        k_rowdot<<<kw, 256, 0, s>>>(F->X, k, k, k, 1, nullptr, g, nullptr, v);    // v = X g
        IHS_LAUNCH_CHECK();
    }
    k_rowdot<<<kw, 256, 0, s>>>(F->XT, k, k, k, 2, v, nullptr, nullptr, u);        // u0 = X^T v
    IHS_LAUNCH_CHECK();
    if (F->woodbury) {
        IHS_TRY(sat(u, w, nullptr));                                                // w = SA^T u0
        k_rowdot<<<mw, 256, 0, s>>>(F->SA, m, d, d, 0, w, nullptr, nullptr, w2);   // w2 = SA w
    } else {
        k_rowdot<<<mw, 256, 0, s>>>(F->SA, m, d, d, 0, u, nullptr, nullptr, w);    // w = SA u0
        IHS_LAUNCH_CHECK();
        IHS_TRY(sat(w, w2, nullptr));                                               // w2 = SA^T w
    }
    IHS_LAUNCH_CHECK();
    k_res_df<<<kb, 256, 0, s>>>(t, u, nu2, w2, k, res);                            // res = t - K u0
    IHS_LAUNCH_CHECK();
    k_rowdot<<<kw, 256, 0, s>>>(F->X, k, k, k, 1, res, nullptr, nullptr, v);       // v = X res
    IHS_LAUNCH_CHECK();
    k_rowdot<<<kw, 256, 0, s>>>(F->XT, k, k, k, 2, v, nullptr, u, u);              // u1 = u0 + X^T v
    IHS_LAUNCH_CHECK();
    if (F->woodbury) {
        IHS_TRY(sat(u, nullptr, g));                                                // gt = (g - SA^T u1) / nu^2
    } else {
        k_direct_out<<<db, 256, 0, s>>>(g, u, d, gt, rpart);                        // gt = u1
        IHS_LAUNCH_CHECK();
    }
    if (d_r) {
        k_sum_half<<<1, 1, 0, s>>>(rpart, (int)db, d_r);
        IHS_LAUNCH_CHECK();
    }
    return IHS_OK;
}

// apply scratch, in 8-byte units: t, v, u, res (k each), w, w2 (max(m, d) each),
// 32 x max(m, d) column-dot partials, 4096 decrement partials, 64 spare
static size_t factor_work_doubles(int64_t k, int64_t m, int64_t d) {
    const size_t mx = (size_t)std::max(m, d);
    return 4 * (size_t)k + 34 * mx + 4096 + 64;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Byte offsets of a factor's buffers in one block: K/L (FP64 k x k), the
// diagonal-block inverses W, X = L^{-1} and X^T (FP32), the multi-launch
// apply's work area, and for the fused apply SA^T and four partial-sum
// buffers (+ one FP64 slot per CTA).
struct FactorLayout {
    size_t L, W, X, XT, work, SAT, Y, total;
};

static FactorLayout factor_layout(int64_t k, int64_t m, int64_t d, bool fused, int sm_count) {
    const int64_t T = ceil_div64(k, FB);
    const size_t kk = (size_t)k * k;
    FactorLayout l;
    size_t o = 0;
    l.L = o;
    o += align256(kk * sizeof(double));
    l.W = o;
    o += align256((size_t)T * FB * FB * sizeof(double));
    l.X = o;
    o += align256(kk * sizeof(float));
    l.XT = o;
    o += align256(kk * sizeof(float));
    l.work = o;
    o += align256(factor_work_doubles(k, m, d) * sizeof(double));
    l.SAT = l.Y = 0;
    if (fused) {
        l.SAT = o;
        o += align256((size_t)m * d * sizeof(float));
        l.Y = o;
        o += align256((4 * ihs_apply_partials(k, m, d)) * sizeof(float2) + (size_t)sm_count * sizeof(double));
    }
    l.total = o;
    return l;
}

static void factor_init(ihs_factor_t* F, ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, int owned,
                        bool allow_fused) {
    memset(F, 0, sizeof(*F));
    F->ctx = ctx;
    F->SA = SA;
    F->m = m;
    F->d = d;
    F->nu = nu;
    F->woodbury = m < d ? 1 : 0;
    F->k = F->woodbury ? m : d;
    F->owned = owned;
    F->fused = (allow_fused && !ctx->no_coop && ((uintptr_t)SA % 16) == 0 && ihs_apply_fused_ok(F->k, m, d)) ? 1 : 0;
}

static void factor_bind(ihs_factor_t* F, char* base, const FactorLayout& l) {
    F->L = reinterpret_cast<double*>(base + l.L);
    F->W = reinterpret_cast<double*>(base + l.W);
    F->X = reinterpret_cast<float*>(base + l.X);
    F->XT = reinterpret_cast<float*>(base + l.XT);
    F->work = reinterpret_cast<double*>(base + l.work);
    if (F->fused) {
        F->SAT = reinterpret_cast<float*>(base + l.SAT);
        F->Y = reinterpret_cast<float2*>(base + l.Y);
    }
}

int ihs_factor_scratch(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t* F,
                       bool check) {
    if (!ctx || !SA || !F || m < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    factor_init(F, ctx, SA, m, d, nu, 0, true);
    const FactorLayout l = factor_layout(F->k, m, d, F->fused, ctx->sm_count);
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_FACTOR, l.total, &ws));
    factor_bind(F, static_cast<char*>(ws), l);
    return check ? ihs_factor_build(ctx, F) : ihs_factor_enqueue(ctx, F);
}

int ihs_factor_alloc(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** out) {
    if (!ctx || !SA || !out || m < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    *out = nullptr;
    ihs_factor_t* F = new (std::nothrow) ihs_factor_t;
    if (!F) return IHS_ENOMEM;
    factor_init(F, ctx, SA, m, d, nu, 1, true);
    const FactorLayout l = factor_layout(F->k, m, d, F->fused, ctx->sm_count);
    void* base = nullptr;
    if (cudaMalloc(&base, l.total) != cudaSuccess) {
        cudaGetLastError();
        delete F;
        return IHS_ENOMEM;
    }
    factor_bind(F, static_cast<char*>(base), l);
    *out = F;
    return IHS_OK;
}

// Factor storage in one block from a stream-ordered memory pool, allocated
// on ctx's stream (owned = 2; release with ihs_factor_release_pool).  These
// factors serve contexts that run many solves side by side and take the
// multi-launch apply.
int ihs_factor_alloc_pool(ihs_ctx* ctx, cudaMemPool_t pool, const float* SA, int64_t m, int64_t d, double nu,
                          ihs_factor_t* F) {
    if (!ctx || !SA || !F || m < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu)) return IHS_EINVAL;
    factor_init(F, ctx, SA, m, d, nu, 2, false);
    const FactorLayout l = factor_layout(F->k, m, d, false, ctx->sm_count);
    void* base = nullptr;
    if (cudaMallocFromPoolAsync(&base, l.total, pool, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return IHS_ENOMEM;
    }
    factor_bind(F, static_cast<char*>(base), l);
    return IHS_OK;
}

void ihs_factor_release_pool(ihs_factor_t* F, cudaStream_t s) {
    if (F && F->owned == 2 && F->L) cudaFreeAsync(F->L, s);
    if (F) memset(F, 0, sizeof(*F));
}

extern "C" int ihs_factor(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** out) {
    IhsRange range("ihs_factor");
    if (!out) return IHS_EINVAL;
    *out = nullptr;
    ihs_factor_t* F = nullptr;
    IHS_TRY(ihs_factor_alloc(ctx, SA, m, d, nu, &F));
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
    if (F->owned != 1) return IHS_EINVAL;   // scratch- or pool-backed factors are released by their owner
    // cudaFree waits for the device's outstanding work on the block; the context
    // is not touched (it may already be destroyed)
    if (F->L) cudaFree(F->L);   // the start of the factor's one block
    delete F;
    return IHS_OK;
}

extern "C" int ihs_apply_hinv(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* r_h) {
    IhsRange range("ihs_apply_hinv");
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
