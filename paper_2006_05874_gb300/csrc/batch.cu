// Batched adaptive IHS: many ridge problems in one solve (gradient-IHS variant).
//
// Every problem follows the same controller as ihs_solve (Sec. 5 variant of
// Algorithm 1: gradient-IHS candidate, accept if r+/r <= c_gd, else m <- 2m
// with a fresh sketch keyed by (seed, level)), but the problems advance in
// lock step, one round per iteration, and every per-iteration step runs as one
// launch over all problems:
//   * candidate x+ = x - mu gt (and ||x+||^2);
//   * gradient g+ = A^T (A x+ - b) + nu^2 x+ (and ||A x+||^2):
//       - problems that share one A (a regularisation path: many nu and b)
//         take one multi-right-hand-side pass over A, R = A X+ - B and
//         G = A^T R, so A is read once per round for all of them;
//       - the other problems take one persistent kernel over a work list of
//         row tiles of all their matrices; the tile height is chosen by timing
//         the candidates on the first call (autotuned);
//   * H_S^{-1} g+ and the decrement r+ (Lemma 4.1): the apply of the single
//     solver, each of its steps one launch over all problems (per-problem
//     descriptors: Woodbury or direct form, own factor, own sketch);
//   * the FP64 scalars of all problems come back in one copy, and the host
//     takes the accept / double / stop decisions in FP64.
// The round (candidate, gradient, apply, scalars) is captured once into a CUDA
// graph and replayed; descriptors and flags live in device tables updated by
// one small copy per round.  Sketches and FP64 factorisations happen only at
// level changes; they run concurrently on a pool of lanes (streams), and the
// sketch of a level is computed once for all problems that share A.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kLanes = 32;

// ---------------------------------------------------------------------------
// Per-problem descriptors (device)

struct BVec {            // the problem's vectors and scalars
    const float* A;
    const float* b;
    float *x, *xc, *g, *gc, *gt, *gtc;
    double* sc;          // [0] r+, [1] ||A x+||^2, [2] ||x+||^2, [3..] spare
    double* xpart;       // candidate partial sums (one per 256-block)
    int64_t n, d;
    double nu2;
    float mu;            // step of this round (0: evaluate at x)
    int active;          // take part in this round
    int commit;          // at the start of the round: x, g, gt <- xc, gc, gtc
    int path;            // index of its shared-A group, or -1
    int col;             // column in that group
};

struct BRow {            // y = (add ? add : 0) + M x, one warp per row (see k_rowdot)
    const float* M;
    int64_t rows, cols, ld;
    int tri;
    const float2* x;
    const float* xf;
    const float2* add;
    float2* y;
    int on;
};

struct BCol {            // part[chunk][c] = sum_j M[j][c] x[j], then reduce (see k_coldot_*)
    const float* M;
    int64_t rows, cols, rpc, nch;
    const float2* x;
    float2* part;
    float2* w;
    const float* g;
    double inv_nu2;
    float* gt;
    double* rpart;
    int on;
};

struct BElt {            // element-wise steps of the apply
    int op;              // 0: t = df(g); 1: res = t - (nu2 u + w2); 2: gt = u (direct out)
    int64_t k;
    const float* g;
    float2 *t, *u, *w2, *res;
    float* gt;
    double nu2;
    double* rpart;
    int on;
};

struct BSum {            // r = 1/2 sum rpart[0..count)
    const double* rpart;
    int count;
    double* r;
    int on;
};

// The apply of one problem as nine batched steps.
constexpr int kRowSteps = 6, kColSteps = 3, kEltSteps = 3;

struct ApplyDesc {
    BRow row[kRowSteps];   // s1 (Woodbury t = SA g), s2 v = X t, s3 u = X^T v, s4/s5 rowdot part, s7, s8
    BCol col[kColSteps];   // s4/s5 coldot part, s9 (Woodbury out)
    BElt elt[kEltSteps];   // s1 direct, s6, s9 direct
    BSum sum;
};

// ---- double-float helpers (same operations as the single-problem apply) ----
__device__ __forceinline__ void acc_mul(Acc2& acc, float m, float2 x) {
    float p, e, s, es;
    two_prod(m, x.x, p, e);
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fmaf_rn(m, x.y, e), es));
}
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_scale(float2 a, double sc) {
    const float sh = (float)sc, sl = (float)(sc - (double)sh);
    float p, e;
    two_prod(a.x, sh, p, e);
    return df_norm(p, __fadd_rn(e, __fmaf_rn(a.x, sl, __fmul_rn(a.y, sh))));
}

// ---------------------------------------------------------------------------
// Round kernels

// commit (x, g, gt <- xc, gc, gtc for accepted problems), then the candidate
// xc = x - mu gt with per-block partials of ||xc||^2.  grid (blocks, P).
__global__ void __launch_bounds__(256) kb_candidate(BVec* __restrict__ V) {
    __shared__ double sm[8];
    BVec& v = V[blockIdx.y];
    if (!v.active && !v.commit) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (i < v.d) {
        float x = v.x[i], gt = v.gt[i];
        if (v.commit) {
            x = v.xc[i];
            gt = v.gtc[i];
            v.x[i] = x;
            v.g[i] = v.gc[i];
            v.gt[i] = gt;
        }
        if (v.active) {
            const float c = __fmaf_rn(-v.mu, gt, x);
            v.xc[i] = c;
            sq = (double)c * (double)c;
        }
    }
    if (!v.active || (int64_t)blockIdx.x * blockDim.x >= v.d) return;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += sm[k];
        v.xpart[blockIdx.x] = s;
    }
}

__global__ void kb_xfold(BVec* __restrict__ V, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !V[p].active) return;
    const int nb = (int)ceil_div64(V[p].d, 256);
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += V[p].xpart[k];
    V[p].sc[2] = s;
}

// ---- gradient, independent problems: work list of row tiles ----
struct Tile {
    int p;          // problem
    int64_t row0;   // first row
    int rows;
};

// One CTA per tile (grid-stride over the list): phase 1, warp per row, Dot2
// r_i = a_i . x - b_i and FP64 ||a_i . x||^2; phase 2, thread per column,
// sum_i r_i a_ic (FMA chains of eight rows, then TwoSum).  Partials (hi, lo)
// per tile; R = rows per tile (<= 256).
__global__ void __launch_bounds__(256) kb_grad_tiles(const BVec* __restrict__ V, const Tile* __restrict__ tiles,
                                                     int ntiles, const int64_t* __restrict__ poff,
                                                     float2* __restrict__ part, double* __restrict__ pax2) {
    __shared__ float rsh[256];
    __shared__ double wsum[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const BVec& v = V[tl.p];
        if (!v.active) continue;
        const int64_t d = v.d;
        const float* __restrict__ x = v.xc;
        double ax2 = 0.0;
        for (int i = warp; i < tl.rows; i += 8) {
            const float* a = v.A + (tl.row0 + i) * d;
            Acc2 acc{0.f, 0.f};
            for (int64_t c = lane; c < d; c += 32) acc.add_prod(a[c], x[c]);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const Acc2 o = acc2_shfl_xor(acc, off);
                acc.add_pair(o.hi, o.lo);
            }
            if (lane == 0) {
                rsh[i] = __fadd_rn(__fsub_rn(acc.hi, v.b[tl.row0 + i]), acc.lo);
                const double s = (double)acc.hi + (double)acc.lo;
                ax2 += s * s;
            }
        }
        if (lane == 0) wsum[warp] = ax2;
        __syncthreads();
        float2* out = part + poff[t];
        for (int64_t c = threadIdx.x; c < d; c += 256) {
            Acc2 acc{0.f, 0.f};
            const float* a = v.A + tl.row0 * d + c;
            int i = 0;
            for (; i + 8 <= tl.rows; i += 8) {
                float s8 = __fmul_rn(rsh[i], a[(int64_t)i * d]);
#pragma unroll
                for (int q = 1; q < 8; ++q) s8 = __fmaf_rn(rsh[i + q], a[(int64_t)(i + q) * d], s8);
                acc.add(s8);
            }
            for (; i < tl.rows; ++i) acc.add(__fmul_rn(rsh[i], a[(int64_t)i * d]));
            out[c] = make_float2(acc.hi, acc.lo);
        }
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += wsum[w];
            pax2[t] = s;
        }
        __syncthreads();
    }
}

// gc = sum of the problem's tile partials + nu^2 xc, in a fixed order as a
// compensated binary32 pair (FP64 runs at a small fraction of the FP32 rate);
// sc[1] = sum pax2 (FP64, lane strides and a butterfly in warp 0).
// grid (ceil(dmax / 256), P).
__global__ void kb_grad_reduce(BVec* __restrict__ V, const int* __restrict__ tbeg, const int* __restrict__ tcnt,
                               const int64_t* __restrict__ poff, const float2* __restrict__ part,
                               const double* __restrict__ pax2) {
    const int p = blockIdx.y;
    BVec& v = V[p];
    if (!v.active || v.path >= 0) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int t0 = tbeg[p], nt = tcnt[p];
    if (c < v.d) {
        Acc2 a{0.f, 0.f};
        for (int t = 0; t < nt; ++t) {
            const float2 q = part[poff[t0 + t] + c];
            a.add_pair(q.x, q.y);
        }
        const float nh = (float)v.nu2;
        const float2 e = df_mul(v.xc[c], 0.f, nh, (float)(v.nu2 - (double)nh));
        a.add_pair(e.x, e.y);
        v.gc[c] = __fadd_rn(a.hi, a.lo);
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double s = 0.0;
        for (int t = threadIdx.x; t < nt; t += 32) s += pax2[t0 + t];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) v.sc[1] = s;
    }
}

// ---- gradient, shared A (multi right-hand side) ----
// X (d x K, row-major) <- the candidates of the group's problems.
__global__ void kb_gather_x(const BVec* __restrict__ V, const int* __restrict__ members, int K, int64_t d,
                            float* __restrict__ X) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= d * K) return;
    const int64_t c = e / K;
    const int k = (int)(e % K);
    const BVec& v = V[members[k]];
    X[e] = v.active ? v.xc[c] : 0.f;
}

constexpr int MR_T = 64;   // rows (or columns of A) per tile
constexpr int MR_K = 64;   // right-hand sides per pass
constexpr int MR_C = 32;   // inner chunk

// R = A X - B on tiles of 64 rows x 64 right-hand sides: FMA chains of eight
// along the inner dimension, each chain added to a (hi, lo) pair by TwoSum;
// r = (hi - b) + lo; per-tile FP64 sums of (hi + lo)^2 per right-hand side.
__global__ void __launch_bounds__(256) kb_mrhs_resid(const float* __restrict__ A, int64_t n, int64_t d,
                                                     const float* __restrict__ X, const float* __restrict__ B,
                                                     int K, float* __restrict__ R, double* __restrict__ pax2) {
    __shared__ float as[MR_C][MR_T + 1];
    __shared__ float xs[MR_C][MR_K + 1];
    __shared__ double red[16][MR_K];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t r0 = (int64_t)blockIdx.x * MR_T;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    for (int64_t c0 = 0; c0 < d; c0 += MR_C) {
        __syncthreads();
        for (int e = threadIdx.x; e < MR_T * MR_C; e += 256) {
            const int rr = e / MR_C, cc = e % MR_C;
            const int64_t row = r0 + rr, col = c0 + cc;
            as[cc][rr] = (row < n && col < d) ? A[row * d + col] : 0.f;
        }
        for (int e = threadIdx.x; e < MR_C * MR_K; e += 256) {
            const int cc = e / MR_K, k = e % MR_K;
            const int64_t col = c0 + cc;
            xs[cc][k] = (col < d && k < K) ? X[col * K + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q0 = 0; q0 < MR_C; q0 += 8) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float s8 = __fmul_rn(as[q0][ty + 16 * a], xs[q0][tx + 16 * b]);
#pragma unroll
                    for (int q = 1; q < 8; ++q) s8 = __fmaf_rn(as[q0 + q][ty + 16 * a], xs[q0 + q][tx + 16 * b], s8);
                    float s, e;
                    two_sum(hi[a][b], s8, s, e);
                    hi[a][b] = s;
                    lo[a][b] = __fadd_rn(lo[a][b], e);
                }
        }
    }
    double colsq[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t row = r0 + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = tx + 16 * b;
            if (row < n && k < K) {
                R[row * K + k] = __fadd_rn(__fsub_rn(hi[a][b], B[row * K + k]), lo[a][b]);
                const double s = (double)hi[a][b] + (double)lo[a][b];
                colsq[b] += s * s;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 4; ++b) red[ty][tx + 16 * b] = colsq[b];
    __syncthreads();
    if (threadIdx.x < MR_K) {
        double s = 0.0;
        for (int y = 0; y < 16; ++y) s += red[y][threadIdx.x];
        pax2[(size_t)blockIdx.x * MR_K + threadIdx.x] = s;
    }
}

// Gpart[split][c][k] = sum over the split's rows of A[row][c] R[row][k]
// (64 columns of A x 64 right-hand sides per CTA, chains of eight rows, TwoSum).
__global__ void __launch_bounds__(256) kb_mrhs_atr(const float* __restrict__ A, int64_t n, int64_t d,
                                                   const float* __restrict__ R, int K, int64_t rows_per_split,
                                                   float2* __restrict__ Gpart) {
    __shared__ float as[MR_C][MR_T + 1];
    __shared__ float rs[MR_C][MR_K + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t c0 = (int64_t)blockIdx.x * MR_T;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t i1 = min(n, i0 + rows_per_split);
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    for (int64_t r = i0; r < i1; r += MR_C) {
        __syncthreads();
        for (int e = threadIdx.x; e < MR_C * MR_T; e += 256) {
            const int rr = e / MR_T, cc = e % MR_T;
            const int64_t row = r + rr, col = c0 + cc;
            as[rr][cc] = (row < i1 && col < d) ? A[row * d + col] : 0.f;
        }
        for (int e = threadIdx.x; e < MR_C * MR_K; e += 256) {
            const int rr = e / MR_K, k = e % MR_K;
            const int64_t row = r + rr;
            rs[rr][k] = (row < i1 && k < K) ? R[row * K + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q0 = 0; q0 < MR_C; q0 += 8) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float s8 = __fmul_rn(as[q0][ty + 16 * a], rs[q0][tx + 16 * b]);
#pragma unroll
                    for (int q = 1; q < 8; ++q) s8 = __fmaf_rn(as[q0 + q][ty + 16 * a], rs[q0 + q][tx + 16 * b], s8);
                    float s, e;
                    two_sum(hi[a][b], s8, s, e);
                    hi[a][b] = s;
                    lo[a][b] = __fadd_rn(lo[a][b], e);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t col = c0 + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = tx + 16 * b;
            if (col < d && k < K)
                Gpart[((size_t)blockIdx.y * d + col) * K + k] = make_float2(hi[a][b], lo[a][b]);
        }
    }
}

// gc of member k = sum over splits + nu_k^2 xc (fixed order, compensated
// binary32 pair); sc[1] from the residual tiles (FP64, warp 0).
__global__ void kb_mrhs_reduce(BVec* __restrict__ V, const int* __restrict__ members, int K, int64_t d, int splits,
                               const float2* __restrict__ Gpart, int rtiles, const double* __restrict__ pax2) {
    const int k = blockIdx.y;
    BVec& v = V[members[k]];
    if (!v.active) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < d) {
        Acc2 a{0.f, 0.f};
        for (int sp = 0; sp < splits; ++sp) {
            const float2 q = Gpart[((size_t)sp * d + c) * K + k];
            a.add_pair(q.x, q.y);
        }
        const float nh = (float)v.nu2;
        const float2 e = df_mul(v.xc[c], 0.f, nh, (float)(v.nu2 - (double)nh));
        a.add_pair(e.x, e.y);
        v.gc[c] = __fadd_rn(a.hi, a.lo);
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double s = 0.0;
        for (int t = threadIdx.x; t < rtiles; t += 32) s += pax2[(size_t)t * MR_K + k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) v.sc[1] = s;
    }
}

// ---- batched apply steps (the single-problem kernels with a problem index) ----
// Steps run for problem blockIdx.y when its descriptor is on and, with
// V != NULL, the problem takes part in the round.
__device__ __forceinline__ bool skip(const BVec* V, int p) { return V != nullptr && !V[p].active; }

// Rows are grid-strided (one warp per row) so that the launch does not depend
// on the sketch sizes of the round.
__global__ void kb_rowdot(const ApplyDesc* __restrict__ D, const BVec* __restrict__ V, int step) {
    const BRow& o = D[blockIdx.y].row[step];
    if (!o.on || skip(V, blockIdx.y)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < o.rows; i += wstride) {
        const int64_t l0 = o.tri == 2 ? i : 0, l1 = o.tri == 1 ? i + 1 : o.cols;
        const float* row = o.M + i * o.ld;
        Acc2 acc{0.f, 0.f};
        if (o.xf) {
            for (int64_t l = l0 + lane; l < l1; l += 32) acc_mul(acc, row[l], make_float2(o.xf[l], 0.f));
        } else {
            for (int64_t l = l0 + lane; l < l1; l += 32) acc_mul(acc, row[l], o.x[l]);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const Acc2 q = acc2_shfl_xor(acc, off);
            acc.add_pair(q.hi, q.lo);
        }
        if (lane == 0) {
            float2 r = df_norm(acc.hi, acc.lo);
            if (o.add) r = df_add(r, o.add[i]);
            o.y[i] = r;
        }
    }
}

// grid (ceil(colsmax / 256), P, nchmax)
__global__ void kb_coldot_part(const ApplyDesc* __restrict__ D, const BVec* __restrict__ V, int step) {
    const BCol& o = D[blockIdx.y].col[step];
    if (!o.on || skip(V, blockIdx.y) || blockIdx.z >= o.nch) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.z * o.rpc;
    const int64_t j1 = o.rows < j0 + o.rpc ? o.rows : j0 + o.rpc;
    if (c >= o.cols) return;
    Acc2 acc{0.f, 0.f};
    for (int64_t j = j0; j < j1; ++j) acc_mul(acc, o.M[j * o.cols + c], o.x[j]);
    o.part[blockIdx.z * o.cols + c] = df_norm(acc.hi, acc.lo);
}

__global__ void kb_coldot_reduce(const ApplyDesc* __restrict__ D, const BVec* __restrict__ V, int step) {
    __shared__ double sm[256];
    const BCol& o = D[blockIdx.y].col[step];
    if (!o.on || skip(V, blockIdx.y)) return;
    if ((int64_t)blockIdx.x * blockDim.x >= o.cols) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double prod = 0.0;
    if (c < o.cols) {
        float2 sum = o.part[c];
        for (int q = 1; q < o.nch; ++q) sum = df_add(sum, o.part[q * o.cols + c]);
        if (o.w) o.w[c] = sum;
        if (o.g) {
            const double v = ((double)o.g[c] - ((double)sum.x + (double)sum.y)) * o.inv_nu2;
            o.gt[c] = (float)v;
            prod = (double)o.g[c] * v;
        }
    }
    if (o.g) {
        sm[threadIdx.x] = prod;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < 256; ++i) t += sm[i];
            o.rpart[blockIdx.x] = t;
        }
    }
}

__global__ void kb_elt(const ApplyDesc* __restrict__ D, const BVec* __restrict__ V, int step) {
    __shared__ double sm[256];
    const BElt& o = D[blockIdx.y].elt[step];
    if (!o.on || skip(V, blockIdx.y)) return;
    if ((int64_t)blockIdx.x * blockDim.x >= o.k) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o.op == 0) {
        if (i < o.k) o.t[i] = make_float2(o.g[i], 0.f);
    } else if (o.op == 1) {
        if (i < o.k) o.res[i] = df_add(o.t[i], df_neg(df_add(df_scale(o.u[i], o.nu2), o.w2[i])));
    } else {
        double prod = 0.0;
        if (i < o.k) {
            const double v = (double)o.u[i].x + (double)o.u[i].y;
            o.gt[i] = (float)v;
            prod = (double)o.g[i] * v;
        }
        sm[threadIdx.x] = prod;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < 256; ++q) t += sm[q];
            o.rpart[blockIdx.x] = t;
        }
    }
}

__global__ void kb_sum(const ApplyDesc* __restrict__ D, const BVec* __restrict__ V, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const BSum& o = D[p].sum;
    if (!o.on || skip(V, p)) return;
    double s = 0.0;
    for (int q = 0; q < o.count; ++q) s += o.rpart[q];
    *o.r = 0.5 * s;
}

// ---------------------------------------------------------------------------
// Host side

struct Params {
    double lam, Lam, mu_gd, c_gd;
};

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
    return p;
}

enum State { NEED_LEVEL = 0, READY = 1, DONE = 2 };

struct Prob {
    ihs_problem in;
    int64_t m, m_cap;
    int level;
    int state;
    int t;
    double r, r1, ax2, xx;
    float* SA;             // own sketch (independent problems)
    ihs_factor_t Fs;       // factor of the current level (storage from the batch's pool)
    ihs_factor_t* F;       // &Fs once built
    ihs_report rep;
    int lane;
    int group;             // shared-A group or -1
};

struct Group {             // problems sharing one A
    const float* A = nullptr;
    int64_t n = 0, d = 0;
    std::vector<int> members;
    std::map<int, float*> sa;   // level -> shared sketch
    float* X = nullptr;         // d x K candidates
    float* B = nullptr;         // n x K right-hand sides
    float* R = nullptr;         // n x K residuals
    float2* Gpart = nullptr;    // splits x d x K
    double* pax2 = nullptr;     // row tiles x K
    int* dmembers = nullptr;    // device copy of members
    int splits = 1;
    int64_t rows_per_split = 0;
};

// Sub-contexts (each with its own scratch arena), their streams and events,
// and the memory pool of level changes: created on the first batched solve of
// a context and kept until the context is destroyed, so that later batches
// find grown arenas and a warm pool.
struct Lanes {
    ihs_ctx* lane[kLanes] = {};
    cudaStream_t lstream[kLanes] = {};
    cudaEvent_t lev[kLanes] = {};
    cudaMemPool_t pool = nullptr;
};

struct Batch {
    ihs_ctx* ctx = nullptr;
    int P = 0;
    std::vector<Prob> pr;
    std::vector<Group> gr;
    ihs_ctx** lane = nullptr;       // the context's lanes
    cudaStream_t* lstream = nullptr;
    cudaEvent_t* lev = nullptr;
    cudaEvent_t mev = nullptr;
    cudaStream_t sm = nullptr;  // the batch's own stream (capturable; ordered after the context's stream)
    cudaMemPool_t pool = nullptr;   // stream-ordered pool for sketches and factors of level changes (the lanes')
    // device tables
    BVec* dV = nullptr;
    std::vector<BVec> hV;
    ApplyDesc* dD = nullptr;    // candidate apply (gc -> gtc)
    ApplyDesc* dR = nullptr;    // re-apply (g -> gt)
    std::vector<ApplyDesc> hD, hR;
    // independent gradient work list
    Tile* dT = nullptr;
    int ntiles = 0;
    int64_t* dpoff = nullptr;
    int* dtbeg = nullptr;
    int* dtcnt = nullptr;
    float2* tpart = nullptr;
    double* tpax2 = nullptr;
    int tile_rows = 0;
    int tile_grid = 1;
    // per-problem vectors and scalars
    void* arena = nullptr;
    double* sc_all = nullptr;
    double* hsc = nullptr;      // pinned copy of sc_all
    int64_t dmax = 1;
    cudaGraphExec_t graph = nullptr;
    bool have_graph = false;
    int64_t graph_kernels = 0;
    float ms_rounds = 0.f;
    double ms_levels = 0.0;     // wall time of level changes (sketches, factors, re-applies)
};

// b of the group's members as the n x K right-hand-side matrix.
__global__ void kb_gather_b(const BVec* __restrict__ V, const int* __restrict__ members, int K, int64_t n,
                            float* __restrict__ Bm) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    Bm[e] = V[members[e % K]].b[e / K];
}

void free_batch(Batch& B) {
    if (B.sm) cudaStreamSynchronize(B.sm);
    cudaStream_t fs = B.lstream ? B.lstream[0] : B.sm;
    for (auto& p : B.pr) {
        if (p.F) ihs_factor_release_pool(&p.Fs, fs);
        p.F = nullptr;
        if (p.SA) cudaFreeAsync(p.SA, fs);
    }
    for (auto& g : B.gr) {
        for (auto& kv : g.sa) cudaFreeAsync(kv.second, fs);
        cudaFree(g.X);
        cudaFree(g.B);
        cudaFree(g.R);
        cudaFree(g.Gpart);
        cudaFree(g.pax2);
        cudaFree(g.dmembers);
    }
    if (B.lstream)
        for (int l = 0; l < kLanes; ++l) cudaStreamSynchronize(B.lstream[l]);
    if (B.mev) cudaEventDestroy(B.mev);
    if (B.sm) cudaStreamDestroy(B.sm);
    cudaFree(B.dV);
    cudaFree(B.dD);
    cudaFree(B.dR);
    cudaFree(B.dT);
    cudaFree(B.dpoff);
    cudaFree(B.dtbeg);
    cudaFree(B.dtcnt);
    cudaFree(B.tpart);
    cudaFree(B.tpax2);
    cudaFree(B.arena);
    if (B.hsc) cudaFreeHost(B.hsc);
    if (B.have_graph) cudaGraphExecDestroy(B.graph);
}

// Descriptors of the apply of problem p (gin -> gout, decrement into r).
ApplyDesc make_apply(const Prob& p, const float* gin, float* gout, double* r) {
    ApplyDesc D;
    memset(&D, 0, sizeof(D));
    const ihs_factor_t* F = p.F;
    const int64_t k = F->k, d = F->d, m = F->m;
    const int64_t mx = std::max(m, d);
    float2* t = reinterpret_cast<float2*>(F->work);
    float2* v = t + k;
    float2* u = v + k;
    float2* res = u + k;
    float2* w = res + k;
    float2* w2 = w + mx;
    float2* part = w2 + mx;
    double* rpart = reinterpret_cast<double*>(part + 32 * mx);
    const int64_t chunks = std::min<int64_t>(32, std::max<int64_t>(1, m / 64));
    const int64_t rpc = ceil_div64(m, chunks);
    const int64_t nch = ceil_div64(m, rpc);
    const double nu2 = F->nu * F->nu;
    auto row = [&](int i, const float* M, int64_t rows, int64_t cols, int64_t ld, int tri, const float2* x,
                   const float* xf, const float2* add, float2* y) {
        D.row[i] = BRow{M, rows, cols, ld, tri, x, xf, add, y, 1};
    };
    auto col = [&](int i, const float2* x, float2* wout, const float* g, float* gt) {
        D.col[i] = BCol{F->SA, m, d, rpc, nch, x, part, wout, g, 1.0 / nu2, gt, rpart, 1};
    };
    if (F->woodbury) {
        row(0, F->SA, m, d, d, 0, nullptr, gin, nullptr, t);            // t = SA g
        row(1, F->X, k, k, k, 1, t, nullptr, nullptr, v);               // v = X t
    } else {
        D.elt[0] = BElt{0, k, gin, t, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, 1};   // t = g
        row(1, F->X, k, k, k, 1, nullptr, gin, nullptr, v);             // v = X g
    }
    row(2, F->XT, k, k, k, 2, v, nullptr, nullptr, u);                  // u0 = X^T v
    if (F->woodbury) {
        col(0, u, w, nullptr, nullptr);                                 // w = SA^T u0
        row(3, F->SA, m, d, d, 0, w, nullptr, nullptr, w2);             // w2 = SA w
    } else {
        row(3, F->SA, m, d, d, 0, u, nullptr, nullptr, w);              // w = SA u0
        col(1, w, w2, nullptr, nullptr);                                // w2 = SA^T w
    }
    D.elt[1] = BElt{1, k, nullptr, t, u, w2, res, nullptr, nu2, nullptr, 1};   // res = t - K u0
    row(4, F->X, k, k, k, 1, res, nullptr, nullptr, v);                 // v = X res
    row(5, F->XT, k, k, k, 2, v, nullptr, u, u);                        // u1 = u0 + X^T v
    if (F->woodbury) {
        col(2, u, nullptr, gin, gout);                                  // gt = (g - SA^T u1) / nu^2
    } else {
        D.elt[2] = BElt{2, k, gin, nullptr, u, nullptr, nullptr, gout, 0.0, rpart, 1};   // gt = u1
    }
    D.sum = BSum{rpart, (int)ceil_div64(d, 256), r, 1};
    return D;
}

// Enqueue the batched apply (descriptor table dtab, P problems) on stream s.
int enqueue_apply(Batch& B, const ApplyDesc* dtab, const BVec* V, cudaStream_t s) {
    const int P = B.P;
    // rows per problem are grid-strided: enough warps per problem to fill the
    // GPU about four times over, at most one per row of the widest matrix
    const int64_t want = std::max<int64_t>(1, ceil_div64(4 * (int64_t)B.ctx->sm_count, P));
    const unsigned rw = (unsigned)std::min<int64_t>(want, ceil_div64(B.dmax * 32, 256) * 64);
    const unsigned cb = (unsigned)ceil_div64(B.dmax, 256);
    const unsigned eb = (unsigned)ceil_div64(B.dmax, 256);
    auto rowk = [&](int st) -> int {
        kb_rowdot<<<dim3(rw, P), 256, 0, s>>>(dtab, V, st);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    auto colk = [&](int st) -> int {
        kb_coldot_part<<<dim3(cb, P, 32), 256, 0, s>>>(dtab, V, st);
        IHS_LAUNCH_CHECK();
        kb_coldot_reduce<<<dim3(cb, P), 256, 0, s>>>(dtab, V, st);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    auto eltk = [&](int st) -> int {
        kb_elt<<<dim3(eb, P), 256, 0, s>>>(dtab, V, st);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    IHS_TRY(rowk(0));    // Woodbury: t = SA g
    IHS_TRY(eltk(0));    // direct: t = g
    IHS_TRY(rowk(1));    // v = X t
    IHS_TRY(rowk(2));    // u0 = X^T v
    IHS_TRY(colk(0));    // Woodbury: w = SA^T u0
    IHS_TRY(rowk(3));    // Woodbury: w2 = SA w / direct: w = SA u0
    IHS_TRY(colk(1));    // direct: w2 = SA^T w
    IHS_TRY(eltk(1));    // res = t - K u0
    IHS_TRY(rowk(4));    // v = X res
    IHS_TRY(rowk(5));    // u1 = u0 + X^T v
    IHS_TRY(colk(2));    // Woodbury: gt = (g - SA^T u1) / nu^2
    IHS_TRY(eltk(2));    // direct: gt = u1
    kb_sum<<<(unsigned)ceil_div64(P, 128), 128, 0, s>>>(dtab, V, P);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

int enqueue_grad(Batch& B, cudaStream_t s) {
    const int P = B.P;
    if (B.ntiles > 0) {
        kb_grad_tiles<<<(unsigned)B.tile_grid, 256, 0, s>>>(B.dV, B.dT, B.ntiles, B.dpoff, B.tpart, B.tpax2);
        IHS_LAUNCH_CHECK();
        kb_grad_reduce<<<dim3((unsigned)ceil_div64(B.dmax, 256), P), 256, 0, s>>>(B.dV, B.dtbeg, B.dtcnt, B.dpoff,
                                                                                  B.tpart, B.tpax2);
        IHS_LAUNCH_CHECK();
    }
    for (auto& g : B.gr) {
        const int K = (int)g.members.size();
        kb_gather_x<<<(unsigned)ceil_div64(g.d * K, 256), 256, 0, s>>>(B.dV, g.dmembers, K, g.d, g.X);
        IHS_LAUNCH_CHECK();
        const int64_t rtiles = ceil_div64(g.n, MR_T);
        kb_mrhs_resid<<<(unsigned)rtiles, 256, 0, s>>>(g.A, g.n, g.d, g.X, g.B, K, g.R, g.pax2);
        IHS_LAUNCH_CHECK();
        kb_mrhs_atr<<<dim3((unsigned)ceil_div64(g.d, MR_T), (unsigned)g.splits), 256, 0, s>>>(
            g.A, g.n, g.d, g.R, K, g.rows_per_split, g.Gpart);
        IHS_LAUNCH_CHECK();
        kb_mrhs_reduce<<<dim3((unsigned)ceil_div64(g.d, 256), K), 256, 0, s>>>(B.dV, g.dmembers, K, g.d, g.splits,
                                                                              g.Gpart, (int)rtiles, g.pax2);
        IHS_LAUNCH_CHECK();
    }
    return IHS_OK;
}

// The round: candidate (with commit), gradient, apply, scalars.
int enqueue_round(Batch& B, cudaStream_t s) {
    const int P = B.P;
    kb_candidate<<<dim3((unsigned)ceil_div64(B.dmax, 256), P), 256, 0, s>>>(B.dV);
    IHS_LAUNCH_CHECK();
    kb_xfold<<<(unsigned)ceil_div64(P, 128), 128, 0, s>>>(B.dV, P);
    IHS_LAUNCH_CHECK();
    IHS_TRY(enqueue_grad(B, s));
    IHS_TRY(enqueue_apply(B, B.dD, B.dV, s));
    return IHS_OK;
}

// Build the independent problems' tile list for tile height R.
int build_tiles(Batch& B, int R) {
    std::vector<Tile> tl;
    std::vector<int64_t> poff;
    std::vector<int> tbeg(B.P, 0), tcnt(B.P, 0);
    int64_t off = 0;
    for (int p = 0; p < B.P; ++p) {
        const Prob& q = B.pr[p];
        tbeg[p] = (int)tl.size();
        if (q.group >= 0) continue;
        for (int64_t r0 = 0; r0 < q.in.n; r0 += R) {
            tl.push_back(Tile{p, r0, (int)std::min<int64_t>(R, q.in.n - r0)});
            poff.push_back(off);
            off += q.in.d;
        }
        tcnt[p] = (int)tl.size() - tbeg[p];
    }
    cudaFree(B.dT);
    cudaFree(B.dpoff);
    cudaFree(B.tpart);
    cudaFree(B.tpax2);
    B.dT = nullptr;
    B.dpoff = nullptr;
    B.tpart = nullptr;
    B.tpax2 = nullptr;
    B.ntiles = (int)tl.size();
    B.tile_rows = R;
    if (B.ntiles == 0) return IHS_OK;
    if (cudaMalloc(&B.dT, tl.size() * sizeof(Tile)) != cudaSuccess ||
        cudaMalloc(&B.dpoff, poff.size() * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&B.tpart, (size_t)off * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&B.tpax2, tl.size() * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return IHS_ENOMEM;
    }
    IHS_CUDA_TRY(cudaMemcpy(B.dT, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    IHS_CUDA_TRY(cudaMemcpy(B.dpoff, poff.data(), poff.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    IHS_CUDA_TRY(cudaMemcpy(B.dtbeg, tbeg.data(), B.P * sizeof(int), cudaMemcpyHostToDevice));
    IHS_CUDA_TRY(cudaMemcpy(B.dtcnt, tcnt.data(), B.P * sizeof(int), cudaMemcpyHostToDevice));
    B.tile_grid = (int)std::min<int64_t>(B.ntiles, 4 * (int64_t)B.ctx->sm_count);
    return IHS_OK;
}

// Autotune the tile height of the independent gradient: time each candidate
// on the actual problems (all active, x as candidate) and keep the fastest.
int autotune_tiles(Batch& B) {
    bool any = false;
    for (auto& q : B.pr) any |= q.group < 0;
    if (!any) return IHS_OK;
    const int cand[4] = {32, 64, 128, 256};
    float best = 1e30f;
    int best_r = 64;
    cudaStream_t s = B.sm;
    for (int R : cand) {
        IHS_TRY(build_tiles(B, R));
        for (int w = 0; w < 2; ++w) {
            kb_grad_tiles<<<(unsigned)B.tile_grid, 256, 0, s>>>(B.dV, B.dT, B.ntiles, B.dpoff, B.tpart, B.tpax2);
            IHS_LAUNCH_CHECK();
        }
        IHS_CUDA_TRY(cudaEventRecord(B.ctx->ev[0], s));
        for (int w = 0; w < 3; ++w) {
            kb_grad_tiles<<<(unsigned)B.tile_grid, 256, 0, s>>>(B.dV, B.dT, B.ntiles, B.dpoff, B.tpart, B.tpax2);
            IHS_LAUNCH_CHECK();
        }
        IHS_CUDA_TRY(cudaEventRecord(B.ctx->ev[1], s));
        IHS_CUDA_TRY(cudaEventSynchronize(B.ctx->ev[1]));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, B.ctx->ev[0], B.ctx->ev[1]);
        if (ms < best) {
            best = ms;
            best_r = R;
        }
    }
    return build_tiles(B, best_r);
}

// Sketch and factor the problems in NEED_LEVEL state at their (new) m, on the
// lanes; shared-A groups sketch each level once.  Then re-apply the new
// factors to the current gradients (gt_t and r_t).
int level_change_impl(Batch& B, bool first);

int level_change(Batch& B, bool first) {
    IHS_CUDA_TRY(cudaStreamSynchronize(B.sm));
    const auto t0 = std::chrono::steady_clock::now();
    const int st = level_change_impl(B, first);
    cudaStreamSynchronize(B.sm);
    B.ms_levels += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

int level_change_impl(Batch& B, bool first) {
    ihs_ctx* ctx = B.ctx;
    const ihs_params& prm = ctx->p;
    std::vector<int> todo;
    for (int p = 0; p < B.P; ++p)
        if (B.pr[p].state == NEED_LEVEL) todo.push_back(p);
    if (todo.empty()) return IHS_OK;
    // the lanes start after everything queued on the main stream
    IHS_CUDA_TRY(cudaEventRecord(B.mev, B.sm));
    for (int l = 0; l < kLanes; ++l) IHS_CUDA_TRY(cudaStreamWaitEvent(B.lstream[l], B.mev, 0));
    // shared sketches first (lane 0), one per (group, level)
    for (int p : todo) {
        Prob& q = B.pr[p];
        if (q.group < 0) continue;
        Group& g = B.gr[q.group];
        if (g.sa.count(q.level)) continue;
        void* SA0 = nullptr;
        if (cudaMallocFromPoolAsync(&SA0, (size_t)q.m * g.d * sizeof(float), B.pool, B.lstream[0]) != cudaSuccess) {
            cudaGetLastError();
            return IHS_ENOMEM;
        }
        float* SA = static_cast<float*>(SA0);
        IHS_TRY(ihs_sketch_enqueue(B.lane[0], g.A, g.n, g.d, q.m, prm.kind, prm.seed, prm.nested ? 0 : q.level, SA));
        g.sa[q.level] = SA;
    }
    IHS_CUDA_TRY(cudaEventRecord(B.lev[0], B.lstream[0]));
    // one host thread per lane enqueues the sketches and factorisations of its
    // problems (each factorisation is dozens of small launches)
    auto work = [&](int p, int l) -> int {
        Prob& q = B.pr[p];
        ihs_ctx* lc = B.lane[l];
        if (q.group >= 0) IHS_CUDA_TRY(cudaStreamWaitEvent(B.lstream[l], B.lev[0], 0));
        if (q.F) {
            ihs_factor_release_pool(&q.Fs, B.lstream[l]);
            q.F = nullptr;
        }
        const float* SA;
        if (q.group >= 0) {
            SA = B.gr[q.group].sa.find(q.level)->second;
        } else {
            if (q.SA) cudaFreeAsync(q.SA, B.lstream[l]);
            q.SA = nullptr;
            void* sa = nullptr;
            if (cudaMallocFromPoolAsync(&sa, (size_t)q.m * q.in.d * sizeof(float), B.pool, B.lstream[l]) !=
                cudaSuccess) {
                cudaGetLastError();
                return IHS_ENOMEM;
            }
            q.SA = static_cast<float*>(sa);
            IHS_TRY(ihs_sketch_enqueue(lc, q.in.A, q.in.n, q.in.d, q.m, prm.kind, prm.seed, prm.nested ? 0 : q.level,
                                       q.SA));
            SA = q.SA;
        }
        IHS_TRY(ihs_factor_alloc_pool(lc, B.pool, SA, q.m, q.in.d, q.in.nu, &q.Fs));
        q.F = &q.Fs;
        IHS_TRY(ihs_factor_enqueue(lc, q.F));
        q.lane = l;
        if (!first) {
            if (q.rep.n_levels < IHS_REPORT_MAX_LEVELS) q.rep.m_levels[q.rep.n_levels] = q.m;
            q.rep.n_levels++;
        } else {
            q.rep.m_levels[0] = q.m;
            q.rep.n_levels = 1;
        }
        B.hD[p] = make_apply(q, B.hV[p].gc, B.hV[p].gtc, B.hV[p].sc + 0);
        B.hR[p] = make_apply(q, B.hV[p].g, B.hV[p].gt, B.hV[p].sc + 0);
        return IHS_OK;
    };
    std::vector<int> lane_st(kLanes, IHS_OK);
    std::vector<std::string> lane_msg(kLanes);
    {
        std::vector<std::thread> th;
        const int nl = (int)std::min<size_t>(kLanes, todo.size());
        for (int l = 0; l < nl; ++l) {
            th.emplace_back([&, l]() {
                const cudaError_t e = cudaSetDevice(ctx->device);
                if (e != cudaSuccess) {
                    ihs_set_last_cuda_error(e, "lane thread device", __FILE__, __LINE__);
                    lane_st[l] = IHS_ECUDA;
                    return;
                }
                for (size_t i = l; i < todo.size(); i += nl) {
                    const int st = work(todo[i], l);
                    if (st != IHS_OK) {
                        lane_st[l] = st;
                        lane_msg[l] = ihs_last_error();   // thread-local: carried to the caller below
                        return;
                    }
                }
            });
        }
        for (auto& t : th) t.join();
    }
    for (int l = 0; l < kLanes; ++l) {
        if (lane_st[l] != IHS_OK) {
            ihs_set_error(lane_msg[l].c_str());
            return lane_st[l];
        }
    }
    for (int l = 0; l < kLanes; ++l) {
        IHS_CUDA_TRY(cudaEventRecord(B.lev[l], B.lstream[l]));
        IHS_CUDA_TRY(cudaStreamWaitEvent(B.sm, B.lev[l], 0));
    }
    for (int l = 0; l < kLanes; ++l) IHS_TRY(ihs_check_status(B.lane[l]));
    // release sketches of shared levels no member uses any more
    for (auto& g : B.gr) {
        for (auto it = g.sa.begin(); it != g.sa.end();) {
            bool used = false;
            for (int p : g.members) used |= B.pr[p].level == it->first && B.pr[p].state != DONE;
            if (!used) {
                cudaFreeAsync(it->second, B.lstream[0]);
                it = g.sa.erase(it);
            } else {
                ++it;
            }
        }
    }
    IHS_CUDA_TRY(cudaMemcpyAsync(B.dD, B.hD.data(), B.P * sizeof(ApplyDesc), cudaMemcpyHostToDevice, B.sm));
    if (!first) {
        // re-apply to the current gradient for the problems that changed level
        std::vector<ApplyDesc> sel(B.P);
        memset(sel.data(), 0, B.P * sizeof(ApplyDesc));
        for (int p : todo) sel[p] = B.hR[p];
        IHS_CUDA_TRY(cudaMemcpyAsync(B.dR, sel.data(), B.P * sizeof(ApplyDesc), cudaMemcpyHostToDevice,
                                     B.sm));
        IHS_TRY(enqueue_apply(B, B.dR, nullptr, B.sm));
        IHS_CUDA_TRY(cudaMemcpyAsync(B.hsc, B.sc_all, (size_t)B.P * 8 * sizeof(double), cudaMemcpyDeviceToHost,
                                     B.sm));
        IHS_CUDA_TRY(cudaStreamSynchronize(B.sm));
        for (int p : todo) {
            B.pr[p].r = B.hsc[8 * p + 0];
            B.pr[p].state = READY;
        }
    } else {
        for (int p : todo) B.pr[p].state = READY;
    }
    return IHS_OK;
}

int run_round(Batch& B) {
    cudaStream_t s = B.sm;
    IHS_CUDA_TRY(cudaMemcpyAsync(B.dV, B.hV.data(), B.P * sizeof(BVec), cudaMemcpyHostToDevice, s));
    if (!B.have_graph) {
        cudaGraph_t g;
        IHS_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int st = enqueue_round(B, s);
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        IHS_TRY(st);
        if (e != cudaSuccess) {
            ihs_set_last_cuda_error(e, "stream capture of the batched round", __FILE__, __LINE__);
            return IHS_ECUDA;
        }
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        B.graph_kernels = (int64_t)nodes;
        const cudaError_t e2 = cudaGraphInstantiate(&B.graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            ihs_set_last_cuda_error(e2, "instantiating the batched round", __FILE__, __LINE__);
            return IHS_ECUDA;
        }
        B.have_graph = true;
    }
    IHS_CUDA_TRY(cudaEventRecord(B.ctx->ev[2], s));
    IHS_CUDA_TRY(cudaGraphLaunch(B.graph, s));
    ihs_count_launches(B.graph_kernels);
    IHS_CUDA_TRY(cudaEventRecord(B.ctx->ev[3], s));
    IHS_CUDA_TRY(cudaMemcpyAsync(B.hsc, B.sc_all, (size_t)B.P * 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    IHS_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, B.ctx->ev[2], B.ctx->ev[3]);
    B.ms_rounds += ms;
    return IHS_OK;
}

int solve_batched(Batch& B, double tol) {
    ihs_ctx* ctx = B.ctx;
    const ihs_params& prm = ctx->p;
    const Params pp = make_params(prm.kind, prm.rho, prm.eta);
    // level of every problem at m_init
    for (auto& q : B.pr) {
        q.m = std::min<int64_t>(q.in.m_init > 0 ? q.in.m_init : prm.m_init, q.m_cap);
        q.level = 0;
        while (((int64_t)1 << q.level) < q.m) ++q.level;
        q.state = NEED_LEVEL;
    }
    IHS_TRY(level_change(B, true));
    for (int p = 0; p < B.P; ++p) {
        B.hV[p].active = 1;
        B.hV[p].commit = 0;
        B.hV[p].mu = 0.f;
    }
    IHS_CUDA_TRY(cudaMemcpyAsync(B.dV, B.hV.data(), B.P * sizeof(BVec), cudaMemcpyHostToDevice, B.sm));
    IHS_TRY(autotune_tiles(B));
    // evaluate at x_1: mu = 0, every problem commits its first candidate
    for (int p = 0; p < B.P; ++p) {
        B.hV[p].mu = 0.f;
        B.hV[p].active = 1;
        B.hV[p].commit = 0;
    }
    IHS_TRY(run_round(B));
    for (int p = 0; p < B.P; ++p) {
        Prob& q = B.pr[p];
        q.r = q.r1 = B.hsc[8 * p + 0];
        q.ax2 = B.hsc[8 * p + 1];
        q.xx = B.hsc[8 * p + 2];
        q.rep.r1 = q.r1;
        q.rep.grad_passes = 1;
        q.t = 1;
        B.hV[p].commit = 1;   // x stays, g and gt take the evaluated values
    }
    while (true) {
        int n_active = 0;
        for (int p = 0; p < B.P; ++p) {
            Prob& q = B.pr[p];
            BVec& v = B.hV[p];
            v.active = 0;
            if (q.state == DONE) continue;
            if (!isfinite(q.r) || !isfinite(q.ax2)) {
                q.rep.status = IHS_ENONFINITE;
                q.state = DONE;
                continue;
            }
            if (q.r <= 0.0 || sqrt(2.0 * pp.Lam * q.r) <= tol * sqrt(q.ax2 + q.in.nu * q.in.nu * q.xx)) {
                q.rep.status = IHS_OK;
                q.state = DONE;
                continue;
            }
            if (q.t >= prm.max_iter) {
                q.rep.status = IHS_EMAXITER;
                q.state = DONE;
                continue;
            }
            v.active = 1;
            v.mu = (float)pp.mu_gd;
            ++n_active;
        }
        if (n_active == 0) break;
        IHS_TRY(run_round(B));
        bool any_level = false;
        for (int p = 0; p < B.P; ++p) {
            Prob& q = B.pr[p];
            BVec& v = B.hV[p];
            if (!v.active) {
                v.commit = 0;
                continue;
            }
            q.rep.grad_passes++;
            const double rc = B.hsc[8 * p + 0];
            v.commit = 0;
            if (!isfinite(rc)) {
                q.rep.status = IHS_ENONFINITE;
                q.state = DONE;
                continue;
            }
            const double ratio = rc / q.r;
            if (ratio <= pp.c_gd || q.m >= q.m_cap) {
                if (!(ratio <= pp.c_gd)) q.rep.flags |= 1;
                v.commit = 1;
                q.r = rc;
                q.ax2 = B.hsc[8 * p + 1];
                q.xx = B.hsc[8 * p + 2];
                q.rep.accepted_gd++;
                ++q.t;
            } else if (prm.floor > 0.0 && q.r <= prm.floor * prm.floor * q.r1) {
                q.rep.flags |= 2;
                q.rep.status = IHS_OK;
                q.state = DONE;
            } else {
                q.rep.rejected++;
                q.m = std::min<int64_t>(2 * q.m, q.m_cap);
                q.level += 1;
                q.state = NEED_LEVEL;
                any_level = true;
            }
        }
        if (any_level) {
            // accepted candidates of this round are committed by the next round's
            // first kernel; the re-apply below reads g of problems that did not move
            IHS_TRY(level_change(B, false));
        }
    }
    // final commit of the last accepted candidates
    bool pending = false;
    for (int p = 0; p < B.P; ++p) {
        pending |= B.hV[p].commit != 0;
        B.hV[p].active = B.hV[p].commit;
        B.hV[p].mu = 0.f;
    }
    if (pending) {
        IHS_CUDA_TRY(cudaMemcpyAsync(B.dV, B.hV.data(), B.P * sizeof(BVec), cudaMemcpyHostToDevice, B.sm));
        kb_candidate<<<dim3((unsigned)ceil_div64(B.dmax, 256), B.P), 256, 0, B.sm>>>(B.dV);
        IHS_LAUNCH_CHECK();
        IHS_CUDA_TRY(cudaStreamSynchronize(B.sm));
    }
    for (auto& q : B.pr) {
        q.rep.iterations = q.t;
        q.rep.m_final = q.m;
        q.rep.r_final = q.r;
        q.rep.axnorm_final = sqrt(q.ax2 + q.in.nu * q.in.nu * q.xx);
        q.rep.ms_iterate = B.ms_rounds;
        q.rep.ms_sketch = B.ms_levels;
    }
    return IHS_OK;
}

}  // namespace

void ihs_lanes_destroy(void* lanes) {
    Lanes* L = static_cast<Lanes*>(lanes);
    if (!L) return;
    for (int l = 0; l < kLanes; ++l) {
        if (L->lane[l]) {
            cudaStreamSynchronize(L->lstream[l]);
            ihs_ctx_destroy(L->lane[l]);
        }
        if (L->lstream[l]) cudaStreamDestroy(L->lstream[l]);
        if (L->lev[l]) cudaEventDestroy(L->lev[l]);
    }
    if (L->pool) cudaMemPoolDestroy(L->pool);
    delete L;
}

extern "C" int ihs_solve_batched(ihs_ctx* ctx, const ihs_problem* probs_h, int32_t count, double tol,
                                 ihs_report* reps_h) {
    IhsRange range("ihs_solve_batched");
    if (!ctx || !probs_h || count < 1) return IHS_EINVAL;
    if (ctx->p.variant != IHS_VARIANT_GD) {
        ihs_set_error("ihs_solve_batched runs the gradient-IHS variant only");
        return IHS_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        const ihs_problem& q = probs_h[i];
        if (!q.A || !q.b || !q.x || q.n < 1 || q.d < 1 || q.n < q.d || !(q.nu > 0.0) || !isfinite(q.nu))
            return IHS_EINVAL;
        if (q.m_init < 0 || (q.m_init > 0 && (q.m_init & (q.m_init - 1)) != 0)) return IHS_EINVAL;
    }
    if (!(tol > 0.0)) tol = ctx->p.tol;
    Batch B;
    B.ctx = ctx;
    B.P = count;
    B.pr.resize(count);
    B.hV.resize(count);
    B.hD.resize(count);
    B.hR.resize(count);
    int st = IHS_OK;
    // false (and the error recorded for ihs_last_error) when e is not cudaSuccess
    auto ok = [](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return true;
        ihs_set_last_cuda_error(e, what, __FILE__, __LINE__);
        return false;
    };
    do {
        // the batch runs on its own stream, after the work queued on the context's
        if (!ok(cudaStreamCreateWithFlags(&B.sm, cudaStreamNonBlocking), "batch stream") ||
            !ok(cudaEventCreateWithFlags(&B.mev, cudaEventDisableTiming), "batch event") ||
            !ok(cudaEventRecord(B.mev, ctx->stream), "record on the context stream") ||
            !ok(cudaStreamWaitEvent(B.sm, B.mev, 0), "batch stream wait")) {
            st = IHS_ECUDA;
            break;
        }
        // groups of at least two problems with the same A (and shape), at most MR_K each
        std::map<const float*, std::vector<int>> byA;
        for (int i = 0; i < count; ++i) byA[probs_h[i].A].push_back(i);
        for (int i = 0; i < count; ++i) {
            Prob& p = B.pr[i];
            memset(&p.rep, 0, sizeof(p.rep));
            p.in = probs_h[i];
            p.m_cap = ctx->p.kind == IHS_SKETCH_SRHT ? next_pow2_64(p.in.n) : p.in.n;
            p.SA = nullptr;
            p.F = nullptr;
            p.group = -1;
            p.lane = 0;
        }
        for (auto& kv : byA) {
            std::vector<int> same;
            for (int i : kv.second)
                if (probs_h[i].n == probs_h[kv.second[0]].n && probs_h[i].d == probs_h[kv.second[0]].d) same.push_back(i);
            for (size_t c0 = 0; c0 + 1 < same.size(); c0 += MR_K) {
                const size_t c1 = std::min(same.size(), c0 + (size_t)MR_K);
                if (c1 - c0 < 2) break;
                Group g;
                g.A = kv.first;
                g.n = probs_h[same[c0]].n;
                g.d = probs_h[same[c0]].d;
                for (size_t j = c0; j < c1; ++j) {
                    g.members.push_back(same[j]);
                    B.pr[same[j]].group = (int)B.gr.size();
                }
                B.gr.push_back(g);
            }
        }
        for (auto& q : B.pr) B.dmax = std::max(B.dmax, q.in.d);
        // per-problem vectors: xc, g, gc, gt, gtc (d each) + candidate partials
        std::vector<size_t> off(count);
        size_t tot = 0;
        for (int i = 0; i < count; ++i) {
            off[i] = tot;
            const size_t vb = ((size_t)B.pr[i].in.d * sizeof(float) + 255) & ~(size_t)255;
            tot += 5 * vb + (((size_t)ceil_div64(B.pr[i].in.d, 256) * sizeof(double) + 255) & ~(size_t)255);
        }
        if (cudaMalloc(&B.arena, tot) != cudaSuccess ||
            cudaMalloc(&B.sc_all, (size_t)count * 8 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&B.hsc, (size_t)count * 8 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&B.dV, count * sizeof(BVec)) != cudaSuccess ||
            cudaMalloc(&B.dD, count * sizeof(ApplyDesc)) != cudaSuccess ||
            cudaMalloc(&B.dR, count * sizeof(ApplyDesc)) != cudaSuccess ||
            cudaMalloc(&B.dtbeg, count * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&B.dtcnt, count * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            st = IHS_ENOMEM;
            break;
        }
        for (int i = 0; i < count; ++i) {
            char* base = static_cast<char*>(B.arena) + off[i];
            const size_t vb = ((size_t)B.pr[i].in.d * sizeof(float) + 255) & ~(size_t)255;
            BVec& v = B.hV[i];
            memset(&v, 0, sizeof(v));
            v.A = B.pr[i].in.A;
            v.b = B.pr[i].in.b;
            v.x = B.pr[i].in.x;
            v.xc = reinterpret_cast<float*>(base);
            v.g = reinterpret_cast<float*>(base + vb);
            v.gc = reinterpret_cast<float*>(base + 2 * vb);
            v.gt = reinterpret_cast<float*>(base + 3 * vb);
            v.gtc = reinterpret_cast<float*>(base + 4 * vb);
            v.sc = B.sc_all + 8 * i;
            v.xpart = reinterpret_cast<double*>(base + 5 * vb);
            v.n = B.pr[i].in.n;
            v.d = B.pr[i].in.d;
            v.nu2 = B.pr[i].in.nu * B.pr[i].in.nu;
            v.path = B.pr[i].group;
            v.col = -1;
        }
        if (!ok(cudaMemsetAsync(B.arena, 0, tot, B.sm), "arena clear") ||
            !ok(cudaMemsetAsync(B.sc_all, 0, (size_t)count * 8 * sizeof(double), B.sm), "scalars clear") ||
            !ok(cudaMemcpyAsync(B.dV, B.hV.data(), count * sizeof(BVec), cudaMemcpyHostToDevice, B.sm),
                "descriptor upload")) {
            st = IHS_ECUDA;
            break;
        }
        // shared-A groups: members, right-hand sides, work buffers
        for (size_t gi = 0; gi < B.gr.size() && st == IHS_OK; ++gi) {
            Group& g = B.gr[gi];
            const int K = (int)g.members.size();
            for (int k = 0; k < K; ++k) B.hV[g.members[k]].col = k;
            const int64_t rtiles = ceil_div64(g.n, MR_T);
            const int64_t ctiles = ceil_div64(g.d, MR_T);
            g.splits = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(2 * (int64_t)ctx->sm_count, ctiles),
                                                                    ceil_div64(g.n, 1024)));
            g.rows_per_split = ceil_div64(ceil_div64(g.n, g.splits), MR_C) * MR_C;
            g.splits = (int)ceil_div64(g.n, g.rows_per_split);
            if (cudaMalloc(&g.X, (size_t)g.d * K * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&g.B, (size_t)g.n * K * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&g.R, (size_t)g.n * K * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&g.Gpart, (size_t)g.splits * g.d * K * sizeof(float2)) != cudaSuccess ||
                cudaMalloc(&g.pax2, (size_t)rtiles * MR_K * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&g.dmembers, K * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                st = IHS_ENOMEM;
                break;
            }
            if (!ok(cudaMemcpy(g.dmembers, g.members.data(), K * sizeof(int), cudaMemcpyHostToDevice), "members")) {
                st = IHS_ECUDA;
                break;
            }
            kb_gather_b<<<(unsigned)ceil_div64(g.n * K, 256), 256, 0, B.sm>>>(B.dV, g.dmembers, K, g.n, g.B);
            if (!ok(cudaGetLastError(), "gather of right-hand sides")) {
                st = IHS_ECUDA;
                break;
            }
        }
        if (st != IHS_OK) break;
        // lanes (created once per context)
        if (!ctx->lanes) {
            Lanes* L = new (std::nothrow) Lanes;
            if (!L) {
                st = IHS_ENOMEM;
                break;
            }
            ctx->lanes = L;
            for (int l = 0; l < kLanes && st == IHS_OK; ++l) {
                if (!ok(cudaStreamCreateWithFlags(&L->lstream[l], cudaStreamNonBlocking), "lane stream") ||
                    !ok(cudaEventCreateWithFlags(&L->lev[l], cudaEventDisableTiming), "lane event")) {
                    st = IHS_ECUDA;
                    break;
                }
                st = ihs_ctx_create(&L->lane[l], L->lstream[l], &ctx->p);
                if (st == IHS_OK) L->lane[l]->no_coop = 1;   // 32 lanes factor side by side
            }
            if (st == IHS_OK) {
                cudaMemPoolProps pp;
                memset(&pp, 0, sizeof(pp));
                pp.allocType = cudaMemAllocationTypePinned;
                pp.handleTypes = cudaMemHandleTypeNone;
                pp.location.type = cudaMemLocationTypeDevice;
                pp.location.id = ctx->device;
                if (!ok(cudaMemPoolCreate(&L->pool, &pp), "memory pool")) {
                    st = IHS_ECUDA;
                } else {
                    uint64_t keep = ~0ull;   // keep freed blocks for reuse
                    cudaMemPoolSetAttribute(L->pool, cudaMemPoolAttrReleaseThreshold, &keep);
                }
            }
            if (st != IHS_OK) {
                ihs_lanes_destroy(L);
                ctx->lanes = nullptr;
                break;
            }
        }
        {
            Lanes* L = static_cast<Lanes*>(ctx->lanes);
            B.lane = L->lane;
            B.lstream = L->lstream;
            B.lev = L->lev;
            B.pool = L->pool;
            for (int l = 0; l < kLanes; ++l) L->lane[l]->p = ctx->p;   // the batch's parameters
        }
        st = solve_batched(B, tol);
    } while (0);
    if (reps_h)
        for (int i = 0; i < count; ++i) reps_h[i] = B.pr[i].rep;
    free_batch(B);
    if (st == IHS_OK) {
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return st;
}
