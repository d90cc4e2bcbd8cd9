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
            int64_t grow0 /* global index of A's row 0, a multiple of Q */,
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
            const uint64_t i = (uint64_t)(grow0 + p * Q + q);
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
            const float sv = (__popcll(hi & (uint64_t)(grow0 / Q + p)) & 1) ? -v : v;
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

// (x, y) <- (x + y, x - y) lane-wise on two packed FP32x2 registers (sm_100+:
// two IEEE binary32 operations per instruction, each rounded as a scalar one).
__device__ __forceinline__ void bfly_x2(unsigned long long& x, unsigned long long& y) {
    unsigned long long s, t;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(x), "l"(y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x), "l"(y));
    x = s;
    y = t;
}

// 32-point unnormalised WHT in registers.  The stages on index bits 0..3 run
// on the packed pairs (v[i], v[i + 16]), the stage on bit 4 last on scalars;
// every output is the same sequence of rounded additions as the radix-2
// stages taken in the order h = 1, 2, 4, 8, 16.
__device__ __forceinline__ void wht32(float (&v)[32]) {
    unsigned long long q[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) asm("mov.b64 %0, {%1, %2};" : "=l"(q[i]) : "f"(v[i]), "f"(v[i + 16]));
#pragma unroll
    for (int h = 1; h < 16; h <<= 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if ((i & h) == 0) bfly_x2(q[i], q[i + h]);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(q[i]));
        v[i] = __fadd_rn(a, b);
        v[i + 16] = __fsub_rn(a, b);
    }
}

// Shared memory of k_srht_r32: two TMA stages of 1024 x 16 floats, the padded
// transpose buffer, sign words, two mbarriers, one (T byte offset, block-index
// bits) pair per accumulator slot (32 MA slots; slots >= m point at T[0]).
constexpr size_t kR32Stage = 1024 * kR32C * sizeof(float);   // 64 KiB
__host__ __device__ inline size_t r32_smem_bytes(int ma) {
    return 2 * kR32Stage + (size_t)32 * kR32Stride * sizeof(float) + 32 * sizeof(uint32_t) + 2 * sizeof(uint64_t) +
           (size_t)32 * ma * sizeof(int2);
}

// MA accumulators per thread: this launch handles m <= 32 MA selected rows;
// thread (c, ql) accumulates rows ql + 32 i (i < MA) of column c in registers.
// Blocks of 1024 x 16 arrive by TMA (four 256-row boxes) into a two-stage
// ring; rows >= n and columns >= d read as zero.
template <int MA>
__global__ void __launch_bounds__(kR32T, 1)
k_srht_r32(const __grid_constant__ CUtensorMap amap, int d, int64_t m, int64_t m_total, int64_t row_off, int64_t P,
           int PG, const int32_t* __restrict__ rows, uint32_t level, uint32_t k0, uint32_t k1, int64_t gblk,
           unsigned* status,
           float* __restrict__ out /* PG x m_total x d partials; this launch writes rows [row_off, row_off + m) */) {
    extern __shared__ __align__(128) unsigned char smraw[];
    float* stage = reinterpret_cast<float*>(smraw);                                   // 2 x 1024 x 16
    float* T = reinterpret_cast<float*>(smraw + 2 * kR32Stage);                      // 32 x 528
    uint32_t* sbits = reinterpret_cast<uint32_t*>(T + 32 * kR32Stride);              // 32 sign words
    uint64_t* full = reinterpret_cast<uint64_t*>(sbits + 32);                        // 2 mbarriers
    int2* sel = reinterpret_cast<int2*>(full + 2);                                  // 32 MA slots
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
    for (int j = tid; j < 32 * MA; j += kR32T) {
        int2 e = make_int2(0, 0);
        if (j < m) {
            const uint32_t r = (uint32_t)rows[j];
            const uint32_t lo = r & 1023u;
            e.x = (int)(((lo >> 5) * kR32Stride + (lo & 31u) * 16) * sizeof(float));
            e.y = (int)(r >> 10);
        }
        sel[j] = e;
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
            const uint4 w = srht_sign_words((uint64_t)(gblk + p) * 8 + tid, level, k0, k1);
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
        // every slot accumulates (slots >= m read T[0] and are never stored):
        // no branches on the gather path
        const int pb = (int)(gblk + p);   // global 1024-row block index
        const unsigned char* Tc = reinterpret_cast<const unsigned char*>(T + c);
#pragma unroll
        for (int i = 0; i < MA; ++i) {
            const int2 e = sel[ql + 32 * i];
            const float val = *reinterpret_cast<const float*>(Tc + e.x);
            acc[i] += __int_as_float(__float_as_int(val) ^ (int)((unsigned)__popc(e.y & pb) << 31));
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

// Small-m variant: blocks of 512 rows (H_512 = H_32 (x) H_16, row 16 k + ql
// with k the high five and ql the low four index bits), CTAs of 256 threads
// = 16 columns x 16 ql, two CTAs per SM so that one CTA's shared-memory phases
// overlap the other's arithmetic.  Each TMA stage (512 x 16 floats) is also
// its block's transpose buffer: Z[K][ql] and then Y[16 K + L] sit at float
// offset q5_pos(K, L) + c, swizzled (L ^ (K & 1)) so that both the transposed
// reads and writes are free of bank conflicts.  The selected rows are then
// summed with the sign (-1)^popc(hi & q) of their high bits hi = r >> 9
// against the 512-row block index q (H_n = H_{n/512} (x) H_512).  The sign of
// row 512 q + 16 k + ql is bit 16 (q & 1) + (k >> 1) of word 16 (k & 1) + ql of
// the 1024-row block q >> 1: the same signs as every other SRHT path.
constexpr int kQ5C = 16, kQ5T = 256, kQ5S = 3;
constexpr size_t kQ5Stage = 512 * kQ5C * sizeof(float);   // 32 KiB
__host__ __device__ constexpr int q5_pos(int K, int L) { return K * 256 + ((L ^ (K & 1)) * 16); }
__host__ __device__ inline size_t q5_smem_bytes(int ma) {
    return kQ5S * kQ5Stage + 32 * sizeof(uint32_t) + kQ5S * sizeof(uint64_t) + (size_t)16 * ma * sizeof(int2);
}

// 16-point WHTs of two independent vectors a and b, packed lane-wise: every
// stage on (a[i], b[i]) pairs, stages in the order h = 1, 2, 4, 8.
__device__ __forceinline__ void wht16_pair(float (&a)[16], float (&b)[16]) {
    unsigned long long q[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) asm("mov.b64 %0, {%1, %2};" : "=l"(q[i]) : "f"(a[i]), "f"(b[i]));
#pragma unroll
    for (int h = 1; h < 16; h <<= 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if ((i & h) == 0) bfly_x2(q[i], q[i + h]);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) asm("mov.b64 {%0, %1}, %2;" : "=f"(a[i]), "=f"(b[i]) : "l"(q[i]));
}

// MA accumulators per thread: m <= 16 MA selected rows, thread (c, ql)
// accumulating rows ql + 16 i of column c; slots >= m read T[0] and are never
// stored.  Rows >= n and columns >= d arrive as zeros from the TMA.
template <int MA>
__global__ void __launch_bounds__(kQ5T, 2)
k_srht_q512(const __grid_constant__ CUtensorMap amap, int d, int64_t m, int64_t m_total, int64_t row_off,
            int64_t P5, int PG, const int32_t* __restrict__ rows, uint32_t level, uint32_t k0, uint32_t k1,
            int64_t gblk /* global 1024-row block of A's row 0 */, unsigned* status,
            float* __restrict__ out /* PG x m_total x d partials */) {
    extern __shared__ __align__(128) unsigned char smraw[];
    float* stage = reinterpret_cast<float*>(smraw);                                   // 3 x 512 x 16
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smraw + kQ5S * kQ5Stage);           // 32 sign words
    uint64_t* full = reinterpret_cast<uint64_t*>(sbits + 32);                        // 3 mbarriers
    int2* sel = reinterpret_cast<int2*>(full + kQ5S);                                // 16 MA slots
    const int tid = threadIdx.x;
    const int c = tid & 15, ql = tid >> 4;
    const int col0 = blockIdx.x * kQ5C;
    const int pg = blockIdx.y;
    const int64_t q0 = (int64_t)pg * P5 / PG, q1 = (int64_t)(pg + 1) * P5 / PG;
    const int64_t nblk = q1 - q0;

    if (tid == 0) {
        for (int i = 0; i < kQ5S; ++i) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    for (int j = tid; j < 16 * MA; j += kQ5T) {
        int2 e = make_int2(0, 0);
        if (j < m) {
            const uint32_t r = (uint32_t)rows[j];
            const int lo = (int)(r & 511u);
            e.x = q5_pos(lo >> 4, lo & 15) * (int)sizeof(float);
            e.y = (int)(r >> 9);
        }
        sel[j] = e;
    }
    __syncthreads();
    auto issue = [&](int64_t bb) {   // block q0 + bb into stage bb % 3
        const int sidx = (int)(bb % kQ5S);
        float* dst = stage + (size_t)sidx * (512 * kQ5C);
        mbar_arrive_expect_tx(&full[sidx], (uint32_t)kQ5Stage);
        const int y0 = (int)((q0 + bb) * 512);
        tma_load_2d(dst, &amap, col0, y0, &full[sidx]);
        tma_load_2d(dst + 256 * kQ5C, &amap, col0, y0 + 256, &full[sidx]);
    };
    int64_t issued = 0;
    if (tid == 0) {
        for (; issued < kQ5S && issued < nblk; ++issued) issue(issued);
    }
    float acc[MA];
#pragma unroll
    for (int i = 0; i < MA; ++i) acc[i] = 0.f;
    // this thread's transposed offsets: writes of Z[K][ql] (even / odd K), and
    // the two K = ql, ql + 16 it transforms next (even / odd L)
    const int wE = ql * 16 + c, wO = (ql ^ 1) * 16 + c;
    const int sw = (ql & 1) * 16;
    const int rE = ql * 256 + c + sw, rO = ql * 256 + c - sw;
    int64_t b = 0;
    int sidx = 0;
    uint32_t ph = 0;
    for (; b < nblk; ++b) {
        const int64_t q = q0 + b;
        if (tid < 8) {
            const uint4 w = srht_sign_words((uint64_t)(gblk + (q >> 1)) * 8 + tid, level, k0, k1);
            sbits[4 * tid + 0] = w.x;
            sbits[4 * tid + 1] = w.y;
            sbits[4 * tid + 2] = w.z;
            sbits[4 * tid + 3] = w.w;
        }
        const bool ok = mbar_wait_bounded(&full[sidx], ph, status);
        if (__syncthreads_or(!ok)) break;   // also: sign words ready, block b - 1 fully gathered
        if (tid == 0 && b >= 1 && issued < nblk) issue(issued++);   // into the stage of block b - 1
        float* st = stage + (size_t)sidx * (512 * kQ5C);
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = st[(16 * k + ql) * kQ5C + c];
        const int hsh = (int)(q & 1) * 16;
        const uint32_t w0 = sbits[ql] >> hsh, w1 = sbits[16 + ql] >> hsh;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint32_t w = (k & 1) ? w1 : w0;
            v[k] = __int_as_float(__float_as_int(v[k]) ^ (int)((w << (31 - (k >> 1))) & 0x80000000u));
        }
        wht32(v);   // over k: v[K] = Z[K][ql]
        __syncthreads();   // the stage is fully read: overwrite it with Z
#pragma unroll
        for (int K = 0; K < 32; ++K) st[K * 256 + ((K & 1) ? wO : wE)] = v[K];
        __syncthreads();
        float a[16], bb[16];
#pragma unroll
        for (int L = 0; L < 16; ++L) {
            const int o = L * 16 + ((L & 1) ? rO : rE);
            a[L] = st[o];
            bb[L] = st[o + 16 * 256];
        }
        wht16_pair(a, bb);   // over ql: Y[16 K + L] for K = ql and ql + 16
#pragma unroll
        for (int L = 0; L < 16; ++L) {   // back to the positions this thread read
            const int o = L * 16 + ((L & 1) ? rO : rE);
            st[o] = a[L];
            st[o + 16 * 256] = bb[L];
        }
        // order these generic writes before the TMA load that will refill the stage
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int qb = (int)(2 * gblk + q);   // global 512-row block index
        const unsigned char* Tc = reinterpret_cast<const unsigned char*>(st + c);
#pragma unroll
        for (int i = 0; i < MA; ++i) {
            const int2 e = sel[ql + 16 * i];
            const float val = *reinterpret_cast<const float*>(Tc + e.x);
            acc[i] += __int_as_float(__float_as_int(val) ^ (int)((unsigned)__popc(e.y & qb) << 31));
        }
        if (++sidx == kQ5S) {
            sidx = 0;
            ph ^= 1u;
        }
    }
    if (b < nblk) {
        // a wait gave up: let the copies in flight land before exiting
        if (tid == 0) {
            for (int64_t t = b; t < issued; ++t)
                mbar_wait_bounded(&full[t % kQ5S], (uint32_t)((t / kQ5S) & 1), status);
        }
        __syncthreads();
        return;
    }
    const int col = col0 + c;
    if (col < d) {
        float* outp = out + ((size_t)pg * m_total + row_off) * d + col;
#pragma unroll
        for (int i = 0; i < MA; ++i) {
            const int64_t j = ql + 16 * i;
            if (j < m) outp[j * d] = acc[i];
        }
    }
}

template <int MA>
int launch_q512(ihs_ctx* ctx, const CUtensorMap& amap, int d, int64_t mc, int64_t m, int64_t c0, int64_t P5, int PG,
                const int32_t* rows, int32_t level, uint64_t seed, int64_t gblk, float* part) {
    const size_t smem = q5_smem_bytes(MA);
    auto kern = k_srht_q512<MA>;
    IHS_CUDA_TRY(ihs_allow_smem(kern, smem));
    // two CTAs per SM need the largest shared-memory carveout
    IHS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    dim3 grid((unsigned)ceil_div64(d, kQ5C), (unsigned)PG);
    kern<<<grid, kQ5T, smem, ctx->stream>>>(amap, d, mc, m, c0, P5, PG, rows, (uint32_t)level, (uint32_t)seed,
                                           (uint32_t)(seed >> 32), gblk, ctx->d_status, part);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

template <int MA>
int launch_r32(ihs_ctx* ctx, const CUtensorMap& amap, int d, int64_t mc, int64_t m, int64_t c0, int64_t P, int PG,
               const int32_t* rows, int32_t level, uint64_t seed, int64_t gblk, float* part) {
    const size_t smem = r32_smem_bytes(MA);
    auto kern = k_srht_r32<MA>;
    IHS_CUDA_TRY(ihs_allow_smem(kern, smem));
    dim3 grid((unsigned)ceil_div64(d, kR32C), (unsigned)PG);
    kern<<<grid, kR32T, smem, ctx->stream>>>(amap, d, mc, m, c0, P, PG, rows, (uint32_t)level, (uint32_t)seed,
                                            (uint32_t)(seed >> 32), gblk, ctx->d_status, part);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

// out[e] = fl32(scale * colscale[e % d] * sum_k part_k[e]).  The K partials
// are summed in a fixed order into a compensated binary32 pair (TwoSum), then
// scaled in double-float arithmetic and rounded once: FP64 runs at a small
// fraction of the FP32 rate on this GPU, and a double accumulator made the
// reduction FP64-bound (about 1 TB/s) instead of HBM-bound.  PAIRS: each
// element is a (hi, lo) float2.  16-byte streaming loads when every partial
// starts on a 16-byte boundary (count a multiple of the elements per load).
template <bool PAIRS>
__global__ void __launch_bounds__(256)
k_reduce_parts(const float* __restrict__ part, int K, int64_t count, int d, float sh, float sl,
               const float* __restrict__ colscale, float* __restrict__ out) {
    constexpr int EV = PAIRS ? 2 : 4;   // elements per float4
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    auto finish = [&](const Acc2& a, int64_t e) {
        float2 v = df_mul(a.hi, a.lo, sh, sl);
        if (colscale != nullptr) v = df_mul(v.x, v.y, colscale[e % d], 0.f);
        out[e] = v.x;
    };
    // the partials in batches of eight independent loads ahead of the
    // dependent compensated additions
    constexpr int BK = 8;
    if (count % EV == 0) {
        const int64_t nv = count / EV;   // float4 per partial
        const float4* src = reinterpret_cast<const float4*>(part);
        for (int64_t v = t0; v < nv; v += stride) {
            Acc2 a[EV] = {};
            for (int k0 = 0; k0 < K; k0 += BK) {
                float4 q[BK];
#pragma unroll
                for (int u = 0; u < BK; ++u)
                    if (k0 + u < K) q[u] = __ldcs(src + (size_t)(k0 + u) * nv + v);
#pragma unroll
                for (int u = 0; u < BK; ++u) {
                    if (k0 + u >= K) break;
                    if constexpr (PAIRS) {
                        a[0].add_pair(q[u].x, q[u].y);
                        a[1].add_pair(q[u].z, q[u].w);
                    } else {
                        a[0].add(q[u].x);
                        a[1].add(q[u].y);
                        a[2].add(q[u].z);
                        a[3].add(q[u].w);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < EV; ++i) finish(a[i], v * EV + i);
        }
    } else {
        for (int64_t e = t0; e < count; e += stride) {
            Acc2 a{0.f, 0.f};
            for (int k0 = 0; k0 < K; k0 += BK) {
                float2 q[BK];
#pragma unroll
                for (int u = 0; u < BK; ++u) {
                    if (k0 + u >= K) continue;
                    if constexpr (PAIRS) q[u] = reinterpret_cast<const float2*>(part)[(size_t)(k0 + u) * count + e];
                    else q[u] = make_float2(part[(size_t)(k0 + u) * count + e], 0.f);
                }
#pragma unroll
                for (int u = 0; u < BK; ++u) {
                    if (k0 + u >= K) break;
                    if constexpr (PAIRS) a.add_pair(q[u].x, q[u].y);
                    else a.add(q[u].x);
                }
            }
            finish(a, e);
        }
    }
}

// Gaussian sketch, FP32 SIMT: tile BM x BN of SA over a K range of rows of A;
// z tile generated in shared memory from Philox, compensated accumulation per
// BK-chunk.
constexpr int kGBM = 64, kGBN = 64, kGBK = 32, kGThreads = 256;

__global__ void __launch_bounds__(kGThreads)
k_gauss_simt(const float* __restrict__ A, int64_t n, int d, int64_t m, int64_t rows_per_split, uint32_t level,
             uint32_t k0, uint32_t k1, uint32_t zq0 /* first z row / 4 */, uint32_t ibase /* global row of A's row 0 */,
             float2* __restrict__ part /* KS x m x d */) {
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
            if (i < i_end) z = gauss4(ibase + (uint32_t)i, zq0 + (uint32_t)((j0 >> 2) + qq), level, k0, k1);
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

// A holds rows [grow0, grow0 + n) of a matrix of n_total rows (a row shard;
// grow0 = 0 and n_total = n for the whole matrix): the sketch of the whole
// matrix restricted to these rows, i.e. this shard's term of SA = sum over
// shards.  grow0 must be a multiple of 1024 (whole transform blocks).
int srht_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                 float* SA, int64_t grow0 = 0, int64_t n_total = 0) {
    if (n_total <= 0) n_total = n;
    const int64_t n_pad = next_pow2_64(n_total);
    if (m > n_pad) return IHS_EINVAL;
    const int Q = (int)std::min<int64_t>(n_pad, kSrhtQmax);
    int logQ = 0;
    while ((1 << logQ) < Q) ++logQ;
    if (grow0 % Q) return IHS_EINVAL;
    // the whole matrix: every block of the padded n_pad rows; a shard: its own blocks
    const int64_t P = (grow0 == 0 && n == n_total) ? n_pad / Q : ceil_div64(n, Q);
    const int64_t gblk = grow0 / 1024;
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
        // Selected rows go in chunks of at most 2048 (64 register accumulators
        // per thread); each chunk re-reads A.  Chunks of <= 256 rows run the
        // 512-row-block kernel at two CTAs per SM, larger ones the 1024-row one.
        const int64_t chunk = std::min<int64_t>(m, 2048);
        const int64_t CT32 = ceil_div64(d, kR32C);
        const bool small = m <= 256;
        // a grid of CT32 x PG32 CTAs in whole waves when the block ranges allow
        // it (PG32 = slots / gcd(CT32, slots), slots = SMs x CTAs per SM), else
        // >= 1 wave
        const int64_t slots = (int64_t)ctx->sm_count * (small ? 2 : 1);
        int64_t g = CT32, h = slots;
        while (h) {
            const int64_t t = g % h;
            g = h;
            h = t;
        }
        int64_t PG32 = slots / g;
        if (PG32 > P || PG32 * m * d * 4 > ((int64_t)1 << 30)) PG32 = std::max<int64_t>(1, ceil_div64(slots, CT32));
        PG32 = std::min<int64_t>(PG32, P);
        if (PG32 > PG) {
            IHS_TRY(ihs_scratch(ctx, SLOT_SKETCH_PART, (size_t)PG32 * m * d * sizeof(float), &pws));
            part = static_cast<float*>(pws);
        }
        PG = PG32;
        for (int64_t c0 = 0; c0 < m; c0 += chunk) {
            const int64_t mc = std::min<int64_t>(chunk, m - c0);
            int st;
            if (mc <= 16) st = launch_q512<1>(ctx, amap, (int)d, mc, m, c0, 2 * P, (int)PG, rows + c0, level, seed, gblk, part);
            else if (mc <= 64) st = launch_q512<4>(ctx, amap, (int)d, mc, m, c0, 2 * P, (int)PG, rows + c0, level, seed, gblk, part);
            else if (mc <= 128) st = launch_q512<8>(ctx, amap, (int)d, mc, m, c0, 2 * P, (int)PG, rows + c0, level, seed, gblk, part);
            else if (mc <= 256) st = launch_q512<16>(ctx, amap, (int)d, mc, m, c0, 2 * P, (int)PG, rows + c0, level, seed, gblk, part);
            else if (mc <= 32 * 16) st = launch_r32<16>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, gblk, part);
            else if (mc <= 32 * 32) st = launch_r32<32>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, gblk, part);
            else st = launch_r32<64>(ctx, amap, (int)d, mc, m, c0, P, (int)PG, rows + c0, level, seed, gblk, part);
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
                                                              (uint32_t)(seed >> 32), acc_in_smem, grow0, part);
        IHS_LAUNCH_CHECK();
    }
    return ihs_reduce_parts_enqueue(ctx, part, false, (int)PG, m * d, d, 1.0 / sqrt((double)m), nullptr, SA);
}

// Rows [zrow0, zrow0 + m) of the Gaussian sketch of size m_scale (zrow0 % 4 == 0).
int gauss_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed, int32_t level,
                  float* SA, int64_t zrow0 = 0, int64_t m_scale = 0, int64_t grow0 = 0) {
    if (m_scale <= 0) m_scale = m;
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
                                                     (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)(zrow0 >> 2),
                                                     (uint32_t)grow0, part);
    IHS_LAUNCH_CHECK();
    return ihs_reduce_parts_enqueue(ctx, reinterpret_cast<const float*>(part), true, (int)KS, m * d, d,
                                    1.0 / sqrt((double)m_scale), nullptr, SA);
}

}  // namespace

int ihs_reduce_parts_enqueue(ihs_ctx* ctx, const float* part, bool pairs, int K, int64_t count, int64_t d,
                             double scale, const float* colscale, float* out) {
    if (K < 1 || count < 1 || d < 1) return IHS_EINVAL;
    const int ev = pairs ? 2 : 4;
    const int64_t work = count % ev == 0 ? count / ev : count;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div64(work, 256), 8 * (int64_t)ctx->sm_count);
    const DfConst s = df_const(scale);
    if (pairs) {
        k_reduce_parts<true><<<grid, 256, 0, ctx->stream>>>(part, K, count, (int)d, s.hi, s.lo, colscale, out);
    } else {
        k_reduce_parts<false><<<grid, 256, 0, ctx->stream>>>(part, K, count, (int)d, s.hi, s.lo, colscale, out);
    }
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

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

int ihs_sketch_shard_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t row0, int64_t n_total,
                             int64_t m, int32_t kind, uint64_t seed, int32_t level, float* SA_part) {
    if (n < 1 || d < 1 || m < 1 || level < 0 || m > ((int64_t)1 << 31)) return IHS_EINVAL;
    if (row0 < 0 || n_total < row0 + n || n_total > ((int64_t)1 << 32)) return IHS_EINVAL;
    if (kind == IHS_SKETCH_SRHT) {
        // whole transform blocks: the shard starts on a block, and ends on one
        // unless it holds the last rows
        if (row0 % 1024 || (n % 1024 && row0 + n != n_total)) return IHS_EINVAL;
        return srht_enqueue(ctx, A, n, d, m, seed, level, SA_part, row0, n_total);
    }
    if (kind == IHS_SKETCH_GAUSS) {
        if (m > n_total) return IHS_EINVAL;
        if (ctx->p.precision == IHS_PREC_BF16)
            return ihs_gauss_tc_enqueue(ctx, A, n, d, m, seed, level, SA_part, 0, 0, 0, row0);
        if (ctx->p.precision == IHS_PREC_FP8)
            return ihs_gauss_tc_enqueue(ctx, A, n, d, m, seed, level, SA_part, 1, 0, 0, row0);
        return gauss_enqueue(ctx, A, n, d, m, seed, level, SA_part, 0, 0, row0);
    }
    return IHS_EINVAL;
}

extern "C" int ihs_sketch_shard(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t row0, int64_t n_total,
                                int64_t m, int32_t kind, uint64_t seed, int32_t level, float* SA_part) {
    IhsRange range("ihs_sketch_shard");
    if (!ctx || !A || !SA_part) return IHS_EINVAL;
    IHS_TRY(ihs_sketch_shard_enqueue(ctx, A, n, d, row0, n_total, m, kind, seed, level, SA_part));
    return IHS_OK;
}

int ihs_sketch_rows_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                            int32_t level, int64_t row0, int64_t mrows, float* SA_rows) {
    if (n < 1 || d < 1 || m < 1 || level < 0 || m > ((int64_t)1 << 31)) return IHS_EINVAL;
    if (row0 < 0 || row0 % 4 || mrows < 1 || row0 + mrows > m) return IHS_EINVAL;
    if (ctx->p.precision == IHS_PREC_BF16) return ihs_gauss_tc_enqueue(ctx, A, n, d, mrows, seed, level, SA_rows, 0, row0, m);
    if (ctx->p.precision == IHS_PREC_FP8) return ihs_gauss_tc_enqueue(ctx, A, n, d, mrows, seed, level, SA_rows, 1, row0, m);
    return gauss_enqueue(ctx, A, n, d, mrows, seed, level, SA_rows, row0, m);
}

extern "C" int ihs_sketch_rows(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                               int32_t level, int64_t row0, int64_t mrows, float* SA_rows) {
    IhsRange range("ihs_sketch_rows");
    if (!ctx || !A || !SA_rows) return IHS_EINVAL;
    return ihs_sketch_rows_enqueue(ctx, A, n, d, m, seed, level, row0, mrows, SA_rows);
}

extern "C" int ihs_sketch(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, int32_t kind,
                          uint64_t seed, int32_t level, float* SA) {
    IhsRange range("ihs_sketch");
    if (!ctx || !A || !SA) return IHS_EINVAL;
    IHS_TRY(ihs_sketch_enqueue(ctx, A, n, d, m, kind, seed, level, SA));
    return IHS_OK;
}
