// Internal definitions shared by the CUDA translation units of the library.
// Nothing here is part of the public C ABI (include/ihs.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ihs.h"

#define IHS_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) {                            \
            ihs_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return IHS_ECUDA;                               \
        }                                                   \
    } while (0)

#define IHS_TRY(expr)                   \
    do {                                \
        int _s = (expr);                \
        if (_s != IHS_OK) return _s;    \
    } while (0)

void ihs_count_launch();
void ihs_count_launches(int64_t n);   // kernels of one replayed CUDA graph
#define IHS_LAUNCH_CHECK()                    \
    do {                                      \
        ihs_count_launch();                   \
        IHS_CUDA_TRY(cudaGetLastError());     \
    } while (0)

void ihs_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void ihs_set_error(const char* msg);   // message for ihs_last_error()

// ---------------------------------------------------------------------------
// Scratch arena: grow-only device buffers keyed by slot.
enum ScratchSlot {
    SLOT_GRAD_PART = 0,   // per-CTA gradient partials (float2 x G x d) + G doubles
    SLOT_GRAD_R,          // residual vector of the generic gradient path (n floats)
    SLOT_SELECT,          // radix-select histograms and compaction counters
    SLOT_SKETCH_PART,     // split partial sums of the sketch
    SLOT_SKETCH_ROWS,     // selected SRHT rows
    SLOT_SOLVE,           // solver state vectors
    SLOT_SOLVE_SA,        // solver-owned SA (m x d)
    SLOT_MISC,            // small device scalars (status word, reductions)
    SLOT_FACTOR,          // the solver's factor (K/L, block inverses, X, X^T, apply scratch)
    SLOT_DUAL,            // underdetermined solves: A^T and the dual gradient's scratch
    SLOT_SOLVE_SA2,       // nested sketches: the previous level's SA while the next one is formed
    SLOT_HOST_IN,         // ihs_solve_host: device copies of the caller's A, b and x
    SLOT_COUNT
};

// Device-side status word bits (set by kernels that give up a bounded wait).
#define IHS_DEV_TIMEOUT 1u
#define IHS_DEV_NOTPD   2u

struct ihs_ctx {
    int device;
    int sm_count;
    cudaStream_t stream;
    ihs_params p;
    void* buf[SLOT_COUNT];
    size_t buf_bytes[SLOT_COUNT];
    double* pinned;          // host pinned scratch (64 doubles)
    unsigned* d_status;      // device status word (IHS_DEV_*)
    cudaEvent_t ev[6];       // [4], [5]: the solver's sketch + factor interval
    cudaStream_t aux;        // private stream for the look-ahead Cholesky (joined back before return)
    cudaEvent_t fev[8];      // fork/join events of the look-ahead Cholesky
    void* lanes;             // batched solves: sub-contexts, streams and memory pool kept across calls
    int no_coop;             // 1: factorisations use the multi-launch form (many run side by side)
    void* trace;             // decision log of the last solve (api.cu), NULL until first use
    uint64_t apply_epoch;    // arrivals so far on the fused apply's grid-barrier counter
    // Test-only fault injection on the host side, read from the environment at
    // creation and off by default: IHS_TEST_BARRIER_UNREACHABLE=1 makes the
    // first grid barrier of this context's first persistent Cholesky ask for one
    // arrival more than the grid can give (a wait that nothing completes);
    // IHS_BARRIER_LIMIT_MS (default 1000) bounds the persistent Cholesky's
    // barrier waits.
    int test_bar_unreachable;
    uint64_t bar_limit_ns;
    // CTAs per SM of the persistent Cholesky: 2 (default; the second CTA's
    // warps hide the latencies of the double-float tile updates) or 1
    // (IHS_CHOL_CTAS_PER_SM=1, a launch-shape setting read at creation)
    int chol_per_sm;
    // CTAs of the fused apply (IHS_APPLY_CTAS, 1 .. SM count; 0: one per SM)
    int apply_ctas;
    // 1: the Gram of a factorisation on the CUDA cores (compensated FP32 FMA
    // chains) instead of the tensor cores (IHS_GRAM_SIMT=1)
    int gram_simt;
};

// Decision log of the controller (api.cu): cleared at the start of a solve,
// one entry per decision, mirrored to the context's JSON-lines file if set.
void ihs_trace_reset(ihs_ctx* ctx);
void ihs_trace_add(ihs_ctx* ctx, int kind, int t, int64_t m, double r, double ratio);
void ihs_trace_free(ihs_ctx* ctx);

// NVTX range for the scope of a library call or phase (a no-op unless a
// profiler is attached).
struct IhsRange {
    explicit IhsRange(const char* name) { nvtxRangePushA(name); }
    ~IhsRange() { nvtxRangePop(); }
    IhsRange(const IhsRange&) = delete;
    IhsRange& operator=(const IhsRange&) = delete;
};

void ihs_lanes_destroy(void* lanes);   // batch.cu

struct ihs_factor {
    ihs_ctx* ctx;
    const float* SA;
    int64_t m, d, k;      // k = m (Woodbury) or d (direct)
    double nu;
    int woodbury;
    double* L;            // k x k: K, then its lower Cholesky factor (row-major; FP64, or
                          // double-float pairs in the same 8 bytes when l_df)
    int l_df;             // 1: L holds (hi, lo) binary32 pairs (persistent Cholesky)
    double* W;            // inverses of the 64 x 64 diagonal blocks of L (FP64)
    float* X;             // k x k lower inverse L^{-1} (FP32)
    float* XT;            // its transpose (upper)
    double* work;         // apply scratch vectors and reduction slots
    int owned;            // 1: the buffers above are this handle's own allocations
    // fused apply (one cooperative launch, apply.cu); fused == 0 takes the
    // multi-launch apply and leaves the two buffers below unset
    int fused;
    float* SAT;           // (SA)^T, d x m FP32
    float2* Y;            // four partial-sum buffers of ihs_apply_partials(k, m, d) pairs each
};

// Fused apply (apply.cu).
bool ihs_apply_fused_ok(int64_t k, int64_t m, int64_t d);
size_t ihs_apply_partials(int64_t k, int64_t m, int64_t d);   // float2 entries per partial buffer
int ihs_apply_prepare(ihs_ctx* ctx, ihs_factor_t* F);          // SA^T
int ihs_apply_fused(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* d_r);

int ihs_scratch(ihs_ctx* ctx, int slot, size_t bytes, void** out);

// Let `kern` use up to the device's opt-in maximum of dynamic shared memory
// (`need` must fit).  The attribute is per function: setting it to one fixed
// value keeps launches from several host threads with different sizes from
// racing on it.
template <typename K>
inline cudaError_t ihs_allow_smem(K kern, size_t need) {
    int dev = 0, mx = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (need > (size_t)mx) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}
int ihs_check_status(ihs_ctx* ctx);   // reads and clears the device status word

// Internal launch helpers (enqueue only, no synchronisation).
int ihs_grad_enqueue(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d,
                     double nu, const float* x, float* g, double* d_axnorm2);
int ihs_sketch_rows_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                            int32_t level, int64_t row0, int64_t mrows, float* SA_rows);
int ihs_sketch_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m,
                       int32_t kind, uint64_t seed, int32_t level, float* SA);
int ihs_gauss_fp32_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                           int32_t level, float* SA);   // FP32 SIMT Gaussian sketch
int ihs_gauss_tc_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                         int32_t level, float* SA, int fp8, int64_t zrow0 = 0, int64_t m_scale = 0,
                         int64_t grow0 = 0);   // rows [zrow0, zrow0 + m) of the sketch of size m_scale; A's row 0 is global row grow0
// out[e] = fl32(scale * colscale[e % d] * sum_k part_k[e]) over K partials of
// `count` elements (float, or hi + lo float2 pairs when `pairs`), summed in a
// fixed order; colscale may be NULL.
int ihs_reduce_parts_enqueue(ihs_ctx* ctx, const float* part, bool pairs, int K, int64_t count, int64_t d,
                             double scale, const float* colscale, float* out);
// K = X X^T + nu^2 I (X = SA, Woodbury, or (SA)^T, direct; kdim rows of X,
// K inner entries) on the tensor cores into G (lower part; double-float pairs
// when out_df, else FP64), on stream s (gram_tc.cu).
int ihs_gram_tc_enqueue(ihs_ctx* ctx, const float* SA, int64_t d, int woodbury, int64_t kdim, int64_t K, double nu2,
                        int out_df, double* G, cudaStream_t s);
// A row shard's term of the sketch (rows [row0, row0 + n) of n_total) and of
// the gradient (FP64 partial sums, d + 1 doubles: A^T (A x - b) and ||A x||^2).
int ihs_sketch_shard_enqueue(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t row0, int64_t n_total,
                             int64_t m, int32_t kind, uint64_t seed, int32_t level, float* SA_part);
int ihs_grad_partial_enqueue(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, const float* x,
                             double* gp);
int ihs_grad_finish_enqueue(ihs_ctx* ctx, const double* gp, int64_t d, double nu, const float* x, float* g,
                            double* d_axnorm2);
int ihs_rows_enqueue(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint64_t seed, int32_t level,
                     int32_t* rows);
int ihs_factor_build(ihs_ctx* ctx, ihs_factor_t* F);       // enqueue + check pivots (syncs)
int ihs_factor_enqueue(ihs_ctx* ctx, ihs_factor_t* F);     // enqueue only (pivot failures in d_status)
int ihs_factor_alloc(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** out);
int ihs_factor_alloc_pool(ihs_ctx* ctx, cudaMemPool_t pool, const float* SA, int64_t m, int64_t d, double nu,
                          ihs_factor_t* F);
void ihs_factor_release_pool(ihs_factor_t* F, cudaStream_t s);
// Factor into the context's scratch (no allocation once the slot is large
// enough); F is caller storage, valid until the next call with the same ctx.
int ihs_factor_scratch(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t* F,
                       bool check = true);   // check = false: enqueue only, the caller reads the status word later
int ihs_apply_enqueue(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt,
                      double* d_r);

// ---------------------------------------------------------------------------
// Device helpers.

// Philox4x32-10 (Salmon et al., SC'11): two 32x32->64 multiplies per round,
// Weyl-sequence key schedule, ten rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

enum { STREAM_SIGNS = 0, STREAM_ROWS = 1, STREAM_GAUSS = 2, STREAM_PROBE = 3 };

// SRHT signs: rows form blocks of 1024; block b owns the 32 words of Philox
// counters 8b .. 8b+7 (word 4t + k = output word k of counter 8b + t), and row
// i = 1024 b + q takes bit (q >> 5) of word (q & 31) (1 -> eps = -1).
__device__ __forceinline__ uint4 srht_sign_words(uint64_t ctr, uint32_t level, uint32_t k0, uint32_t k1) {
    return philox4x32_10(make_uint4((uint32_t)ctr, (uint32_t)(ctr >> 32), level, STREAM_SIGNS), k0, k1);
}

__device__ __forceinline__ int srht_sign_bit(uint64_t i, uint32_t level, uint32_t k0, uint32_t k1) {
    const uint32_t q = (uint32_t)(i & 1023u);
    const uint32_t wi = q & 31u;
    const uint4 w = srht_sign_words((i >> 10) * 8 + (wi >> 2), level, k0, k1);
    const uint32_t sel = wi & 3u;
    const uint32_t word = sel == 0 ? w.x : (sel == 1 ? w.y : (sel == 2 ? w.z : w.w));
    return (int)((word >> (q >> 5)) & 1u);
}

__device__ __forceinline__ uint64_t srht_row_key(uint64_t i, uint32_t level, uint32_t k0, uint32_t k1) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), level, STREAM_ROWS), k0, k1);
    return ((uint64_t)w.y << 32) | (uint64_t)w.x;
}

// Box-Muller pair from two Philox words: u1 = (w/2^8 + 1) 2^-24 in (0, 1],
// u2 = (w'/2^8) 2^-24 in [0, 1); both exact in binary32.
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
    const float u1 = (float)((wa >> 8) + 1u) * 5.9604644775390625e-8f;
    const float u2 = (float)(wb >> 8) * 5.9604644775390625e-8f;
    const float radius = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(radius * c, radius * s);
}

// Four standard normals z[4q .. 4q+3] of column i at `level`.
__device__ __forceinline__ float4 gauss4(uint32_t i, uint32_t q, uint32_t level, uint32_t k0, uint32_t k1) {
    const uint4 w = philox4x32_10(make_uint4(i, q, level, STREAM_GAUSS), k0, k1);
    const float2 a = box_muller(w.x, w.y);
    const float2 b = box_muller(w.z, w.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Same draws with the fast hardware approximations of log and sin/cos (used
// where the sketch is rounded to BF16 / FP8 anyway); differences from gauss4
// are a few binary32 ulps.
__device__ __forceinline__ float4 gauss4_fast(uint32_t i, uint32_t q, uint32_t level, uint32_t k0, uint32_t k1) {
    const uint4 w = philox4x32_10(make_uint4(i, q, level, STREAM_GAUSS), k0, k1);
    float4 z;
    {
        const float u1 = (float)((w.x >> 8) + 1u) * 5.9604644775390625e-8f;
        const float u2 = (float)(w.y >> 8) * 5.9604644775390625e-8f;
        const float rad = sqrtf(-2.0f * __logf(u1));
        float sn, cs;
        __sincosf(6.283185307179586f * u2, &sn, &cs);
        z.x = rad * cs;
        z.y = rad * sn;
    }
    {
        const float u1 = (float)((w.z >> 8) + 1u) * 5.9604644775390625e-8f;
        const float u2 = (float)(w.w >> 8) * 5.9604644775390625e-8f;
        const float rad = sqrtf(-2.0f * __logf(u1));
        float sn, cs;
        __sincosf(6.283185307179586f * u2, &sn, &cs);
        z.z = rad * cs;
        z.w = rad * sn;
    }
    return z;
}

// Error-free transformations (Knuth TwoSum; TwoProduct through FMA).  The
// _rn intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Compensated accumulator (hi + lo) of float terms.
struct Acc2 {
    float hi, lo;
    __device__ __forceinline__ void add(float v) {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_prod(float a, float b) {   // Dot2 step
        float p, ep, s, es;
        two_prod(a, b, p, ep);
        two_sum(hi, p, s, es);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(ep, es));
    }
    __device__ __forceinline__ void add_pair(float h2, float l2) {
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, l2));
    }
};

// packed FP32x2 (sm_100+): two independent IEEE binary32 operations per instruction
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// Two Acc2 accumulators in packed form.
struct Acc2x2 {
    f2 hi, lo;
    // Dot2 step on both lanes: (hi, lo) += a * x exactly up to the final
    // rounding of lo; xn = -x.  Same operations as Acc2::add_prod.
    __device__ __forceinline__ void add_prod(f2 a, f2 x, f2 xn) {
        const f2 np = f2_mul(a, xn);        // -p, p = fl(a x)
        const f2 ep = f2_fma(a, x, np);     // a x - p
        const f2 s = f2_sub(hi, np);        // hi + p
        const f2 z = f2_sub(s, hi);
        const f2 e1 = f2_sub(hi, f2_sub(s, z));
        const f2 e2n = f2_add(np, z);       // -(p - z)
        const f2 es = f2_sub(e1, e2n);
        hi = s;
        lo = f2_add(lo, f2_add(ep, es));
    }
    // Same operations as Acc2::add_pair.
    __device__ __forceinline__ void add_pair(f2 h2, f2 l2) {
        const f2 s = f2_add(hi, h2);
        const f2 z = f2_sub(s, hi);
        const f2 e = f2_add(f2_sub(hi, f2_sub(s, z)), f2_sub(h2, z));
        hi = s;
        lo = f2_add(lo, f2_add(e, l2));
    }
    // Same operations as Acc2::add.
    __device__ __forceinline__ void add(f2 v) {
        const f2 s = f2_add(hi, v);
        const f2 z = f2_sub(s, hi);
        const f2 e = f2_add(f2_sub(hi, f2_sub(s, z)), f2_sub(v, z));
        hi = s;
        lo = f2_add(lo, e);
    }
};

// A double as an unevaluated binary32 pair (hi + lo), on the host.
struct DfConst {
    float hi, lo;
};
inline DfConst df_const(double v) {
    const float hi = (float)v;
    return DfConst{hi, (float)(v - (double)hi)};
}

// (hi + lo) * (sh + sl) as a normalised pair: the product of two double-float
// numbers with the lo * sl term dropped (below 2^-46 relative).
__device__ __forceinline__ float2 df_mul(float hi, float lo, float sh, float sl) {
    float p, e;
    two_prod(hi, sh, p, e);
    e = __fmaf_rn(hi, sl, __fmaf_rn(lo, sh, e));
    const float s = __fadd_rn(p, e);
    return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

// v as hi + lo with integer operations (no FP64 instruction: conversions from
// double run at the FP64 rate): hi keeps the sign, the exponent and the top 23
// stored mantissa bits (truncated), lo the remaining 29 bits rounded to 24,
// 48 bits in all.  Magnitudes outside [2^-74, 2^127] take the FP64 conversion.
__device__ __forceinline__ float2 df_split(double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned h32 = (unsigned)(bits >> 32), l32 = (unsigned)bits;
    const int e32 = (int)((h32 >> 20) & 0x7FFu) - 1023 + 127;   // binary32 biased exponent of v
    if (e32 < 53 || e32 > 254) {
        if (v == 0.0) return make_float2(0.f, 0.f);
        const float hi = __double2float_rn(v);
        return make_float2(hi, __double2float_rn(v - (double)hi));
    }
    const unsigned sign = h32 & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)e32 << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
    const float scale = __uint_as_float((unsigned)(e32 - 52) << 23);   // 2^(exponent of v - 52)
    const float lo = __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale);
    return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ Acc2 acc2_shfl_xor(Acc2 a, int mask) {
    Acc2 o;
    o.hi = __shfl_xor_sync(0xffffffffu, a.hi, mask);
    o.lo = __shfl_xor_sync(0xffffffffu, a.lo, mask);
    return o;
}

// ---- shared-memory barriers and bulk copies (sm_90+ PTX) -------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 4-byte asynchronous global -> shared copy; cp_async_mbar_arrive_noinc makes
// `bar` receive one arrival once all earlier cp.async of this thread landed
// (count that arrival in the barrier's expected count).
__device__ __forceinline__ void cp_async_4(void* dst_smem, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)),
                 "l"((unsigned long long)__cvta_generic_to_global(src))
                 : "memory");
}

__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` for at most ~limit_ns; on expiry set the
// timeout bit of the device status word and return false.
// try_wait with a suspend-time hint: the warp sleeps in hardware until the
// phase completes or about `hint_ns` passed, instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* status,
                                                  uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
        if (global_timer_ns() - t0 > limit_ns) {
            atomicOr(status, IHS_DEV_TIMEOUT);
            return false;
        }
    }
}

// 1-D bulk copy global -> shared, completing on `bar` (bytes % 16 == 0, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 2-D tiled bulk tensor load (TMA) into shared memory, completing on `bar`.
// x is the innermost coordinate (elements), y the row.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Host: encode a row-major FP32 matrix (rows x cols, leading dimension ld
// elements) as a 2-D tensor map with box (box_cols, box_rows); out-of-range
// elements read as zero.  Returns IHS_EINVAL if the layout is not TMA-able.
int ihs_tensor_map_f32(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows);

__host__ __device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

__host__ __device__ __forceinline__ int64_t next_pow2_64(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}
