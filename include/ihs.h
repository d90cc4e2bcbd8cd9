/*
 * ihs.h - C ABI of the GB300 adaptive Hessian-sketch ridge solver.
 *
 * Method: Lacotte & Pilanci, "Effective Dimension Adaptive Sketching Methods for
 * Faster Regularized Least-Squares Optimization" (NeurIPS 2020).  The library
 * solves the ridge problem of Eq. 1,
 *
 *     x* = argmin_x  1/2 ||A x - b||^2 + nu^2/2 ||x||^2 ,   A in R^{n x d}, n >= d,
 *
 * with the adaptive Polyak-IHS of Algorithm 1 or its gradient-only variant
 * (Sec. 5), preconditioning with the sketched Hessian H_S = (SA)^T SA + nu^2 I
 * of Eq. 3 applied through the Woodbury identity of App. B.4.
 *
 * Conventions shared by every entry point:
 *  - Matrices are row-major with leading dimension equal to their column count
 *    (A: n x d, SA: m x d).  Vectors are contiguous.
 *  - Pointers without a `_h` suffix are DEVICE pointers (cudaMalloc'd or torch
 *    CUDA tensors) on the current device; `_h` pointers are host pointers.
 *    float buffers must be 4-byte aligned; the fast kernels also want 16-byte
 *    alignment and d % 4 == 0, and fall back to slower kernels otherwise.
 *  - The caller owns every input and output buffer.  The library owns only the
 *    opaque handles (ihs_ctx, ihs_factor_t) and the scratch memory they hold;
 *    the matching *_destroy call frees them.
 *  - All device work is ordered on the stream given to ihs_ctx_create.  A call
 *    that returns a host scalar (`*_h` outputs) synchronises that stream before
 *    returning; others return as soon as the work is enqueued.
 *  - Every call returns an int status: IHS_OK (0) or a negative IHS_E* code.  A
 *    failing call leaves its outputs unspecified.  Device faults and launch
 *    failures surface as IHS_ECUDA.
 *  - A context is not thread-safe; use one per host thread / stream.
 */
#ifndef IHS_H
#define IHS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define IHS_OK          0
#define IHS_EINVAL     (-1)  /* bad argument (sizes, nu <= 0, n < d, m < 1, ...) */
#define IHS_ENOMEM     (-2)  /* device or pinned-host allocation failed          */
#define IHS_ENOTPD     (-3)  /* Cholesky met a non-positive or non-finite pivot   */
#define IHS_ENONFINITE (-4)  /* NaN/Inf in an input or in the decrement r_t       */
#define IHS_EMCAP      (-5)  /* sketch size reached its cap (report flag only)    */
#define IHS_EMAXITER   (-6)  /* iteration limit reached; x holds the last iterate */
#define IHS_ETIMEOUT   (-7)  /* a bounded device wait gave up                     */
#define IHS_ECUDA      (-8)  /* CUDA runtime error                                */

/* ---- enumerations -------------------------------------------------------- */
#define IHS_SKETCH_SRHT   0  /* subsampled randomized Hadamard transform (App. C.2) */
#define IHS_SKETCH_GAUSS  1  /* i.i.d. N(0, 1/m) entries (Sec. 1, App. C.1)        */

#define IHS_VARIANT_GD     0 /* gradient-IHS candidates only (Sec. 5 variant)   */
#define IHS_VARIANT_POLYAK 1 /* Algorithm 1: Polyak candidate, then gradient-IHS */

#define IHS_PREC_FP32  0     /* Gaussian sketch arithmetic: FP32 products       */
#define IHS_PREC_BF16  1     /* BF16 operands, FP32 accumulation (tensor cores)  */
#define IHS_PREC_FP8   2     /* FP8 e4m3 operands + per-column scales, FP32 acc. */

#define IHS_REPORT_MAX_LEVELS 40

/* Solver parameters (Algorithm 1's inputs plus the build's choices). */
typedef struct ihs_params {
    int32_t  kind;       /* IHS_SKETCH_*                                         */
    int32_t  variant;    /* IHS_VARIANT_*                                        */
    int32_t  precision;  /* IHS_PREC_* (Gaussian sketch only)                    */
    int32_t  max_iter;   /* limit on accepted iterations t                       */
    int64_t  m_init;     /* initial sketch size, a power of two >= 1             */
    double   rho;        /* aspect-ratio target of Def 3.1 / 3.2 (default 0.1)   */
    double   eta;        /* Gaussian concentration slack of Def 3.1 (0.01)       */
    double   tol;        /* stop when sqrt(2 Lambda r_t) <= tol ||Abar x_t||      */
    double   floor;      /* noise-floor guard: a rejected step with
                            r_t <= floor^2 r_1 stops instead of doubling (0: off) */
    uint64_t seed;       /* Philox key of every random draw                      */
    int32_t  nested;     /* 1: every level of ihs_solve draws with the key of
                            level 0, so the sketches are nested (Gaussian: the
                            first m rows of S_2m are S_m / sqrt 2 and are reused,
                            only the new rows are computed; SRHT: the rows of S_m
                            are a subset of those of S_2m).  Default 0: an
                            independent draw per level, as the paper samples S. */
    int32_t  reserved;   /* 0                                                    */
} ihs_params;

/* What ihs_solve did. */
typedef struct ihs_report {
    int32_t status;          /* IHS_OK, IHS_EMAXITER, ...                        */
    int32_t iterations;      /* final t                                          */
    int32_t grad_passes;     /* gradient evaluations (passes over A)             */
    int32_t n_levels;        /* number of sketches drawn                         */
    int32_t accepted_polyak;
    int32_t accepted_gd;
    int32_t rejected;        /* doublings of m                                   */
    int32_t flags;           /* bit 0: m reached its cap; bit 1: floor guard hit */
    int64_t m_final;
    int64_t m_levels[IHS_REPORT_MAX_LEVELS]; /* sketch size of each level drawn   */
    double  r1;              /* sketched Newton decrement at x_1 (Lemma 4.1)     */
    double  r_final;         /* decrement at the returned iterate                */
    double  axnorm_final;    /* ||Abar x_T||                                     */
    double  ms_sketch;       /* device time in sketch + factor (CUDA events)     */
    double  ms_iterate;      /* device time in gradient passes + applies         */
    double  ms_grad;         /* device time in the gradient passes alone          */
} ihs_report;

typedef struct ihs_ctx ihs_ctx;
typedef struct ihs_factor ihs_factor_t;

/* Library version string (static storage). */
const char* ihs_version(void);

/* Text of the last CUDA runtime error seen by this host thread (static
 * storage; empty if none). */
const char* ihs_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts); a diagnostic for counting device work. */
int64_t ihs_kernel_launches(void);

/* Fill *p with the defaults: SRHT, gradient-only, FP32, rho = 0.1, eta = 0.01,
 * m_init = 1, tol = 1e-5, floor = 0, max_iter = 500, seed = 0. */
int ihs_params_default(ihs_params* p_h);

/* Create a context bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current device.  *p_h may be NULL (defaults).  The context
 * owns its scratch memory and a pinned host buffer. */
int ihs_ctx_create(ihs_ctx** ctx_h, void* stream, const ihs_params* p_h);
int ihs_ctx_destroy(ihs_ctx* ctx);
/* Replace the parameters of an existing context. */
int ihs_ctx_set_params(ihs_ctx* ctx, const ihs_params* p_h);

/* ---- random draws (App. C.2) --------------------------------------------- */
/* Rademacher signs eps_i in {-1,+1}, i < n_pad (int8, device).  Philox4x32-10
 * with key (seed_lo, seed_hi) and counter (c_lo, c_hi, level, 0): rows form
 * blocks of 1024; block b owns the 32 words of counters 8b .. 8b+7 (word
 * 4t + k is output word k of counter 8b + t); row i = 1024 b + q takes bit
 * (q >> 5) of word (q & 31), and eps_i = +1 iff that bit is 0. */
int ihs_srht_signs(ihs_ctx* ctx, int64_t n_pad, uint64_t seed, int32_t level, int8_t* eps);

/* The m row indices of [0, n_pad) with the smallest 64-bit keys
 * key_i = (w1 << 32) | w0 of Philox counter (i_lo, i_hi, level, 1), ties broken
 * by index, written in ascending index order (int32, device): a uniformly
 * random m-subset drawn without replacement (App. C.2).  1 <= m <= n_pad <= 2^31. */
int ihs_srht_rows(ihs_ctx* ctx, int64_t n_pad, int64_t m, uint64_t seed, int32_t level, int32_t* rows);

/* ---- the three hot kernels ----------------------------------------------- */
/* SA = S A for the embedding S of `kind` drawn at (seed, level) (Sec. 1, Eq. 3):
 *  SRHT : S = sqrt(n_pad/m) R H_norm diag(eps) on A zero-padded to
 *         n_pad = 2^ceil(log2 n) rows, i.e. SA_j = m^-1/2 sum_i
 *         (-1)^popcount(r_j & i) eps_i a_i, rows r_j from ihs_srht_rows.
 *  GAUSS: S_ji = z_ji / sqrt(m), z from Philox counter (i, j/4, level, 2) by
 *         Box-Muller; arithmetic per the context's precision.
 * A: n x d (device), SA: m x d FP32 (device, overwritten).  1 <= m; for SRHT
 * m <= n_pad.  Uses context scratch. */
int ihs_sketch(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m,
               int32_t kind, uint64_t seed, int32_t level, float* SA);

/* Rows [row0, row0 + mrows) of the Gaussian SA of size m (S_ji = z_ji / sqrt(m),
 * z as for ihs_sketch, arithmetic per the context's precision) into SA_rows
 * (mrows x d FP32, device).  Row j of z does not depend on m, so with a level
 * fixed the sketch of size 2m is [S_m A / sqrt 2; these new rows]: the nested
 * sketches of the solver's nested mode.  row0 % 4 == 0, row0 + mrows <= m;
 * IHS_EINVAL otherwise. */
int ihs_sketch_rows(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, int64_t m, uint64_t seed,
                    int32_t level, int64_t row0, int64_t mrows, float* SA_rows);

/* Factor H_S = (SA)^T SA + nu^2 I (Eq. 3) for repeated applies: m < d caches
 * the Cholesky factor of nu^2 I_m + SA SA^T (Woodbury, App. B.4); m >= d
 * the Cholesky factor of H_S itself.  The Gram is formed on the tensor cores
 * from an exact three-piece BF16 split of SA's entries; the factor is held as
 * double-float pairs of binary32 (about 2^-46 relative; FP64 in contexts that
 * factor side by side).  SA (m x d, device) must stay valid
 * and unchanged while *F_h is in use.  nu > 0.  IHS_ENOTPD on breakdown. */
int ihs_factor(ihs_ctx* ctx, const float* SA, int64_t m, int64_t d, double nu, ihs_factor_t** F_h);
int ihs_factor_destroy(ihs_factor_t* F);

/* gt = H_S^{-1} g (d-vectors, device FP32) and, if r_h != NULL, the sketched
 * Newton decrement r = 1/2 g^T gt (Lemma 4.1) in FP64 (host; synchronises). */
int ihs_apply_hinv(ihs_ctx* ctx, const ihs_factor_t* F, const float* g, float* gt, double* r_h);

/* One fused pass over A: g = A^T (A x - b) + nu^2 x (gradient of Eq. 1, App.
 * B.1 stacked form) with compensated FP32 accumulation and a fixed-order
 * reduction (bitwise reproducible).  If axnorm2_h != NULL also returns
 * ||A x||^2 (FP64, host; synchronises).  A n x d, b n, x d, g d: device FP32. */
int ihs_grad(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d,
             double nu, const float* x, float* g, double* axnorm2_h);

/* Allocation-free variant of ihs_grad, for callers that cannot let a library
 * call cudaMalloc/cudaFree: code whose device memory belongs to another
 * allocator (a framework's caching pool, a fixed arena sized up front) and
 * latency-critical loops that must not block in cudaMalloc/cudaFree, which
 * synchronise the device.  The paper has no counterpart.
 *
 * It launches the same kernels with the same grid and the same fixed-order
 * reduction as ihs_grad for these inputs, so on a GPU with at most 160 SMs
 * (GB300 has 152) the two return the same bits; on a larger GPU the grid is
 * sized as if it had 160 SMs and the results agree within the gradient pass's
 * rounding bound.  It takes no context and allocates nothing: its
 * scratch is a file-scope device array of about 10 MiB (partials of at most
 * 160 x 8192 columns) that every GPU which loads the library holds until the
 * process exits.
 *  - stream: a cudaStream_t (NULL = legacy default stream) on the current
 *    device.  Asynchronous: returns once the work is enqueued.
 *  - A (n x d), b (n), x (d), g (d): device FP32 on the current device;
 *    axnorm2: device double receiving ||A x||^2, or NULL.
 *  - Limits: 4 <= d <= 8192, d % 4 == 0, n >= 1, A and x 16-byte aligned,
 *    nu >= 0 and finite; anything else returns IHS_EINVAL before any work.
 *  - Each call made outside stream capture looks up the device address of the
 *    scratch array (cudaGetSymbolAddress, with the stream's device current),
 *    so calls stay valid across cudaDeviceReset.  A call on a capturing stream
 *    reuses the address found by an earlier call on that device: make one call
 *    before any stream capture (IHS_EINVAL otherwise).
 *  - Every call on a device shares the one scratch array (each call rewrites
 *    it fully and clears its status word first): calls that overlap on the
 *    GPU, e.g. from two streams at once, race and must be serialised.
 *  - If the kernel's bounded wait ever gives up, g and *axnorm2 are NaN. */
int ihs_grad_noalloc(void* stream, const float* A, const float* b, int64_t n, int64_t d,
                     double nu, const float* x, float* g, double* axnorm2);

/* ---- the solver ---------------------------------------------------------- */
/* Adaptive IHS (Algorithm 1 or its gradient-only variant, per the context's
 * parameters; `tol` overrides params.tol when > 0).  x (device, d): on entry
 * x_1 (also x_0), on exit the last iterate.  rep_h may be NULL.  Returns IHS_OK
 * on convergence, IHS_EMAXITER if the limit was hit. */
int ihs_solve(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d,
              double nu, double tol, float* x, ihs_report* rep_h);

/* ihs_solve with HOST buffers, end to end: A_h (n x d), b_h (n) and x_h (d,
 * x_1 on entry, the last iterate on exit) are host FP32 arrays; the call copies
 * them into device memory the context owns (grown as needed, kept for the next
 * call), solves, copies x back and synchronises.  Page-locked host memory
 * (cudaHostAlloc / cudaHostRegister) gives the copies the full host-device
 * bandwidth; pageable memory works but is staged.  Errors as ihs_solve. */
int ihs_solve_host(ihs_ctx* ctx, const float* A_h, const float* b_h, int64_t n, int64_t d,
                   double nu, double tol, float* x_h, ihs_report* rep_h);

/* Underdetermined case, n <= d (App. A.2): the same controller on the dual
 * z* = argmin 1/2 ||A^T z||^2 + nu^2/2 ||z||^2 - b^T z, whose data matrix is A^T
 * (d x n) and whose gradient is A A^T z - b + nu^2 z; sketches are drawn over
 * the d rows of A^T with the context's kind, seed and levels.  z starts at 0;
 * on return x = A^T z (device, d floats; its content on entry is ignored).
 * A (n x d, row-major FP32) and b (n) are device buffers owned by the caller;
 * A^T is formed in context scratch (4nd bytes).  tol and rep_h as for
 * ihs_solve, applied to the dual iteration (rep_h->m_levels are dual sketch
 * sizes).  IHS_EINVAL when n > d, nu <= 0 or a pointer is NULL. */
int ihs_solve_dual(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d,
                   double nu, double tol, float* x, ihs_report* rep_h);

/* ---- decision trace and resumable solves --------------------------------- */
/* The controller's decisions, in order, as Algorithm 1 takes them (an auxiliary
 * record: the paper prints no trace).  `ratio` is the quantity the decision
 * tested: (r_p / r_1)^(1/t) against cbar_p for the Polyak candidate, r_gd / r_t
 * against cbar_gd for the gradient-IHS candidate (and for a doubling), and for
 * a stop the stopping test's value sqrt(2 Lambda r_t) / (tol ||Abar x_t||) <= 1. */
#define IHS_EV_STOP           0  /* stopping rule met before iteration t           */
#define IHS_EV_POLYAK         1  /* Polyak candidate accepted                      */
#define IHS_EV_POLYAK_REJECT  2  /* Polyak candidate rejected                      */
#define IHS_EV_GD             3  /* gradient-IHS candidate accepted                */
#define IHS_EV_GD_AT_CAP      4  /* rejected at the cap of m, accepted anyway       */
#define IHS_EV_DOUBLE         5  /* both rejected: m <- 2m, a new sketch           */
#define IHS_EV_FLOOR          6  /* rejected at the noise floor: stop              */

typedef struct ihs_event {
    int32_t kind;    /* IHS_EV_*                                                */
    int32_t t;       /* iteration index the decision belongs to                 */
    int64_t m;       /* sketch size in force when it was taken                  */
    double  r;       /* r_t at that moment (Lemma 4.1 decrement)                */
    double  ratio;   /* the tested value (see above)                            */
} ihs_event;

/* Copy up to `cap` events of the context's last solve (ihs_solve,
 * ihs_solve_resume or ihs_solve_dual) to ev_h (host) and their total count to
 * *count_h (host; may exceed cap).  ev_h may be NULL when cap == 0. */
int ihs_trace_events(const ihs_ctx* ctx, ihs_event* ev_h, int32_t cap, int32_t* count_h);

/* Also append every decision to a text file as one JSON object per line
 * ({"t":..,"m":..,"event":"gd","r":..,"ratio":..}), flushed per line, so that a
 * long solve can be followed while it runs.  path_h (host string) NULL or ""
 * closes the file.  IHS_EINVAL if the file cannot be opened. */
int ihs_ctx_set_trace_file(ihs_ctx* ctx, const char* path_h);

/* Where a solve stands between iterations: enough to continue it later with
 * the same result (an auxiliary facility; the paper's warm starts along a
 * regularisation path, Sec. 5, restart from x_t).  The sketch in force is not
 * stored: it is keyed by (seed, level) and redrawn on resume. */
typedef struct ihs_state {
    int32_t t;           /* iteration index of x_t; 0 = not started           */
    int32_t level;       /* log2 of the sketch size in force                   */
    int64_t m;           /* that sketch size                                   */
    double  r1;          /* r_1 of the run (base of the Polyak ratio)          */
    int32_t grad_passes; /* gradient passes so far                             */
    int32_t n_levels;    /* sketches drawn so far                              */
} ihs_state;

/* ihs_solve that starts from, and returns, an ihs_state.  x (device, d): x_t on
 * entry, the last iterate on exit.  x_prev (device, d): x_{t-1} on entry (read
 * by the Polyak candidate) and on exit.  st_h (host): st_h->t == 0 starts a new
 * run from x_1 = x (x_prev is then set to x, level from params.m_init);
 * otherwise the run continues at (t, level, r1) with the sketch of that level
 * redrawn.  params.max_iter bounds the total t, so a run split into calls with
 * rising limits takes the decisions of one uninterrupted run and, in the
 * default (non-nested) mode, returns the same bits; a nested-mode resume draws
 * the level's sketch in one piece, equal up to rounding.  On return *st_h
 * holds the state at exit (IHS_EMAXITER: resumable; IHS_OK: converged).
 * Errors as ihs_solve; IHS_EINVAL for an inconsistent state (m != 2^level,
 * t < 0, r1 <= 0 when t > 0). */
int ihs_solve_resume(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d,
                     double nu, double tol, float* x, float* x_prev, ihs_state* st_h,
                     ihs_report* rep_h);

/* ---- row-sharded data path (several GPUs, one process each) ------------- */
/* The method's data-parallel structure: the gradient of Eq. 1 is a sum over
 * row blocks, A^T (A x - b) = sum_p A_p^T (A_p x - b_p), and so is the sketch,
 * S A = sum_p S_{:,p} A_p (Sec. 1: the per-iteration products are where
 * distributed computation is needed).  A rank holds rows [row0, row0 + n) of a
 * matrix of n_total rows; its terms are summed over ranks, and the factor and
 * the controller run replicated on the summed values.  The draws are keyed by
 * global row index, so the summed sketch is the whole matrix's sketch: SRHT
 * signs and Hadamard parities of global rows (row0 a multiple of 1024, and a
 * shard ends on a multiple of 1024 unless it holds the last rows), Gaussian
 * columns z_{:,i} of global i.  FP8 Gaussian sketches scale each shard's
 * columns by that shard's own maxima (its term matches the unsharded FP8
 * sketch only to the E4M3 rounding). */

/* This shard's term of SA (m x d, device FP32, with the definition's 1/sqrt(m)
 * factor): the sum over shards is ihs_sketch of the whole A.
 * kind and seed/level as ihs_sketch; m <= n_pad(n_total) (SRHT) or n_total
 * (Gaussian).  Asynchronous. */
int ihs_sketch_shard(ihs_ctx* ctx, const float* A_local, int64_t n, int64_t d, int64_t row0,
                     int64_t n_total, int64_t m, int32_t kind, uint64_t seed, int32_t level,
                     float* SA_part);

/* This shard's gradient terms in FP64, unrounded (d + 1 doubles, device):
 * gp[0..d) = A_p^T (A_p x - b_p), gp[d] = ||A_p x||^2.  The gradient of Eq. 1
 * is sum_p gp[0..d) + nu^2 x.  Asynchronous. */
int ihs_grad_shard(ihs_ctx* ctx, const float* A_local, const float* b_local, int64_t n, int64_t d,
                   const float* x, double* gp);

/* In-place sum of a device buffer over the ranks of a sharded solve:
 * `count` elements of IHS_DTYPE_F32 or IHS_DTYPE_F64 at `buf`, whose contents
 * come from work already enqueued on `stream` (a cudaStream_t).  The callback
 * must order the sum after that work (e.g. an NCCL all-reduce enqueued on the
 * stream, or a synchronisation first) and have finished it, or enqueued it on
 * the stream, when it returns; every rank must receive the same sums.  Return
 * 0 on success; anything else makes the solve return IHS_ECUDA. */
#define IHS_DTYPE_F32 0
#define IHS_DTYPE_F64 1
typedef int (*ihs_allreduce_fn)(void* user, void* buf, int64_t count, int32_t dtype, void* stream);

/* ihs_solve on a row shard: every rank calls it with its rows (A_local n x d,
 * b_local n, device FP32) and the same ctx parameters, nu, tol and x_1; the
 * sketch of each level (m x d floats) and the gradient partials of each pass
 * (d + 1 doubles) are summed by `allreduce` (called from this host thread,
 * user passed through), and every rank takes the same decisions and returns
 * the same x.  Requirements as ihs_sketch_shard; params.nested must be 0.
 * Returns as ihs_solve. */
int ihs_solve_sharded(ihs_ctx* ctx, const float* A_local, const float* b_local, int64_t n, int64_t d,
                      int64_t row0, int64_t n_total, double nu, double tol, float* x,
                      ihs_report* rep_h, ihs_allreduce_fn allreduce, void* user);

/* ---- batched solves ------------------------------------------------------- */
/* One ridge problem of a batch.  A (n x d, row-major FP32), b (n) and x (d)
 * are device buffers owned by the caller; x holds x_1 on entry and x_T on
 * exit.  Problems may share A (a regularisation path: one A, many nu and b). */
typedef struct ihs_problem {
    const float* A;
    const float* b;
    int64_t n, d;
    double nu;
    float* x;
    int64_t m_init;   /* initial sketch size of this problem (a power of two),
                         e.g. from ihs_warm_start; 0 = params.m_init */
} ihs_problem;

/* Solves every problem of probs_h[0..count) with the gradient-IHS variant
 * (Sec. 5) under the context's parameters (kind, precision, rho, eta, m_init,
 * max_iter, floor, seed; params.variant must be IHS_VARIANT_GD, else
 * IHS_EINVAL).  Each problem runs the controller of ihs_solve, sketches keyed
 * by (seed, level) as there; the batch advances all problems one iteration
 * per round.  Problems that share A (same pointer, n and d; up to 64 per
 * group) share each level's sketch and take one multi-right-hand-side
 * gradient pass over A per round; the others take one launch over a work list
 * of their row tiles, whose height is autotuned on the first round.  The round
 * is captured once as a CUDA graph and replayed.  FP64 factorisations of
 * level changes run concurrently on internal streams.  tol > 0 overrides
 * params.tol.  reps_h (count entries, may be NULL): per-problem reports
 * (for the whole batch: ms_iterate = device time of all rounds, ms_sketch =
 * wall time of all level changes).  Returns IHS_OK when
 * the batch ran; per-problem outcomes (IHS_OK, IHS_EMAXITER, IHS_ENONFINITE)
 * are in reps_h[i].status.  Synchronous.  Device memory: the problems'
 * factors and sketches live at the same time. */
int ihs_solve_batched(ihs_ctx* ctx, const ihs_problem* probs_h, int32_t count, double tol,
                      ihs_report* reps_h);

/* m0_h[i] (and pred_h[i], may be NULL) as ihs_warm_start for every problem of
 * a batch (the x, b and m_init fields are not read): the features of all
 * problems, one forward pass of the network over them, one copy back.
 * Synchronous.  The result can be passed as the problems' m_init. */
int ihs_warm_start_batched(ihs_ctx* ctx, const float* params, const ihs_problem* probs_h, int32_t count,
                           uint64_t seed, int64_t* m0_h, float* pred_h);

/* ---- comparators (Sec. 5) ------------------------------------------------ */
/* Conjugate gradient on the normal equations (A^T A + nu^2 I) x = A^T b, or,
 * with precond_kind = IHS_SKETCH_SRHT / IHS_SKETCH_GAUSS, sketch-preconditioned
 * CG whose preconditioner is H_S of a sketch of size ceil(d / rho) (Gaussian)
 * or ceil(d ln d / rho) (SRHT) drawn at level 0 of params.seed, capped at n
 * (Gaussian) or n_pad (SRHT); precond_kind = -1 gives plain CG.  Sec. 5 names
 * the comparators and these sketch sizes; the preconditioner form and the
 * stopping rule ||r|| <= tol ||A^T b|| (r = A^T b - (A^T A + nu^2 I) x) are
 * this library's.  x (device, d): on entry x_0, on exit the last iterate.
 * rep_h (may be NULL): iterations, grad_passes (Hessian-vector products + 2),
 * m_final (sketch size), r_final (= ||r|| / ||A^T b||), ms_sketch
 * (preconditioner set-up), ms_iterate.  IHS_EMAXITER if max_iter is reached. */
int ihs_cg(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu, double tol,
           int32_t max_iter, int32_t precond_kind, float* x, ihs_report* rep_h);

/* ---- learned warm start ------------------------------------------------- */
/* Algorithm 1 may start the doubling of m at any power of two; the paper
 * starts at m = 1.  These calls predict the level the doubling settles at
 * (log2 m_T of a cold run) with a small network, so that a solve can start
 * just below it.  The paper has no counterpart: this is an addition of the
 * library.  A wrong prediction costs time only (the doubling still runs).
 *
 * Features (11 floats): log n, log d, log nu, then log sigma_k(P) for
 * k = 1, 2, 3, 4, 6, 8, 12, 16, where P = G A (32 x d) is the Gaussian sketch
 * of size 32 (N(0, 1/32) entries, the i.i.d. Gaussian draw of the sketch
 * module at level 200 of `seed`, FP32 products) and sigma_k(P)^2 are the
 * eigenvalues of P P^T in descending order (FP64 Gram, cyclic Jacobi),
 * clamped below at 1e-10 lambda_1.
 *
 * Network (parameters: one flat FP32 device vector of ihs_mlp_num_params()
 * entries): mu[11], sd[11], W1[64][11], b1[64], W2[64][64], b2[64], w3[64],
 * b3; y = w3 . tanh(W2 tanh(W1 (x - mu) / sd + b1) + b2) + b3.  mu and sd are
 * the feature normalisation, fixed by training and never updated.
 * Every call runs one CTA on ctx's stream; X is B x 11 row-major. */
int ihs_mlp_num_params(void);

/* feat (device, 11 floats) <- the features of (A, nu).  A device FP32 n x d,
 * nu > 0.  Asynchronous. */
int ihs_probe_features(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, double nu,
                       uint64_t seed, float* feat);

/* y[B] <- network(X).  All device pointers.  Asynchronous. */
int ihs_mlp_forward(ihs_ctx* ctx, const float* params, const float* X, int32_t B, float* y);

/* grad (device, num_params) <- gradient of the mean squared error
 * (1/B) sum_b (y_b - target_b)^2 with respect to params (zero for mu, sd);
 * *loss_h (host, may be NULL) <- that loss, which makes the call synchronous. */
int ihs_mlp_grad(ihs_ctx* ctx, const float* params, const float* X, const float* target,
                 int32_t B, float* grad, double* loss_h);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step >= 1 the 1-based
 * count for the bias corrections) on that loss, in place on params, adam_m and
 * adam_v (device, num_params each, zero before step 1).  *loss_h (may be NULL)
 * receives the loss at the parameters before the step. */
int ihs_mlp_train_step(ihs_ctx* ctx, float* params, float* adam_m, float* adam_v, int32_t step,
                       const float* X, const float* target, int32_t B, double lr, double* loss_h);

/* *m0_h <- 2^clamp(floor(y) - 1, 0, floor(log2 n)) where y is the network's
 * prediction for (A, nu) (optionally returned in *pred_h).  Synchronous.
 * IHS_ENONFINITE if y is not finite. */
int ihs_warm_start(ihs_ctx* ctx, const float* params, const float* A, int64_t n, int64_t d,
                   double nu, uint64_t seed, int64_t* m0_h, float* pred_h);

#ifdef __cplusplus
}
#endif

#endif /* IHS_H */
