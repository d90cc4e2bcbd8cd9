// Comparators of Sec. 5 on the GPU: conjugate gradient on the normal
// equations (A^T A + nu^2 I) x = A^T b and sketch-preconditioned CG.  The
// Hessian-vector product H p = A^T (A p) + nu^2 p is one fused gradient pass
// with a zero right-hand side; the preconditioner is the factored sketched
// Hessian of a sketch of size ceil(d / rho) (Gaussian) or ceil(d ln d / rho)
// (SRHT), capped at n (Gaussian) or n_pad (SRHT).  Stop when
// ||r|| <= tol ||A^T b||.  Scalars are FP64; vectors FP32.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace {

// partial sums (FP64) of a . b over blocks of 256
__global__ void k_dot_part(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
    __shared__ double sm[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    sm[threadIdx.x] = i < n ? (double)a[i] * (double)b[i] : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 256; ++k) s += sm[k];
        part[blockIdx.x] = s;
    }
}

__global__ void k_fold_to(const double* __restrict__ part, int count, double* __restrict__ out) {
    double s = 0.0;
    for (int k = 0; k < count; ++k) s += part[k];
    *out = s;
}

// x += alpha p; r -= alpha q; partials of ||r||^2
__global__ void k_cg_update(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                            const float* __restrict__ q, double alpha, int64_t n, double* __restrict__ part) {
    __shared__ double sm[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rr = 0.0;
    if (i < n) {
        x[i] = (float)((double)x[i] + alpha * (double)p[i]);
        const float ri = (float)((double)r[i] - alpha * (double)q[i]);
        r[i] = ri;
        rr = (double)ri * (double)ri;
    }
    sm[threadIdx.x] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 256; ++k) s += sm[k];
        part[blockIdx.x] = s;
    }
}

// p = z + beta p
__global__ void k_cg_dir(float* __restrict__ p, const float* __restrict__ z, double beta, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = (float)((double)z[i] + beta * (double)p[i]);
}

__global__ void k_neg_inplace(float* a, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = -a[i];
}

}  // namespace

extern "C" int ihs_cg(ihs_ctx* ctx, const float* A, const float* b, int64_t n, int64_t d, double nu, double tol,
                      int32_t max_iter, int32_t precond_kind, float* x, ihs_report* rep_h) {
    IhsRange range("ihs_cg");
    if (!ctx || !A || !b || !x || n < 1 || d < 1 || !(nu > 0.0) || !isfinite(nu) || !(tol > 0.0) || max_iter < 1)
        return IHS_EINVAL;
    if (precond_kind != -1 && precond_kind != IHS_SKETCH_SRHT && precond_kind != IHS_SKETCH_GAUSS) return IHS_EINVAL;
    cudaStream_t s = ctx->stream;
    ihs_report rep;
    memset(&rep, 0, sizeof(rep));
    const size_t vb = ((size_t)d * sizeof(float) + 255) & ~(size_t)255;
    const size_t nb = ((size_t)n * sizeof(float) + 255) & ~(size_t)255;
    const int64_t blocks = ceil_div64(d, 256);
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE, 5 * vb + nb + (size_t)(blocks + 64) * sizeof(double), &ws));
    char* base = static_cast<char*>(ws);
    float* r = reinterpret_cast<float*>(base);
    float* z = reinterpret_cast<float*>(base + vb);
    float* p = reinterpret_cast<float*>(base + 2 * vb);
    float* q = reinterpret_cast<float*>(base + 3 * vb);
    float* tmp = reinterpret_cast<float*>(base + 4 * vb);
    float* zero_b = reinterpret_cast<float*>(base + 5 * vb);
    double* part = reinterpret_cast<double*>(base + 5 * vb + nb);
    double* sc = part + blocks;   // device scalars
    IHS_CUDA_TRY(cudaMemsetAsync(zero_b, 0, (size_t)n * sizeof(float), s));
    IHS_CUDA_TRY(cudaMemsetAsync(tmp, 0, (size_t)d * sizeof(float), s));
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[2], s));

    // optional preconditioner
    ihs_factor_t Fs;
    const ihs_factor_t* F = nullptr;
    if (precond_kind >= 0) {
        const double rho = ctx->p.rho;
        int64_t m;
        if (precond_kind == IHS_SKETCH_GAUSS) m = std::min<int64_t>((int64_t)ceil(d / rho), n);
        else m = std::min<int64_t>((int64_t)ceil(d * log((double)d) / rho), next_pow2_64(n));
        void* sws = nullptr;
        IHS_TRY(ihs_scratch(ctx, SLOT_SOLVE_SA, (size_t)m * d * sizeof(float), &sws));
        float* SA = static_cast<float*>(sws);
        IHS_TRY(ihs_sketch_enqueue(ctx, A, n, d, m, precond_kind, ctx->p.seed, 0, SA));
        IHS_TRY(ihs_factor_scratch(ctx, SA, m, d, nu, &Fs));
        F = &Fs;
        rep.m_final = m;
        rep.m_levels[0] = m;
        rep.n_levels = 1;
    }
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[3], s));
    auto dot = [&](const float* a, const float* bb, double* out) -> int {
        k_dot_part<<<(unsigned)blocks, 256, 0, s>>>(a, bb, d, part);
        IHS_LAUNCH_CHECK();
        k_fold_to<<<1, 1, 0, s>>>(part, (int)blocks, out);
        IHS_LAUNCH_CHECK();
        return IHS_OK;
    };
    auto read = [&](int count) -> int {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, sc, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        IHS_CUDA_TRY(cudaStreamSynchronize(s));
        return IHS_OK;
    };
    // ||A^T b|| from the gradient at 0, r0 = -grad(x0)
    IHS_TRY(ihs_grad_enqueue(ctx, A, b, n, d, nu, tmp, q, nullptr));
    IHS_TRY(dot(q, q, sc + 0));
    IHS_TRY(ihs_grad_enqueue(ctx, A, b, n, d, nu, x, r, nullptr));
    k_neg_inplace<<<(unsigned)blocks, 256, 0, s>>>(r, d);
    IHS_LAUNCH_CHECK();
    IHS_TRY(dot(r, r, sc + 1));
    rep.grad_passes = 2;
    double rz;
    if (F) {
        IHS_TRY(ihs_apply_enqueue(ctx, F, r, z, sc + 2));   // z = M^{-1} r, sc[2] = r.z / 2
        IHS_TRY(read(3));
        rz = 2.0 * ctx->pinned[2];
        IHS_CUDA_TRY(cudaMemcpyAsync(p, z, (size_t)d * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
        IHS_TRY(read(2));
        rz = ctx->pinned[1];
        IHS_CUDA_TRY(cudaMemcpyAsync(p, r, (size_t)d * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    const double norm0 = sqrt(ctx->pinned[0]);
    double rnorm = sqrt(ctx->pinned[1]);
    int it = 0;
    int status = IHS_EMAXITER;
    while (true) {
        if (!isfinite(rnorm)) {
            status = IHS_ENONFINITE;
            break;
        }
        if (rnorm <= tol * norm0) {
            status = IHS_OK;
            break;
        }
        if (it >= max_iter) break;
        IHS_TRY(ihs_grad_enqueue(ctx, A, zero_b, n, d, nu, p, q, nullptr));   // q = H p
        rep.grad_passes++;
        IHS_TRY(dot(p, q, sc + 3));
        IHS_TRY(read(4));
        const double alpha = rz / ctx->pinned[3];
        k_cg_update<<<(unsigned)blocks, 256, 0, s>>>(x, r, p, q, alpha, d, part);
        IHS_LAUNCH_CHECK();
        k_fold_to<<<1, 1, 0, s>>>(part, (int)blocks, sc + 1);
        IHS_LAUNCH_CHECK();
        ++it;
        double rz_new;
        const float* zz = r;
        if (F) {
            IHS_TRY(ihs_apply_enqueue(ctx, F, r, z, sc + 2));
            IHS_TRY(read(3));
            rz_new = 2.0 * ctx->pinned[2];
            zz = z;
        } else {
            IHS_TRY(read(2));
            rz_new = ctx->pinned[1];
        }
        rnorm = sqrt(ctx->pinned[1]);
        if (rnorm <= tol * norm0) continue;   // converged: loop top reports it
        k_cg_dir<<<(unsigned)blocks, 256, 0, s>>>(p, zz, rz_new / rz, d);
        IHS_LAUNCH_CHECK();
        rz = rz_new;
    }
    IHS_CUDA_TRY(cudaEventRecord(ctx->ev[1], s));
    IHS_CUDA_TRY(cudaEventSynchronize(ctx->ev[1]));
    float ms_pre = 0.f, ms_it = 0.f;
    cudaEventElapsedTime(&ms_pre, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&ms_it, ctx->ev[3], ctx->ev[1]);
    rep.status = status;
    rep.iterations = it;
    rep.r_final = rnorm / norm0;
    rep.ms_sketch = ms_pre;
    rep.ms_iterate = ms_it;
    if (rep_h) *rep_h = rep;
    if (status == IHS_OK || status == IHS_EMAXITER) {
        const int s2 = ihs_check_status(ctx);
        if (s2 != IHS_OK) return s2;
    }
    return status;
}
