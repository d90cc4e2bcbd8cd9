// Learned warm start: predict the initial sketch size of the adaptive IHS.
//
// The paper starts the doubling at m = 1 (Algorithm 1 allows any initial size);
// this library adds a small network that predicts log2 of the size the doubling
// settles at, from cheap features of (A, nu), so that the solve can start a few
// levels below it.  The doubling still runs from the predicted size, so a wrong
// guess costs time, never accuracy.
//
// Features (11): log n, log d, log nu, and log sigma_k, k in {1,2,3,4,6,8,12,16},
// the singular values of a 32-row Gaussian probe P = G A / sqrt(32) (Philox
// stream GAUSS at the reserved level 200): eigenvalues of P P^T (FP64 Gram,
// cyclic Jacobi in one CTA).
//
// Network: x -> (x - mu) / sd -> tanh(W1 . + b1) (64) -> tanh(W2 . + b2) (64)
// -> w3 . + b3.  Parameters are one flat FP32 vector (layout below); training
// minimises the mean squared error to log2(m_settled) with Adam, all in one
// CTA per step (deterministic order).
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace {

constexpr int NF = 11, NH = 64;
// flat parameter layout
constexpr int OFF_MU = 0, OFF_SD = OFF_MU + NF, OFF_W1 = OFF_SD + NF, OFF_B1 = OFF_W1 + NH * NF,
              OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH,
              NPARAM = OFF_B3 + 1;
constexpr int kSamplesPerChunk = 4;   // 4 samples x 64 units = 256 threads

// Q = P P^T (32 x 32, FP64 from FP32 products), one warp per entry.
__global__ void k_probe_gram(const float* __restrict__ P, int d, double* __restrict__ Q) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= 32 * 32) return;
    const int r = w / 32, c = w % 32;
    double s = 0.0;
    for (int k = lane; k < d; k += 32) s = fma((double)P[r * d + k], (double)P[c * d + k], s);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) Q[r * 32 + c] = s;
}

// Eigenvalues of the symmetric 32 x 32 Q by cyclic Jacobi (round-robin pairs,
// 16 disjoint rotations per round, 31 rounds per sweep, at most 16 sweeps,
// stopping when the off-diagonal part is negligible), then the 11 features.
// One CTA per problem (blockIdx.x): Q of problem i at Q + 1024 i, its three
// size features at logs + 3 i, its features to feat + 11 i.
__global__ void __launch_bounds__(256) k_probe_features(const double* __restrict__ Qall,
                                                        const double* __restrict__ logs, float* __restrict__ featall) {
    const double* Q = Qall + (size_t)blockIdx.x * 1024;
    float* feat = featall + (size_t)blockIdx.x * NF;
    const double logn = logs[3 * blockIdx.x], logd = logs[3 * blockIdx.x + 1], lognu = logs[3 * blockIdx.x + 2];
    __shared__ double a[32][33];
    __shared__ double cs[16], sn[16];
    __shared__ int pp[16], qq[16];
    __shared__ double ev[32];
    __shared__ double red[2][8];
    __shared__ int done;
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * 32; e += 256) a[e / 32][e % 32] = 0.5 * (Q[e] + Q[(e % 32) * 32 + e / 32]);
    __syncthreads();
    for (int sweep = 0; sweep < 16; ++sweep) {
        // stop once the off-diagonal mass is below (1e-15)^2 of the diagonal's
        double off = 0.0, dia = 0.0;
        for (int e = tid; e < 32 * 32; e += 256) {
            const double v = a[e / 32][e % 32];
            if (e / 32 == e % 32)
                dia += v * v;
            else
                off += v * v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = off;
            red[1][tid >> 5] = dia;
        }
        __syncthreads();
        if (tid == 0) {
            double so = 0.0, sd = 0.0;
            for (int w = 0; w < 8; ++w) {
                so += red[0][w];
                sd += red[1][w];
            }
            done = so <= 1e-30 * sd;
        }
        __syncthreads();
        if (done) break;
        for (int r = 0; r < 31; ++r) {
            if (tid < 16) {
                int p, q;
                if (tid == 0) {
                    p = r % 31;
                    q = 31;
                } else {
                    p = (r + tid) % 31;
                    q = (r - tid + 31) % 31;
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                const double apq = a[p][q];
                double c = 1.0, s = 0.0;
                if (fabs(apq) > 1e-300) {
                    const double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                pp[tid] = p;
                qq[tid] = q;
                cs[tid] = c;
                sn[tid] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < 16 * 32; e += 256) {
                const int k = e / 32, col = e % 32;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = a[p][col], aq = a[q][col];
                a[p][col] = c * ap - s * aq;
                a[q][col] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J
            for (int e = tid; e < 16 * 32; e += 256) {
                const int k = e / 32, row = e % 32;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = a[row][p], aq = a[row][q];
                a[row][p] = c * ap - s * aq;
                a[row][q] = s * ap + c * aq;
            }
            __syncthreads();
        }
    }
    if (tid < 32) ev[tid] = a[tid][tid];
    __syncthreads();
    if (tid == 0) {
        // descending insertion sort of the 32 eigenvalues
        for (int i = 1; i < 32; ++i) {
            const double v = ev[i];
            int j = i - 1;
            while (j >= 0 && ev[j] < v) {
                ev[j + 1] = ev[j];
                --j;
            }
            ev[j + 1] = v;
        }
        const int ks[8] = {1, 2, 3, 4, 6, 8, 12, 16};
        // eigenvalues below 1e-10 lambda_1 (rank deficiency, d < 16) are clamped there
        const double floor_lam = fmax(ev[0] * 1e-10, 1e-300);
        feat[0] = (float)logn;
        feat[1] = (float)logd;
        feat[2] = (float)lognu;
        for (int i = 0; i < 8; ++i) feat[3 + i] = (float)(0.5 * log(fmax(ev[ks[i] - 1], floor_lam)));
    }
}

// Forward for up to kSamplesPerChunk samples at a time; thread = (sample, unit).
// mode 0: inference (y only); 1: gradient (grad, loss); 2: gradient + Adam step.
__global__ void __launch_bounds__(256) k_mlp(float* __restrict__ params, const float* __restrict__ X,
                                             const float* __restrict__ target, int B, int mode,
                                             float* __restrict__ y_out, float* __restrict__ grad_out,
                                             float* __restrict__ adam_m, float* __restrict__ adam_v, int step,
                                             float lr, double* __restrict__ loss_out) {
    __shared__ float p[NPARAM];
    __shared__ float g[NPARAM];
    __shared__ float xn[kSamplesPerChunk][NF];
    __shared__ float h1[kSamplesPerChunk][NH], h2[kSamplesPerChunk][NH];
    __shared__ float dz1[kSamplesPerChunk][NH], dz2[kSamplesPerChunk][NH];
    __shared__ float ysum[kSamplesPerChunk][2];
    __shared__ float dy[kSamplesPerChunk];
    __shared__ double loss_acc;
    const int tid = threadIdx.x;
    const int s = tid / NH, u = tid % NH;
    for (int e = tid; e < NPARAM; e += 256) {
        p[e] = params[e];
        g[e] = 0.f;
    }
    if (tid == 0) loss_acc = 0.0;
    __syncthreads();
    for (int b0 = 0; b0 < B; b0 += kSamplesPerChunk) {
        const int nb = min(kSamplesPerChunk, B - b0);
        if (tid < kSamplesPerChunk * NF) {
            const int ss = tid / NF, i = tid % NF;
            float v = 0.f;
            if (ss < nb) v = (X[(b0 + ss) * NF + i] - p[OFF_MU + i]) / p[OFF_SD + i];
            xn[ss][i] = v;
        }
        __syncthreads();
        {
            float z = p[OFF_B1 + u];
#pragma unroll
            for (int i = 0; i < NF; ++i) z = fmaf(p[OFF_W1 + u * NF + i], xn[s][i], z);
            h1[s][u] = tanhf(z);
        }
        __syncthreads();
        float yv;
        {
            float z = p[OFF_B2 + u];
            for (int k = 0; k < NH; ++k) z = fmaf(p[OFF_W2 + u * NH + k], h1[s][k], z);
            const float h = tanhf(z);
            h2[s][u] = h;
            float c = p[OFF_W3 + u] * h;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
            if ((tid & 31) == 0) ysum[s][(u >> 5)] = c;
        }
        __syncthreads();
        yv = p[OFF_B3] + ysum[s][0] + ysum[s][1];
        if (u == 0 && s < nb) {
            if (y_out) y_out[b0 + s] = yv;
            if (mode > 0) dy[s] = 2.0f * (yv - target[b0 + s]) / (float)B;
        }
        if (mode == 0) {
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            for (int ss = 0; ss < nb; ++ss) {
                const double e = (double)(p[OFF_B3] + ysum[ss][0] + ysum[ss][1]) - (double)target[b0 + ss];
                loss_acc += e * e;
            }
        }
        __syncthreads();
        {
            const float dys = s < nb ? dy[s] : 0.f;
            const float h = h2[s][u];
            dz2[s][u] = dys * p[OFF_W3 + u] * (1.f - h * h);
        }
        __syncthreads();
        {
            float dh = 0.f;
            for (int k = 0; k < NH; ++k) dh = fmaf(p[OFF_W2 + k * NH + u], dz2[s][k], dh);
            const float h = h1[s][u];
            dz1[s][u] = dh * (1.f - h * h);
        }
        __syncthreads();
        // accumulate gradients; each parameter has one owner thread that adds
        // the samples of the chunk in order (deterministic)
        for (int e = tid; e < NPARAM; e += 256) {
            float acc = 0.f;
            for (int ss = 0; ss < nb; ++ss) {
                float v = 0.f;
                if (e >= OFF_W1 && e < OFF_B1) {
                    const int uu = (e - OFF_W1) / NF, i = (e - OFF_W1) % NF;
                    v = dz1[ss][uu] * xn[ss][i];
                } else if (e >= OFF_B1 && e < OFF_W2) {
                    v = dz1[ss][e - OFF_B1];
                } else if (e >= OFF_W2 && e < OFF_B2) {
                    const int uu = (e - OFF_W2) / NH, k = (e - OFF_W2) % NH;
                    v = dz2[ss][uu] * h1[ss][k];
                } else if (e >= OFF_B2 && e < OFF_W3) {
                    v = dz2[ss][e - OFF_B2];
                } else if (e >= OFF_W3 && e < OFF_B3) {
                    v = dy[ss] * h2[ss][e - OFF_W3];
                } else if (e == OFF_B3) {
                    v = dy[ss];
                }
                acc += v;
            }
            g[e] += acc;
        }
        __syncthreads();
    }
    if (mode == 0) return;
    if (tid == 0 && loss_out) *loss_out = loss_acc / (double)B;
    if (grad_out)
        for (int e = tid; e < NPARAM; e += 256) grad_out[e] = g[e];
    if (mode == 2) {
        // Adam (Kingma & Ba): beta1 0.9, beta2 0.999, eps 1e-8; normalisation constants stay fixed
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
        for (int e = tid; e < NPARAM; e += 256) {
            if (e < OFF_W1) continue;
            const float ge = g[e];
            const float mm = b1 * adam_m[e] + (1.f - b1) * ge;
            const float vv = b2 * adam_v[e] + (1.f - b2) * ge * ge;
            adam_m[e] = mm;
            adam_v[e] = vv;
            params[e] = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        }
    }
}

}  // namespace

extern "C" int ihs_mlp_num_params(void) { return NPARAM; }

// The probe Gram of (A, d) into Q (32 x 32 FP64), using P (32 x d FP32).
static int probe_gram(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, uint64_t seed, float* P, double* Q) {
    IHS_TRY(ihs_gauss_fp32_enqueue(ctx, A, n, d, 32, seed, 200, P));
    k_probe_gram<<<(32 * 32 * 32 + 255) / 256, 256, 0, ctx->stream>>>(P, (int)d, Q);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

extern "C" int ihs_probe_features(ihs_ctx* ctx, const float* A, int64_t n, int64_t d, double nu, uint64_t seed,
                                  float* feat) {
    if (!ctx || !A || !feat || n < 1 || d < 1 || !(nu > 0.0)) return IHS_EINVAL;
    const size_t pbytes = ((size_t)32 * d * sizeof(float) + 255) & ~(size_t)255;
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_MISC, pbytes + 32 * 32 * sizeof(double) + 256, &ws));
    float* P = static_cast<float*>(ws);
    double* Q = reinterpret_cast<double*>(static_cast<char*>(ws) + pbytes);
    double* logs = Q + 32 * 32;
    IHS_TRY(probe_gram(ctx, A, n, d, seed, P, Q));
    const double hl[3] = {log((double)n), log((double)d), log(nu)};
    IHS_CUDA_TRY(cudaMemcpyAsync(logs, hl, sizeof(hl), cudaMemcpyHostToDevice, ctx->stream));
    k_probe_features<<<1, 256, 0, ctx->stream>>>(Q, logs, feat);
    IHS_LAUNCH_CHECK();
    IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));   // hl lives on this stack frame
    return IHS_OK;
}

extern "C" int ihs_mlp_forward(ihs_ctx* ctx, const float* params, const float* X, int32_t B, float* y) {
    if (!ctx || !params || !X || !y || B < 1) return IHS_EINVAL;
    k_mlp<<<1, 256, 0, ctx->stream>>>(const_cast<float*>(params), X, nullptr, B, 0, y, nullptr, nullptr, nullptr, 0,
                                      0.f, nullptr);
    IHS_LAUNCH_CHECK();
    return IHS_OK;
}

extern "C" int ihs_mlp_grad(ihs_ctx* ctx, const float* params, const float* X, const float* target, int32_t B,
                            float* grad, double* loss_h) {
    if (!ctx || !params || !X || !target || !grad || B < 1) return IHS_EINVAL;
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_MISC, 256, &ws));
    double* d_loss = static_cast<double*>(ws);
    k_mlp<<<1, 256, 0, ctx->stream>>>(const_cast<float*>(params), X, target, B, 1, nullptr, grad, nullptr, nullptr, 0,
                                      0.f, d_loss);
    IHS_LAUNCH_CHECK();
    if (loss_h) {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, d_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *loss_h = ctx->pinned[0];
    }
    return IHS_OK;
}

extern "C" int ihs_mlp_train_step(ihs_ctx* ctx, float* params, float* adam_m, float* adam_v, int32_t step,
                                  const float* X, const float* target, int32_t B, double lr, double* loss_h) {
    if (!ctx || !params || !adam_m || !adam_v || !X || !target || B < 1 || step < 1 || !(lr > 0.0))
        return IHS_EINVAL;
    void* ws = nullptr;
    IHS_TRY(ihs_scratch(ctx, SLOT_MISC, 256, &ws));
    double* d_loss = static_cast<double*>(ws);
    k_mlp<<<1, 256, 0, ctx->stream>>>(params, X, target, B, 2, nullptr, nullptr, adam_m, adam_v, step, (float)lr,
                                      d_loss);
    IHS_LAUNCH_CHECK();
    if (loss_h) {
        IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, d_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *loss_h = ctx->pinned[0];
    }
    return IHS_OK;
}

extern "C" int ihs_warm_start(ihs_ctx* ctx, const float* params, const float* A, int64_t n, int64_t d, double nu,
                              uint64_t seed, int64_t* m0, float* pred_h) {
    IhsRange range("ihs_warm_start");
    if (!ctx || !params || !A || !m0 || n < 1 || d < 1 || !(nu > 0.0)) return IHS_EINVAL;
    void* ws = nullptr;
    // features and prediction live past the probe's scratch in the same slot
    const size_t pbytes = ((size_t)32 * d * sizeof(float) + 255) & ~(size_t)255;
    const size_t off = pbytes + 32 * 32 * sizeof(double) + 256;
    IHS_TRY(ihs_scratch(ctx, SLOT_MISC, off + 256, &ws));
    float* feat = reinterpret_cast<float*>(static_cast<char*>(ws) + off);
    float* y = feat + 16;
    IHS_TRY(ihs_probe_features(ctx, A, n, d, nu, seed, feat));
    k_mlp<<<1, 256, 0, ctx->stream>>>(const_cast<float*>(params), feat, nullptr, 1, 0, y, nullptr, nullptr, nullptr,
                                      0, 0.f, nullptr);
    IHS_LAUNCH_CHECK();
    float pred = 0.f;
    IHS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, y, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    IHS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    memcpy(&pred, ctx->pinned, sizeof(float));
    if (!isfinite(pred)) return IHS_ENONFINITE;
    // start one level below the predicted settled level (the doubling corrects
    // an under-estimate; an over-estimate only costs a larger sketch)
    int lvl = (int)floorf(pred) - 1;
    int cap = 0;
    while (cap < 62 && ((int64_t)1 << (cap + 1)) <= n) ++cap;
    lvl = lvl < 0 ? 0 : (lvl > cap ? cap : lvl);
    *m0 = (int64_t)1 << lvl;
    if (pred_h) *pred_h = pred;
    return IHS_OK;
}

extern "C" int ihs_warm_start_batched(ihs_ctx* ctx, const float* params, const ihs_problem* probs_h, int32_t count,
                                      uint64_t seed, int64_t* m0_h, float* pred_h) {
    if (!ctx || !params || !probs_h || !m0_h || count < 1) return IHS_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!probs_h[i].A || probs_h[i].n < 1 || probs_h[i].d < 1 || !(probs_h[i].nu > 0.0)) return IHS_EINVAL;
    // features of all problems (one row each), then one forward pass and one copy
    float* feat = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&feat), (size_t)count * 16 * sizeof(float), ctx->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return IHS_ENOMEM;
    }
    float* y = feat + (size_t)count * NF;
    int st = IHS_OK;
    // probe Grams one by one (P reused in stream order), then the eigenvalues of
    // all problems in one launch (one CTA each)
    int64_t dmax = 1;
    for (int i = 0; i < count; ++i) dmax = probs_h[i].d > dmax ? probs_h[i].d : dmax;
    double* Qall = nullptr;
    float* P = nullptr;
    std::vector<double> hl(3 * (size_t)count);
    for (int i = 0; i < count; ++i) {
        hl[3 * i] = log((double)probs_h[i].n);
        hl[3 * i + 1] = log((double)probs_h[i].d);
        hl[3 * i + 2] = log(probs_h[i].nu);
    }
    if (cudaMallocAsync(reinterpret_cast<void**>(&Qall), (size_t)count * (1024 + 3) * sizeof(double), ctx->stream) !=
            cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&P), (size_t)32 * dmax * sizeof(float), ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        st = IHS_ENOMEM;
    }
    double* logs = Qall + (size_t)count * 1024;
    // the probe depends on (A, seed) only: problems sharing A share its Gram
    std::vector<int> first(count, -1);
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i && first[i] < 0; ++j)
            if (first[j] < 0 && probs_h[j].A == probs_h[i].A && probs_h[j].n == probs_h[i].n &&
                probs_h[j].d == probs_h[i].d)
                first[i] = j;
    for (int i = 0; i < count && st == IHS_OK; ++i) {
        if (first[i] < 0) {
            st = probe_gram(ctx, probs_h[i].A, probs_h[i].n, probs_h[i].d, seed, P, Qall + (size_t)i * 1024);
        } else if (cudaMemcpyAsync(Qall + (size_t)i * 1024, Qall + (size_t)first[i] * 1024, 1024 * sizeof(double),
                                   cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            st = IHS_ECUDA;
        }
    }
    if (st == IHS_OK &&
        cudaMemcpyAsync(logs, hl.data(), hl.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        st = IHS_ECUDA;
    if (st == IHS_OK) {
        k_probe_features<<<(unsigned)count, 256, 0, ctx->stream>>>(Qall, logs, feat);
        if (cudaGetLastError() != cudaSuccess) st = IHS_ECUDA;
        ihs_count_launch();
    }
    if (st == IHS_OK) {
        k_mlp<<<1, 256, 0, ctx->stream>>>(const_cast<float*>(params), feat, nullptr, count, 0, y, nullptr, nullptr,
                                          nullptr, 0, 0.f, nullptr);
        if (cudaGetLastError() != cudaSuccess) st = IHS_ECUDA;
        ihs_count_launch();
    }
    float* hy = nullptr;
    if (st == IHS_OK && cudaMallocHost(reinterpret_cast<void**>(&hy), (size_t)count * sizeof(float)) != cudaSuccess)
        st = IHS_ENOMEM;
    if (st == IHS_OK && (cudaMemcpyAsync(hy, y, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream) !=
                             cudaSuccess ||
                         cudaStreamSynchronize(ctx->stream) != cudaSuccess))
        st = IHS_ECUDA;
    cudaFreeAsync(feat, ctx->stream);
    if (Qall) cudaFreeAsync(Qall, ctx->stream);
    if (P) cudaFreeAsync(P, ctx->stream);
    if (st == IHS_OK) {
        for (int i = 0; i < count; ++i) {
            const float pred = hy[i];
            if (!isfinite(pred)) {
                st = IHS_ENONFINITE;
                break;
            }
            int lvl = (int)floorf(pred) - 1;
            int cap = 0;
            while (cap < 62 && ((int64_t)1 << (cap + 1)) <= probs_h[i].n) ++cap;
            lvl = lvl < 0 ? 0 : (lvl > cap ? cap : lvl);
            m0_h[i] = (int64_t)1 << lvl;
            if (pred_h) pred_h[i] = pred;
        }
    }
    if (hy) cudaFreeHost(hy);
    return st;
}
