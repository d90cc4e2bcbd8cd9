// Context, scratch arena, parameters and status plumbing of the C ABI.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <new>

#include "common.cuh"

#include <atomic>
#include <vector>

namespace {
thread_local char g_last_error[512];
std::atomic<int64_t> g_launches{0};
}

void ihs_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void ihs_count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t ihs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void ihs_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s (%d) at %s:%d: %s", cudaGetErrorString(e), (int)e, file,
             line, what);
}

void ihs_set_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

extern "C" const char* ihs_last_error(void) { return g_last_error; }

extern "C" const char* ihs_version(void) { return "ihs-gb300 0.1 (sm_103a)"; }

extern "C" int ihs_params_default(ihs_params* p) {
    if (!p) return IHS_EINVAL;
    memset(p, 0, sizeof(*p));
    p->kind = IHS_SKETCH_SRHT;
    p->variant = IHS_VARIANT_GD;
    p->precision = IHS_PREC_FP32;
    p->max_iter = 500;
    p->m_init = 1;
    p->rho = 0.1;
    p->eta = 0.01;
    p->tol = 1e-5;
    p->floor = 0.0;
    p->seed = 0;
    return IHS_OK;
}

static int validate_params(const ihs_params* p) {
    if (p->kind != IHS_SKETCH_SRHT && p->kind != IHS_SKETCH_GAUSS) return IHS_EINVAL;
    if (p->variant != IHS_VARIANT_GD && p->variant != IHS_VARIANT_POLYAK) return IHS_EINVAL;
    if (p->precision < IHS_PREC_FP32 || p->precision > IHS_PREC_FP8) return IHS_EINVAL;
    if (p->m_init < 1 || (p->m_init & (p->m_init - 1))) return IHS_EINVAL;
    if (!(p->rho > 0.0 && p->rho < 1.0)) return IHS_EINVAL;
    if (p->kind == IHS_SKETCH_GAUSS && !(p->rho <= 0.18 && p->eta > 0.0 && p->eta <= 0.01)) return IHS_EINVAL;
    if (!(p->tol >= 0.0) || !(p->floor >= 0.0) || p->max_iter < 1) return IHS_EINVAL;
    return IHS_OK;
}

extern "C" int ihs_ctx_create(ihs_ctx** out, void* stream, const ihs_params* p) {
    if (!out) return IHS_EINVAL;
    *out = nullptr;
    ihs_params prm;
    if (p) {
        prm = *p;
    } else {
        ihs_params_default(&prm);
    }
    IHS_TRY(validate_params(&prm));
    ihs_ctx* c = new (std::nothrow) ihs_ctx;
    if (!c) return IHS_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->p = prm;
    c->stream = static_cast<cudaStream_t>(stream);
    {
        const char* e = getenv("IHS_TEST_BARRIER_UNREACHABLE");
        c->test_bar_unreachable = (e && e[0] == '1') ? 1 : 0;
        const char* l = getenv("IHS_BARRIER_LIMIT_MS");
        const long ms = l ? strtol(l, nullptr, 10) : 0;
        c->bar_limit_ns = (ms >= 1 && ms <= 60000) ? (uint64_t)ms * 1000000ull : 1000000000ull;
        const char* cp = getenv("IHS_CHOL_CTAS_PER_SM");
        c->chol_per_sm = (cp && cp[0] == '1') ? 1 : 2;
        const char* ac = getenv("IHS_APPLY_CTAS");
        c->apply_ctas = ac ? (int)strtol(ac, nullptr, 10) : 0;
        const char* gs = getenv("IHS_GRAM_SIMT");
        c->gram_simt = (gs && gs[0] == '1') ? 1 : 0;
    }
    int st = IHS_OK;
    do {
        if (cudaGetDevice(&c->device) != cudaSuccess) { st = IHS_ECUDA; break; }
        if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            st = IHS_ECUDA;
            break;
        }
        if (cudaMallocHost(&c->pinned, 64 * sizeof(double)) != cudaSuccess) { st = IHS_ENOMEM; break; }
        if (cudaMalloc(&c->d_status, 256) != cudaSuccess) { st = IHS_ENOMEM; break; }
        if (cudaMemsetAsync(c->d_status, 0, 256, c->stream) != cudaSuccess) { st = IHS_ECUDA; break; }
        for (int i = 0; i < 6; ++i)
            if (cudaEventCreate(&c->ev[i]) != cudaSuccess) { st = IHS_ECUDA; break; }
        if (st != IHS_OK) break;
        if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess) { st = IHS_ECUDA; break; }
        for (int i = 0; i < 8; ++i)
            if (cudaEventCreateWithFlags(&c->fev[i], cudaEventDisableTiming) != cudaSuccess) { st = IHS_ECUDA; break; }
    } while (0);
    if (st != IHS_OK) {
        ihs_ctx_destroy(c);
        return st;
    }
    *out = c;
    return IHS_OK;
}

extern "C" int ihs_ctx_destroy(ihs_ctx* c) {
    if (!c) return IHS_OK;
    cudaStreamSynchronize(c->stream);
    if (c->lanes) ihs_lanes_destroy(c->lanes);
    for (int i = 0; i < SLOT_COUNT; ++i)
        if (c->buf[i]) cudaFree(c->buf[i]);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->d_status) cudaFree(c->d_status);
    for (int i = 0; i < 6; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (int i = 0; i < 8; ++i)
        if (c->fev[i]) cudaEventDestroy(c->fev[i]);
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaStreamDestroy(c->aux);
    }
    ihs_trace_free(c);
    delete c;
    return IHS_OK;
}

extern "C" int ihs_ctx_set_params(ihs_ctx* c, const ihs_params* p) {
    if (!c || !p) return IHS_EINVAL;
    IHS_TRY(validate_params(p));
    c->p = *p;
    return IHS_OK;
}

int ihs_scratch(ihs_ctx* c, int slot, size_t bytes, void** out) {
    if (slot < 0 || slot >= SLOT_COUNT) return IHS_EINVAL;
    if (bytes == 0) bytes = 16;
    if (c->buf_bytes[slot] < bytes) {
        if (c->buf[slot]) {
            // in-flight kernels may still use the old buffer
            IHS_CUDA_TRY(cudaStreamSynchronize(c->stream));
            cudaFree(c->buf[slot]);
            c->buf[slot] = nullptr;
            c->buf_bytes[slot] = 0;
        }
        const size_t grow = bytes + bytes / 4 + 4096;
        if (cudaMalloc(&c->buf[slot], grow) != cudaSuccess) {
            cudaGetLastError();
            return IHS_ENOMEM;
        }
        c->buf_bytes[slot] = grow;
    }
    *out = c->buf[slot];
    return IHS_OK;
}

int ihs_tensor_map_f32(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return IHS_ECUDA;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (((uintptr_t)base & 15) || ((ld * 4) & 15) || rows < 1 || cols < 1) return IHS_EINVAL;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? IHS_OK : IHS_EINVAL;
}

int ihs_check_status(ihs_ctx* c) {
    unsigned h = 0;
    IHS_CUDA_TRY(cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    IHS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (h) {
        IHS_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
        if (h & IHS_DEV_TIMEOUT) {
            // a fused apply that gave up leaves its barrier counter and last-CTA
            // ticket (words 32..41) behind: start both again from zero
            IHS_CUDA_TRY(cudaMemsetAsync(c->d_status + 32, 0, 10 * sizeof(unsigned), c->stream));
            IHS_CUDA_TRY(cudaStreamSynchronize(c->stream));
            c->apply_epoch = 0;
            return IHS_ETIMEOUT;
        }
        if (h & IHS_DEV_NOTPD) return IHS_ENOTPD;
    }
    IHS_CUDA_TRY(cudaGetLastError());
    return IHS_OK;
}

// ---------------------------------------------------------------------------
// Decision log of the controller.

namespace {

struct TraceLog {
    std::vector<ihs_event> ev;
    FILE* file = nullptr;
};

TraceLog* trace_of(ihs_ctx* c, bool create) {
    if (!c->trace && create) c->trace = new (std::nothrow) TraceLog;
    return static_cast<TraceLog*>(c->trace);
}

const char* event_name(int kind) {
    switch (kind) {
        case IHS_EV_STOP: return "stop";
        case IHS_EV_POLYAK: return "polyak";
        case IHS_EV_POLYAK_REJECT: return "polyak_reject";
        case IHS_EV_GD: return "gd";
        case IHS_EV_GD_AT_CAP: return "gd_at_cap";
        case IHS_EV_DOUBLE: return "double";
        case IHS_EV_FLOOR: return "floor";
        default: return "unknown";
    }
}

}  // namespace

void ihs_trace_reset(ihs_ctx* c) {
    TraceLog* T = trace_of(c, true);
    if (T) T->ev.clear();
}

void ihs_trace_add(ihs_ctx* c, int kind, int t, int64_t m, double r, double ratio) {
    TraceLog* T = trace_of(c, true);
    if (!T) return;
    ihs_event e;
    e.kind = kind;
    e.t = t;
    e.m = m;
    e.r = r;
    e.ratio = ratio;
    T->ev.push_back(e);
    if (T->file) {
        fprintf(T->file, "{\"t\": %d, \"m\": %lld, \"event\": \"%s\", \"r\": %.17g, \"ratio\": %.17g}\n", t,
                (long long)m, event_name(kind), r, ratio);
        fflush(T->file);
    }
}

void ihs_trace_free(ihs_ctx* c) {
    TraceLog* T = trace_of(c, false);
    if (!T) return;
    if (T->file) fclose(T->file);
    delete T;
    c->trace = nullptr;
}

extern "C" int ihs_trace_events(const ihs_ctx* c, ihs_event* ev, int32_t cap, int32_t* count) {
    if (!c || !count || cap < 0 || (cap > 0 && !ev)) return IHS_EINVAL;
    const TraceLog* T = static_cast<const TraceLog*>(c->trace);
    const size_t total = T ? T->ev.size() : 0;
    *count = (int32_t)total;
    for (size_t i = 0; i < total && i < (size_t)cap; ++i) ev[i] = T->ev[i];
    return IHS_OK;
}

extern "C" int ihs_ctx_set_trace_file(ihs_ctx* c, const char* path) {
    if (!c) return IHS_EINVAL;
    TraceLog* T = trace_of(c, true);
    if (!T) return IHS_ENOMEM;
    if (T->file) {
        fclose(T->file);
        T->file = nullptr;
    }
    if (path && path[0]) {
        T->file = fopen(path, "a");
        if (!T->file) return IHS_EINVAL;
    }
    return IHS_OK;
}
