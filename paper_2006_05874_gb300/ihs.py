"""Thin Python binding of the C ABI in include/ihs.h (argument marshalling only).

Every computation happens in libihs.so (hand-written CUDA for sm_103a).  There is
no fallback: if the library is missing, `load()` raises.  Tensors are torch CUDA
tensors; their device pointers are passed through unchanged.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libihs.so")

IHS_OK, IHS_EINVAL, IHS_ENOMEM, IHS_ENOTPD = 0, -1, -2, -3
IHS_ENONFINITE, IHS_EMCAP, IHS_EMAXITER, IHS_ETIMEOUT, IHS_ECUDA = -4, -5, -6, -7, -8
SKETCH_SRHT, SKETCH_GAUSS = 0, 1
VARIANT_GD, VARIANT_POLYAK = 0, 1
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
REPORT_MAX_LEVELS = 40

STATUS_NAMES = {0: "IHS_OK", -1: "IHS_EINVAL", -2: "IHS_ENOMEM", -3: "IHS_ENOTPD", -4: "IHS_ENONFINITE",
                -5: "IHS_EMCAP", -6: "IHS_EMAXITER", -7: "IHS_ETIMEOUT", -8: "IHS_ECUDA"}
KINDS = {"srht": SKETCH_SRHT, "gauss": SKETCH_GAUSS}
VARIANTS = {"gd": VARIANT_GD, "polyak": VARIANT_POLYAK}
PRECISIONS = {"fp32": PREC_FP32, "bf16": PREC_BF16, "fp8": PREC_FP8}


class IHSError(RuntimeError):
    def __init__(self, func, status, detail=""):
        self.status = status
        super().__init__("%s returned %s%s" % (func, STATUS_NAMES.get(status, status),
                                              (": " + detail) if detail else ""))


class Params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("m_init", ctypes.c_int64), ("rho", ctypes.c_double),
                ("eta", ctypes.c_double), ("tol", ctypes.c_double), ("floor", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("nested", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("grad_passes", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("accepted_polyak", ctypes.c_int32),
                ("accepted_gd", ctypes.c_int32), ("rejected", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("m_final", ctypes.c_int64), ("m_levels", ctypes.c_int64 * REPORT_MAX_LEVELS),
                ("r1", ctypes.c_double), ("r_final", ctypes.c_double), ("axnorm_final", ctypes.c_double),
                ("ms_sketch", ctypes.c_double), ("ms_iterate", ctypes.c_double), ("ms_grad", ctypes.c_double)]

    def levels(self):
        return [int(self.m_levels[i]) for i in range(min(self.n_levels, REPORT_MAX_LEVELS))]


EVENT_NAMES = {0: "stop", 1: "polyak", 2: "polyak_reject", 3: "gd", 4: "gd_at_cap", 5: "double", 6: "floor"}


class Event(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t", ctypes.c_int32), ("m", ctypes.c_int64), ("r", ctypes.c_double),
                ("ratio", ctypes.c_double)]

    def as_tuple(self):
        """(event name, t, m, ratio), the layout of the oracle's trace entries."""
        return (EVENT_NAMES.get(self.kind, str(self.kind)), int(self.t), int(self.m), float(self.ratio))


class State(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int32), ("level", ctypes.c_int32), ("m", ctypes.c_int64), ("r1", ctypes.c_double),
                ("grad_passes", ctypes.c_int32), ("n_levels", ctypes.c_int32)]


# ihs_allreduce_fn: int (*)(void* user, void* buf, int64_t count, int32_t dtype, void* stream)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_void_p)

_vp, _i64, _i32, _u64, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
_SIGNATURES = {
    "ihs_version": ([], ctypes.c_char_p),
    "ihs_last_error": ([], ctypes.c_char_p),
    "ihs_kernel_launches": ([], ctypes.c_int64),
    "ihs_params_default": ([ctypes.POINTER(Params)], ctypes.c_int),
    "ihs_ctx_create": ([ctypes.POINTER(_vp), _vp, ctypes.POINTER(Params)], ctypes.c_int),
    "ihs_ctx_destroy": ([_vp], ctypes.c_int),
    "ihs_ctx_set_params": ([_vp, ctypes.POINTER(Params)], ctypes.c_int),
    "ihs_srht_signs": ([_vp, _i64, _u64, _i32, _vp], ctypes.c_int),
    "ihs_srht_rows": ([_vp, _i64, _i64, _u64, _i32, _vp], ctypes.c_int),
    "ihs_sketch": ([_vp, _vp, _i64, _i64, _i64, _i32, _u64, _i32, _vp], ctypes.c_int),
    "ihs_sketch_rows": ([_vp, _vp, _i64, _i64, _i64, _u64, _i32, _i64, _i64, _vp], ctypes.c_int),
    "ihs_factor": ([_vp, _vp, _i64, _i64, _dbl, ctypes.POINTER(_vp)], ctypes.c_int),
    "ihs_factor_destroy": ([_vp], ctypes.c_int),
    "ihs_apply_hinv": ([_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl)], ctypes.c_int),
    "ihs_grad": ([_vp, _vp, _vp, _i64, _i64, _dbl, _vp, _vp, ctypes.POINTER(_dbl)], ctypes.c_int),
    "ihs_solve": ([_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _vp, ctypes.POINTER(Report)], ctypes.c_int),
    "ihs_solve_host": ([_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _vp, ctypes.POINTER(Report)], ctypes.c_int),
    "ihs_solve_resume": ([_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _vp, _vp, ctypes.POINTER(State),
                          ctypes.POINTER(Report)], ctypes.c_int),
    "ihs_sketch_shard": ([_vp, _vp, _i64, _i64, _i64, _i64, _i64, _i32, _u64, _i32, _vp], ctypes.c_int),
    "ihs_grad_shard": ([_vp, _vp, _vp, _i64, _i64, _vp, _vp], ctypes.c_int),
    "ihs_solve_sharded": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _dbl, _dbl, _vp, ctypes.POINTER(Report),
                           ALLREDUCE_FN, _vp], ctypes.c_int),
    "ihs_trace_events": ([_vp, ctypes.POINTER(Event), _i32, ctypes.POINTER(_i32)], ctypes.c_int),
    "ihs_ctx_set_trace_file": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "ihs_solve_dual": ([_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _vp, ctypes.POINTER(Report)], ctypes.c_int),
    "ihs_cg": ([_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _i32, _i32, _vp, ctypes.POINTER(Report)], ctypes.c_int),
    "ihs_grad_noalloc": ([_vp, _vp, _vp, _i64, _i64, _dbl, _vp, _vp, _vp], ctypes.c_int),
    "ihs_solve_batched": ([_vp, _vp, _i32, _dbl, _vp], ctypes.c_int),
    "ihs_warm_start_batched": ([_vp, _vp, _vp, _i32, _u64, _vp, _vp], ctypes.c_int),
    "ihs_mlp_num_params": ([], ctypes.c_int),
    "ihs_probe_features": ([_vp, _vp, _i64, _i64, _dbl, _u64, _vp], ctypes.c_int),
    "ihs_mlp_forward": ([_vp, _vp, _vp, _i32, _vp], ctypes.c_int),
    "ihs_mlp_grad": ([_vp, _vp, _vp, _vp, _i32, _vp, ctypes.POINTER(_dbl)], ctypes.c_int),
    "ihs_mlp_train_step": ([_vp, _vp, _vp, _vp, _i32, _vp, _vp, _i32, _dbl, ctypes.POINTER(_dbl)], ctypes.c_int),
    "ihs_warm_start": ([_vp, _vp, _vp, _i64, _i64, _dbl, _u64, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_float)],
                       ctypes.c_int),
}

_lib = None


def load(path=LIB_PATH):
    """Load libihs.so (built by paper_2006_05874_gb300.build.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libihs.so not built (%s); run paper_2006_05874_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(func, status):
    if status != IHS_OK:
        detail = ""
        if status == IHS_ECUDA:
            detail = _lib.ihs_last_error().decode()
        raise IHSError(func, status, detail)
    return status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def version():
    return load().ihs_version().decode()


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load().ihs_kernel_launches())


def grad_noalloc(A, b, nu, x, g, axnorm2=None, stream=None):
    """ihs_grad_noalloc: the gradient pass without a context and without any
    allocation (scratch in a fixed device array; see include/ihs.h)."""
    import torch

    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream() if stream is None else stream
    if stream.device.index != dev:
        raise ValueError("the stream is on cuda:%d, the current device is cuda:%d" % (stream.device.index, dev))
    for name, t, dtype in (("A", A, torch.float32), ("b", b, torch.float32), ("x", x, torch.float32),
                           ("g", g, torch.float32), ("axnorm2", axnorm2, torch.float64)):
        if t is None:
            continue
        if t.device.type != "cuda" or t.device.index != dev:
            raise ValueError("%s must be on the current device cuda:%d (got %s)" % (name, dev, t.device))
        if t.dtype != dtype:
            raise ValueError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    n, d = A.shape
    if b.numel() != n or x.numel() != d or g.numel() != d or (axnorm2 is not None and axnorm2.numel() < 1):
        raise ValueError("shapes: A %s, b %d, x %d, g %d" % (tuple(A.shape), b.numel(), x.numel(), g.numel()))
    _check("ihs_grad_noalloc", load().ihs_grad_noalloc(ctypes.c_void_p(stream.cuda_stream), _ptr(A), _ptr(b), n, d,
                                                       float(nu), _ptr(x), _ptr(g), _ptr(axnorm2)))


def default_params(**kw):
    p = Params()
    load().ihs_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "kind":
            v = KINDS.get(v, v)
        elif k == "variant":
            v = VARIANTS.get(v, v)
        elif k == "precision":
            v = PRECISIONS.get(v, v)
        setattr(p, k, v)
    return p


class Factor:
    def __init__(self, ctx, handle, SA):
        self.ctx, self.handle, self.SA = ctx, handle, SA

    def apply_hinv(self, g, gt, want_r=True):
        r = ctypes.c_double(0.0)
        _check("ihs_apply_hinv", _lib.ihs_apply_hinv(self.ctx.handle, self.handle, _ptr(g), _ptr(gt),
                                                     ctypes.byref(r) if want_r else None))
        return r.value if want_r else None

    def destroy(self):
        if self.handle:
            _lib.ihs_factor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Problem(ctypes.Structure):
    """One problem of ihs_solve_batched (device pointers)."""
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int64),
                ("nu", ctypes.c_double), ("x", ctypes.c_void_p), ("m_init", ctypes.c_int64)]


class Context:
    """An ihs_ctx bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, params=None, stream=None, **kw):
        import torch

        import weakref

        lib = load()
        self._factors = weakref.WeakSet()
        self.params = params if params is not None else default_params(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check("ihs_ctx_create", lib.ihs_ctx_create(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream),
                                                    ctypes.byref(self.params)))
        self.handle = h

    def set_params(self, **kw):
        for k, v in kw.items():
            if k == "kind":
                v = KINDS.get(v, v)
            elif k == "variant":
                v = VARIANTS.get(v, v)
            elif k == "precision":
                v = PRECISIONS.get(v, v)
            setattr(self.params, k, v)
        _check("ihs_ctx_set_params", _lib.ihs_ctx_set_params(self.handle, ctypes.byref(self.params)))

    def srht_signs(self, n_pad, seed, level, eps):
        _check("ihs_srht_signs", _lib.ihs_srht_signs(self.handle, n_pad, seed, level, _ptr(eps)))

    def srht_rows(self, n_pad, m, seed, level, rows):
        _check("ihs_srht_rows", _lib.ihs_srht_rows(self.handle, n_pad, m, seed, level, _ptr(rows)))

    def sketch_rows(self, A, m, seed, level, row0, mrows, SA_rows):
        """Rows [row0, row0 + mrows) of the Gaussian sketch of size m."""
        n, d = A.shape
        _check("ihs_sketch_rows", _lib.ihs_sketch_rows(self.handle, _ptr(A), n, d, m, seed, level, row0, mrows,
                                                       _ptr(SA_rows)))

    def sketch(self, A, m, kind, seed, level, SA):
        n, d = A.shape
        _check("ihs_sketch", _lib.ihs_sketch(self.handle, _ptr(A), n, d, m, KINDS.get(kind, kind), seed, level,
                                             _ptr(SA)))

    def factor(self, SA, nu):
        m, d = SA.shape
        h = ctypes.c_void_p()
        _check("ihs_factor", _lib.ihs_factor(self.handle, _ptr(SA), m, d, float(nu), ctypes.byref(h)))
        f = Factor(self, h, SA)
        self._factors.add(f)
        return f

    def grad(self, A, b, nu, x, g, want_axnorm2=True):
        n, d = A.shape
        ax2 = ctypes.c_double(0.0)
        _check("ihs_grad", _lib.ihs_grad(self.handle, _ptr(A), _ptr(b), n, d, float(nu), _ptr(x), _ptr(g),
                                         ctypes.byref(ax2) if want_axnorm2 else None))
        return ax2.value if want_axnorm2 else None

    def solve(self, A, b, nu, x, tol=0.0, raise_on_maxiter=False):
        n, d = A.shape
        rep = Report()
        st = _lib.ihs_solve(self.handle, _ptr(A), _ptr(b), n, d, float(nu), float(tol), _ptr(x), ctypes.byref(rep))
        if st != IHS_OK and (st != IHS_EMAXITER or raise_on_maxiter):
            _check("ihs_solve", st)
        return rep

    def solve_host(self, A_h, b_h, nu, x_h, tol=0.0, raise_on_maxiter=False):
        """ihs_solve_host: A_h, b_h, x_h are contiguous float32 CPU tensors (pinned
        for full copy bandwidth); x_h is updated in place."""
        for t in (A_h, b_h, x_h):
            if t.is_cuda or not t.is_contiguous() or t.dtype != __import__("torch").float32:
                raise ValueError("expected contiguous float32 host tensors")
        n, d = A_h.shape
        rep = Report()
        st = _lib.ihs_solve_host(self.handle, ctypes.c_void_p(A_h.data_ptr()), ctypes.c_void_p(b_h.data_ptr()), n, d,
                                 float(nu), float(tol), ctypes.c_void_p(x_h.data_ptr()), ctypes.byref(rep))
        if st != IHS_OK and (st != IHS_EMAXITER or raise_on_maxiter):
            _check("ihs_solve_host", st)
        return rep

    def solve_resume(self, A, b, nu, x, x_prev, state=None, tol=0.0):
        """ihs_solve_resume: continue a run from `state` (None or t == 0: start
        from x).  Returns (report, state); x and x_prev are updated in place."""
        n, d = A.shape
        state = State() if state is None else state
        rep = Report()
        st = _lib.ihs_solve_resume(self.handle, _ptr(A), _ptr(b), n, d, float(nu), float(tol), _ptr(x),
                                   _ptr(x_prev), ctypes.byref(state), ctypes.byref(rep))
        if st not in (IHS_OK, IHS_EMAXITER):
            _check("ihs_solve_resume", st)
        return rep, state

    def sketch_shard(self, A_local, row0, n_total, m, kind, seed, level, SA_part):
        """This shard's term of the sketch of the whole matrix (ihs_sketch_shard)."""
        n, d = A_local.shape
        _check("ihs_sketch_shard", _lib.ihs_sketch_shard(self.handle, _ptr(A_local), n, d, row0, n_total, m,
                                                         KINDS.get(kind, kind), seed, level, _ptr(SA_part)))

    def grad_shard(self, A_local, b_local, x, gp):
        """This shard's FP64 gradient terms, d + 1 doubles (ihs_grad_shard)."""
        n, d = A_local.shape
        _check("ihs_grad_shard", _lib.ihs_grad_shard(self.handle, _ptr(A_local), _ptr(b_local), n, d, _ptr(x),
                                                     _ptr(gp)))

    def solve_sharded(self, A_local, b_local, row0, n_total, nu, x, allreduce_cb, tol=0.0):
        """ihs_solve_sharded with an ALLREDUCE_FN callback (see shard.make_allreduce)."""
        n, d = A_local.shape
        rep = Report()
        st = _lib.ihs_solve_sharded(self.handle, _ptr(A_local), _ptr(b_local), n, d, row0, n_total, float(nu),
                                    float(tol), _ptr(x), ctypes.byref(rep), allreduce_cb, None)
        if st not in (IHS_OK, IHS_EMAXITER):
            _check("ihs_solve_sharded", st)
        return rep

    def trace(self):
        """Decisions of the last solve as (event, t, m, ratio) tuples."""
        count = _i32(0)
        _check("ihs_trace_events", _lib.ihs_trace_events(self.handle, None, 0, ctypes.byref(count)))
        buf = (Event * max(1, count.value))()
        _check("ihs_trace_events", _lib.ihs_trace_events(self.handle, buf, count.value, ctypes.byref(count)))
        return [buf[i].as_tuple() for i in range(count.value)]

    def set_trace_file(self, path):
        """Append each decision to `path` as a JSON line (None closes the file)."""
        _check("ihs_ctx_set_trace_file",
               _lib.ihs_ctx_set_trace_file(self.handle, None if path is None else str(path).encode()))

    def solve_dual(self, A, b, nu, x, tol=0.0, raise_on_maxiter=False):
        """Underdetermined A (n <= d): the dual iteration, x = A^T z on return."""
        n, d = A.shape
        rep = Report()
        st = _lib.ihs_solve_dual(self.handle, _ptr(A), _ptr(b), n, d, float(nu), float(tol), _ptr(x),
                                 ctypes.byref(rep))
        if st != IHS_OK and (st != IHS_EMAXITER or raise_on_maxiter):
            _check("ihs_solve_dual", st)
        return rep

    def solve_batched(self, problems, tol=0.0, m_init=None):
        """problems: sequence of (A, b, nu, x) device tensors (A may be shared);
        m_init: optional per-problem initial sketch sizes (powers of two).
        Returns one Report per problem (each with its own status)."""
        arr = (Problem * len(problems))()
        for i, (A, b, nu, x) in enumerate(problems):
            n, d = A.shape
            m0 = 0 if m_init is None else int(m_init[i])
            arr[i] = Problem(_ptr(A).value, _ptr(b).value, n, d, float(nu), _ptr(x).value, m0)
        reps = (Report * len(problems))()
        _check("ihs_solve_batched", _lib.ihs_solve_batched(self.handle, ctypes.byref(arr), len(problems),
                                                           float(tol), ctypes.byref(reps)))
        return list(reps)

    def warm_start_batched(self, params, problems, seed=None):
        """m0 for every (A, nu) (or (A, b, nu, x)) of a batch: one forward pass over all."""
        arr = (Problem * len(problems))()
        for i, pr in enumerate(problems):
            A, nu = pr[0], pr[2] if len(pr) > 2 else pr[1]
            n, d = A.shape
            arr[i] = Problem(_ptr(A).value, None, n, d, float(nu), None, 0)
        m0 = (ctypes.c_int64 * len(problems))()
        pred = (ctypes.c_float * len(problems))()
        seed = self.params.seed if seed is None else seed
        _check("ihs_warm_start_batched", _lib.ihs_warm_start_batched(self.handle, _ptr(params), ctypes.byref(arr),
                                                                     len(problems), int(seed), ctypes.byref(m0),
                                                                     ctypes.byref(pred)))
        return list(m0), list(pred)

    def cg(self, A, b, nu, x, tol=1e-6, max_iter=1000, precond=None, raise_on_maxiter=False):
        """CG (precond=None) or sketch-preconditioned CG (precond="srht"/"gauss")."""
        n, d = A.shape
        rep = Report()
        kind = -1 if precond is None else KINDS.get(precond, precond)
        st = _lib.ihs_cg(self.handle, _ptr(A), _ptr(b), n, d, float(nu), float(tol), int(max_iter), kind, _ptr(x),
                         ctypes.byref(rep))
        if st != IHS_OK and (st != IHS_EMAXITER or raise_on_maxiter):
            _check("ihs_cg", st)
        return rep

    # ---- learned warm start (no counterpart in the paper) ----
    def probe_features(self, A, nu, seed, feat):
        """feat (device float32, 11) <- the warm-start features of (A, nu)."""
        n, d = A.shape
        _check("ihs_probe_features", _lib.ihs_probe_features(self.handle, _ptr(A), n, d, float(nu), int(seed),
                                                             _ptr(feat)))

    def mlp_forward(self, params, X, y):
        _check("ihs_mlp_forward", _lib.ihs_mlp_forward(self.handle, _ptr(params), _ptr(X), X.shape[0], _ptr(y)))

    def mlp_grad(self, params, X, target, grad):
        loss = ctypes.c_double(0.0)
        _check("ihs_mlp_grad", _lib.ihs_mlp_grad(self.handle, _ptr(params), _ptr(X), _ptr(target), X.shape[0],
                                                 _ptr(grad), ctypes.byref(loss)))
        return loss.value

    def mlp_train_step(self, params, adam_m, adam_v, step, X, target, lr, want_loss=True):
        loss = ctypes.c_double(0.0)
        _check("ihs_mlp_train_step", _lib.ihs_mlp_train_step(self.handle, _ptr(params), _ptr(adam_m), _ptr(adam_v),
                                                             int(step), _ptr(X), _ptr(target), X.shape[0],
                                                             float(lr), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def warm_start(self, params, A, nu, seed=None):
        """(m0, prediction): the initial sketch size the network suggests for (A, nu)."""
        n, d = A.shape
        m0 = ctypes.c_int64(0)
        pred = ctypes.c_float(0.0)
        seed = self.params.seed if seed is None else seed
        _check("ihs_warm_start", _lib.ihs_warm_start(self.handle, _ptr(params), _ptr(A), n, d, float(nu), int(seed),
                                                     ctypes.byref(m0), ctypes.byref(pred)))
        return m0.value, pred.value

    def destroy(self):
        if getattr(self, "handle", None):
            for f in list(getattr(self, "_factors", ())):   # factors first: they were made on this context
                f.destroy()
            _lib.ihs_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
