"""Python binding of librtr.so: argument marshalling only.

Every function here has the name of the C entry point it calls
(``include/rtr.h``), takes torch CUDA tensors for device buffers, and does no
arithmetic of its own.  If the compiled library is missing, ``lib()`` raises:
there is no CPU or PyTorch fallback.
"""
import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librtr.so")

RTR_OK, RTR_EINVAL, RTR_ENOMEM, RTR_ECUDA, RTR_ENONFINITE, RTR_ENOTCONV, RTR_ETIMEOUT, RTR_EUNSUPPORTED = range(8)
RTR_FP64, RTR_FP32, RTR_BF16, RTR_FP8 = 0, 1, 2, 3
PREC = {"fp64": RTR_FP64, "fp32": RTR_FP32, "bf16": RTR_BF16, "fp8": RTR_FP8}
FLAG_NONFINITE, FLAG_QR_FALLBACK, FLAG_GRAM_PINV, FLAG_TIMEOUT = 1, 2, 4, 8
PARAM_NO_GRAPH, PARAM_PAIR = 1, 2

# every entry point of include/rtr.h
ENTRY_POINTS = (
    "rtr_params_default", "rtr_last_error", "rtr_kernel_launches", "rtr_plan_create", "rtr_plan_destroy", "rtr_plan_info",
    "rtr_plan_flags", "rtr_plan_sketch_passes", "rtr_sketch", "rtr_project", "rtr_project_sequential", "rtr_project_host", "rtr_als", "rtr_svd", "rtr_backproject",
    "rtr_reconstruct_work_bytes", "rtr_reconstruct", "rtr_rse", "rtr_draw_omega", "rtr_gaussian_table",
    "rtr_sketch_mode_noalloc", "rtr_batch_create", "rtr_batch_destroy", "rtr_batch_run",
    "rtr_batch_graph_kernels", "rtr_batch_flags", "rtr_mlp_param_count", "rtr_mlp_work_bytes", "rtr_spectrum_features",
    "rtr_mlp_forward", "rtr_mlp_grad", "rtr_mlp_adam", "rtr_mlp_status", "rtr_propose", "rtr_test_bounded_wait",
)


class RtrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rtr status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("seed", ctypes.c_uint64), ("sweeps", ctypes.c_int),
                ("tol", ctypes.c_double), ("flags", ctypes.c_int), ("chain_order", ctypes.c_int * 8),
                ("power_iters", ctypes.c_int)]


_lib = None
_VP = ctypes.c_void_p
_VPP = ctypes.POINTER(ctypes.c_void_p)
_I64P = ctypes.POINTER(ctypes.c_int64)
_IP = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load librtr.so (built by ``paper_1901_01652_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1901_01652_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "rtr_params_default": (None, [ctypes.POINTER(Params)]),
        "rtr_last_error": (ctypes.c_char_p, []),
        "rtr_kernel_launches": (ctypes.c_ulonglong, []),
        "rtr_plan_create": (ctypes.c_int, [_VPP, ctypes.c_int, _I64P, _IP, _IP, ctypes.POINTER(Params)]),
        "rtr_plan_destroy": (ctypes.c_int, [_VP]),
        "rtr_plan_info": (ctypes.c_int, [_VP, _IP, _IP]),
        "rtr_plan_flags": (ctypes.c_int, [_VP, _IP]),
        "rtr_plan_sketch_passes": (ctypes.c_int, [_VP, _IP]),
        "rtr_sketch": (ctypes.c_int, [_VP, _VP, _VPP, _VP]),
        "rtr_project": (ctypes.c_int, [_VP, _VP, _VPP, _VPP, _VP, _VP]),
        "rtr_project_sequential": (ctypes.c_int, [_VP, _VP, _VPP, _VPP, _VP, _VP]),
        "rtr_project_host": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VPP, ctypes.c_size_t, _VPP, _VPP, _VP,
                                            _VP]),
        "rtr_als": (ctypes.c_int, [_VP, _VP, _VPP, ctypes.c_int, _VP, _VP]),
        "rtr_svd": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VPP, _IP, _VP]),
        "rtr_backproject": (ctypes.c_int, [_VP, _VPP, _VPP, _VPP, _IP, _VP]),
        "rtr_reconstruct_work_bytes": (ctypes.c_size_t, [ctypes.c_int, _I64P, _IP]),
        "rtr_reconstruct": (ctypes.c_int, [ctypes.c_int, _I64P, _IP, _VPP, ctypes.c_int, _VP, _VP,
                                           ctypes.c_size_t, _VP]),
        "rtr_rse": (ctypes.c_int, [_VP, _VP, _VPP, _IP, _VP, _VP]),
        "rtr_draw_omega": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _VP, _VP]),
        "rtr_gaussian_table": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "rtr_sketch_mode_noalloc": (ctypes.c_int, [ctypes.c_int, _VP, ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                   _VP, _VP]),
        "rtr_batch_create": (ctypes.c_int, [_VPP, ctypes.c_int, ctypes.c_int, _I64P, _IP, _IP,
                                            ctypes.POINTER(Params), ctypes.c_int]),
        "rtr_batch_destroy": (ctypes.c_int, [_VP]),
        "rtr_batch_run": (ctypes.c_int, [_VP, _VPP, _VPP, _VP, _VP]),
        "rtr_batch_graph_kernels": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
        "rtr_batch_flags": (ctypes.c_int, [_VP, _IP]),
        "rtr_mlp_param_count": (ctypes.c_size_t, []),
        "rtr_mlp_work_bytes": (ctypes.c_size_t, [ctypes.c_int]),
        "rtr_spectrum_features": (ctypes.c_int, [ctypes.c_int, _I64P, _IP, _VPP, _VP, _VP]),
        "rtr_mlp_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t, _VP]),
        "rtr_mlp_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
        "rtr_mlp_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP]),
        "rtr_mlp_status": (ctypes.c_int, [_VP, _IP]),
        "rtr_propose": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_int, _I64P, ctypes.c_int, _IP, _IP]),
        "rtr_test_bounded_wait": (ctypes.c_int, [ctypes.c_int, _VP, _VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != RTR_OK:
        raise RtrError(status, lib().rtr_last_error().decode())


def _dev(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t


def _ptr(t):
    return _VP(0 if t is None else t.data_ptr())


def _ptrs(ts, dtype=None, name="buffers"):
    arr = (_VP * len(ts))()
    for i, t in enumerate(ts):
        _dev(t, dtype, f"{name}[{i}]")
        arr[i] = 0 if t is None else t.data_ptr()
    return arr


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return _VP(s.cuda_stream)


def _i64(xs):
    return (ctypes.c_int64 * len(xs))(*[int(x) for x in xs])


def _i32(xs):
    return (ctypes.c_int * len(xs))(*[int(x) for x in xs])


class Plan:
    """Owning handle of an rtr_plan."""

    def __init__(self, handle, dims, K, R, params):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        self.R = tuple(int(r) for r in R)
        self.params = params
        ke = (ctypes.c_int * self.N)()
        order = (ctypes.c_int * self.N)()
        _check(lib().rtr_plan_info(handle, ke, order))
        self.K = tuple(ke)
        self.order = tuple(order)
        self.prec = params.prec
        self.x_dtype = torch.float64 if params.prec == RTR_FP64 else torch.float32
        self.projected = tuple(k < d for k, d in zip(self.K, self.dims))

    def close(self):
        if self.handle:
            lib().rtr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rtr_kernel_launches():
    return int(lib().rtr_kernel_launches())


def rtr_params_default():
    p = Params()
    lib().rtr_params_default(ctypes.byref(p))
    return p


def make_params(prec="fp32", seed=0, sweeps=20, tol=1e-2, chain_order=None, power=0, flags=0):
    p = rtr_params_default()
    p.flags = int(flags)
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    p.seed = int(seed)
    p.sweeps = int(sweeps)
    p.tol = float(tol)
    p.power_iters = int(power)
    if chain_order is not None:
        for i, m in enumerate(chain_order):
            p.chain_order[i] = int(m)
    return p


def rtr_plan_create(dims, K, R, params):
    h = _VP()
    N = len(dims)
    _check(lib().rtr_plan_create(ctypes.byref(h), N, _i64(dims), _i32(K), _i32(R), ctypes.byref(params)))
    return Plan(h, dims, K, R, params)


def rtr_plan_destroy(plan):
    plan.close()


def rtr_plan_flags(plan):
    f = ctypes.c_int(0)
    _check(lib().rtr_plan_flags(plan.handle, ctypes.byref(f)))
    return f.value


def rtr_plan_sketch_passes(plan):
    """Passes over X that rtr_sketch makes for this plan (16-byte aligned X)."""
    n = ctypes.c_int(0)
    _check(lib().rtr_plan_sketch_passes(plan.handle, ctypes.byref(n)))
    return n.value


def rtr_sketch(plan, X, Y, stream=None):
    _dev(X, plan.x_dtype, "X")
    _check(lib().rtr_sketch(plan.handle, _ptr(X), _ptrs(Y, torch.float64, "Y"), _stream(stream)))


def rtr_project(plan, X, Y, Q, P, stream=None):
    _dev(X, plan.x_dtype, "X")
    _dev(P, plan.x_dtype, "P")
    _check(lib().rtr_project(plan.handle, _ptr(X), _ptrs(Y, torch.float64, "Y"), _ptrs(Q, torch.float64, "Q"),
                             _ptr(P), _stream(stream)))


def rtr_project_sequential(plan, X, Y, Q, P, stream=None):
    _dev(X, plan.x_dtype, "X")
    _dev(P, plan.x_dtype, "P")
    _check(lib().rtr_project_sequential(plan.handle, _ptr(X), _ptrs(Y, torch.float64, "Y"),
                                        _ptrs(Q, torch.float64, "Q"), _ptr(P), _stream(stream)))


def rtr_project_host(plan, X_host, slab_rows, stage, Y, Q, P, stream=None):
    """Out-of-core steps 3-8: X_host a CPU tensor (pinned for overlapped
    copies), stage two CUDA tensors of equal size (bytes >= slab_rows rows)."""
    if not isinstance(X_host, torch.Tensor) or X_host.is_cuda or not X_host.is_contiguous():
        raise TypeError("X_host must be a contiguous CPU tensor")
    if X_host.dtype != plan.x_dtype:
        raise TypeError(f"X_host must be {plan.x_dtype}")
    if tuple(X_host.shape) != tuple(plan.dims):
        raise ValueError(f"X_host has shape {tuple(X_host.shape)}, the plan {tuple(plan.dims)}")
    if len(stage) != 2:
        raise ValueError("stage must hold two device buffers")
    for t in stage:
        _dev(t, None, "stage")
    nbytes = min(t.numel() * t.element_size() for t in stage)
    arr = (_VP * 2)(_ptr(stage[0]), _ptr(stage[1]))
    _dev(P, plan.x_dtype, "P")
    _check(lib().rtr_project_host(plan.handle, ctypes.c_void_p(X_host.data_ptr()), int(slab_rows), arr, nbytes,
                                  _ptrs(Y, torch.float64, "Y"), _ptrs(Q, torch.float64, "Q"), _ptr(P),
                                  _stream(stream)))


def rtr_als(plan, P, Z, init_given, err=None, stream=None):
    _dev(P, plan.x_dtype, "P")
    _dev(err, torch.float64, "err")
    _check(lib().rtr_als(plan.handle, _ptr(P), _ptrs(Z, torch.float64, "Z"), int(bool(init_given)), _ptr(err),
                         _stream(stream)))


def rtr_svd(plan, P, tol, Z, ranks=None, stream=None):
    _dev(P, plan.x_dtype, "P")
    r = _i32(ranks if ranks is not None else [0] * plan.N)
    _check(lib().rtr_svd(plan.handle, _ptr(P), float(tol), _ptrs(Z, torch.float64, "Z"), r, _stream(stream)))
    return list(r)


def rtr_backproject(plan, Z, Q, G, ranks=None, stream=None):
    r = None if ranks is None else _i32(ranks)
    _check(lib().rtr_backproject(plan.handle, _ptrs(Z, torch.float64, "Z"), _ptrs(Q, torch.float64, "Q"),
                                 _ptrs(G, torch.float64, "G"), r, _stream(stream)))


def rtr_reconstruct_work_bytes(dims, R):
    return int(lib().rtr_reconstruct_work_bytes(len(dims), _i64(dims), _i32(R)))


def rtr_reconstruct(dims, R, G, out_prec, Xhat, work, stream=None):
    op = PREC[out_prec] if isinstance(out_prec, str) else int(out_prec)
    _dev(Xhat, torch.float64 if op == RTR_FP64 else torch.float32, "Xhat")
    _dev(work, None, "work")
    _check(lib().rtr_reconstruct(len(dims), _i64(dims), _i32(R), _ptrs(G, torch.float64, "G"), op, _ptr(Xhat),
                                 _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def rtr_rse(plan, P, Z, out, ranks=None, stream=None):
    _dev(P, plan.x_dtype, "P")
    _dev(out, torch.float64, "out")
    r = None if ranks is None else _i32(ranks)
    _check(lib().rtr_rse(plan.handle, _ptr(P), _ptrs(Z, torch.float64, "Z"), r, _ptr(out), _stream(stream)))


def rtr_draw_omega(plan, mode, row0, nrows, K, out, stream=None):
    _dev(out, torch.float64, "out")
    _check(lib().rtr_draw_omega(plan.handle, int(mode), int(row0), int(nrows), int(K), _ptr(out), _stream(stream)))


def rtr_gaussian_table(prec):
    out = (ctypes.c_double * 4096)()
    op = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(lib().rtr_gaussian_table(op, out))
    return np.frombuffer(out, dtype=np.float64).copy()


def rtr_test_bounded_wait(limit_us, flags, stream=None):
    """Test support: a device wait on a barrier nothing completes, bounded by
    limit_us; returns the status code (RTR_ETIMEOUT expected) without raising."""
    _dev(flags, torch.int32, "flags")
    return int(lib().rtr_test_bounded_wait(int(limit_us), _ptr(flags), _stream(stream)))


def rtr_sketch_mode_noalloc(prec, X, view, K, seed, mode, Y, stream=None):
    """Allocation-free one-mode sketch; view = (A, I, B) of X around the mode.

    The C entry point cannot see the buffers' sizes, so the view is checked
    here against X (A*I*B elements) and Y (I*K float64) before any launch.
    Every call shares the library's one static scratch array: calls must not
    overlap on the GPU (other streams or threads)."""
    op = PREC[prec] if isinstance(prec, str) else int(prec)
    A, I, B = (int(v) for v in view)
    if X.numel() != A * I * B:
        raise ValueError(f"view {(A, I, B)} does not match X with {X.numel()} elements")
    if Y.numel() != I * int(K):
        raise ValueError(f"Y has {Y.numel()} elements, the sketch writes I*K = {I * int(K)}")
    _dev(X, torch.float64 if op == RTR_FP64 else torch.float32, "X")
    _dev(Y, torch.float64, "Y")
    _check(lib().rtr_sketch_mode_noalloc(op, _ptr(X), A, I, B, int(K), int(seed), int(mode), _ptr(Y),
                                         _stream(stream)))


class Batch:
    """Owning handle of an rtr_batch."""

    def __init__(self, handle, shapes, K, R, params):
        self.handle = handle
        self.shapes = [tuple(int(d) for d in s) for s in shapes]
        self.count = len(self.shapes)
        self.N = len(self.shapes[0])
        self.K = [tuple(int(k) for k in ks) for ks in K]
        self.R = [tuple(int(r) for r in rs) for rs in R]
        self.params = params
        self.x_dtype = torch.float64 if params.prec == RTR_FP64 else torch.float32

    def close(self):
        if self.handle:
            lib().rtr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rtr_batch_create(shapes, K, R, params, nstreams=8):
    """shapes, K, R: one sequence of N values per tensor."""
    if len(shapes) == 0:
        raise ValueError("a batch needs at least one tensor")
    N = len(shapes[0])
    if any(len(s) != N for s in list(shapes) + list(K) + list(R)) or not (len(shapes) == len(K) == len(R)):
        raise ValueError("every tensor needs N dims, K and R values")
    h = _VP()
    flat = lambda xs: [v for s in xs for v in s]
    _check(lib().rtr_batch_create(ctypes.byref(h), len(shapes), N, _i64(flat(shapes)), _i32(flat(K)),
                                  _i32(flat(R)), ctypes.byref(params), int(nstreams)))
    return Batch(h, shapes, K, R, params)


def rtr_batch_destroy(batch):
    batch.close()


def rtr_batch_run(batch, X, G, rse=None, stream=None):
    """X: list of count device tensors; G: list of count lists of N float64 core buffers."""
    if len(X) != batch.count or len(G) != batch.count:
        raise ValueError("X and G need one entry per tensor")
    xs = _ptrs(X, batch.x_dtype, "X")
    gs = _ptrs([g for gt in G for g in gt], torch.float64, "G")
    _dev(rse, torch.float64, "rse")
    _check(lib().rtr_batch_run(batch.handle, xs, gs, _ptr(rse), _stream(stream)))


def rtr_batch_flags(batch):
    f = ctypes.c_int(0)
    _check(lib().rtr_batch_flags(batch.handle, ctypes.byref(f)))
    return f.value


def rtr_batch_graph_kernels(batch):
    n = ctypes.c_uint64(0)
    _check(lib().rtr_batch_graph_kernels(batch.handle, ctypes.byref(n)))
    return int(n.value)


# ----------------------------------------------------------------------------- learned proposer

def rtr_mlp_param_count():
    return int(lib().rtr_mlp_param_count())


def rtr_mlp_work_bytes(batch):
    return int(lib().rtr_mlp_work_bytes(int(batch)))


def rtr_spectrum_features(dims, Kf, Y, f, stream=None):
    """Y: list of N float64 sketches (I_n x Kf_n); f: float32 device tensor of 320."""
    _dev(f, torch.float32, "f")
    _check(lib().rtr_spectrum_features(len(dims), _i64(dims), _i32(Kf), _ptrs(Y, torch.float64, "Y"), _ptr(f),
                                       _stream(stream)))


def rtr_mlp_forward(theta, F, out, work, stream=None):
    for t, n in ((theta, "theta"), (F, "F"), (out, "out")):
        _dev(t, torch.float32, n)
    _dev(work, None, "work")
    batch = F.shape[0]
    _check(lib().rtr_mlp_forward(_ptr(theta), _ptr(F), int(batch), _ptr(out), _ptr(work),
                                 work.numel() * work.element_size(), _stream(stream)))


def rtr_mlp_grad(theta, F, T, M, grad, loss, work, stream=None):
    for t, n in ((theta, "theta"), (F, "F"), (T, "T"), (M, "M"), (grad, "grad")):
        _dev(t, torch.float32, n)
    _dev(loss, torch.float64, "loss")
    _dev(work, None, "work")
    _check(lib().rtr_mlp_grad(_ptr(theta), _ptr(F), _ptr(T), _ptr(M), int(F.shape[0]), _ptr(grad), _ptr(loss),
                              _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def rtr_mlp_adam(theta, grad, m, v, step, lr, stream=None):
    for t, n in ((theta, "theta"), (grad, "grad"), (m, "m"), (v, "v")):
        _dev(t, torch.float32, n)
    _check(lib().rtr_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)))


def rtr_mlp_status(work):
    f = ctypes.c_int(0)
    st = lib().rtr_mlp_status(_ptr(_dev(work, None, "work")), ctypes.byref(f))
    _check(st)
    return f.value


def rtr_propose(out_row, dims, r_max=16):
    """out_row: 10 host floats -> (K list, R list)."""
    o = (ctypes.c_float * 10)(*[float(x) for x in out_row])
    N = len(dims)
    K = (ctypes.c_int * N)()
    R = (ctypes.c_int * N)()
    _check(lib().rtr_propose(o, N, _i64(dims), int(r_max), K, R))
    return list(K), list(R)
