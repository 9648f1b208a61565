"""Python binding of the C ABI in ``include/slk.h`` (argument marshalling only).

Every computation runs in ``libslk.so``; this module converts tensors and
arrays to pointers, passes torch's current CUDA stream and raises on a
non-OK status.  It has no fallback: without the built library every call
raises ``SlkError``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

try:  # torch is used for device memory and streams only
    import torch
except ImportError:  # pragma: no cover
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libslk.so")

KERNELS = {"gaussian": 0, "laplacian": 1, "negdist": 2, "matern32": 3}
PRECISIONS = {"f64": 0, "f32": 1, "bf16": 2, "f16x3": 3}
METHODS = {"auto": 0, "nfft": 1, "ndft": 2, "cheb": 3}
STATUS = {0: "SLK_OK", 1: "SLK_ERR_INVALID", 2: "SLK_ERR_OOM", 3: "SLK_ERR_CUDA", 4: "SLK_ERR_ACCURACY",
          5: "SLK_ERR_TIMEOUT", 6: "SLK_ERR_BUSY", 7: "SLK_ERR_UNSUPPORTED", 8: "SLK_ERR_NOT_FOUND"}


class SlkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class PlanDesc(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("precision", ctypes.c_int32), ("param", ctypes.c_double),
                ("d", ctypes.c_int32), ("P", ctypes.c_int32), ("n_coeff", ctypes.c_int32),
                ("method", ctypes.c_int32), ("seed", ctypes.c_uint64), ("directions", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("radius", ctypes.c_double), ("slice_batch", ctypes.c_int32),
                ("slice_offset", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("precision", ctypes.c_int32), ("d", ctypes.c_int32),
                ("P", ctypes.c_int32), ("N", ctypes.c_int64), ("method", ctypes.c_int32),
                ("n_coeff", ctypes.c_int32), ("n_grid", ctypes.c_int32), ("window", ctypes.c_int32),
                ("k_lo", ctypes.c_int32), ("k_hi", ctypes.c_int32), ("cheb_terms", ctypes.c_int32),
                ("cheb_horner", ctypes.c_int32), ("sort_buckets", ctypes.c_int32), ("period", ctypes.c_double),
                ("radius", ctypes.c_double), ("model_error", ctypes.c_double), ("c_d", ctypes.c_double),
                ("device_bytes", ctypes.c_int64)]


class RffDesc(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("precision", ctypes.c_int32), ("param", ctypes.c_double),
                ("d", ctypes.c_int32), ("D", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("seed", ctypes.c_uint64), ("features", ctypes.c_void_p),
                ("reserved", ctypes.c_int32 * 4)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None

# exported names of include/slk.h with their ctypes signatures
_SIGNATURES = {
    "slk_version": (ctypes.c_int32, []),
    "slk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "slk_last_error": (ctypes.c_char_p, []),
    "slk_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlanDesc), ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "slk_sum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p]),
    "slk_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "slk_sum_derivs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "slk_grad_derivs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "slk_plan_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "slk_plan_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "slk_plan_get_center": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "slk_plan_get_directions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "slk_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "slk_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "slk_fourier_params": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.c_double, ctypes.POINTER(PlanInfo)]),
    "slk_sum_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "slk_rff_sum": (ctypes.c_int, [ctypes.POINTER(RffDesc), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "slk_rff_features": (ctypes.c_int, [ctypes.POINTER(RffDesc), ctypes.c_void_p]),
    "slk_launch_count": (ctypes.c_int64, []),
    "slk_device_alloc_count": (ctypes.c_int64, []),
    "slk_timing_enable": (ctypes.c_int, [ctypes.c_int32]),
    "slk_timing_read": (ctypes.c_int, [ctypes.POINTER(KernelTime), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "slk_timing_reset": (ctypes.c_int, []),
    "slk_kernel_sum": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Load libslk.so (raises SlkError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise SlkError(3, f"{path} is missing: build it with paper_2401_08260_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int):
    if st != 0:
        raise SlkError(st, load().slk_last_error().decode(errors="replace"))


def _stream_of(t) -> Optional[int]:
    if torch is not None and isinstance(t, torch.Tensor) and t.is_cuda:
        return torch.cuda.current_stream(t.device).cuda_stream
    return None


def _dtype_for(precision: str):
    return np.float64 if precision == "f64" else np.float32


class _Arr:
    """Pointer, leading dimension and keep-alive for a 2-D (or 1-D) argument."""

    def __init__(self, a, dtype, ndim):
        self.keep = a
        if torch is not None and isinstance(a, torch.Tensor):
            want = torch.float64 if dtype == np.float64 else torch.float32
            if a.dtype != want:
                raise TypeError(f"expected {want}, got {a.dtype}")
            if ndim == 2:
                if a.dim() != 2 or a.stride(1) != 1:
                    a = a.contiguous()
                self.ld = a.stride(0)
            else:
                a = a.contiguous()
                self.ld = 1
            self.keep = a
            self.ptr = a.data_ptr()
            self.rows = a.shape[0]
            self.cols = a.shape[1] if ndim == 2 else 1
        else:
            a = np.asarray(a)
            if a.dtype != dtype:
                raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
            a = np.ascontiguousarray(a)
            self.keep = a
            self.ptr = a.ctypes.data
            self.ld = a.shape[1] if ndim == 2 else 1
            self.rows = a.shape[0]
            self.cols = a.shape[1] if ndim == 2 else 1


def _plan_desc(kernel: str, param: float, d: int, P: int, precision: str, n_coeff: int = 0, method: str = "auto",
               seed: int = 0, directions=None, tol: float = 0.0, radius: float = 0.0, slice_offset: int = 0,
               slice_batch: int = 0):
    """A filled PlanDesc and the FP64 copy of `directions` it points to (keep it alive)."""
    desc = PlanDesc()
    desc.kernel = KERNELS[kernel]
    desc.precision = PRECISIONS[precision]
    desc.param = float(param)
    desc.d = int(d)
    desc.P = int(P)
    desc.n_coeff = int(n_coeff)
    desc.method = METHODS[method]
    desc.seed = int(seed)
    dirs = None
    if directions is not None:
        if torch is not None and isinstance(directions, torch.Tensor):
            dirs = directions.to(torch.float64).contiguous()
            desc.directions = dirs.data_ptr()
        else:
            dirs = np.ascontiguousarray(np.asarray(directions, dtype=np.float64))
            desc.directions = dirs.ctypes.data
        if tuple(dirs.shape) != (int(P), int(d)):
            raise ValueError("directions must be P x d")
    desc.tol = float(tol)
    desc.radius = float(radius)
    desc.slice_offset = int(slice_offset)
    desc.slice_batch = int(slice_batch)
    return desc, dirs


class Plan:
    """A sliced kernel-summation plan over the sources x (N x d) with weights w.

    kernel: "gaussian" (param = sigma), "laplacian" (param = alpha, F = exp(-alpha r))
    or "negdist" or "matern32" (param = beta).  precision: "f64", "f32", "bf16" or "f16x3".  directions: optional
    P x d unit directions (FP64); otherwise the library draws rows slice_offset .. slice_offset + P - 1 of
    the direction sequence of ``seed``."""

    def __init__(self, x, w, kernel: str, param: float = 0.0, P: int = 256, precision: str = "f32",
                 n_coeff: int = 0, method: str = "auto", seed: int = 0, directions=None, tol: float = 0.0,
                 radius: float = 0.0, slice_offset: int = 0):
        lib = load()
        self.precision = precision
        self.dtype = _dtype_for(precision)
        xa = _Arr(x, self.dtype, 2)
        wa = _Arr(w, self.dtype, 1)
        d = int(x.shape[1])
        desc, self._dirs = _plan_desc(kernel, param, d, P, precision, n_coeff, method, seed, directions, tol,
                                      radius, slice_offset)
        self.kernel, self.param, self.d, self.P = kernel, param, d, int(P)
        self.N = int(x.shape[0])
        self._desc = desc
        self._stream = _stream_of(x)
        h = ctypes.c_void_p()
        _check(lib.slk_plan_create(ctypes.byref(h), ctypes.byref(desc), xa.ptr, xa.rows, xa.ld, wa.ptr,
                                   self._stream))
        self._h = h

    @property
    def handle(self):
        return self._h

    def sum(self, y, out=None, sync: bool = True):
        """s_m for every row of y.  Returns a tensor/array like y."""
        lib = load()
        ya = _Arr(y, self.dtype, 2)
        if out is None:
            if torch is not None and isinstance(y, torch.Tensor):
                out = torch.empty(ya.rows, dtype=ya.keep.dtype, device=ya.keep.device)
            else:
                out = np.empty(ya.rows, dtype=self.dtype)
        oa = _Arr(out, self.dtype, 1)
        _check(lib.slk_sum(self._h, ya.ptr, ya.rows, ya.ld, oa.ptr, _stream_of(y)))
        if sync:
            _check(lib.slk_plan_sync(self._h))
        return out

    def grad(self, y, gs=None, out=None, sync: bool = True):
        """Gradient of sum_m gs_m s_m with respect to y (M x d)."""
        lib = load()
        ya = _Arr(y, self.dtype, 2)
        ga = _Arr(gs, self.dtype, 1) if gs is not None else None
        if out is None:
            if torch is not None and isinstance(y, torch.Tensor):
                out = torch.empty(ya.rows, self.d, dtype=ya.keep.dtype, device=ya.keep.device)
            else:
                out = np.empty((ya.rows, self.d), dtype=self.dtype)
        oa = _Arr(out, self.dtype, 2)
        _check(lib.slk_grad(self._h, ya.ptr, ya.rows, ya.ld, ga.ptr if ga else None, oa.ptr, oa.ld, _stream_of(y)))
        if sync:
            _check(lib.slk_plan_sync(self._h))
        return out

    def sum_derivs(self, y, out=None, g=None, sync: bool = True):
        """(s, g): the sums at the rows of y and the per-slice derivatives g (P x M,
        g[p, m] = t_p'(<xi_p, y_m - mu>)) from one projection and one evaluation.  out and g
        may be given (device or host, independently of y)."""
        lib = load()
        ya = _Arr(y, self.dtype, 2)
        on_dev = torch is not None and isinstance(y, torch.Tensor)
        if out is None:
            out = torch.empty(ya.rows, dtype=ya.keep.dtype, device=ya.keep.device) if on_dev else \
                np.empty(ya.rows, dtype=self.dtype)
        if g is None:
            g = torch.empty(self.P, ya.rows, dtype=ya.keep.dtype, device=ya.keep.device) if on_dev else \
                np.empty((self.P, ya.rows), dtype=self.dtype)
        s = out
        sa, gd = _Arr(s, self.dtype, 1), _Arr(g, self.dtype, 2)
        _check(lib.slk_sum_derivs(self._h, ya.ptr, ya.rows, ya.ld, sa.ptr, gd.ptr, gd.ld, _stream_of(y)))
        if sync:
            _check(lib.slk_plan_sync(self._h))
        return s, g

    def grad_derivs(self, g, gs=None, out=None, sync: bool = True):
        """Gradient of sum_m gs_m s_m with respect to y from the derivatives g (P x M) that
        sum_derivs returned: gy_m = gs_m (1/P) sum_p g[p, m] xi_p."""
        lib = load()
        gd = _Arr(g, self.dtype, 2)
        M = gd.cols
        ga = _Arr(gs, self.dtype, 1) if gs is not None else None
        if out is None:
            if torch is not None and isinstance(g, torch.Tensor):
                out = torch.empty(M, self.d, dtype=gd.keep.dtype, device=gd.keep.device)
            else:
                out = np.empty((M, self.d), dtype=self.dtype)
        oa = _Arr(out, self.dtype, 2)
        _check(lib.slk_grad_derivs(self._h, gd.ptr, M, gd.ld, ga.ptr if ga else None, oa.ptr, oa.ld, _stream_of(g)))
        if sync:
            _check(lib.slk_plan_sync(self._h))
        return out

    def project(self, x, out=None, sync: bool = True):
        """Z[p, i] = <xi_p, x_i - mu> on the plan's projection path (P x n)."""
        lib = load()
        xa = _Arr(x, self.dtype, 2)
        if out is None:
            if torch is not None and isinstance(x, torch.Tensor):
                out = torch.empty(self.P, xa.rows, dtype=xa.keep.dtype, device=xa.keep.device)
            else:
                out = np.empty((self.P, xa.rows), dtype=self.dtype)
        oa = _Arr(out, self.dtype, 2)
        _check(lib.slk_plan_project(self._h, xa.ptr, xa.rows, xa.ld, oa.ptr, oa.ld, _stream_of(x)))
        if sync:
            _check(lib.slk_plan_sync(self._h))
        return out

    def center(self) -> np.ndarray:
        mu = np.empty(self.d, dtype=np.float64)
        _check(load().slk_plan_get_center(self._h, mu.ctypes.data))
        return mu

    def sync(self):
        _check(load().slk_plan_sync(self._h))

    def directions(self) -> np.ndarray:
        xi = np.empty((self.P, self.d), dtype=np.float64)
        _check(load().slk_plan_get_directions(self._h, xi.ctypes.data))
        return xi

    def info(self) -> dict:
        inf = PlanInfo()
        _check(load().slk_plan_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in PlanInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().slk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fourier_params(kernel: str, param: float, d: int, radius: float, precision: str = "f32", n_coeff: int = 0,
                   method: str = "auto", tol: float = 0.0) -> dict:
    """Host-only: the Fourier parameters a plan would choose for projected points in [-radius, radius]."""
    desc = PlanDesc()
    desc.kernel, desc.precision, desc.param, desc.d, desc.P = KERNELS[kernel], PRECISIONS[precision], param, d, 1
    desc.n_coeff, desc.method, desc.tol = n_coeff, METHODS[method], tol
    inf = PlanInfo()
    _check(load().slk_fourier_params(ctypes.byref(desc), float(radius), ctypes.byref(inf)))
    return {f: getattr(inf, f) for f, _ in PlanInfo._fields_}


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().slk_launch_count())


def timing_enable(on: bool = True):
    _check(load().slk_timing_enable(1 if on else 0))


def timing_reset():
    _check(load().slk_timing_reset())


def timing_read() -> dict:
    """{kernel name: (launches, total device ms)} for the launches recorded while enabled."""
    lib = load()
    cap = 128
    buf = (KernelTime * cap)()
    n = ctypes.c_int32()
    _check(lib.slk_timing_read(buf, cap, ctypes.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, cap))}


def kernel_sum(x, w, y, kernel: str, param: float = 0.0, P: int = 256, precision: str = "f32",
               slice_batch: int = 0, out=None, **kw):
    """One-shot s = sum_n w_n F(|x_n - y_m|) via slicing (slk_kernel_sum: plan, sum, destroy).

    slice_batch: 0 < B < P processes the slices in batches of at most B, one batch's plan in
    device memory at a time; the other keywords are those of `Plan`."""
    lib = load()
    dtype = _dtype_for(precision)
    xa, wa, ya = _Arr(x, dtype, 2), _Arr(w, dtype, 1), _Arr(y, dtype, 2)
    desc, dirs = _plan_desc(kernel, param, int(x.shape[1]), P, precision, slice_batch=slice_batch, **kw)
    if out is None:
        if torch is not None and isinstance(y, torch.Tensor):
            out = torch.empty(ya.rows, dtype=ya.keep.dtype, device=ya.keep.device)
        else:
            out = np.empty(ya.rows, dtype=dtype)
    oa = _Arr(out, dtype, 1)
    _check(lib.slk_kernel_sum(ctypes.byref(desc), xa.ptr, xa.rows, xa.ld, wa.ptr, ya.ptr, ya.rows, ya.ld, oa.ptr,
                              _stream_of(x)))
    del dirs
    return out


def _rff_desc(kernel: str, param: float, d: int, D: int, variant: int, precision: str, seed: int, features):
    if kernel not in ("gaussian", "laplacian"):
        raise ValueError("random Fourier features need the Gaussian or the Laplacian kernel")
    desc = RffDesc()
    desc.kernel = KERNELS[kernel]
    desc.precision = PRECISIONS[precision]
    desc.param = float(param)
    desc.d = int(d)
    desc.D = int(D)
    desc.variant = int(variant)
    desc.seed = int(seed)
    keep = None
    if features is not None:
        keep = np.ascontiguousarray(np.asarray(features, dtype=np.float64))
        if keep.shape != (D, d + 1):
            raise ValueError(f"features must be D x (d + 1) = {D} x {d + 1}")
        desc.features = keep.ctypes.data
    return desc, keep


def rff_sum(x, w, y, kernel: str, param: float, D: int, variant: int = 2, precision: str = "f32", seed: int = 0,
            features=None, out=None):
    """Random Fourier feature estimate of s_m = sum_n w_n K(x_n, y_m) (Section 4.3; RFF-1 for
    variant 1, RFF-2 for variant 2) on the library's kernels (slk_rff_sum).  features: an
    optional D x (d + 1) array of rows (v_p, b_p); None = the library's draw from seed."""
    lib = load()
    dtype = _dtype_for(precision)
    xa, wa, ya = _Arr(x, dtype, 2), _Arr(w, dtype, 1), _Arr(y, dtype, 2)
    desc, keep = _rff_desc(kernel, param, int(x.shape[1]), D, variant, precision, seed, features)
    if out is None:
        if torch is not None and isinstance(y, torch.Tensor):
            out = torch.empty(ya.rows, dtype=ya.keep.dtype, device=ya.keep.device)
        else:
            out = np.empty(ya.rows, dtype=dtype)
    oa = _Arr(out, dtype, 1)
    _check(lib.slk_rff_sum(ctypes.byref(desc), xa.ptr, xa.rows, xa.ld, wa.ptr, ya.ptr, ya.rows, ya.ld, oa.ptr,
                           _stream_of(x)))
    del keep
    return out


def rff_features(kernel: str, param: float, d: int, D: int, seed: int = 0) -> np.ndarray:
    """The D x (d + 1) features (v_p, b_p) the library draws for these arguments."""
    desc, _ = _rff_desc(kernel, param, d, D, 2, "f64", seed, None)
    out = np.empty((D, d + 1), dtype=np.float64)
    _check(load().slk_rff_features(ctypes.byref(desc), out.ctypes.data))
    return out


if torch is not None:

    class SlicedKernelSum(torch.autograd.Function):
        """s = sliced kernel sum at targets y; the forward pass also keeps the per-slice
        derivatives (sign(0) = 0), from which backward forms the y-gradient by the backward
        product alone."""

        @staticmethod
        def forward(ctx, y, plan: Plan):
            ctx.plan = plan
            if not y.requires_grad:
                return plan.sum(y.detach())
            # the per-slice derivatives come from the same pass and are kept for backward
            s, g = plan.sum_derivs(y.detach())
            ctx.save_for_backward(g)
            return s

        @staticmethod
        def backward(ctx, grad_s):
            (g,) = ctx.saved_tensors
            gy = ctx.plan.grad_derivs(g, gs=grad_s.contiguous().to(g.dtype))
            return gy, None

    def sliced_kernel_sum(y, plan: Plan):
        """Differentiable (in y) sliced kernel sum."""
        return SlicedKernelSum.apply(y, plan)


# ---------------------------------------------------------------- serving (include/slk_serve.h)

class ServeDesc(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("memory_budget", ctypes.c_int64), ("plan_cache_bytes", ctypes.c_int64),
                ("reserved", ctypes.c_int32 * 8)]


class RequestDesc(ctypes.Structure):
    _fields_ = [("desc", PlanDesc), ("x", ctypes.c_void_p), ("N", ctypes.c_int64), ("ldx", ctypes.c_int64),
                ("w", ctypes.c_void_p), ("y", ctypes.c_void_p), ("M", ctypes.c_int64), ("ldy", ctypes.c_int64),
                ("s", ctypes.c_void_p), ("source_key", ctypes.c_uint64)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("plan_cached", ctypes.c_int32), ("batch_requests", ctypes.c_int32),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("message", ctypes.c_char * 128)]


_SERVE_SIGNATURES = {
    "slk_serve_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ServeDesc)]),
    "slk_serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(RequestDesc), ctypes.POINTER(ctypes.c_uint64)]),
    "slk_serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(RequestResult)]),
    "slk_serve_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "slk_request_bytes": (ctypes.c_int64, [ctypes.POINTER(PlanDesc), ctypes.c_int64, ctypes.c_int64]),
}


def _serve_lib():
    lib = load()
    if not getattr(lib, "_serve_ready", False):
        for name, (res, args) in _SERVE_SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        lib._serve_ready = True
    return lib


def make_desc(kernel: str, param: float, d: int, P: int, precision: str = "f32", n_coeff: int = 0,
              method: str = "auto", seed: int = 0, tol: float = 0.0, radius: float = 0.0) -> PlanDesc:
    desc = PlanDesc()
    desc.kernel, desc.precision, desc.param, desc.d, desc.P = KERNELS[kernel], PRECISIONS[precision], param, d, P
    desc.n_coeff, desc.method, desc.seed, desc.tol, desc.radius = n_coeff, METHODS[method], seed, tol, radius
    return desc


def request_bytes(desc: PlanDesc, N: int, M: int) -> int:
    """Conservative device bytes of one request (plan build plus one sum); host-only."""
    return int(_serve_lib().slk_request_bytes(ctypes.byref(desc), N, M))


class Server:
    """Concurrent request server on the current device (admission by a memory budget,
    worker streams, a cache of source-side plans keyed by `source_key`, and batches of the
    queued requests that query one cached plan)."""

    def __init__(self, workers: int = 0, memory_budget: int = 0, plan_cache_bytes: int = 0):
        lib = _serve_lib()
        sd = ServeDesc()
        sd.workers, sd.memory_budget, sd.plan_cache_bytes = workers, memory_budget, plan_cache_bytes
        h = ctypes.c_void_p()
        _check(lib.slk_serve_create(ctypes.byref(h), ctypes.byref(sd)))
        self._h = h
        self._keep = {}

    def submit(self, x, w, y, out, desc: PlanDesc, source_key: int = 0) -> int:
        """Queue s = kernel sums of (x, w) at y into `out`; returns the request id.
        x, w, y and out stay referenced until the request is polled; an array that
        desc.directions points to must be kept alive by the caller until then too."""
        dtype = np.float64 if desc.precision == PRECISIONS["f64"] else np.float32
        xa, wa, ya, oa = _Arr(x, dtype, 2), _Arr(w, dtype, 1), _Arr(y, dtype, 2), _Arr(out, dtype, 1)
        r = RequestDesc()
        r.desc = desc
        r.x, r.N, r.ldx, r.w = xa.ptr, xa.rows, xa.ld, wa.ptr
        r.y, r.M, r.ldy, r.s = ya.ptr, ya.rows, ya.ld, oa.ptr
        r.source_key = source_key
        rid = ctypes.c_uint64()
        _check(_serve_lib().slk_serve_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (xa, wa, ya, oa)
        return rid.value

    def poll(self, rid: int, timeout_us: int = -1):
        """Result dict when finished, None on timeout."""
        res = RequestResult()
        st = _serve_lib().slk_serve_poll(self._h, rid, timeout_us, ctypes.byref(res))
        if st == 5:
            return None
        _check(st)
        self._keep.pop(rid, None)
        return {"status": int(res.status), "plan_cached": bool(res.plan_cached),
                "batch_requests": int(res.batch_requests), "queue_ms": res.queue_ms,
                "run_ms": res.run_ms, "total_ms": res.total_ms, "message": res.message.decode(errors="replace")}

    def close(self):
        if getattr(self, "_h", None):
            _serve_lib().slk_serve_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
