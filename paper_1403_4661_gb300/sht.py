"""Thin Python binding of libsht (include/sht.h): argument marshalling only.

Every step of the transforms runs in the CUDA library; this module passes device pointers of
torch tensors and the current CUDA stream through the C ABI.  There is no fallback: if
libsht.so is missing or fails to load, the first call raises.

Functions with the C names (``sht_plan``, ``sht_forward``, ...) mirror the ABI one to one; the
``Plan`` class wraps a plan handle, and ``SHTForward`` / ``SHTInverse`` are the
``torch.autograd.Function``s whose backward passes call the adjoint entry points (PyTorch's
complex convention: grad_input = M^H grad_output for a linear map M).
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsht.so")

SHT_OK = 0
SHT_STATUS = {0: "SHT_OK", 1: "SHT_ERR_INVALID_ARG", 2: "SHT_ERR_UNSUPPORTED", 3: "SHT_ERR_OOM",
              4: "SHT_ERR_CUDA", 5: "SHT_ERR_NOT_CONVERGED", 6: "SHT_ERR_TIMEOUT"}
SHT_F64 = 0
SHT_F64_TENSOR = 1
SHT_BF16_REFINED = 2
SHT_BF16X2_REFINED = 3
SHT_TF32_REFINED = 4
SHT_F32 = 5
DTYPES = {"f64": SHT_F64, "f64_tensor": SHT_F64_TENSOR, "bf16_refined": SHT_BF16_REFINED,
          "bf16x2_refined": SHT_BF16X2_REFINED, "tf32_refined": SHT_TF32_REFINED, "f32": SHT_F32}
SHT_ORDER_GREEDY = 0
SHT_ORDER_SIMPLE = 1
MEASURES = {"uniform": 0, "sin": 2, "tan13": 4}   # SHT_MEASURE_* flags
SHT_PLAN_NO_PTILDE = 8
EXPORTED = ["sht_plan", "sht_plan_with_thetas", "sht_plan_thetas", "sht_plan_bandlimit",
            "sht_plan_reserve", "sht_plan_destroy", "sht_forward", "sht_inverse",
            "sht_inverse_adjoint", "sht_forward_adjoint", "sht_get_info", "sht_status_string",
            "sht_last_error_message", "sht_plan_set_timing", "sht_plan_stage_times",
            "sht_forward_noalloc", "sht_plan_check", "sht_plan_set_refinement",
            "sht_forward_uneven", "sht_inverse_uneven", "sht_plan_set_wait_limit",
            "sht_plan_set_paths", "sht_plan_autotune", "sht_plan_save", "sht_plan_load",
            "sht_plan_spin", "sht_plan_spin_with_thetas", "sht_uneven_create", "sht_uneven_forward",
            "sht_uneven_inverse", "sht_uneven_set_wait_limit", "sht_uneven_check", "sht_uneven_destroy",
            "sht_ring_analysis", "sht_ring_synthesis"]
SHT_PATH_DEFAULT = 0
SHT_PATH_TENSOR = 1
SHT_PATH_SIMT = 2
PATHS = {"default": SHT_PATH_DEFAULT, "tensor": SHT_PATH_TENSOR, "simt": SHT_PATH_SIMT}
STAGES = ["ring_dft", "solve", "alias", "layout", "synthesis", "ring_idft"]


class SHTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{SHT_STATUS.get(status, status)}: {msg}")
        self.status = status


class ShtInfo(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("dtype", ctypes.c_int), ("table_bytes", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("workspace_batch", ctypes.c_int64),
                ("plan_seconds", ctypes.c_double), ("order_seconds", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("refine_iterations", ctypes.c_int),
                ("refine_last_update", ctypes.c_double), ("spin", ctypes.c_int)]


class ShtTuning(ctypes.Structure):
    _fields_ = [("forward_path", ctypes.c_int), ("inverse_path", ctypes.c_int), ("split_cap", ctypes.c_int),
                ("forward_ms", ctypes.c_double), ("inverse_ms", ctypes.c_double)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libsht.so (once) and declare the ABI's signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsht.so not found at {path}; build it with "
                           "`python -m paper_1403_4661_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.sht_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(P)]
    lib.sht_plan_with_thetas.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_uint32, ctypes.POINTER(P)]
    lib.sht_plan_spin.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(P)]
    lib.sht_plan_spin_with_thetas.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double), ctypes.c_uint32, ctypes.POINTER(P)]
    lib.sht_plan_thetas.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.sht_plan_bandlimit.argtypes = [P]
    lib.sht_plan_bandlimit.restype = ctypes.c_int
    lib.sht_plan_reserve.argtypes = [P, i64]
    lib.sht_plan_destroy.argtypes = [P]
    for name in ("sht_forward", "sht_inverse", "sht_inverse_adjoint", "sht_forward_adjoint",
                 "sht_forward_noalloc", "sht_ring_analysis", "sht_ring_synthesis"):
        getattr(lib, name).argtypes = [P, P, P, i64, P]
    lib.sht_get_info.argtypes = [P, ctypes.POINTER(ShtInfo)]
    lib.sht_status_string.argtypes = [ctypes.c_int]
    lib.sht_status_string.restype = ctypes.c_char_p
    lib.sht_plan_check.argtypes = [P]
    lib.sht_plan_set_refinement.argtypes = [P, ctypes.c_int, ctypes.c_double]
    lib.sht_plan_set_wait_limit.argtypes = [P, ctypes.c_double]
    for name in ("sht_forward_uneven", "sht_inverse_uneven"):
        getattr(lib, name).argtypes = [ctypes.POINTER(P), ctypes.c_int, i64, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(i64), P, P, P]
    lib.sht_plan_set_paths.argtypes = [P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.sht_uneven_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, i64, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(i64), ctypes.POINTER(P)]
    lib.sht_uneven_forward.argtypes = [P, P, P, P]
    lib.sht_uneven_inverse.argtypes = [P, P, P, P]
    lib.sht_uneven_set_wait_limit.argtypes = [P, ctypes.c_double]
    lib.sht_uneven_check.argtypes = [P]
    lib.sht_uneven_destroy.argtypes = [P]
    lib.sht_plan_save.argtypes = [P, ctypes.c_char_p]
    lib.sht_plan_load.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(P)]
    lib.sht_plan_autotune.argtypes = [P, i64, ctypes.POINTER(ShtTuning)]
    lib.sht_plan_set_timing.argtypes = [P, ctypes.c_int]
    lib.sht_plan_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.sht_last_error_message.argtypes = []
    lib.sht_last_error_message.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("sht_plan_bandlimit", "sht_status_string", "sht_last_error_message"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != SHT_OK:
        msg = _lib.sht_last_error_message().decode(errors="replace")
        raise SHTError(status, msg)


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# -------------------------------------------------------------------------------------------
# C-named wrappers
# -------------------------------------------------------------------------------------------

def sht_plan(L, dtype=SHT_F64, flags=SHT_ORDER_GREEDY):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sht_plan(int(L), int(dtype), int(flags), ctypes.byref(h)))
    return h


def sht_plan_with_thetas(L, theta, dtype=SHT_F64, flags=0):
    lib = load_library()
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    if th.shape != (L,):
        raise ValueError("theta must have L entries")
    h = ctypes.c_void_p()
    _check(lib.sht_plan_with_thetas(int(L), int(dtype),
                                    th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    int(flags), ctypes.byref(h)))
    return h


def sht_plan_spin(L, spin, dtype=SHT_F64, flags=SHT_ORDER_GREEDY):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sht_plan_spin(int(L), int(spin), int(dtype), int(flags), ctypes.byref(h)))
    return h


def sht_plan_spin_with_thetas(L, spin, theta, dtype=SHT_F64, flags=0):
    lib = load_library()
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    if th.shape != (L,):
        raise ValueError("theta must have L entries")
    h = ctypes.c_void_p()
    _check(lib.sht_plan_spin_with_thetas(int(L), int(spin), int(dtype),
                                         th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(flags), ctypes.byref(h)))
    return h


def sht_plan_thetas(h, L):
    out = np.zeros(L, dtype=np.float64)
    _check(load_library().sht_plan_thetas(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def sht_plan_destroy(h):
    _check(load_library().sht_plan_destroy(h))


def sht_plan_reserve(h, batch):
    _check(load_library().sht_plan_reserve(h, int(batch)))


def sht_get_info(h):
    info = ShtInfo()
    _check(load_library().sht_get_info(h, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in ShtInfo._fields_}


def sht_plan_set_refinement(h, max_iters, tol):
    _check(load_library().sht_plan_set_refinement(h, int(max_iters), float(tol)))


def sht_plan_check(h):
    _check(load_library().sht_plan_check(h))


def sht_plan_set_timing(h, enable):
    _check(load_library().sht_plan_set_timing(h, 1 if enable else 0))


def sht_plan_stage_times(h):
    """{stage: (milliseconds, spans)} summed since the last query; clears the record."""
    ms = (ctypes.c_double * len(STAGES))()
    n = (ctypes.c_int64 * len(STAGES))()
    _check(load_library().sht_plan_stage_times(h, ms, n))
    return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}


def _call(name, h, inp, out, batch, stream=None):
    fn = getattr(load_library(), name)
    _check(fn(h, ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(batch),
              _stream_ptr(stream)))


def _as_batch(x, L, name, cdtype=torch.complex128):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != cdtype:
        raise TypeError(f"{name} must be {str(cdtype).replace('torch.', '')} for this plan")
    if x.shape[-1] != L * L:
        raise ValueError(f"{name}: last dimension must be L^2 = {L * L}")
    return x.contiguous()


def sht_forward(h, L, samples, out=None, stream=None, cdtype=torch.complex128):
    x = _as_batch(samples, L, "samples", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_forward", h, x, y, x.numel() // (L * L), stream)
    return y


def sht_forward_noalloc(h, L, samples, out=None, stream=None):
    """sht_forward with its scratch in the library's fixed device array (no allocation)."""
    x = _as_batch(samples, L, "samples")
    y = torch.empty_like(x) if out is None else out
    _call("sht_forward_noalloc", h, x, y, x.numel() // (L * L), stream)
    return y


def sht_inverse(h, L, coeffs, out=None, stream=None, cdtype=torch.complex128):
    x = _as_batch(coeffs, L, "coeffs", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_inverse", h, x, y, x.numel() // (L * L), stream)
    return y


def sht_ring_analysis(h, L, samples, out=None, stream=None, cdtype=torch.complex128):
    """Forward ring DFTs alone: ring-major bins, bin j of ring k at k^2 + k + j, 1/(2k+1) scaled."""
    x = _as_batch(samples, L, "samples", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_ring_analysis", h, x, y, x.numel() // (L * L), stream)
    return y


def sht_ring_synthesis(h, L, bins, out=None, stream=None, cdtype=torch.complex128):
    """Inverse ring DFTs alone (unscaled) from ring-major bins."""
    x = _as_batch(bins, L, "bins", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_ring_synthesis", h, x, y, x.numel() // (L * L), stream)
    return y


def _uneven(name, plans, plan_index, offsets, x, out, stream):
    """Signals of different band-limits packed in one flat complex128 tensor: signal i uses
    plans[plan_index[i]] and occupies L^2 values at element offset offsets[i]."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.complex128:
        raise TypeError("input must be a complex128 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x) if out is None else out
    n = len(plan_index)
    if len(offsets) != n:
        raise ValueError("plan_index and offsets differ in length")
    hs = (ctypes.c_void_p * max(1, len(plans)))(*[pl.handle for pl in plans])
    idx = (ctypes.c_int * max(1, n))(*[int(i) for i in plan_index])
    off = (ctypes.c_int64 * max(1, n))(*[int(o) for o in offsets])
    # the library validates indices and offsets; here only the extent of the valid signals
    ends = [int(o) + plans[int(i)].L ** 2 for i, o in zip(plan_index, offsets) if 0 <= int(i) < len(plans)]
    if ends and max(ends) > x.numel():
        raise ValueError("signals extend past the end of the input")
    _check(getattr(load_library(), name)(hs, len(plans), n, idx, off, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream)))
    return y


class UnevenBatch:
    """A batch of signals of different band-limits transformed in one persistent launch per
    direction (sht_uneven_create / sht_uneven_forward / sht_uneven_inverse).  The plans must stay
    alive while the batch exists; signal i uses plans[plan_index[i]] at complex offset offsets[i]."""

    def __init__(self, plans, plan_index, offsets):
        lib = load_library()
        self.plans = list(plans)
        n = len(plan_index)
        hs = (ctypes.c_void_p * max(1, len(self.plans)))(*[p.handle for p in self.plans])
        pi = (ctypes.c_int * max(1, n))(*[int(i) for i in plan_index])
        of = (ctypes.c_int64 * max(1, n))(*[int(o) for o in offsets])
        self.handle = ctypes.c_void_p()
        _check(lib.sht_uneven_create(hs, len(self.plans), n, pi, of, ctypes.byref(self.handle)))

    def _run(self, name, x, out, stream):
        if x.dtype != torch.complex128 or not x.is_cuda:
            raise ValueError("uneven batches take complex128 CUDA tensors")
        x = x.contiguous()
        if out is None:
            out = torch.zeros_like(x)
        _check(getattr(load_library(), name)(self.handle, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def forward(self, samples, out=None, stream=None):
        return self._run("sht_uneven_forward", samples, out, stream)

    def inverse(self, coeffs, out=None, stream=None):
        return self._run("sht_uneven_inverse", coeffs, out, stream)

    def set_wait_limit(self, seconds):
        _check(load_library().sht_uneven_set_wait_limit(self.handle, float(seconds)))

    def check(self):
        _check(load_library().sht_uneven_check(self.handle))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.sht_uneven_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward_uneven(plans, plan_index, offsets, samples, out=None, stream=None):
    """Forward SHT of signals of different band-limits in one call (sht_forward_uneven)."""
    return _uneven("sht_forward_uneven", plans, plan_index, offsets, samples, out, stream)


def inverse_uneven(plans, plan_index, offsets, coeffs, out=None, stream=None):
    """Inverse SHT of signals of different band-limits in one call (sht_inverse_uneven)."""
    return _uneven("sht_inverse_uneven", plans, plan_index, offsets, coeffs, out, stream)


def sht_forward_adjoint(h, L, coeffs, out=None, stream=None, cdtype=torch.complex128):
    x = _as_batch(coeffs, L, "coeffs", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_forward_adjoint", h, x, y, x.numel() // (L * L), stream)
    return y


def sht_inverse_adjoint(h, L, samples, out=None, stream=None, cdtype=torch.complex128):
    x = _as_batch(samples, L, "samples", cdtype)
    y = torch.empty_like(x) if out is None else out
    _call("sht_inverse_adjoint", h, x, y, x.numel() // (L * L), stream)
    return y


# -------------------------------------------------------------------------------------------
# Plan object and autograd
# -------------------------------------------------------------------------------------------

class Plan:
    """A libsht plan for band-limit L on the current CUDA device.

    Plan(L)                           greedy condition-number ring ordering (Sec. III-E)
    Plan(L, ordering="simple")        the ordering of Eq. (20)
    Plan(L, measure="sin" | "tan13")  rings from the sets of the alternative measures (Sec. III-F)
    Plan(L, theta=array_of_L_values)  caller-given ring co-latitudes
    Plan(L, spin=s)                   spin-s functions (Sec. III-H), float64 only
    Plan(L, keep_ptilde=False)        no P~ table (only uneven batches, which regenerate it)
    """

    def __init__(self, L, theta=None, ordering="greedy", dtype=SHT_F64, measure="uniform", spin=0,
                 keep_ptilde=True):
        self.L = int(L)
        dtype = DTYPES.get(dtype, dtype)
        self.dtype = dtype
        self.spin = int(spin)
        # element type of the plan's signals: complex64 for SHT_F32, complex128 otherwise
        self.cdtype = torch.complex64 if dtype == SHT_F32 else torch.complex128
        flags = {"greedy": SHT_ORDER_GREEDY, "simple": SHT_ORDER_SIMPLE}[ordering] | MEASURES[measure]
        if not keep_ptilde:
            flags |= SHT_PLAN_NO_PTILDE
        if self.spin != 0:
            self.handle = (sht_plan_spin_with_thetas(self.L, self.spin, theta, dtype) if theta is not None
                           else sht_plan_spin(self.L, self.spin, dtype, flags))
        elif theta is not None:
            self.handle = sht_plan_with_thetas(self.L, theta, dtype, flags & SHT_PLAN_NO_PTILDE)
        else:
            self.handle = sht_plan(self.L, dtype, flags)
        self.theta = sht_plan_thetas(self.handle, self.L)

    @classmethod
    def load(cls, path, dtype=SHT_F64):
        """A plan on the co-latitudes stored by Plan.save (sht_plan_load): no ring ordering."""
        dtype = DTYPES.get(dtype, dtype)
        h = ctypes.c_void_p()
        _check(load_library().sht_plan_load(os.fsencode(path), int(dtype), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle = h
        self.L = load_library().sht_plan_bandlimit(h)
        self.dtype = dtype
        self.cdtype = torch.complex64 if dtype == SHT_F32 else torch.complex128
        self.theta = sht_plan_thetas(h, self.L)
        return self

    def save(self, path):
        """Store the plan's ring co-latitudes in a checksummed file (sht_plan_save)."""
        _check(load_library().sht_plan_save(self.handle, os.fsencode(path)))

    def close(self):
        if getattr(self, "handle", None) is not None:
            sht_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, batch):
        sht_plan_reserve(self.handle, batch)

    def info(self):
        return sht_get_info(self.handle)

    def set_refinement(self, max_iters=10, tol=1e-11):
        """Iteration control of refined plans (tol = 0: fixed iterations, no synchronisation)."""
        sht_plan_set_refinement(self.handle, max_iters, tol)

    def set_paths(self, batch, forward="default", inverse="default", split_cap=0):
        """Pin the execution paths used for calls with this batch size (sht_plan_set_paths)."""
        _check(load_library().sht_plan_set_paths(self.handle, int(batch), PATHS.get(forward, forward),
                                                 PATHS.get(inverse, inverse), int(split_cap)))

    def autotune(self, batch):
        """Time every execution path the plan offers at this batch size and keep the fastest
        (sht_plan_autotune); returns the choice and its measured times."""
        t = ShtTuning()
        _check(load_library().sht_plan_autotune(self.handle, int(batch), ctypes.byref(t)))
        names = {v: k for k, v in PATHS.items()}
        return {"forward_path": names[t.forward_path], "inverse_path": names[t.inverse_path],
                "split_cap": t.split_cap, "forward_ms": t.forward_ms, "inverse_ms": t.inverse_ms}

    def set_wait_limit(self, seconds=1.0):
        """Limit of the tensor kernels' waits on other CTAs and on their pipeline."""
        _check(load_library().sht_plan_set_wait_limit(self.handle, float(seconds)))

    def check(self):
        """Synchronise and raise if a bounded device wait gave up since the last check."""
        sht_plan_check(self.handle)

    def set_timing(self, enable=True):
        sht_plan_set_timing(self.handle, enable)

    def stage_times(self):
        return sht_plan_stage_times(self.handle)

    def forward(self, samples, out=None, stream=None):
        return sht_forward(self.handle, self.L, samples, out, stream, self.cdtype)

    def inverse(self, coeffs, out=None, stream=None):
        return sht_inverse(self.handle, self.L, coeffs, out, stream, self.cdtype)

    def forward_adjoint(self, coeffs, out=None, stream=None):
        return sht_forward_adjoint(self.handle, self.L, coeffs, out, stream, self.cdtype)

    def ring_analysis(self, samples, out=None, stream=None):
        return sht_ring_analysis(self.handle, self.L, samples, out, stream, self.cdtype)

    def ring_synthesis(self, bins, out=None, stream=None):
        return sht_ring_synthesis(self.handle, self.L, bins, out, stream, self.cdtype)

    def inverse_adjoint(self, samples, out=None, stream=None):
        return sht_inverse_adjoint(self.handle, self.L, samples, out, stream, self.cdtype)


class SHTForward(torch.autograd.Function):
    """coeffs = F(samples); backward: grad_samples = F^H grad_coeffs."""

    @staticmethod
    def forward(ctx, plan, samples):
        ctx.plan = plan
        return plan.forward(samples)

    @staticmethod
    def backward(ctx, grad):
        return None, ctx.plan.forward_adjoint(grad.contiguous())


class SHTInverse(torch.autograd.Function):
    """samples = A(coeffs); backward: grad_coeffs = A^H grad_samples."""

    @staticmethod
    def forward(ctx, plan, coeffs):
        ctx.plan = plan
        return plan.inverse(coeffs)

    @staticmethod
    def backward(ctx, grad):
        return None, ctx.plan.inverse_adjoint(grad.contiguous())


def forward(plan, samples):
    """Differentiable forward SHT; real input is promoted to the plan's complex type (complex128,
    or complex64 for float32 plans)."""
    if not samples.is_complex():
        samples = samples.to(plan.cdtype)
    return SHTForward.apply(plan, samples)


def inverse(plan, coeffs):
    """Differentiable inverse SHT."""
    if not coeffs.is_complex():
        coeffs = coeffs.to(plan.cdtype)
    return SHTInverse.apply(plan, coeffs)
