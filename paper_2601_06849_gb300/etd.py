"""Python binding of the ETD2RK-DS CUDA library (include/etd.h).

Argument marshalling only: every step of the time integration runs in the
sm_103a kernels of ``libetd.so``. The functions named ``etd_*`` mirror the C ABI
one to one (pointers are passed as integers); :class:`Plan` wraps them for
torch tensors. PyTorch provides device memory and the stream; nothing here
computes. If the library has not been built, every call raises
:class:`EtdError` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libetd.so")

ETD_OK, ETD_ERR_INVALID_ARG, ETD_ERR_OOM, ETD_ERR_CUDA, ETD_ERR_UNSUPPORTED, ETD_ERR_DIVERGED, ETD_ERR_TIMEOUT = range(7)
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16x3": 4, "bf16x6": 5, "tf32x6": 6, "dst32": 7,
             "fp64split": 8, "fp64split40": 9, "fp64split32": 10}
# precisions whose fields and state are FP64
F64_PRECISIONS = ("fp64", "fp64split", "fp64split40", "fp64split32")
REACTION = {"none": 0, "linear": 1, "allen_cahn": 2, "fhn": 3, "singular": 4, "ac_forced": 5}
FAMILY = {"exact": 0, 2: 2, 4: 4, 0: 0}

# every symbol include/etd.h declares
SYMBOLS = (
    "etd_options_default", "etd_plan_create", "etd_step", "etd_step_host", "etd_transform",
    "etd_plan_invalidate", "etd_set_time", "etd_sync", "etd_field_stats", "etd_get_plan_info",
    "etd_set_timing", "etd_kernel_times", "etd_plan_destroy", "etd_status_string", "etd_last_error",
    "etd_transform_noalloc", "etd_batch_create", "etd_batch_step", "etd_step_adjoint",
    "etd_selftest_wait_timeout",
)
ETD_NOALLOC_MAX_ELEMS = 4194304
ETD_FLAG_AUTOTUNE = 1


class EtdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class etd_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("reaction", ctypes.c_int),
        ("rx_params", ctypes.c_double * 8),
        ("n_comp", ctypes.c_int),
        ("kappa_comp", ctypes.c_double * 2),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_int),
        ("diag_every", ctypes.c_int),
        ("diag_max_abs", ctypes.c_double),
    ]


class etd_plan_info(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("n", ctypes.c_int), ("n_comp", ctypes.c_int), ("precision", ctypes.c_int),
        ("products", ctypes.c_int), ("gemms_per_step", ctypes.c_int),
        ("unknowns", ctypes.c_longlong), ("gemm_flops", ctypes.c_double), ("step_flops", ctypes.c_double),
        ("workspace_bytes", ctypes.c_longlong), ("pass_persistent", ctypes.c_int * 2),
        ("pass_tile_n", ctypes.c_int * 2), ("step_bytes", ctypes.c_double), ("kernels_per_pass", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libetd.so; raise if it is missing (build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise EtdError(ETD_ERR_UNSUPPORTED,
                           f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "etd_options_default": ([ctypes.POINTER(etd_options)], i),
            "etd_plan_create": ([ctypes.POINTER(vp), i, i, d, d, d, i, ctypes.POINTER(etd_options)], i),
            "etd_step": ([vp, vp, i], i),
            "etd_step_host": ([vp, vp, i], i),
            "etd_transform": ([vp, vp, vp], i),
            "etd_plan_invalidate": ([vp], i),
            "etd_set_time": ([vp, d], i),
            "etd_sync": ([vp], i),
            "etd_field_stats": ([vp, vp, ctypes.POINTER(d), ctypes.POINTER(ll)], i),
            "etd_get_plan_info": ([vp, ctypes.POINTER(etd_plan_info)], i),
            "etd_set_timing": ([vp, i], i),
            "etd_kernel_times": ([vp, i, ctypes.POINTER(d), ctypes.POINTER(ll)], i),
            "etd_plan_destroy": ([vp], i),
            "etd_status_string": ([i], ctypes.c_char_p),
            "etd_last_error": ([], ctypes.c_char_p),
            "etd_transform_noalloc": ([i, i, i, vp, vp, vp], i),
            "etd_batch_create": ([ctypes.POINTER(vp), i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d),
                                  ctypes.POINTER(d), ctypes.POINTER(d), i, ctypes.POINTER(etd_options)], i),
            "etd_batch_step": ([vp, ctypes.POINTER(vp), i], i),
            "etd_step_adjoint": ([vp, vp, vp, i, ctypes.POINTER(d), ctypes.POINTER(d)], i),
            "etd_selftest_wait_timeout": ([vp, d], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return _lib


def _check(status: int) -> None:
    if status != ETD_OK:
        L = lib()
        raise EtdError(status, f"{L.etd_status_string(status).decode()}: {L.etd_last_error().decode()}")


# ---- the C ABI, one Python function per entry point --------------------------

def etd_options_default() -> etd_options:
    o = etd_options()
    _check(lib().etd_options_default(ctypes.byref(o)))
    return o


def etd_plan_create(d: int, m: int, kappa: float, q: float, dt: float, pade_order: int,
                    opt: Optional[etd_options] = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().etd_plan_create(ctypes.byref(h), d, m, kappa, q, dt, pade_order,
                                 ctypes.byref(opt) if opt is not None else None))
    return h.value


def etd_step(plan: int, u_dev: int, n_steps: int) -> None:
    _check(lib().etd_step(plan, u_dev, n_steps))


def etd_step_host(plan: int, u_host: int, n_steps: int) -> None:
    _check(lib().etd_step_host(plan, u_host, n_steps))


def etd_transform(plan: int, in_dev: int, out_dev: int) -> None:
    _check(lib().etd_transform(plan, in_dev, out_dev))


def etd_plan_invalidate(plan: int) -> None:
    _check(lib().etd_plan_invalidate(plan))


def etd_set_time(plan: int, t: float) -> None:
    _check(lib().etd_set_time(plan, t))


def etd_sync(plan: int) -> None:
    _check(lib().etd_sync(plan))


def etd_field_stats(plan: int, u_dev: int):
    m, bad = ctypes.c_double(), ctypes.c_longlong()
    st = lib().etd_field_stats(plan, u_dev, ctypes.byref(m), ctypes.byref(bad))
    if st not in (ETD_OK, ETD_ERR_DIVERGED):
        _check(st)
    return m.value, bad.value


def etd_get_plan_info(plan: int) -> etd_plan_info:
    info = etd_plan_info()
    _check(lib().etd_get_plan_info(plan, ctypes.byref(info)))
    return info


def etd_set_timing(plan: int, enable: bool) -> None:
    _check(lib().etd_set_timing(plan, int(bool(enable))))


def etd_kernel_times(plan: int, kind: int):
    ms, cnt = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().etd_kernel_times(plan, kind, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def etd_transform_noalloc(d: int, n: int, n_comp: int, in_dev: int, out_dev: int, stream: int = 0) -> None:
    """T(in) into out (float32 device fields) with no device allocation: the
    workspace is a fixed 16 MiB device array inside the library. For callers
    that must not allocate device memory during the call (a framework allocator
    owns the GPU's memory, or cudaFree's device-wide synchronisation cannot be
    afforded). Concurrent calls on the GPU share that array and race."""
    _check(lib().etd_transform_noalloc(d, n, n_comp, in_dev, out_dev, stream))


def etd_batch_create(d, m, kappa, q, dt, pade_order: int, opt: Optional[etd_options] = None) -> int:
    count = len(m)
    arr = lambda T, xs: (T * count)(*xs)
    h = ctypes.c_void_p()
    _check(lib().etd_batch_create(ctypes.byref(h), count, arr(ctypes.c_int, d), arr(ctypes.c_int, m),
                                  arr(ctypes.c_double, kappa), arr(ctypes.c_double, q), arr(ctypes.c_double, dt),
                                  pade_order, ctypes.byref(opt) if opt is not None else None))
    return h.value


def etd_batch_step(plan: int, u_dev_ptrs, n_steps: int) -> None:
    ptrs = (ctypes.c_void_p * len(u_dev_ptrs))(*u_dev_ptrs)
    _check(lib().etd_batch_step(plan, ptrs, n_steps))


def etd_step_adjoint(plan: int, u_ckpt: int, lambda_dev: int, n_steps: int):
    """Backpropagate lambda_dev (in place) through n_steps from u_ckpt; returns
    (dL/dkappa per component [2], dL/d rx_params [4])."""
    gk = (ctypes.c_double * 2)()
    gr = (ctypes.c_double * 4)()
    _check(lib().etd_step_adjoint(plan, u_ckpt, lambda_dev, n_steps, gk, gr))
    return list(gk), list(gr)


def etd_selftest_wait_timeout(plan: int, limit_ms: float) -> None:
    _check(lib().etd_selftest_wait_timeout(plan, limit_ms))


def etd_plan_destroy(plan: int) -> None:
    _check(lib().etd_plan_destroy(plan))


# ---- torch-facing wrappers ----------------------------------------------------

class Batch:
    """An ensemble of independent problems (one etd_batch_create handle).

    ``n``, ``kappa``, ``q``, ``dt`` are per-instance sequences; the reaction,
    precision, Pade order and component count are shared."""

    def __init__(self, d, n, kappa, q, dt, pade=2, precision="fp64split", reaction="fhn", rx_params=(), n_comp=2,
                 kappa_v=None, stream=None, autotune=False, diag_every=0, diag_max_abs=0.0):
        import torch

        count = len(n)
        d = [d] * count if isinstance(d, int) else list(d)
        self.n, self.d, self.n_comp = list(n), d, n_comp
        self.dtype = torch.float64 if precision in F64_PRECISIONS else torch.float32
        opt = etd_options_default()
        opt.precision = PRECISION[precision]
        opt.reaction = REACTION[reaction]
        for i, v in enumerate(rx_params):
            opt.rx_params[i] = float(v)
        opt.n_comp = n_comp
        if kappa_v is not None:
            opt.kappa_comp[1] = float(kappa_v)
        if autotune:
            opt.flags |= ETD_FLAG_AUTOTUNE
        opt.diag_every = int(diag_every)
        opt.diag_max_abs = float(diag_max_abs)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        self.handle = etd_batch_create(d, self.n, kappa, q, dt, FAMILY[pade], opt)

    def step(self, fields, n_steps: int = 1):
        for i, u in enumerate(fields):
            shape = (self.n_comp,) + (self.n[i],) * self.d[i]
            if not u.is_cuda or u.dtype != self.dtype or tuple(u.shape) != shape or not u.is_contiguous():
                raise EtdError(ETD_ERR_INVALID_ARG, f"field {i} must be a contiguous {self.dtype} CUDA tensor {shape}")
        etd_batch_step(self.handle, [u.data_ptr() for u in fields], n_steps)
        return fields

    def sync(self):
        etd_sync(self.handle)

    def invalidate(self):
        etd_plan_invalidate(self.handle)

    def info(self) -> etd_plan_info:
        return etd_get_plan_info(self.handle)

    def set_timing(self, enable: bool):
        etd_set_timing(self.handle, enable)

    def kernel_times(self, kind: int):
        return etd_kernel_times(self.handle, kind)

    def close(self):
        if getattr(self, "handle", None):
            etd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Plan:
    """One ETD2RK-DS problem on (0,1)^d with n interior points per axis.

    ``pade``: 2 (P_{0,2}), 4 (P_{0,4}) or "exact" (eq. (9)-(10)).
    ``precision``: one of PRECISION; fields are float64 for the F64_PRECISIONS, else float32.
    ``diag_every``, ``diag_max_abs``: the in-step field check of etd_options
    (0 = off); a failed check makes the next ``sync()`` raise ETD_ERR_DIVERGED.
    """

    def __init__(self, d: int, n: int, kappa: float, q: float, dt: float, pade=2, precision: str = "fp64split",
                 reaction: str = "allen_cahn", rx_params: Sequence[float] = (), n_comp: int = 1,
                 kappa_comp: Optional[Sequence[float]] = None, stream=None, autotune: bool = False,
                 diag_every: int = 0, diag_max_abs: float = 0.0):
        import torch

        self.d, self.n, self.dt, self.n_comp = d, n, dt, n_comp
        self.precision = precision
        self.dtype = torch.float64 if precision in F64_PRECISIONS else torch.float32
        opt = etd_options_default()
        opt.precision = PRECISION[precision]
        opt.reaction = REACTION[reaction]
        for i, v in enumerate(rx_params):
            opt.rx_params[i] = float(v)
        opt.n_comp = n_comp
        if kappa_comp is not None:
            for i, v in enumerate(kappa_comp):
                opt.kappa_comp[i] = float(v)
        if autotune:
            opt.flags |= ETD_FLAG_AUTOTUNE
        opt.diag_every = int(diag_every)
        opt.diag_max_abs = float(diag_max_abs)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        self.handle = etd_plan_create(d, n, kappa, q, dt, FAMILY[pade], opt)

    @property
    def shape(self):
        return (self.n_comp,) + (self.n,) * self.d

    def _check_field(self, u, name="u"):
        if not u.is_cuda or u.dtype != self.dtype or tuple(u.shape) != self.shape or not u.is_contiguous():
            raise EtdError(ETD_ERR_INVALID_ARG,
                           f"{name} must be a contiguous {self.dtype} CUDA tensor of shape {self.shape}, "
                           f"got {u.dtype} {tuple(u.shape)} on {u.device}")

    def step(self, u, n_steps: int = 1):
        """Advance u (CUDA tensor, shape (n_comp, n, ..)) in place; asynchronous."""
        self._check_field(u)
        etd_step(self.handle, u.data_ptr(), n_steps)
        return u

    def step_host(self, u_host, n_steps: int = 1):
        """Advance a CPU tensor in place through etd_step_host (copies inside the call)."""
        if u_host.is_cuda or u_host.dtype != self.dtype or tuple(u_host.shape) != self.shape or \
                not u_host.is_contiguous():
            raise EtdError(ETD_ERR_INVALID_ARG, f"u_host must be a contiguous CPU {self.dtype} tensor {self.shape}")
        etd_step_host(self.handle, u_host.data_ptr(), n_steps)
        return u_host

    def transform(self, x):
        import torch

        self._check_field(x, "x")
        out = torch.empty_like(x)
        etd_transform(self.handle, x.data_ptr(), out.data_ptr())
        return out

    def invalidate(self):
        etd_plan_invalidate(self.handle)

    def set_time(self, t: float):
        etd_set_time(self.handle, t)

    def sync(self):
        etd_sync(self.handle)

    def adjoint(self, u_ckpt, lam, n_steps: int):
        """lam <- dL/dU at u_ckpt given dL/dU n_steps later; returns (dL/dkappa, dL/drx)."""
        self._check_field(u_ckpt, "u_ckpt")
        self._check_field(lam, "lam")
        return etd_step_adjoint(self.handle, u_ckpt.data_ptr(), lam.data_ptr(), n_steps)

    def stats(self, u):
        self._check_field(u)
        return etd_field_stats(self.handle, u.data_ptr())

    def info(self) -> etd_plan_info:
        return etd_get_plan_info(self.handle)

    def set_timing(self, enable: bool):
        etd_set_timing(self.handle, enable)

    def kernel_times(self, kind: int):
        return etd_kernel_times(self.handle, kind)

    def close(self):
        if getattr(self, "handle", None):
            etd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
