"""Python binding of libbspline.so (the C ABI in include/bspline.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Functions named like the ABI take raw integers/pointers; the Plan
class accepts torch tensors (device memory and streams come from PyTorch) and
passes their data pointers and the current stream to the ABI.  There is no
fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import math
import os

from . import _build

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_N = -2
ERR_UNSUPPORTED_ORDER = -3
ERR_CUDA = -4
ERR_NONFINITE_INPUT = -5
ERR_TIMEOUT = -6
ERR_NOT_IMPLEMENTED = -7
ERR_OUT_OF_MEMORY = -8
ERR_TOO_LARGE = -9
ERR_BOUNDS = -10
NOALLOC_MAX_N = 256
NOALLOC_MAX_PARTICLES = 131072

F64, F32, BF16 = 0, 1, 2
PREFILTER_INTERP, PREFILTER_L2 = 0, 1
INTERP_NO_GRAD = 0x1
INTERP_SORTED = 0x2
GATHER_SPLIT_AUTO = 0xFFFFFFFE

DTYPES = {"f64": F64, "f32": F32, "bf16": BF16}

_lib = None


class BSplineError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    # BSPLINE_LIBRARY selects another build of the same ABI (the BSPLINE_CHECKS=1 variant)
    path = os.environ.get("BSPLINE_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1201_4060_gb300._build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "bspline_plan": (i32, [ctypes.POINTER(vp), i32, i32, i32]),
        "bspline_plan_set_length": (i32, [vp, ctypes.c_double]),
        "bspline_plan_set_prefilter": (i32, [vp, i32]),
        "bspline_plan_set_band": (i32, [vp, i32]),
        "bspline_prefilter_values": (i32, [i32, i32, i32, ctypes.POINTER(ctypes.c_double)]),
        "bspline_plan_set_stream": (i32, [vp, vp]),
        "bspline_coeffs_bytes": (i32, [vp, ctypes.POINTER(sz)]),
        "bspline_uhat_bytes": (i32, [vp, ctypes.POINTER(sz)]),
        "bspline_coeffs": (i32, [vp, vp, vp]),
        "bspline_interp": (i32, [vp, vp, vp, i64, vp, vp, i32]),
        "bspline_eval": (i32, [vp, vp, vp, vp, i64, vp, vp, i32]),
        "bspline_spread_adjoint": (i32, [vp, vp, vp, i64, vp, vp, vp, vp, vp]),
        "bspline_sort_order": (i32, [vp, vp, i64, vp]),
        "bspline_workspace_bytes": (i32, [vp, i64, ctypes.POINTER(sz)]),
        "bspline_status": (i32, [vp, ctypes.POINTER(i64)]),
        "bspline_run_host": (i32, [vp, vp, vp, i64, vp, vp]),
        "bspline_run_host_async": (i32, [vp, vp, vp, i64, vp, vp]),
        "bspline_wait": (i32, [vp]),
        "bspline_destroy": (i32, [vp]),
        "bspline_status_string": (ctypes.c_char_p, [i32]),
        "bspline_version": (ctypes.c_char_p, []),
        "bspline_plan_set_timing": (i32, [vp, i32]),
        "bspline_plan_set_test_hooks": (i32, [vp, i32]),
        "bspline_plan_set_gather_split": (i32, [vp, ctypes.c_uint]),
        "bspline_plan_set_deterministic": (i32, [vp, i32]),
        "bspline_plan_autotune": (i32, [vp, vp, vp, i64, vp, vp, ctypes.POINTER(ctypes.c_uint),
                                        ctypes.POINTER(ctypes.c_double)]),
        "bspline_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
        "bspline_interp_noalloc": (i32, [vp, i32, i32, i32, ctypes.c_double, vp, i64, vp, vp, i32, vp]),
        "bspline_batch_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]),
        "bspline_batch_capture": (i32, [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "bspline_batch_launch": (i32, [vp, vp]),
        "bspline_batch_autotune": (i32, [vp, vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]),
        "bspline_batch_destroy": (i32, [vp]),
        "bspline_batch_set_layout": (i32, [vp, i32, i32, i32]),
        "bspline_batch_config": (i32, [vp] + [ctypes.POINTER(i32)] * 5),
        "bspline_batch_status": (i32, [vp, ctypes.POINTER(i64)]),
        "bspline_batch_set_test_hooks": (i32, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lib() -> ctypes.CDLL:
    return _load()


def status_string(code: int) -> str:
    return _load().bspline_status_string(code).decode()


def version() -> str:
    return _load().bspline_version().decode()


def _check(code: int, where: str) -> None:
    if code != OK:
        raise BSplineError(code, where)


def _require(t, name: str, shape, dtype, where: str) -> None:
    """Raise ValueError unless t is a contiguous tensor of this shape and dtype on the given side
    (where = "cuda" or "cpu"): the library reads and writes exactly that many elements through the
    pointer, so a smaller or strided buffer would be overrun."""
    on_side = t.is_cuda if where == "cuda" else t.device.type == "cpu"
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous() or not on_side:
        raise ValueError(f"{name} must be a contiguous {where} {dtype} tensor of shape {tuple(shape)}; got "
                         f"{t.dtype} {tuple(t.shape)} on {t.device}{'' if t.is_contiguous() else ', strided'}")


# ---- ABI-named thin wrappers (raw pointers / ints) --------------------------------

def bspline_plan(N: int, order: int, dtype: int) -> tuple[int, int]:
    h = ctypes.c_void_p()
    rc = _load().bspline_plan(ctypes.byref(h), N, order, dtype)
    return rc, (h.value or 0)


def bspline_plan_set_length(plan: int, L: float) -> int:
    return _load().bspline_plan_set_length(plan, L)


def bspline_plan_set_prefilter(plan: int, kind: int) -> int:
    return _load().bspline_plan_set_prefilter(plan, kind)


def bspline_prefilter_values(N: int, order: int, kind: int) -> tuple[int, list[float]]:
    """(status, [c(k) for k = 0..N-1]) of a plan of this N, order and prefilter kind (host, FP64)."""
    buf = (ctypes.c_double * max(int(N), 1))()
    rc = _load().bspline_prefilter_values(N, order, kind, buf)
    return rc, list(buf)[:max(int(N), 0)]


def bspline_plan_set_stream(plan: int, stream: int) -> int:
    return _load().bspline_plan_set_stream(plan, stream)


def bspline_coeffs(plan: int, u_hat_ptr: int, coeffs_ptr: int) -> int:
    return _load().bspline_coeffs(plan, u_hat_ptr, coeffs_ptr)


def bspline_interp(plan: int, coeffs_ptr: int, x_ptr: int, P: int, u_ptr: int, grad_ptr: int, flags: int) -> int:
    return _load().bspline_interp(plan, coeffs_ptr, x_ptr, P, u_ptr, grad_ptr, flags)


def bspline_run_host_async(plan: int, u_hat_ptr: int, x_ptr: int, P: int, u_ptr: int, grad_ptr: int) -> int:
    return _load().bspline_run_host_async(plan, u_hat_ptr, x_ptr, P, u_ptr, grad_ptr)


def bspline_wait(plan: int) -> int:
    return _load().bspline_wait(plan)


def bspline_eval(plan: int, u_hat_ptr: int, coeffs_ptr: int, x_ptr: int, P: int, u_ptr: int, grad_ptr: int,
                 flags: int) -> int:
    return _load().bspline_eval(plan, u_hat_ptr, coeffs_ptr, x_ptr, P, u_ptr, grad_ptr, flags)


def bspline_sort_order(plan: int, x_ptr: int, P: int, perm_ptr: int) -> int:
    return _load().bspline_sort_order(plan, x_ptr, P, perm_ptr)


def bspline_spread_adjoint(plan, coeffs_ptr, x_ptr, P, gu_ptr, ggrad_ptr, gcoef_ptr, guhat_ptr, gx_ptr) -> int:
    return _load().bspline_spread_adjoint(plan, coeffs_ptr, x_ptr, P, gu_ptr, ggrad_ptr, gcoef_ptr, guhat_ptr, gx_ptr)


def bspline_workspace_bytes(plan: int, P: int) -> tuple[int, int]:
    b = ctypes.c_size_t()
    rc = _load().bspline_workspace_bytes(plan, P, ctypes.byref(b))
    return rc, b.value


def bspline_coeffs_bytes(plan: int) -> tuple[int, int]:
    b = ctypes.c_size_t()
    rc = _load().bspline_coeffs_bytes(plan, ctypes.byref(b))
    return rc, b.value


def bspline_uhat_bytes(plan: int) -> tuple[int, int]:
    b = ctypes.c_size_t()
    rc = _load().bspline_uhat_bytes(plan, ctypes.byref(b))
    return rc, b.value


def bspline_status(plan: int) -> tuple[int, int]:
    n = ctypes.c_int64()
    rc = _load().bspline_status(plan, ctypes.byref(n))
    return rc, n.value


def bspline_run_host(plan: int, uhat_ptr: int, x_ptr: int, P: int, u_ptr: int, grad_ptr: int) -> int:
    return _load().bspline_run_host(plan, uhat_ptr, x_ptr, P, u_ptr, grad_ptr)


def bspline_destroy(plan: int) -> int:
    return _load().bspline_destroy(plan)


def bspline_status_string(code: int) -> str:
    return status_string(code)


NSTAGES = 10
STAGES = ["fft_x", "fft_yz", "bin", "scan", "scatter", "gather", "spread", "grad_x", "adj_fft", "gather_direct"]
TEST_DROP_TRANSFORM_SIGNALS = 0x1
TEST_NO_TMA = 0x2
TEST_SKIP_TMA_ISSUE = 0x4
TEST_DROP_QUEUE_SIGNAL = 0x8


def bspline_plan_set_test_hooks(plan: int, hooks: int) -> int:
    return _load().bspline_plan_set_test_hooks(plan, hooks)


def bspline_plan_set_timing(plan: int, enable: int) -> int:
    return _load().bspline_plan_set_timing(plan, enable)


def bspline_stage_times(plan: int) -> tuple[int, list[float], list[int]]:
    ms = (ctypes.c_double * NSTAGES)()
    n = (ctypes.c_int64 * NSTAGES)()
    rc = _load().bspline_stage_times(plan, ms, n)
    return rc, list(ms), list(n)


def bspline_interp_noalloc(coeffs_ptr: int, N: int, order: int, dtype: int, L: float, x_ptr: int, P: int,
                           u_ptr: int, grad_ptr: int, flags: int, stream: int) -> int:
    """Allocation-free evaluation (fixed scratch inside the library; see include/bspline.h)."""
    return _load().bspline_interp_noalloc(coeffs_ptr, N, order, dtype, L, x_ptr, P, u_ptr, grad_ptr, flags, stream)


# ---- torch-facing plan -------------------------------------------------------------

class Plan:
    """A plan for an N^3 periodic grid, B-spline order `order`, coefficient type `dtype`.

    u_hat: complex half spectrum [3, N, N, N//2+1] (complex128 for "f64", complex64 otherwise)
    coefficients: [3, N, N, N] of float64 / float32 / bfloat16
    positions: float64 [P, 3]; outputs u [P, 3], grad [P, 3, 3] (float64 for "f64", float32 otherwise)
    """

    def __init__(self, N: int, order: int, dtype: str = "f32", L: float = 2.0 * math.pi,
                 prefilter: str = "interp"):
        import torch  # noqa: F401  (device memory and streams)
        self.N, self.order, self.dtype = int(N), int(order), dtype
        rc, h = bspline_plan(self.N, self.order, DTYPES[dtype])
        _check(rc, "bspline_plan")
        self.handle = h
        self.L = float(L)
        if L != 2.0 * math.pi:
            _check(bspline_plan_set_length(h, self.L), "bspline_plan_set_length")
        if prefilter != "interp":
            _check(bspline_plan_set_prefilter(h, PREFILTER_L2), "bspline_plan_set_prefilter")

    def close(self) -> None:
        if getattr(self, "handle", 0):
            bspline_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # dtypes
    @property
    def uhat_dtype(self):
        import torch
        return torch.complex128 if self.dtype == "f64" else torch.complex64

    @property
    def coef_dtype(self):
        import torch
        return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[self.dtype]

    @property
    def out_dtype(self):
        import torch
        return torch.float64 if self.dtype == "f64" else torch.float32

    def _stream(self, stream=None) -> None:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(bspline_plan_set_stream(self.handle, s.cuda_stream), "bspline_plan_set_stream")

    def empty_coeffs(self):
        import torch
        return torch.empty((3, self.N, self.N, self.N), dtype=self.coef_dtype, device="cuda")

    def _require_coef(self, coef) -> None:
        _require(coef, "coef", (3, self.N, self.N, self.N), self.coef_dtype, "cuda")

    def _outputs(self, P, device, out_u, out_grad, grad):
        """The u and grad u buffers: allocated where not given, checked where given."""
        import torch
        if out_u is None:
            out_u = torch.empty((P, 3), dtype=self.out_dtype, device=device)
        _require(out_u, "out_u", (P, 3), self.out_dtype, "cuda")
        if grad:
            if out_grad is None:
                out_grad = torch.empty((P, 3, 3), dtype=self.out_dtype, device=device)
            _require(out_grad, "out_grad", (P, 3, 3), self.out_dtype, "cuda")
        return out_u, out_grad

    def coeffs(self, u_hat, out=None, stream=None):
        import torch
        N = self.N
        if u_hat.shape != (3, N, N, N // 2 + 1) or u_hat.dtype != self.uhat_dtype or not u_hat.is_cuda \
                or not u_hat.is_contiguous():
            raise ValueError(f"u_hat must be contiguous CUDA {self.uhat_dtype} of shape {(3, N, N, N // 2 + 1)}")
        if out is None:
            out = self.empty_coeffs()
        _require(out, "out", (3, N, N, N), self.coef_dtype, "cuda")
        self._stream(stream)
        _check(bspline_coeffs(self.handle, u_hat.data_ptr(), out.data_ptr()), "bspline_coeffs")
        return out

    def interp(self, coef, x, out_u=None, out_grad=None, grad: bool = True, stream=None, sorted: bool = False):
        """u (and grad u) at x; sorted=True passes BSPLINE_INTERP_SORTED (x in the order of sort_order)."""
        import torch
        if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA float64 tensor [P, 3]")
        P = x.shape[0]
        self._require_coef(coef)
        out_u, out_grad = self._outputs(P, x.device, out_u, out_grad, grad)
        self._stream(stream)
        flags = (0 if grad else INTERP_NO_GRAD) | (INTERP_SORTED if sorted else 0)
        rc = bspline_interp(self.handle, coef.data_ptr(), x.data_ptr(), P, out_u.data_ptr(),
                            out_grad.data_ptr() if grad else 0, flags)
        _check(rc, "bspline_interp")
        return (out_u, out_grad) if grad else out_u

    def sort_order(self, x, stream=None):
        """perm (int32 [P], device): original index of the particle evaluated i-th (bspline_sort_order);
        x[perm] can then be passed with sorted=True."""
        import torch
        if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA float64 tensor [P, 3]")
        perm = torch.empty((x.shape[0],), dtype=torch.int32, device=x.device)
        self._stream(stream)
        _check(bspline_sort_order(self.handle, x.data_ptr(), x.shape[0], perm.data_ptr()), "bspline_sort_order")
        return perm

    def eval(self, u_hat, x, coef=None, out_u=None, out_grad=None, grad: bool = True, stream=None,
             sorted: bool = False):
        """coeffs(u_hat) then interp at x in one call, the particle sort overlapping the transform.

        Returns (coef, u, grad_u), or (coef, u) with grad=False.
        """
        import torch
        N = self.N
        if u_hat.shape != (3, N, N, N // 2 + 1) or u_hat.dtype != self.uhat_dtype or not u_hat.is_cuda \
                or not u_hat.is_contiguous():
            raise ValueError(f"u_hat must be contiguous CUDA {self.uhat_dtype} of shape {(3, N, N, N // 2 + 1)}")
        if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA float64 tensor [P, 3]")
        if coef is None:
            coef = self.empty_coeffs()
        self._require_coef(coef)
        P = x.shape[0]
        out_u, out_grad = self._outputs(P, x.device, out_u, out_grad, grad)
        self._stream(stream)
        flags = (0 if grad else INTERP_NO_GRAD) | (INTERP_SORTED if sorted else 0)
        rc = bspline_eval(self.handle, u_hat.data_ptr(), coef.data_ptr(), x.data_ptr(), P, out_u.data_ptr(),
                          out_grad.data_ptr() if grad else 0, flags)
        _check(rc, "bspline_eval")
        return (coef, out_u, out_grad) if grad else (coef, out_u)

    def spread_adjoint(self, x, g_u=None, g_grad=None, coef=None, g_coef=None, u_hat_grad: bool = True,
                       stream=None):
        """Adjoint of coeffs + interp for the loss sum g_u . u + sum g_grad . grad u.

        Returns (g_u_hat, g_x, g_coef): g_coef [3, N, N, N] (out dtype) is accumulated into
        (allocated as zeros if None); g_u_hat (half spectrum, u_hat dtype) if u_hat_grad;
        g_x [P, 3] float64 if coef is given (position gradients need the coefficients).
        """
        import torch
        if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA float64 tensor [P, 3]")
        P, N = x.shape[0], self.N
        for name, tns, shape in (("g_u", g_u, (P, 3)), ("g_grad", g_grad, (P, 3, 3))):
            if tns is not None and (tns.shape != shape or tns.dtype != self.out_dtype or not tns.is_contiguous()
                                    or not tns.is_cuda):
                raise ValueError(f"{name} must be a contiguous CUDA {self.out_dtype} tensor {shape}")
        if coef is not None:
            self._require_coef(coef)
        if g_coef is None:
            g_coef = torch.zeros((3, N, N, N), dtype=self.out_dtype, device=x.device)
        else:
            _require(g_coef, "g_coef", (3, N, N, N), self.out_dtype, "cuda")
        g_u_hat = torch.empty((3, N, N, N // 2 + 1), dtype=self.uhat_dtype, device=x.device) if u_hat_grad \
            else None
        g_x = torch.empty((P, 3), dtype=torch.float64, device=x.device) if coef is not None else None
        self._stream(stream)
        rc = bspline_spread_adjoint(self.handle, coef.data_ptr() if coef is not None else 0, x.data_ptr(), P,
                                    g_u.data_ptr() if g_u is not None else 0,
                                    g_grad.data_ptr() if g_grad is not None else 0, g_coef.data_ptr(),
                                    g_u_hat.data_ptr() if g_u_hat is not None else 0,
                                    g_x.data_ptr() if g_x is not None else 0)
        _check(rc, "bspline_spread_adjoint")
        return g_u_hat, g_x, g_coef

    def status(self) -> int:
        """Count of non-finite positions of the last interp; raises if the last transform timed out."""
        rc, n = bspline_status(self.handle)
        if rc not in (OK, ERR_NONFINITE_INPUT):
            raise BSplineError(rc, "bspline_status")
        return n

    def set_deterministic(self, enable: bool) -> None:
        """Exact fixed-point sums in the adjoint spread: bit-identical results call to call
        (bspline_plan_set_deterministic)."""
        _check(_load().bspline_plan_set_deterministic(self.handle, 1 if enable else 0),
               "bspline_plan_set_deterministic")

    def set_band(self, kmax: int) -> None:
        """Modes with |kx|, |ky| or kz beyond kmax are zero (bspline_plan_set_band; 0 = off)."""
        _check(_load().bspline_plan_set_band(self.handle, int(kmax)), "bspline_plan_set_band")

    def set_gather_split(self, direct_below: int) -> None:
        """Bricks with fewer particles than this use the direct gather (bspline_plan_set_gather_split)."""
        _check(_load().bspline_plan_set_gather_split(self.handle, int(direct_below)), "bspline_plan_set_gather_split")

    def autotune(self, coef, x, out_u=None, out_grad=None, grad: bool = True):
        """Pick the gather split for these particles by timing (bspline_plan_autotune); returns (split, ms)."""
        import torch
        if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA float64 tensor [P, 3]")
        P = x.shape[0]
        self._require_coef(coef)
        out_u, out_grad = self._outputs(P, x.device, out_u, out_grad, grad)
        self._stream(None)
        split = ctypes.c_uint()
        ms = ctypes.c_double()
        rc = _load().bspline_plan_autotune(self.handle, coef.data_ptr(), x.data_ptr(), P, out_u.data_ptr(),
                                          out_grad.data_ptr() if grad else 0, ctypes.byref(split), ctypes.byref(ms))
        _check(rc, "bspline_plan_autotune")
        return split.value, ms.value

    def set_test_hooks(self, hooks: int) -> None:
        _check(bspline_plan_set_test_hooks(self.handle, hooks), "bspline_plan_set_test_hooks")

    def set_timing(self, enable: bool) -> None:
        _check(bspline_plan_set_timing(self.handle, 1 if enable else 0), "bspline_plan_set_timing")

    def stage_times(self) -> dict:
        """{stage: (total ms, launches)} since the last call; synchronises the plan's stream."""
        rc, ms, n = bspline_stage_times(self.handle)
        _check(rc, "bspline_stage_times")
        return {STAGES[i]: (ms[i], n[i]) for i in range(NSTAGES)}

    def workspace_bytes(self, P: int) -> int:
        rc, b = bspline_workspace_bytes(self.handle, P)
        _check(rc, "bspline_workspace_bytes")
        return b

    def run_host(self, u_hat_host, x_host, u_host, grad_host=None, stream=None, wait: bool = True):
        """Whole path on host (ideally pinned) tensors; copies happen inside the library call.

        wait=False queues the work and returns (bspline_run_host_async): the tensors must be left
        alone until wait() returns.
        """
        import torch
        N = self.N
        _require(u_hat_host, "u_hat_host", (3, N, N, N // 2 + 1), self.uhat_dtype, "cpu")
        if x_host.dim() != 2:
            raise ValueError("x_host must be a contiguous cpu torch.float64 tensor [P, 3]")
        P = x_host.shape[0]
        _require(x_host, "x_host", (P, 3), torch.float64, "cpu")
        _require(u_host, "u_host", (P, 3), self.out_dtype, "cpu")
        if grad_host is not None:
            _require(grad_host, "grad_host", (P, 3, 3), self.out_dtype, "cpu")
        self._stream(stream)
        fn = bspline_run_host if wait else bspline_run_host_async
        rc = fn(self.handle, u_hat_host.data_ptr(), x_host.data_ptr(), x_host.shape[0],
                u_host.data_ptr(), grad_host.data_ptr() if grad_host is not None else 0)
        _check(rc, "bspline_run_host" if wait else "bspline_run_host_async")

    def wait(self):
        """Wait for everything queued on the plan (bspline_wait)."""
        _check(bspline_wait(self.handle), "bspline_wait")


# ---- batches of independent fields (one CUDA graph launch) -------------------------

def _ptr_array(vals):
    arr = (ctypes.c_void_p * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = v
    return arr


class Batch:
    """Many fields, each with its own Plan, evaluated by one graph launch (bspline_batch_*).

    capture() takes lists (one entry per field) of u_hat, coefficient buffers, positions and output
    tensors, as Plan.coeffs / Plan.interp would; launch() replays the graph on the current stream.
    """

    def __init__(self, plans):
        self.plans = list(plans)          # keeps the plans alive while the batch exists
        h = ctypes.c_void_p()
        arr = _ptr_array([p.handle for p in self.plans])
        _check(_load().bspline_batch_create(ctypes.byref(h), len(self.plans), arr), "bspline_batch_create")
        self.handle = h.value
        self._keep = None

    def capture(self, u_hats, coeffs, xs, outs_u, outs_grad=None, streams: int = 4):
        n = len(self.plans)
        assert len(u_hats) == len(coeffs) == len(xs) == len(outs_u) == n
        P = (ctypes.c_int64 * n)(*[int(x.shape[0]) for x in xs])
        args = [_ptr_array([t.data_ptr() for t in lst]) for lst in (u_hats, coeffs, xs, outs_u)]
        g = _ptr_array([t.data_ptr() if t is not None else 0 for t in outs_grad]) if outs_grad is not None else None
        self._keep = (u_hats, coeffs, xs, outs_u, outs_grad)
        rc = _load().bspline_batch_capture(self.handle, streams, args[0], args[1], args[2], P, args[3], g)
        _check(rc, "bspline_batch_capture")

    def launch(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(_load().bspline_batch_launch(self.handle, s.cuda_stream), "bspline_batch_launch")

    def autotune(self, stream=None) -> tuple[int, float]:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        k = ctypes.c_int()
        ms = ctypes.c_double()
        _check(_load().bspline_batch_autotune(self.handle, s.cuda_stream, ctypes.byref(k), ctypes.byref(ms)),
               "bspline_batch_autotune")
        return k.value, ms.value

    def set_layout(self, queue: int = -1, brick_y: int = 0, item_particles: int = 2048) -> None:
        """Queue use (-1 auto, 0 never, 1 required), brick y extent and particles per gather item."""
        _check(_load().bspline_batch_set_layout(self.handle, queue, brick_y, item_particles),
               "bspline_batch_set_layout")

    def config(self) -> dict:
        vals = [ctypes.c_int() for _ in range(5)]
        _check(_load().bspline_batch_config(self.handle, *[ctypes.byref(v) for v in vals]), "bspline_batch_config")
        keys = ("queue", "streams", "brick_y", "item_particles", "kernel_nodes")
        return {k: v.value for k, v in zip(keys, vals)}

    def status(self) -> tuple[int, int]:
        """(status code, non-finite positions) of the last launch's queue (bspline_batch_status)."""
        n = ctypes.c_int64()
        rc = _load().bspline_batch_status(self.handle, ctypes.byref(n))
        return rc, n.value

    def set_test_hooks(self, hooks: int) -> None:
        _check(_load().bspline_batch_set_test_hooks(self.handle, hooks), "bspline_batch_set_test_hooks")

    def close(self) -> None:
        if getattr(self, "handle", 0):
            _load().bspline_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
