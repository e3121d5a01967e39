"""Python binding of the wsfft C ABI (include/wsfft.h).

Argument marshalling only: every step of a transform runs in the CUDA
library ``_build/libwsfft.so``.  There is no fallback: if the library is
missing, every call raises.

Tensors:
  complex64 CUDA tensors          -> WSFFT_C32
  float16  CUDA tensors (..., 2)  -> WSFFT_C16F  (re, im pairs)
  bfloat16 CUDA tensors (..., 2)  -> WSFFT_C16BF (re, im pairs)
"""
from __future__ import annotations

import collections
import ctypes
import os
import threading

import torch

C32, C16F, C16BF = 0, 1, 2
FORWARD, INVERSE = -1, 1
NORM_PAPER, NORM_NONE, NORM_ORTHO, NORM_FORWARD = 0, 1, 2, 3
LAYOUT_NATURAL, LAYOUT_SWAPPED, LAYOUT_WAFER = 0, 1, 2
NORMS = {"paper": NORM_PAPER, "none": NORM_NONE, "ortho": NORM_ORTHO, "forward": NORM_FORWARD}

SUCCESS = 0
ERR_INVALID_ARG = -1
ERR_INVALID_SIZE = -2
ERR_UNSUPPORTED = -3
ERR_ALLOC = -4
ERR_CUDA = -5
ERR_DEVICE_TIMEOUT = -6

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libwsfft.so")
_lib = None
_lock = threading.Lock()

EXPORTS = (
    "wsfft_plan_create", "wsfft_plan_set_norm", "wsfft_plan_set_layout", "wsfft_execute", "wsfft_execute_host",
    "wsfft_destroy", "wsfft_plan_create_ragged", "wsfft_execute_ragged", "wsfft_autotune",
    "wsfft_plan_sync_status", "wsfft_plan_passes", "wsfft_plan_profile",
    "wsfft_plan_set_pass_variant", "wsfft_plan_set_engine", "wsfft_plan_set_wait_test",
    "wsfft_plan_launch_times", "wsfft_status_string", "wsfft_plan_create_axis", "wsfft_transpose_outer",
    "wsfft_plan_set_ragged_variant",
)


class WsfftError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"wsfft CUDA library not built ({LIB_PATH}); run "
                               "paper_2209_15040_gb300.build.build_library()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.wsfft_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(i64), ci, ci, ci, i64]
        L.wsfft_plan_set_norm.argtypes = [P, ci]
        L.wsfft_plan_set_layout.argtypes = [P, ci]
        L.wsfft_execute.argtypes = [P, P, P, P]
        L.wsfft_execute_host.argtypes = [P, P, P, P]
        L.wsfft_destroy.argtypes = [P]
        L.wsfft_plan_create_ragged.argtypes = [ctypes.POINTER(P), ci, ctypes.POINTER(i64), ci, ci]
        L.wsfft_execute_ragged.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), P]
        L.wsfft_autotune.argtypes = [P, P]
        L.wsfft_plan_sync_status.argtypes = [P, P]
        L.wsfft_plan_passes.argtypes = [P, ctypes.POINTER(ci), ctypes.POINTER(i64)]
        L.wsfft_plan_profile.argtypes = [P, ci]
        L.wsfft_plan_set_pass_variant.argtypes = [P, ci, ci, ci]
        L.wsfft_plan_set_engine.argtypes = [P, ci]
        L.wsfft_plan_set_wait_test.argtypes = [P, ci, i64]
        L.wsfft_plan_launch_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), ci,
                                              ctypes.POINTER(ci)]
        L.wsfft_plan_create_axis.argtypes = [ctypes.POINTER(P), i64, i64, ci, ci, i64]
        L.wsfft_transpose_outer.argtypes = [P, P, i64, i64, i64, ci, P]
        L.wsfft_plan_set_ragged_variant.argtypes = [P, ci, ci]
        L.wsfft_status_string.argtypes = [ci]
        L.wsfft_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "wsfft_status_string":
                getattr(L, name).restype = ci
        _lib = L
        return L


def status_string(status: int) -> str:
    return lib().wsfft_status_string(int(status)).decode()


def _check(rc: int, what: str) -> None:
    if rc != SUCCESS:
        raise WsfftError(rc, what)


def _stream_handle(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """A plan for ``batch`` transforms of shape ``dims`` (see wsfft_plan_create)."""

    def __init__(self, dims, dtype: int = C32, direction: int = FORWARD, batch: int = 1,
                 norm: int | None = None):
        self.dims = tuple(int(d) for d in dims)
        self.dtype, self.direction, self.batch = int(dtype), int(direction), int(batch)
        arr = (ctypes.c_int64 * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        _check(lib().wsfft_plan_create(ctypes.byref(h), arr, len(self.dims), self.dtype,
                                       self.direction, self.batch), "wsfft_plan_create")
        self._h = h
        self.norm = NORM_PAPER if self.dtype == C32 else NORM_ORTHO
        if norm is not None:
            self.set_norm(norm)

    @property
    def handle(self):
        return self._h

    def set_norm(self, norm: int) -> None:
        _check(lib().wsfft_plan_set_norm(self._h, int(norm)), "wsfft_plan_set_norm")
        self.norm = int(norm)

    def execute(self, in_ptr: int, out_ptr: int, stream=None) -> None:
        _check(lib().wsfft_execute(self._h, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                   ctypes.c_void_p(_stream_handle(stream))), "wsfft_execute")

    def execute_host(self, host_in: int, host_out: int, stream=None) -> None:
        _check(lib().wsfft_execute_host(self._h, ctypes.c_void_p(host_in),
                                        ctypes.c_void_p(host_out),
                                        ctypes.c_void_p(_stream_handle(stream))),
               "wsfft_execute_host")

    def sync_status(self, stream=None) -> int:
        return int(lib().wsfft_plan_sync_status(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def autotune(self, stream=None) -> None:
        _check(lib().wsfft_autotune(self._h, ctypes.c_void_p(_stream_handle(stream))),
               "wsfft_autotune")

    def passes(self):
        n = ctypes.c_int()
        b = ctypes.c_int64()
        _check(lib().wsfft_plan_passes(self._h, ctypes.byref(n), ctypes.byref(b)),
               "wsfft_plan_passes")
        return n.value, b.value

    def set_layout(self, layout: int) -> None:
        """Spectral-side layout: LAYOUT_NATURAL, LAYOUT_SWAPPED (last two axes
        swapped) or LAYOUT_WAFER (rank 3: [n2][n0][n1], the wafer's order)."""
        _check(lib().wsfft_plan_set_layout(self._h, int(layout)), "wsfft_plan_set_layout")

    def set_pass_variant(self, pass_index: int, values_per_thread: int, tile: int) -> None:
        """Kernel shape of one pass (0, 0 = default); see wsfft_plan_set_pass_variant."""
        _check(lib().wsfft_plan_set_pass_variant(self._h, int(pass_index), int(values_per_thread),
                                                 int(tile)), "wsfft_plan_set_pass_variant")

    def set_engine(self, mode) -> None:
        """Schedule of an n0 x n x n transform: 0 one launch per superstep (the
        default), 4 cluster-fused z and y per slab (n in {256, 512}),
        3 warp-per-pencil, 1 persistent, 2 pipelined.  A mode the shape does not
        support runs one launch per superstep."""
        _check(lib().wsfft_plan_set_engine(self._h, int(mode)), "wsfft_plan_set_engine")

    def set_wait_test(self, withhold: bool, timeout_ns: int) -> None:
        """Testing aid: drop one completion signal so bounded waits run out."""
        _check(lib().wsfft_plan_set_wait_test(self._h, int(bool(withhold)), int(timeout_ns)),
               "wsfft_plan_set_wait_test")

    def profile(self, capacity: int) -> None:
        """Record CUDA events around up to ``capacity`` later kernel launches."""
        _check(lib().wsfft_plan_profile(self._h, int(capacity)), "wsfft_plan_profile")

    def launch_times(self, capacity: int = 4096):
        """Milliseconds of each recorded launch (and reset the recording)."""
        buf = (ctypes.c_float * max(1, capacity))()
        n = ctypes.c_int()
        _check(lib().wsfft_plan_launch_times(self._h, buf, capacity, ctypes.byref(n)),
               "wsfft_plan_launch_times")
        return [buf[i] for i in range(min(n.value, capacity))]

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().wsfft_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AxisPlan(Plan):
    """``batch`` x ``inner`` 1D transforms of length ``n`` along the middle
    axis of a [batch][n][inner] array (see wsfft_plan_create_axis)."""

    def __init__(self, n: int, inner: int, dtype: int = C32, direction: int = FORWARD, batch: int = 1,
                 norm: int | None = None):
        self.dims = (int(n),)
        self.inner = int(inner)
        self.dtype, self.direction, self.batch = int(dtype), int(direction), int(batch)
        h = ctypes.c_void_p()
        _check(lib().wsfft_plan_create_axis(ctypes.byref(h), int(n), self.inner, self.dtype, self.direction,
                                            self.batch), "wsfft_plan_create_axis")
        self._h = h
        self.norm = NORM_PAPER if self.dtype == C32 else NORM_ORTHO
        if norm is not None:
            self.set_norm(norm)


def transpose_outer(in_ptr: int, out_ptr: int, a: int, b: int, c: int, dtype: int = C32, stream=None) -> None:
    """out[b][a][c] = in[a][b][c] on the device (see wsfft_transpose_outer)."""
    _check(lib().wsfft_transpose_outer(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(a), int(b), int(c),
                                       int(dtype), ctypes.c_void_p(_stream_handle(stream))),
           "wsfft_transpose_outer")


class RaggedPlan:
    """One persistent launch over ``count`` rank-3 transforms of uneven shapes."""

    def __init__(self, shapes, dtype: int = C32, direction: int = FORWARD):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        flat = [v for s in self.shapes for v in s]
        arr = (ctypes.c_int64 * len(flat))(*flat)
        h = ctypes.c_void_p()
        _check(lib().wsfft_plan_create_ragged(ctypes.byref(h), len(self.shapes), arr, int(dtype),
                                              int(direction)), "wsfft_plan_create_ragged")
        self._h = h

    @property
    def handle(self):
        return self._h

    def execute(self, in_ptrs, out_ptrs, stream=None) -> None:
        n = len(self.shapes)
        ia = (ctypes.c_void_p * n)(*[int(p) for p in in_ptrs])
        oa = (ctypes.c_void_p * n)(*[int(p) for p in out_ptrs])
        _check(lib().wsfft_execute_ragged(self._h, ia, oa, ctypes.c_void_p(_stream_handle(stream))),
               "wsfft_execute_ragged")

    def sync_status(self, stream=None) -> int:
        return int(lib().wsfft_plan_sync_status(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def set_variant(self, shape_select: int, lag: int = 1) -> None:
        """Tile shape per axis length (bit log2(N) - 5) and queue lag (see
        wsfft_plan_set_ragged_variant)."""
        _check(lib().wsfft_plan_set_ragged_variant(self._h, int(shape_select), int(lag)),
               "wsfft_plan_set_ragged_variant")

    def autotune(self, stream=None) -> None:
        _check(lib().wsfft_autotune(self._h, ctypes.c_void_p(_stream_handle(stream))), "wsfft_autotune")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().wsfft_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# torch-level API


def storage_of(x: torch.Tensor):
    """(dtype code, logical shape) of a tensor in one of the storage layouts."""
    if x.dtype == torch.complex64:
        return C32, tuple(x.shape)
    if x.dtype in (torch.float16, torch.bfloat16):
        if x.ndim < 1 or x.shape[-1] != 2:
            raise ValueError("float16/bfloat16 complex storage needs a trailing dimension of 2")
        return (C16F if x.dtype == torch.float16 else C16BF), tuple(x.shape[:-1])
    raise TypeError(f"unsupported dtype {x.dtype}")


_plans: "collections.OrderedDict" = collections.OrderedDict()
_plans_lock = threading.Lock()
_plan_cache_size = 32


def set_plan_cache_size(n: int) -> None:
    """Plans that fftn/ifftn keep (least recently used ones are destroyed
    beyond it: a plan holds its tables and, for long 1D axes or the other
    spectral layouts, a workspace of up to 4 GiB)."""
    global _plan_cache_size
    if n < 1:
        raise ValueError("the plan cache holds at least one plan")
    with _plans_lock:
        _plan_cache_size = int(n)
        _evict_locked()


def clear_plan_cache() -> None:
    """Destroy every plan fftn/ifftn keep (each waits for its own work)."""
    with _plans_lock:
        while _plans:
            _plans.popitem(last=False)[1].close()


def _evict_locked() -> None:
    while len(_plans) > _plan_cache_size:
        _plans.popitem(last=False)[1].close()


def _get_plan_locked(dims, dtype, direction, batch, norm) -> Plan:
    key = (torch.cuda.current_device(), tuple(dims), dtype, direction, batch, norm)
    p = _plans.get(key)
    if p is None:
        p = Plan(dims, dtype, direction, batch, norm)
        _plans[key] = p
        _evict_locked()
    else:
        _plans.move_to_end(key)
    return p


def get_plan(dims, dtype, direction, batch, norm) -> Plan:
    """The cached plan for these parameters (made on first use).  It may be
    destroyed once more than the cache size of other plans have been used
    since; fftn/ifftn enqueue their executes while holding the cache."""
    with _plans_lock:
        return _get_plan_locked(dims, dtype, direction, batch, norm)


def _run(x: torch.Tensor, rank, direction: int, norm, out=None) -> torch.Tensor:
    if not x.is_cuda:
        raise ValueError("wsfft operates on CUDA tensors")
    code, shape = storage_of(x)
    rank = len(shape) if rank is None else int(rank)
    if not 1 <= rank <= min(3, len(shape)):
        raise ValueError(f"rank must be 1..3 and at most the tensor rank, got {rank}")
    dims = shape[len(shape) - rank:]
    batch = 1
    for s in shape[:len(shape) - rank]:
        batch *= s
    if norm is None:
        norm = NORM_PAPER if code == C32 else NORM_ORTHO
    norm = NORMS[norm] if isinstance(norm, str) else int(norm)
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    if x.numel() == 0:
        return out
    with torch.cuda.device(x.device), _plans_lock:
        # enqueue under the cache lock: no other thread can evict the plan
        # between the lookup and the execute
        _get_plan_locked(dims, code, direction, batch, norm).execute(x.data_ptr(), out.data_ptr())
    return out


_ADJOINT_NORM = {  # (direction, norm) -> norm of the adjoint transform (other direction)
    (FORWARD, NORM_PAPER): NORM_NONE, (FORWARD, NORM_NONE): NORM_NONE,
    (FORWARD, NORM_ORTHO): NORM_ORTHO, (FORWARD, NORM_FORWARD): NORM_PAPER,
    (INVERSE, NORM_PAPER): NORM_FORWARD, (INVERSE, NORM_NONE): NORM_NONE,
    (INVERSE, NORM_ORTHO): NORM_ORTHO, (INVERSE, NORM_FORWARD): NORM_NONE,
}


class _FFTN(torch.autograd.Function):
    """Y = F x with the adjoint as backward: for a linear map, the gradient
    of a real loss is F^H applied to the output gradient, and F^H is the
    transform of the opposite direction with conjugated roots and the
    matching scale (Section 4.2 gives the conjugated-roots inverse)."""

    @staticmethod
    def forward(ctx, x, rank, direction, norm):
        ctx.rank, ctx.direction, ctx.norm = rank, direction, norm
        return _run(x, rank, direction, norm)

    @staticmethod
    def backward(ctx, g):
        adj = _ADJOINT_NORM[(ctx.direction, ctx.norm)]
        return _run(g.contiguous(), ctx.rank, -ctx.direction, adj), None, None, None


def _resolve_norm(x, norm):
    if norm is None:
        return NORM_PAPER if x.dtype == torch.complex64 else NORM_ORTHO
    return NORMS[norm] if isinstance(norm, str) else int(norm)


def fftn(x: torch.Tensor, rank: int | None = None, norm=None) -> torch.Tensor:
    """Forward transform over the last ``rank`` logical axes (differentiable)."""
    return _FFTN.apply(x, rank, FORWARD, _resolve_norm(x, norm))


def ifftn(x: torch.Tensor, rank: int | None = None, norm=None) -> torch.Tensor:
    """Inverse transform over the last ``rank`` logical axes (differentiable)."""
    return _FFTN.apply(x, rank, INVERSE, _resolve_norm(x, norm))
