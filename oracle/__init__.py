"""FP64 CPU oracle for the k-superstep multidimensional complex FFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports, links or calls
it, and this package imports nothing from the product.

The arithmetic lives in ``fft_oracle.c`` (plain C, double precision, OpenMP
over pencils); this module only marshals numpy arrays to it and composes a few
of its calls.  What each function follows:

* ``fftn`` / ``ifftn`` -- the DFT of the paper's Section 1 evaluated as one
  superstep per axis (Section 1; Section 4.1 pencil computation; Section 4.2
  inverse with 1/N per compute stage).
* ``fft_axis`` -- one superstep alone (Section 2.2, Section 4.2).
* ``dft_brute`` / ``dft_points`` -- the definition evaluated term by term.
* ``loss_grad`` -- gradient of sum |W * F x|^2 via the adjoint of the
  unnormalised forward transform (the inverse with conjugated roots and no
  scaling, Section 4.2).  Not a result of the paper: its definition is the
  chain rule; pinned by finite differences in the tests.

Parity is pinned in ``tests/test_oracle.py`` against brute force, numpy's
pocketfft (the paper's own validator, Section 4.1), closed forms and
invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_fft.so")
_lib = None

NORM_PAPER = 0   # forward unscaled, inverse 1/n per axis (total 1/N)
NORM_NONE = 1    # never scaled
NORM_ORTHO = 2   # 1/sqrt(n) per axis, both directions


def build(force: bool = False) -> str:
    """Compile fft_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    lib.oracle_fftn.argtypes = [P, P, P, ci, i64, ci, ci]
    lib.oracle_fftn.restype = ci
    lib.oracle_fft_axis.argtypes = [P, P, ci, i64, ci, ci, ctypes.c_double]
    lib.oracle_fft_axis.restype = ci
    lib.oracle_dft_brute.argtypes = [P, P, P, ci, i64, ci]
    lib.oracle_dft_brute.restype = ci
    lib.oracle_dft_points.argtypes = [P, P, ci, ci, P, i64, P]
    lib.oracle_dft_points.restype = ci
    lib.oracle_unit_root.argtypes = [i64, i64, ci, P]
    lib.oracle_unit_root.restype = None
    lib.oracle_set_threads.argtypes = [ci]
    lib.oracle_get_threads.restype = ci
    _lib = lib
    return lib


def _dims_arr(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _c128(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def fftn(x, rank: int | None = None, sign: int = -1, norm: int = NORM_PAPER):
    """k-dimensional DFT over the last ``rank`` axes of ``x`` (leading axes are
    batch).  sign=-1 forward, +1 inverse.  Returns complex128."""
    x = _c128(x)
    rank = x.ndim if rank is None else rank
    dims = _dims_arr(x.shape[x.ndim - rank:])
    batch = int(np.prod(x.shape[:x.ndim - rank], dtype=np.int64))
    out = np.empty_like(x)
    rc = _load().oracle_fftn(x.ctypes.data, out.ctypes.data, dims.ctypes.data, rank,
                             batch, sign, norm)
    _check(rc, "fftn")
    return out


def ifftn(x, rank: int | None = None, norm: int = NORM_PAPER):
    return fftn(x, rank=rank, sign=+1, norm=norm)


def fft_axis(x, axis: int, rank: int | None = None, sign: int = -1, scale: float = 1.0):
    """One superstep: 1D DFTs along ``axis`` (counted within the last ``rank``
    axes, 0 = outermost transform axis)."""
    y = _c128(x).copy()
    rank = y.ndim if rank is None else rank
    dims = _dims_arr(y.shape[y.ndim - rank:])
    batch = int(np.prod(y.shape[:y.ndim - rank], dtype=np.int64))
    rc = _load().oracle_fft_axis(y.ctypes.data, dims.ctypes.data, rank, batch, axis,
                                 sign, float(scale))
    _check(rc, "fft_axis")
    return y


def dft_brute(x, rank: int | None = None, sign: int = -1):
    """O(N^2) DFT from the definition (unnormalised)."""
    x = _c128(x)
    rank = x.ndim if rank is None else rank
    dims = _dims_arr(x.shape[x.ndim - rank:])
    batch = int(np.prod(x.shape[:x.ndim - rank], dtype=np.int64))
    out = np.empty_like(x)
    rc = _load().oracle_dft_brute(x.ctypes.data, out.ctypes.data, dims.ctypes.data,
                                  rank, batch, sign)
    _check(rc, "dft_brute")
    return out


def dft_points(x, kflat, sign: int = -1):
    """Selected coefficients X[k] (flat row-major indices) of the full-rank
    DFT of one array ``x``, each by direct O(N) summation."""
    x = _c128(x)
    dims = _dims_arr(x.shape)
    k = np.ascontiguousarray(np.asarray(kflat, dtype=np.int64))
    out = np.empty(k.shape[0], dtype=np.complex128)
    rc = _load().oracle_dft_points(x.ctypes.data, dims.ctypes.data, x.ndim, sign,
                                   k.ctypes.data, k.shape[0], out.ctypes.data)
    _check(rc, "dft_points")
    return out


def unit_root(m: int, n: int, sign: int = -1) -> complex:
    buf = np.zeros(2, dtype=np.float64)
    _load().oracle_unit_root(int(m), int(n), int(sign), buf.ctypes.data)
    return complex(buf[0], buf[1])


def loss(x, w, rank: int | None = None) -> float:
    """L = sum |w * F x|^2 with F the unnormalised forward transform."""
    y = fftn(x, rank=rank, sign=-1, norm=NORM_NONE)
    return float(np.sum(np.abs(np.asarray(w, dtype=np.float64) * y) ** 2))


def loss_grad(x, w, rank: int | None = None):
    """dL/dx for L = sum |w * F x|^2, as the complex number dL/dRe + i dL/dIm
    (the convention torch uses for real losses of complex inputs).

    With Y = F x, L = sum w^2 |Y|^2, so dL/dY* = w^2 Y and, F being linear,
    dL/dx* = F^H (w^2 Y); F^H is the unnormalised inverse (conjugated roots,
    no 1/N).  The (dRe + i dIm) gradient is twice dL/dx*.
    """
    w2 = np.asarray(w, dtype=np.float64) ** 2
    y = fftn(x, rank=rank, sign=-1, norm=NORM_NONE)
    return 2.0 * fftn(w2 * y, rank=rank, sign=+1, norm=NORM_NONE)


def rel_l2(y, ref) -> float:
    """||y - ref||_2 / ||ref||_2 over all re and im parts."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((y - ref).ravel())
    return float(num / den) if den > 0 else float(num)


def max_abs(y, ref) -> float:
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.max(np.abs(y - ref))) if y.size else 0.0
