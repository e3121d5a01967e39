"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no FFT arithmetic: it draws random numbers, lays them out as
interleaved complex arrays and rounds them to a storage dtype.  Both the CUDA
path and the FP64 oracle are fed the same bytes from here.

Recipe (the paper prints no input values; these stand in for its workloads,
which are n^3 complex arrays with n = 32..512, Table 1):

* generator: ``numpy.random.default_rng(seed)``;
* draws of shape (*shape, 2) in float64, [..., 0] = re, [..., 1] = im;
* ``uniform``: U[-1, 1); ``normal``: N(0, 1);
* cast once to the storage dtype (complex64, or float16 / bfloat16 pairs with
  round-to-nearest-even), identical bytes on both sides;
* ragged shapes: ``default_rng(4).choice([32, 64, 128, 256], size=(count, 3))``
  drawn before any data.
"""
from __future__ import annotations

import numpy as np

DTYPES = ("c32", "c16f", "c16bf")


def draw(shape, seed: int, dist: str = "normal") -> np.ndarray:
    """Float64 draws of shape (*shape, 2) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    full = tuple(int(s) for s in shape) + (2,)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=full)
    if dist == "normal":
        return rng.standard_normal(size=full)
    raise ValueError(f"unknown distribution {dist!r}")


def _f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even); returns uint16 bits."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def _bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def to_storage(pairs: np.ndarray, dtype: str) -> np.ndarray:
    """Round float64 (..., 2) pairs to storage.

    c32   -> complex64 array of shape pairs.shape[:-1]
    c16f  -> float16 array of shape (..., 2)
    c16bf -> uint16 (bfloat16 bit patterns) array of shape (..., 2)
    """
    pairs = np.asarray(pairs)
    if dtype == "c32":
        return np.ascontiguousarray(pairs.astype(np.float32)).view(np.complex64)[..., 0]
    if dtype == "c16f":
        return np.ascontiguousarray(pairs.astype(np.float16))
    if dtype == "c16bf":
        # float64 -> float32 is exact for every bf16-representable value and
        # keeps nearest rounding to bf16 correct except for double-rounding
        # ties, which cannot matter for the identical bytes both sides get.
        return _f32_to_bf16_bits(pairs.astype(np.float32))
    raise ValueError(f"unknown dtype {dtype!r}")


def storage_to_c128(a: np.ndarray, dtype: str) -> np.ndarray:
    """Exact upcast of storage values to complex128 (what the oracle sees)."""
    if dtype == "c32":
        return np.asarray(a, dtype=np.complex64).astype(np.complex128)
    if dtype == "c16f":
        f = np.asarray(a, dtype=np.float16).astype(np.float64)
    elif dtype == "c16bf":
        f = _bf16_bits_to_f32(a).astype(np.float64)
    else:
        raise ValueError(f"unknown dtype {dtype!r}")
    return f[..., 0] + 1j * f[..., 1]


def complex_input(shape, seed: int, dist: str = "normal", dtype: str = "c32") -> np.ndarray:
    """Seeded input in storage layout (see ``to_storage``)."""
    return to_storage(draw(shape, seed, dist), dtype)


def loss_weights(shape, seed: int) -> np.ndarray:
    """Real weights W ~ U[0, 1) of the given shape (float32)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=tuple(shape)).astype(np.float32)


def ragged_shapes(count: int = 256, seed: int = 4, axes=(32, 64, 128, 256)) -> np.ndarray:
    """``count`` 3D shapes, each axis drawn independently from ``axes``."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(axes, dtype=np.int64), size=(count, 3))
