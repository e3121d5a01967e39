"""wsfft for sm_103a: the k-superstep multidimensional complex FFT of
"Wafer-Scale Fast Fourier Transforms", as hand-written CUDA behind a C ABI
(include/wsfft.h).

Submodules load lazily so that ``inputs`` can be imported without the CUDA
library: ``wsfft`` (the binding), ``build`` (compiles the library),
``inputs`` (seeded synthetic inputs).
"""
import importlib

__all__ = ["wsfft", "build", "inputs", "fftn", "ifftn"]


def __getattr__(name):
    if name in ("wsfft", "build", "inputs"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("fftn", "ifftn", "Plan", "RaggedPlan"):
        return getattr(importlib.import_module(f"{__name__}.wsfft"), name)
    raise AttributeError(name)
