"""CPU checks of the C ABI: the library builds, loads, exports every function
that include/wsfft.h declares, and rejects bad arguments on the host before
touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2209_15040_gb300 import build
from paper_2209_15040_gb300 import wsfft as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(wsfft_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return W.lib()


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for must in ("wsfft_plan_create", "wsfft_execute", "wsfft_destroy", "wsfft_plan_set_norm",
                 "wsfft_plan_create_ragged", "wsfft_execute_ragged", "wsfft_autotune",
                 "wsfft_plan_sync_status", "wsfft_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(W.EXPORTS) <= set(declared_functions())


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        s = W.status_string(code)
        assert s and s != "unknown status"
    assert W.status_string(12345) == "unknown status"


def _create(lib, dims, rank=None, dtype=0, direction=-1, batch=1):
    rank = len(dims) if rank is None else rank
    arr = (ctypes.c_int64 * max(1, len(dims)))(*dims)
    h = ctypes.c_void_p()
    return lib.wsfft_plan_create(ctypes.byref(h), arr, rank, dtype, direction, batch), h


def test_host_validation_without_gpu(lib):
    # every one of these is rejected before any CUDA call
    assert _create(lib, [8, 8, 8], rank=0)[0] == W.ERR_INVALID_ARG
    assert _create(lib, [8, 8, 8, 8], rank=4)[0] == W.ERR_INVALID_ARG
    assert _create(lib, [8, 8, 8], batch=0)[0] == W.ERR_INVALID_ARG
    assert _create(lib, [8, 8, 8], dtype=7)[0] == W.ERR_INVALID_ARG
    assert _create(lib, [8, 8, 8], direction=0)[0] == W.ERR_INVALID_ARG
    assert _create(lib, [8, 12, 8])[0] == W.ERR_INVALID_SIZE
    assert _create(lib, [0, 8, 8])[0] == W.ERR_INVALID_SIZE
    assert _create(lib, [8192, 8])[0] == W.ERR_INVALID_SIZE       # rank 2: axes <= 4096
    assert _create(lib, [1 << 25])[0] == W.ERR_INVALID_SIZE       # rank 1: <= 2^24
    assert lib.wsfft_plan_create(None, None, 3, 0, -1, 1) == W.ERR_INVALID_ARG
    assert lib.wsfft_execute(None, None, None, None) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_set_norm(None, 0) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_set_layout(None, W.LAYOUT_SWAPPED) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_sync_status(None, None) == W.ERR_INVALID_ARG
    assert lib.wsfft_destroy(None) == W.SUCCESS


def test_ragged_host_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 6)(32, 64, 128, 32, 48, 32)
    assert lib.wsfft_plan_create_ragged(ctypes.byref(h), 2, dims, 0, -1) in (
        W.ERR_INVALID_SIZE, W.ERR_UNSUPPORTED)
    assert lib.wsfft_plan_create_ragged(ctypes.byref(h), 0, dims, 0, -1) in (
        W.ERR_INVALID_ARG, W.ERR_UNSUPPORTED)


def test_product_path_has_no_oracle_dependency():
    # the product package never imports the oracle, and the library links no
    # oracle object
    pkg = os.path.join(ROOT, "paper_2209_15040_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn), errors="ignore").read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "fft_oracle" not in src, fn


def test_new_entry_points_validate_on_the_host(lib):
    # rejected before any CUDA call: runs without a GPU
    h = ctypes.c_void_p()
    assert lib.wsfft_plan_create_axis(None, 512, 16, W.C32, W.FORWARD, 1) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 512, 16, W.C32, W.FORWARD, 0) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 512, 16, 9, W.FORWARD, 1) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 512, 16, W.C32, 0, 1) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 500, 16, W.C32, W.FORWARD, 1) == W.ERR_INVALID_SIZE
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 8192, 16, W.C32, W.FORWARD, 1) == W.ERR_INVALID_SIZE
    assert lib.wsfft_plan_create_axis(ctypes.byref(h), 512, 24, W.C32, W.FORWARD, 1) == W.ERR_INVALID_SIZE
    buf = (ctypes.c_char * 4096)()
    p = ctypes.addressof(buf)
    assert lib.wsfft_transpose_outer(None, p, 2, 2, 2, W.C32, None) == W.ERR_INVALID_ARG
    assert lib.wsfft_transpose_outer(p, p, 2, 2, 2, W.C32, None) == W.ERR_INVALID_ARG          # in == out
    assert lib.wsfft_transpose_outer(p, p + 32, 2, 2, 2, W.C32, None) == W.ERR_INVALID_ARG     # overlapping
    assert lib.wsfft_transpose_outer(p, p + 2048, 0, 2, 2, W.C32, None) == W.ERR_INVALID_ARG   # empty axis
    assert lib.wsfft_transpose_outer(p, p + 2048, 2, 2, 2, 5, None) == W.ERR_INVALID_ARG       # bad dtype
    assert lib.wsfft_plan_set_ragged_variant(None, 0, 1) == W.ERR_INVALID_ARG
    assert lib.wsfft_plan_set_engine(None, 4) == W.ERR_INVALID_ARG


def test_distributed_rejects_bad_layouts():
    from paper_2209_15040_gb300.distributed import SlabFFT3

    class Dummy:
        pass

    with pytest.raises(ValueError):
        SlabFFT3((64, 64), world=1, rank=0, local_forward=Dummy(), local_inverse=Dummy())
    with pytest.raises(ValueError):
        SlabFFT3((6, 8, 8), world=4, rank=0, local_forward=Dummy(), local_inverse=Dummy())
