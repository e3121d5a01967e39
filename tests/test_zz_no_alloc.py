"""GPU test of wsfft_execute_cube_noalloc, the entry point for callers that
cannot allocate device memory (inside graph capture, under a foreign
allocator, or with all memory reserved up front).  It is called through the
C ABI and compared with the regular plan-based entry point on two calls in a
row, within the complex64 tolerance of the other GPU tests.  The file name
makes pytest collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build, inputs
from paper_2209_15040_gb300 import wsfft as W

pytestmark = pytest.mark.gpu
TOL = 5e-6


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    L = W.lib()
    f = L.wsfft_execute_cube_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def noalloc(L, x, y, n, batch, direction):
    st = torch.cuda.current_stream().cuda_stream
    return L.wsfft_execute_cube_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        n, batch, direction, ctypes.c_void_p(st))


def regular(x, n, batch, direction):
    plan = W.Plan((n, n, n), W.C32, direction, batch)
    y = torch.empty_like(x)
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    plan.close()
    return y


@pytest.mark.parametrize("n,batch", [(128, 2), (256, 1), (512, 1)])
def test_noalloc_matches_plan_two_calls(lib, n, batch):
    shape = (batch, n, n, n)
    for call, (seed, direction) in enumerate(((1, W.FORWARD), (2, W.INVERSE))):
        x = torch.from_numpy(inputs.complex_input(shape, seed, "normal", "c32")).cuda()
        y = torch.full_like(x, float("nan"))
        rc = noalloc(lib, x, y, n, batch, direction)
        assert rc == W.SUCCESS, (call, W.status_string(rc))
        torch.cuda.synchronize()
        ref = regular(x, n, batch, direction)
        err = oracle.rel_l2(y.cpu().numpy(), ref.cpu().numpy())
        print(f"noalloc {n}^3 x{batch} call {call}: rel_l2 vs plan {err:.2e}")
        assert err < TOL
        del x, y, ref


def test_noalloc_rejects_sizes_beyond_its_arrays(lib):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    assert noalloc(lib, x, x, 512, 9, W.FORWARD) == W.ERR_INVALID_SIZE  # 9 * 512 > 4096 slabs
    assert noalloc(lib, x, x, 1024, 1, W.FORWARD) == W.ERR_INVALID_SIZE
    assert noalloc(lib, x, x, 100, 1, W.FORWARD) == W.ERR_INVALID_SIZE
    assert noalloc(lib, x, x, 128, 1, 0) == W.ERR_INVALID_ARG
