"""GPU test of wsfft_execute_cube_noalloc, the entry point for callers that
cannot allocate device memory (code running while a CUDA graph is captured,
code whose memory belongs to another framework's allocator, or programs that
reserve all device memory up front).  It is called through the C ABI, two
calls in a row (a forward then an inverse), and each result is compared with
the regular plan-based entry point and with the FP64 oracle, within the
complex64 tolerance of the other GPU tests; its status word is read back
through wsfft_noalloc_sync_status after every call.  The file name makes
pytest collect it last."""
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
    g = L.wsfft_noalloc_sync_status
    g.argtypes = [ctypes.c_void_p]
    g.restype = ctypes.c_int
    return L


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def noalloc(L, x, y, n, batch, direction):
    return L.wsfft_execute_cube_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        n, batch, direction, _stream())


def regular(x, n, batch, direction):
    plan = W.Plan((n, n, n), W.C32, direction, batch)
    y = torch.empty_like(x)
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    plan.close()
    return y


@pytest.mark.parametrize("n,batch", [(128, 2), (256, 1), (512, 1)])
def test_noalloc_matches_plan_and_oracle_two_calls(lib, n, batch):
    shape = (batch, n, n, n)
    for call, (seed, direction) in enumerate(((1, W.FORWARD), (2, W.INVERSE))):
        xs = inputs.complex_input(shape, seed, "normal", "c32")
        x = torch.from_numpy(xs).cuda()
        y = torch.full_like(x, float("nan"))
        rc = noalloc(lib, x, y, n, batch, direction)
        assert rc == W.SUCCESS, (call, W.status_string(rc))
        assert lib.wsfft_noalloc_sync_status(_stream()) == W.SUCCESS
        got = y.cpu().numpy().astype(np.complex128)
        ref_plan = regular(x, n, batch, direction).cpu().numpy().astype(np.complex128)
        err_plan = oracle.rel_l2(got, ref_plan)
        del x, y
        ref = oracle.fftn(xs.astype(np.complex128), rank=3, sign=direction)
        err = oracle.rel_l2(got, ref)
        print(f"noalloc {n}^3 x{batch} call {call}: rel_l2 vs plan {err_plan:.2e}, vs oracle {err:.2e}")
        assert err_plan < TOL
        assert err < TOL


def test_noalloc_in_place_allocates_nothing(lib):
    n = 128
    xs = inputs.complex_input((n, n, n), 3, "normal", "c32")
    x = torch.from_numpy(xs).cuda()
    w = x.clone()
    assert noalloc(lib, w, w, n, 1, W.FORWARD) == W.SUCCESS  # warm: set-up already done or done here
    torch.cuda.synchronize()
    w.copy_(x)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    assert noalloc(lib, w, w, n, 1, W.FORWARD) == W.SUCCESS  # in place
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    assert lib.wsfft_noalloc_sync_status(_stream()) == W.SUCCESS
    ref = oracle.fftn(xs.astype(np.complex128))
    assert oracle.rel_l2(w.cpu().numpy().astype(np.complex128), ref) < TOL


def test_noalloc_rejects_sizes_beyond_its_arrays(lib):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    assert noalloc(lib, x, x, 512, 9, W.FORWARD) == W.ERR_INVALID_SIZE  # 9 * 512 > 4096 slabs
    assert noalloc(lib, x, x, 1024, 1, W.FORWARD) == W.ERR_INVALID_SIZE
    assert noalloc(lib, x, x, 100, 1, W.FORWARD) == W.ERR_INVALID_SIZE
    assert noalloc(lib, x, x, 128, 1, 0) == W.ERR_INVALID_ARG
    # in and out sharing bytes without being equal: refused before any GPU work
    p = x.data_ptr()
    assert lib.wsfft_execute_cube_noalloc(ctypes.c_void_p(p), ctypes.c_void_p(p + 16), 128, 1, W.FORWARD,
                                          _stream()) == W.ERR_INVALID_ARG
