"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Floating-point bar (relative L2 over all re and im
parts): 5e-6 for complex64 storage, 3e-3 for float16, 2e-2 for bfloat16; the
max-abs error is reported alongside."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build
from paper_2209_15040_gb300 import wsfft as W
from tests._helpers import DT, TOL, run_plan, seeded, to_device, to_host_c128

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()
    torch.cuda.init()


def check(shape_full, rank, dtype="c32", direction=W.FORWARD, norm=None, seed=0,
          dist="normal", inplace=False, ref_fn=None):
    xs, xc = seeded(shape_full, seed, dist, dtype)
    dims = shape_full[len(shape_full) - rank:]
    batch = int(np.prod(shape_full[:len(shape_full) - rank], dtype=np.int64))
    if norm is None:
        norm = W.NORM_PAPER if dtype == "c32" else W.NORM_ORTHO
    y = to_host_c128(run_plan(to_device(xs, dtype), dims, dtype, direction, batch, norm,
                              inplace), dtype)
    ref = ref_fn(xc) if ref_fn else oracle.fftn(xc, rank=rank, sign=direction, norm=norm)
    err = oracle.rel_l2(y, ref)
    print(f"{shape_full} rank={rank} {dtype} dir={direction} norm={norm}: rel_l2={err:.3e} "
          f"max_abs={oracle.max_abs(y, ref):.3e}")
    assert err < TOL[dtype], err
    return err


# -- 3D ---------------------------------------------------------------------

def test_8cubed_against_brute_force():
    # the 8x8x8 check of the 32^3 configuration: the definition, not the FFT
    check((8, 8, 8), 3, seed=0, dist="uniform", norm=W.NORM_NONE,
          ref_fn=lambda x: oracle.dft_brute(x))


def test_32cubed_uniform_seed0():
    check((32, 32, 32), 3, seed=0, dist="uniform")


@pytest.mark.parametrize("shape", [(4, 4, 4), (2, 4, 8), (2, 2, 2), (16, 64, 8), (64, 256, 32),
                                   (256, 32, 64), (32, 128, 256), (4096, 2, 16), (8, 4096, 2),
                                   (2, 8, 4096), (1, 16, 1), (1, 1, 1)])
def test_3d_shapes(shape):
    check(shape, 3, seed=3)


@pytest.mark.parametrize("n", [128, 256])
def test_cubes_forward_inverse(n):
    check((n, n, n), 3, seed=1)
    check((n, n, n), 3, seed=1, direction=W.INVERSE)


def test_batched_3d():
    check((8, 16, 16, 16), 3, seed=4)
    check((3, 32, 64, 16), 3, seed=5, direction=W.INVERSE)


@pytest.mark.parametrize("norm", [W.NORM_PAPER, W.NORM_NONE, W.NORM_ORTHO, W.NORM_FORWARD])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
def test_normalisations(norm, direction):
    if norm == W.NORM_FORWARD:
        # oracle has no forward-scaled mode: forward/N or unscaled inverse
        N = 16 * 32 * 8
        sc = 1.0 / N if direction == W.FORWARD else 1.0
        ref = lambda x: sc * oracle.fftn(x, rank=3, sign=direction, norm=oracle.NORM_NONE)
        check((16, 32, 8), 3, direction=direction, norm=norm, seed=6, ref_fn=ref)
    else:
        check((16, 32, 8), 3, direction=direction, norm=norm, seed=6)


def test_in_place():
    check((32, 64, 128), 3, seed=7, inplace=True)
    check((64, 64), 2, seed=7, inplace=True, direction=W.INVERSE)


def test_input_preserved_out_of_place():
    xs, _ = seeded((32, 32, 32), 8, "normal", "c32")
    x = to_device(xs, "c32")
    before = x.clone()
    run_plan(x, (32, 32, 32), "c32", W.FORWARD, 1)
    assert torch.equal(x, before)


# -- 2D and 1D ----------------------------------------------------------------

@pytest.mark.parametrize("shape", [(64, 64), (4096, 4096), (2, 4096), (4096, 8), (16, 32, 64)])
def test_2d(shape):
    check(shape, 2, seed=1)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_1d_short(n):
    check((7, n), 1, seed=9)
    check((3, n), 1, seed=9, direction=W.INVERSE)


@pytest.mark.parametrize("n", [8192, 1 << 14, 1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20, 1 << 21, 1 << 24])
def test_1d_four_step(n):
    batch = max(1, (1 << 22) // n)
    check((batch, n), 1, seed=1)
    check((min(batch, 2), n), 1, seed=2, direction=W.INVERSE)


def test_1d_2pow20_batch512_full_size():
    # the 1D case of the 512^3 configuration at its full size (512 transforms
    # of 2^20 points, 4 GiB, one workspace chunk): three batch entries against
    # the oracle element by element, and Parseval over the whole batch
    n, b = 1 << 20, 512
    g = torch.Generator(device="cuda")
    g.manual_seed(20)
    x = torch.view_as_complex(torch.randn(b, n, 2, generator=g, device="cuda")).contiguous()
    y = torch.empty_like(x)
    plan = W.Plan((n,), W.C32, W.FORWARD, b)
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    for i in (0, 257, 511):
        xi = x[i].cpu().numpy().astype(np.complex128)
        ref = oracle.fftn(xi, rank=1)
        err = oracle.rel_l2(y[i].cpu().numpy(), ref)
        assert err < TOL["c32"], (i, err)
    ex = torch.linalg.vector_norm(x.view(torch.float32).double()) ** 2
    ey = torch.linalg.vector_norm(y.view(torch.float32).double()) ** 2
    assert abs(float(ey / (n * ex)) - 1.0) < 1e-5


# -- reduced precision ---------------------------------------------------------

@pytest.mark.parametrize("dtype", ["c16f", "c16bf"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (128, 128, 128), (2, 64, 16, 256)])
def test_half_storage(dtype, shape):
    rank = 3
    check(shape, rank, dtype=dtype, seed=0, dist="uniform")
    check(shape, rank, dtype=dtype, seed=0, dist="uniform", direction=W.INVERSE)


@pytest.mark.parametrize("dtype", ["c16f", "c16bf"])
def test_half_storage_1d_and_2d(dtype):
    check((4, 1 << 16), 1, dtype=dtype, seed=2, dist="uniform")
    check((512, 512), 2, dtype=dtype, seed=2, dist="uniform")


# -- host-buffer entry point ----------------------------------------------------

def test_execute_host_buffers():
    xs, xc = seeded((2, 64, 32, 16), 11, "normal", "c32")
    plan = W.Plan((64, 32, 16), W.C32, W.FORWARD, 2)
    hin = torch.from_numpy(xs).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    plan.execute_host(hin.data_ptr(), hout.data_ptr())
    ref = oracle.fftn(xc, rank=3)
    assert oracle.rel_l2(hout.numpy(), ref) < TOL["c32"]
    plan.close()


@pytest.mark.parametrize("dtype", ["c32", "c16f", "c16bf"])
@pytest.mark.parametrize("shape_full", [(1, 64, 32, 16), (3, 2, 128, 64), (1, 16, 8, 8), (1, 128, 128, 128)])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
def test_execute_host_pipelined(dtype, shape_full, direction):
    # rank-3 host-buffer executes overlap the copies with the supersteps in
    # chunks (slab chunks in, inner-index chunks out); shapes cover fewer
    # slabs than chunks, batches, and an inner size at the chunking limit
    xs, xc = seeded(shape_full, 12, "normal" if dtype == "c32" else "uniform", dtype)
    norm = W.NORM_PAPER if dtype == "c32" else W.NORM_ORTHO
    plan = W.Plan(shape_full[1:], DT[dtype], direction, shape_full[0], norm)
    hin = to_device(xs, dtype).cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for inplace in (False, True):
        src = hin.clone().pin_memory() if inplace else hin
        dst = src if inplace else hout
        plan.execute_host(src.data_ptr(), dst.data_ptr())
        got = to_host_c128(dst, dtype)
        ref = oracle.fftn(xc, rank=3, sign=direction, norm=norm)
        err = oracle.rel_l2(got, ref)
        print(f"{shape_full} {dtype} dir={direction} inplace={inplace}: rel_l2={err:.3e}")
        assert err < TOL[dtype], err
    assert plan.sync_status() == W.SUCCESS
    plan.close()


def test_execute_rejects_misaligned_pointers():
    plan = W.Plan((16, 16, 16), W.C32, W.FORWARD, 1)
    x = torch.zeros(16 * 16 * 16 + 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(W.WsfftError) as e:
        plan.execute(x.data_ptr() + 8, x.data_ptr())
    assert e.value.status == W.ERR_INVALID_ARG
    plan.close()


def test_execute_rejects_partially_overlapping_buffers():
    # in == out is the in-place form; arrays that share some bytes are refused
    # (device and host entry points alike) and leave the data untouched
    n = 16 * 16 * 16
    plan = W.Plan((16, 16, 16), W.C32, W.FORWARD, 1)
    x = torch.arange(2 * n, dtype=torch.float32, device="cuda").view(torch.complex64)
    before = x.clone()
    for shift in (2, n // 2, n - 2):  # 16-byte aligned shifts that overlap
        with pytest.raises(W.WsfftError) as e:
            plan.execute(x.data_ptr(), x.data_ptr() + 8 * shift)
        assert e.value.status == W.ERR_INVALID_ARG
        with pytest.raises(W.WsfftError) as e:
            plan.execute(x.data_ptr() + 8 * shift, x.data_ptr())
        assert e.value.status == W.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.equal(x, before)
    plan.execute(x.data_ptr(), x.data_ptr() + 8 * n)  # adjacent, not overlapping
    h = torch.zeros(2 * n, dtype=torch.complex64).pin_memory()
    with pytest.raises(W.WsfftError) as e:
        plan.execute_host(h.data_ptr(), h.data_ptr() + 8 * (n // 2))
    assert e.value.status == W.ERR_INVALID_ARG
    plan.close()
    torch.cuda.synchronize()


# -- plans kept by fftn / ifftn ---------------------------------------------------

def test_fftn_plan_cache_is_bounded_and_thread_safe():
    import threading
    W.clear_plan_cache()
    W.set_plan_cache_size(3)
    try:
        sizes = (8, 16, 32, 64, 128)
        for n in sizes:
            xs, xc = seeded((4, n), 90 + n, "normal", "c32")
            y = W.fftn(torch.from_numpy(xs).cuda(), rank=1)
            assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(xc, rank=1)) < TOL["c32"]
            assert len(W._plans) <= 3
        assert len(W._plans) == 3
        # two threads cycling through more shapes than the cache holds: every
        # execute is enqueued while its plan is held, so none runs on a
        # destroyed plan
        errors = []

        def worker(seed):
            try:
                for k in range(20):
                    n = sizes[(seed + k) % len(sizes)]
                    xs, xc = seeded((2, n), seed * 100 + k, "normal", "c32")
                    y = W.ifftn(W.fftn(torch.from_numpy(xs).cuda(), rank=1), rank=1)
                    torch.cuda.synchronize()
                    if oracle.rel_l2(y.cpu().numpy(), xc) > TOL["c32"]:
                        errors.append((seed, k, n))
            except Exception as e:  # reported below
                errors.append(repr(e))

        threads = [threading.Thread(target=worker, args=(s,)) for s in (1, 2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        assert len(W._plans) <= 3
    finally:
        W.set_plan_cache_size(32)
        W.clear_plan_cache()
