"""GPU parity of the spectral layouts other than natural order: the swapped
layout (the middle axis in memory, as on the wafer after its two
transposes, Section 4.2: the last two axes swapped) and, for rank 3, the
wafer's own arrangement [n2][n0][n1].  The forward writes its result in the
layout, the inverse reads its input in it; the spatial side is natural.  Compared with the FP64 oracle's natural result with those two
axes swapped, for every storage type, rank 2 and 3, batches, in place and
out of place, and sizes that reach the tuned 512-point kernel shapes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build
from paper_2209_15040_gb300 import wsfft as W
from tests._helpers import DT, TOL, seeded, to_device, to_host_c128

pytestmark = pytest.mark.gpu

DTYPES = ["c32", "c16f", "c16bf"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()
    torch.cuda.init()


def _norm(dtype):
    return W.NORM_PAPER if dtype == "c32" else W.NORM_ORTHO


def _run(x, dims, dtype, direction, batch, inplace):
    plan = W.Plan(dims, DT[dtype], direction, batch, _norm(dtype))
    plan.set_layout(W.LAYOUT_SWAPPED)
    out = x.clone() if inplace else torch.empty_like(x)
    plan.execute(out.data_ptr() if inplace else x.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    return out


def _swapped_shape(shape):
    return tuple(shape[:-2]) + (shape[-1], shape[-2])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,rank", [((2, 64, 128, 256), 3), ((1, 128, 64), 3), ((3, 256, 64), 2),
                                        ((2, 512, 512), 2), ((4, 32, 512, 64), 3)])
@pytest.mark.parametrize("inplace", [False, True])
def test_forward_swapped(dtype, shape, rank, inplace):
    xs, xc = seeded(shape, 11, "uniform", dtype)
    x = to_device(xs, dtype)
    dims = shape[len(shape) - rank:]
    batch = int(np.prod(shape[:len(shape) - rank], dtype=np.int64))
    out = _run(x, dims, dtype, W.FORWARD, batch, inplace)
    y = to_host_c128(out, dtype).reshape(_swapped_shape(shape))
    ref = np.swapaxes(oracle.fftn(xc, rank=rank, norm=_norm(dtype)), -1, -2)
    err = oracle.rel_l2(y, ref)
    print(f"{shape} rank {rank} {dtype} forward swapped in_place={inplace}: rel_l2={err:.3e}")
    assert err < TOL[dtype], err


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,rank", [((2, 64, 128, 256), 3), ((3, 256, 64), 2), ((2, 512, 512), 2)])
@pytest.mark.parametrize("inplace", [False, True])
def test_inverse_from_swapped(dtype, shape, rank, inplace):
    # the device buffer holds a spectrum in the swapped layout
    xs, xc = seeded(shape, 12, "uniform", dtype)
    x = to_device(xs, dtype)
    dims = shape[len(shape) - rank:]
    batch = int(np.prod(shape[:len(shape) - rank], dtype=np.int64))
    out = _run(x, dims, dtype, W.INVERSE, batch, inplace)
    y = to_host_c128(out, dtype).reshape(shape)
    spec = np.swapaxes(xc.reshape(_swapped_shape(shape)), -1, -2)
    ref = oracle.fftn(spec, rank=rank, sign=+1, norm=_norm(dtype))
    err = oracle.rel_l2(y, ref)
    print(f"{shape} rank {rank} {dtype} inverse from swapped in_place={inplace}: rel_l2={err:.3e}")
    assert err < TOL[dtype], err


def test_round_trip_512_cube_swapped():
    # forward into the swapped layout and back: the input again (paper
    # normalisation), at the full 512^3 size of the bench workload
    n = 512
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    x = torch.view_as_complex(torch.randn(n, n, n, 2, generator=g, device="cuda")).contiguous()
    f = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    i = W.Plan((n, n, n), W.C32, W.INVERSE, 1)
    f.set_layout(W.LAYOUT_SWAPPED)
    i.set_layout(W.LAYOUT_SWAPPED)
    y = torch.empty_like(x)
    f.execute(x.data_ptr(), y.data_ptr())
    # sampled spectral entries against direct sums: X[k0, k1, k2] sits at [k0][k2][k1]
    rng = np.random.default_rng(4)
    xs = x.cpu().numpy().astype(np.complex128)
    j = np.arange(n)
    for _ in range(3):
        k0, k1, k2 = (int(v) for v in rng.integers(0, n, 3))
        e0 = np.exp(-2j * np.pi * j * k0 / n)
        e1 = np.exp(-2j * np.pi * j * k1 / n)
        e2 = np.exp(-2j * np.pi * j * k2 / n)
        want = ((xs @ e2) @ e1) @ e0
        got = complex(y[k0, k2, k1].item())
        assert abs(got - want) <= 5e-6 * np.sqrt(n ** 3) * 4, (k0, k1, k2, got, want)
    i.execute(y.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert f.sync_status() == W.SUCCESS and i.sync_status() == W.SUCCESS
    err = (torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)).item()
    assert err < 5e-6, err
    f.close()
    i.close()


def test_swapped_layout_rejections():
    p1 = W.Plan((4096,), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        p1.set_layout(W.LAYOUT_SWAPPED)  # rank 1
    p1.close()
    p2 = W.Plan((64, 32), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        p2.set_layout(W.LAYOUT_SWAPPED)  # an axis below 64
    p2.close()
    p3 = W.Plan((64, 64), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        p3.set_layout(7)
    p3.set_layout(W.LAYOUT_SWAPPED)
    p3.set_layout(W.LAYOUT_NATURAL)
    p3.close()


def test_swapped_layout_host_buffers():
    # wsfft_execute_host takes the plain (not pipelined) path for this layout
    shape = (64, 128, 256)
    xs, xc = seeded(shape, 13, "uniform", "c32")
    hx = torch.from_numpy(np.ascontiguousarray(xs)).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    plan = W.Plan(shape, W.C32, W.FORWARD, 1)
    plan.set_layout(W.LAYOUT_SWAPPED)
    plan.execute_host(hx.data_ptr(), hy.data_ptr())
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    y = hy.numpy().astype(np.complex128).reshape(_swapped_shape(shape))
    ref = np.swapaxes(oracle.fftn(xc, rank=3), -1, -2)
    assert oracle.rel_l2(y, ref) < TOL["c32"]


def test_swapped_layout_autotune_cache(tmp_path, monkeypatch):
    # the tuning cache keeps swapped and natural plans of one shape apart
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("WSFFT_TUNE_CACHE", str(cache))
    shape = (2, 256, 512)
    xs, xc = seeded(shape, 14, "normal", "c32")
    x = to_device(xs, "c32")
    y = torch.empty_like(x)
    plan = W.Plan(shape[1:], W.C32, W.FORWARD, 2)
    plan.set_layout(W.LAYOUT_SWAPPED)
    plan.autotune()
    assert len(cache.read_text().strip().splitlines()) == 1
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    plan.close()
    ref = oracle.fftn(xc, rank=2)
    got = to_host_c128(y, "c32").reshape(_swapped_shape(shape))
    assert oracle.rel_l2(got, np.swapaxes(ref, -1, -2)) < TOL["c32"]
    plan2 = W.Plan(shape[1:], W.C32, W.FORWARD, 2)
    plan2.autotune()
    assert len(cache.read_text().strip().splitlines()) == 2
    y.zero_()
    plan2.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    plan2.close()
    assert oracle.rel_l2(to_host_c128(y, "c32"), ref) < TOL["c32"]


# -- the wafer's own rank-3 arrangement [n2][n0][n1] ----------------------------

def _run_wafer(x, dims, dtype, direction, batch, inplace):
    plan = W.Plan(dims, DT[dtype], direction, batch, _norm(dtype))
    plan.set_layout(W.LAYOUT_WAFER)
    assert plan.passes()[0] == 3
    out = x.clone() if inplace else torch.empty_like(x)
    plan.execute(out.data_ptr() if inplace else x.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    return out


def _to_wafer(a):
    """[..., n0, n1, n2] -> [..., n2, n0, n1]"""
    return np.moveaxis(a, -1, -3)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", [(2, 64, 128, 256), (1, 256, 64, 128), (1, 128, 512, 64), (2, 64, 64, 512)])
@pytest.mark.parametrize("inplace", [False, True])
def test_forward_wafer(dtype, shape, inplace):
    xs, xc = seeded(shape, 15, "uniform", dtype)
    x = to_device(xs, dtype)
    out = _run_wafer(x, shape[1:], dtype, W.FORWARD, shape[0], inplace)
    n0, n1, n2 = shape[1:]
    y = to_host_c128(out, dtype).reshape((shape[0], n2, n0, n1))
    ref = _to_wafer(oracle.fftn(xc, rank=3, norm=_norm(dtype)))
    err = oracle.rel_l2(y, ref)
    print(f"{shape} {dtype} forward wafer in_place={inplace}: rel_l2={err:.3e}")
    assert err < TOL[dtype], err


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", [(2, 64, 128, 256), (1, 128, 512, 64), (2, 512, 64, 64)])
@pytest.mark.parametrize("inplace", [False, True])
def test_inverse_from_wafer(dtype, shape, inplace):
    # the device buffer holds a spectrum X[k0][k1][k2] stored as [k2][k0][k1]
    n0, n1, n2 = shape[1:]
    wshape = (shape[0], n2, n0, n1)
    xs, xc = seeded(wshape, 16, "uniform", dtype)
    x = to_device(xs, dtype)
    out = _run_wafer(x, shape[1:], dtype, W.INVERSE, shape[0], inplace)
    y = to_host_c128(out, dtype).reshape(shape)
    spec = np.moveaxis(xc, -3, -1)  # back to [k0][k1][k2]
    ref = oracle.fftn(spec, rank=3, sign=+1, norm=_norm(dtype))
    err = oracle.rel_l2(y, ref)
    print(f"{shape} {dtype} inverse from wafer in_place={inplace}: rel_l2={err:.3e}")
    assert err < TOL[dtype], err


def test_wafer_512_cube_forward_and_round_trip():
    # the bench workload's size: every spectral element against the oracle,
    # then the inverse from the wafer layout back to the input
    n = 512
    xs, xc = seeded((n, n, n), 17, "normal", "c32")
    x = to_device(xs, "c32")
    f = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    i = W.Plan((n, n, n), W.C32, W.INVERSE, 1)
    f.set_layout(W.LAYOUT_WAFER)
    i.set_layout(W.LAYOUT_WAFER)
    y = torch.empty_like(x)
    f.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    ref = _to_wafer(oracle.fftn(xc))
    err = oracle.rel_l2(got, ref)
    del got, ref
    print(f"512^3 wafer forward rel_l2 {err:.3e}")
    assert err < TOL["c32"]
    i.execute(y.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert f.sync_status() == W.SUCCESS and i.sync_status() == W.SUCCESS
    rt = (torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)).item()
    assert rt < 5e-6, rt
    f.close()
    i.close()


def test_wafer_layout_rejections():
    p2 = W.Plan((64, 64), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        p2.set_layout(W.LAYOUT_WAFER)  # rank 2 (its wafer order is LAYOUT_SWAPPED)
    p2.close()
    p3 = W.Plan((64, 32, 64), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        p3.set_layout(W.LAYOUT_WAFER)  # an axis below 64
    p3.set_layout(W.LAYOUT_NATURAL)
    p3.close()
