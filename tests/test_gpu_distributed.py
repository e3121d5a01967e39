"""GPU parity of the pieces of the slab-distributed transform: the axis plan
(one superstep along a strided axis, wsfft_plan_create_axis), the outer-axes
transpose that regroups a slab by destination (wsfft_transpose_outer,
bit-exact), and the whole distributed forward/inverse with the library's
kernels -- G ranks emulated in one process with an in-process exchange (one
GPU per run here), and G = 1 through a real NCCL process group."""
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build, inputs
from paper_2209_15040_gb300 import wsfft as W
from paper_2209_15040_gb300.distributed import SlabFFT3
from tests._helpers import DT, TOL, to_device, to_host_c128

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()


@pytest.mark.parametrize("dtype", ["c32", "c16f", "c16bf"])
@pytest.mark.parametrize("n,inner,batch", [(512, 4096, 2), (64, 16, 3), (128, 1, 5), (1024, 1 << 17, 1),
                                           (8, 2, 7), (4096, 32, 1)])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
def test_axis_plan(dtype, n, inner, batch, direction):
    shape = (batch, n, inner)
    dist = "normal" if dtype == "c32" else "uniform"
    xs = inputs.complex_input(shape, 31, dist, dtype)
    xc = inputs.storage_to_c128(xs, dtype)
    x = to_device(xs, dtype)
    y = torch.empty_like(x)
    plan = W.AxisPlan(n, inner, DT[dtype], direction, batch)
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    assert plan.passes()[0] == 1
    plan.close()
    if dtype == "c32":
        scale = 1.0 / n if direction == W.INVERSE else 1.0
    else:
        scale = 1.0 / np.sqrt(n)
    ref = oracle.fft_axis(xc, axis=0, rank=2, sign=direction, scale=scale)
    err = oracle.rel_l2(to_host_c128(y, dtype), ref)
    assert err < TOL[dtype], err


@pytest.mark.parametrize("dtype", ["c32", "c16f"])
@pytest.mark.parametrize("a,b,c", [(4, 2, 65536), (2, 4, 512), (3, 5, 7), (1, 8, 1), (16, 16, 3), (64, 8, 1024),
                                   (1, 2, (1 << 27) + 6)])
def test_transpose_outer_bit_exact(dtype, a, b, c):
    xs = inputs.complex_input((a, b, c), 41, "normal", dtype)
    x = to_device(xs, dtype)
    y = torch.empty_like(x)
    W.transpose_outer(x.data_ptr(), y.data_ptr(), a, b, c, DT[dtype])
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    want = np.ascontiguousarray(np.asarray(xs).reshape((a, b, c) + xs.shape[3:]).swapaxes(0, 1))
    assert np.array_equal(got.reshape(-1).view(np.uint8), want.reshape(-1).view(np.uint8))


def test_transpose_outer_rejects_overlap():
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert W.lib().wsfft_transpose_outer(x.data_ptr(), x.data_ptr(), 4, 4, 4, W.C32, None) == W.ERR_INVALID_ARG
    assert W.lib().wsfft_transpose_outer(x.data_ptr(), x.data_ptr() + 8, 4, 4, 3, W.C32, None) == W.ERR_INVALID_ARG


def _emulate(dims, world, dtype, seed):
    """Every rank's local steps on this GPU, the exchange done in-process."""
    dist = "normal" if dtype == "c32" else "uniform"
    xs = inputs.complex_input(dims, seed, dist, dtype)
    xc = inputs.storage_to_c128(xs, dtype)
    x = to_device(xs, dtype)
    n0l, n1l = dims[0] // world, dims[1] // world
    ranks = [SlabFFT3(dims, DT[dtype], world=world, rank=r) for r in range(world)]
    blk = n0l * n1l * dims[2] * (1 if dtype == "c32" else 2)

    def exchange(sends):
        outs = []
        for r, f in enumerate(ranks):
            recv = torch.cat([sends[s].reshape(-1)[r * blk:(r + 1) * blk] for s in range(world)])
            outs.append(recv)
        return outs

    sends = [f.forward_pack(x[r * n0l:(r + 1) * n0l].contiguous()) for r, f in enumerate(ranks)]
    recvs = exchange(sends)
    ys = [f.forward_finish(rv) for f, rv in zip(ranks, recvs)]
    torch.cuda.synchronize()
    ys_host = [to_host_c128(y, dtype).reshape(dims[0], n1l, dims[2]) for y in ys]
    sends = [f.inverse_pack(y) for f, y in zip(ranks, ys)]
    recvs = exchange(sends)
    xr = [f.inverse_finish(rv) for f, rv in zip(ranks, recvs)]
    torch.cuda.synchronize()
    xr_host = [to_host_c128(v, dtype).reshape(n0l, dims[1], dims[2]) for v in xr]
    for f in ranks:
        f.close()
    return xc, ys_host, xr_host


@pytest.mark.parametrize("dims,world,dtype", [((64, 64, 64), 2, "c32"), ((128, 64, 32), 4, "c32"),
                                              ((256, 256, 256), 8, "c32"), ((512, 512, 512), 2, "c32"),
                                              ((128, 128, 128), 2, "c16f"), ((64, 128, 64), 4, "c16bf")])
def test_slab_distributed_emulated(dims, world, dtype):
    xc, ys, xr = _emulate(dims, world, dtype, 51)
    norm = oracle.NORM_PAPER if dtype == "c32" else oracle.NORM_ORTHO
    ref = oracle.fftn(xc, norm=norm)
    got = np.concatenate(ys, axis=1)  # y-slabs side by side = the whole spectrum
    err = oracle.rel_l2(got, ref)
    print(f"distributed {dims} over {world} {dtype}: rel_l2 {err:.2e}")
    assert err < TOL[dtype]
    back = np.concatenate(xr, axis=0)
    rt = oracle.rel_l2(back, xc)
    assert rt < (TOL[dtype] if dtype == "c32" else 3 * TOL[dtype])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_distributed_nccl_one_rank():
    import torch.distributed as dist
    dims = (128, 64, 64)
    xs = inputs.complex_input(dims, 61, "normal", "c32")
    x = torch.from_numpy(xs).cuda()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", world_size=1, rank=0)
    try:
        f = SlabFFT3(dims)
        y = f.forward(x)
        xr = f.inverse(y)
        torch.cuda.synchronize()
        f.close()
    finally:
        dist.destroy_process_group()
    ref = oracle.fftn(xs.astype(np.complex128))
    assert oracle.rel_l2(y.cpu().numpy(), ref) < TOL["c32"]
    assert oracle.rel_l2(xr.cpu().numpy(), xs) < TOL["c32"]
