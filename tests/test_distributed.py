"""CPU tests of the slab-distributed transform (paper_2209_15040_gb300.
distributed): the partitioning into x-slabs, the regrouping by destination,
the all-to-all and the spectral y-slab layout, against the FP64 oracle of
the whole array.  World size 2 runs as two gloo ranks; larger worlds are
emulated in one process with a loopback exchange.  The local steps use
numpy's FFT on CPU tensors (tests/_dist_local.py); the GPU kernels of the
same steps are tested in test_gpu_distributed.py."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import inputs
from paper_2209_15040_gb300.distributed import SlabFFT3
from tests._dist_local import NumpyLocal

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _global(dims, seed):
    return inputs.complex_input(dims, seed, "normal", "c32").astype(np.complex128)


def _make(dims, world, rank):
    return SlabFFT3(dims, world=world, rank=rank, local_forward=NumpyLocal(-1), local_inverse=NumpyLocal(+1))


@pytest.mark.parametrize("dims,world", [((8, 8, 4), 1), ((16, 8, 32), 2), ((16, 16, 8), 4), ((32, 8, 16), 8)])
def test_loopback_worlds(dims, world):
    # every rank's pack, an in-process all-to-all, every rank's finish
    x = _global(dims, 3)
    ref = oracle.fftn(x)
    n0l, n1l = dims[0] // world, dims[1] // world
    ranks = [_make(dims, world, r) for r in range(world)]
    sends = [f.forward_pack(torch.from_numpy(np.ascontiguousarray(x[r * n0l:(r + 1) * n0l]))) for r, f in
             enumerate(ranks)]
    blk = n0l * n1l * dims[2]
    ys = []
    for r, f in enumerate(ranks):
        recv = torch.cat([sends[s].reshape(-1)[r * blk:(r + 1) * blk] for s in range(world)])
        ys.append(f.forward_finish(recv.reshape(f.spectral_shape())))
    for r, y in enumerate(ys):
        assert oracle.rel_l2(y.numpy(), ref[:, r * n1l:(r + 1) * n1l, :]) < 1e-12
    # inverse back to x-slabs
    sends = [f.inverse_pack(y) for f, y in zip(ranks, ys)]
    blk = n0l * n1l * dims[2]
    for r, f in enumerate(ranks):
        recv = torch.cat([sends[s].reshape(-1)[r * blk:(r + 1) * blk] for s in range(world)])
        xr = f.inverse_finish(recv.reshape(f.slab_shape()))
        assert oracle.rel_l2(xr.numpy(), x[r * n0l:(r + 1) * n0l]) < 1e-12


def test_rejects_axes_not_divisible():
    with pytest.raises(ValueError):
        _make((12, 8, 8), 8, 0)
    with pytest.raises(ValueError):
        _make((8, 4, 8), 8, 0)


_WORKER = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
import oracle
from paper_2209_15040_gb300 import inputs
from paper_2209_15040_gb300.distributed import SlabFFT3
from tests._dist_local import NumpyLocal
dist.init_process_group("gloo")
r, G = dist.get_rank(), dist.get_world_size()
dims = {dims!r}
x = inputs.complex_input(dims, 5, "normal", "c32").astype(np.complex128)
ref = oracle.fftn(x)
n0l, n1l = dims[0] // G, dims[1] // G
f = SlabFFT3(dims, local_forward=NumpyLocal(-1), local_inverse=NumpyLocal(+1))
y = f.forward(torch.from_numpy(np.ascontiguousarray(x[r * n0l:(r + 1) * n0l])))
e1 = oracle.rel_l2(y.numpy(), ref[:, r * n1l:(r + 1) * n1l, :])
xr = f.inverse(y)
e2 = oracle.rel_l2(xr.numpy(), x[r * n0l:(r + 1) * n0l])
assert e1 < 1e-12 and e2 < 1e-12, (e1, e2)
dist.destroy_process_group()
print("rank", r, "ok", e1, e2, flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("dims", [(16, 8, 32), (8, 16, 4)])
def test_gloo_world_size_2(dims):
    port = _free_port()
    code = _WORKER.format(root=ROOT, dims=dims)
    procs = []
    for r in range(2):
        env = dict(os.environ)
        env.update({"WORLD_SIZE": "2", "RANK": str(r), "LOCAL_RANK": str(r), "MASTER_ADDR": "127.0.0.1",
                    "MASTER_PORT": str(port), "CUDA_VISIBLE_DEVICES": ""})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=180)[0] for p in procs]
    for r, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"rank {r} ok" in out
