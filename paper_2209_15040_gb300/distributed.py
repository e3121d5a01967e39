"""Slab-distributed 3D transform over several GPUs, one process per GPU.

The paper spreads the array over its processors (Section 2.1, data
distribution: one pencil per processor, or slabs when there are fewer
processors than pencils), runs each superstep on the local data and
redistributes the array between supersteps so that the next axis becomes
local (Section 4.3); Section 8 proposes the same structure over several
systems for larger problems.  With G GPUs and an n0 x n1 x n2 array:

  forward (rank r holds x-slab r: rows r*n0/G .. (r+1)*n0/G of axis 0)
    1. z and y supersteps of the local rows: a rank-2 plan (n1, n2) with
       batch n0/G;
    2. regroup by destination, [n0/G][G][n1/G * n2] -> [G][n0/G][n1/G * n2]
       (wsfft_transpose_outer), so the block for rank d is contiguous;
    3. one all-to-all (the only exchange): rank r receives from each rank s
       rows s*n0/G.. of y-range r, i.e. [G][n0/G][n1/G][n2] = [n0][n1/G][n2],
       its y-slab in natural order;
    4. x superstep of the y-slab: an axis plan of length n0 with stride
       n1/G * n2.
  The spectrum stays distributed by y-slabs: rank r holds X[:, r*n1/G ..
  (r+1)*n1/G, :] as [n0][n1/G][n2] (the distributed output of Section 4.2,
  where the spectrum also ends redistributed).  The inverse runs the same
  steps backwards and returns x-slabs.

Every step on the data runs in the library's kernels (the superstep plans
and the transpose); torch.distributed's all_to_all_single moves the blocks
between GPUs (NCCL on GPUs).  The local steps are an object with three
methods, so the partitioning and the exchange can also run on CPU tensors
with another implementation of those steps (the gloo tests do that).
"""
from __future__ import annotations

import torch

from . import wsfft as W


def _elems(t: torch.Tensor) -> int:
    """Complex elements of a tensor in one of the library's storage forms."""
    return t.numel() if t.is_complex() else t.numel() // 2


def _view(t: torch.Tensor, shape) -> torch.Tensor:
    """The same contiguous storage viewed as `shape` complex elements
    (complex dtype) or `shape` x 2 (16-bit storage as re, im pairs)."""
    return t.view(tuple(shape)) if t.is_complex() else t.view(tuple(shape) + (2,))


class CudaLocal:
    """The local steps on one GPU with the library's kernels: the (y, z)
    supersteps of a batch of slabs, the x superstep of a y-slab, and the
    regrouping transpose."""

    def __init__(self, dims, world: int, dtype: int, direction: int, norm=None):
        n0, n1, n2 = dims
        self.dtype = dtype
        self.slabs = W.Plan((n1, n2), dtype, direction, n0 // world, norm)
        self.axis = W.AxisPlan(n0, (n1 // world) * n2, dtype, direction, 1, norm)

    def slab_2d(self, x: torch.Tensor, out: torch.Tensor) -> None:
        self.slabs.execute(x.data_ptr(), out.data_ptr())

    def axis0(self, x: torch.Tensor, out: torch.Tensor) -> None:
        self.axis.execute(x.data_ptr(), out.data_ptr())

    def regroup(self, x: torch.Tensor, out: torch.Tensor, a: int, b: int, c: int) -> None:
        W.transpose_outer(x.data_ptr(), out.data_ptr(), a, b, c, self.dtype)

    def close(self) -> None:
        self.slabs.close()
        self.axis.close()


class SlabFFT3:
    """n0 x n1 x n2 transform distributed by slabs of axis 0 over `world`
    ranks (n0 and n1 multiples of world).  forward() takes this rank's x-slab
    [n0/G][n1][n2] and returns its y-slab of the spectrum [n0][n1/G][n2];
    inverse() does the reverse.  The phases are public so that one process
    can also drive several ranks' local steps with its own exchange."""

    def __init__(self, dims, dtype: int = W.C32, group=None, world: int | None = None, rank: int | None = None,
                 norm=None, local_forward=None, local_inverse=None):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 3:
            raise ValueError("SlabFFT3 needs three axes")
        self.group = group
        if world is None or rank is None:
            import torch.distributed as dist
            world = dist.get_world_size(group) if world is None else world
            rank = dist.get_rank(group) if rank is None else rank
        self.world, self.rank, self.dtype = int(world), int(rank), int(dtype)
        n0, n1, n2 = self.dims
        if n0 % self.world or n1 % self.world:
            raise ValueError(f"axes 0 and 1 ({n0}, {n1}) must be multiples of the world size {self.world}")
        self.n0l, self.n1l = n0 // self.world, n1 // self.world
        self.fwd = local_forward or CudaLocal(self.dims, self.world, self.dtype, W.FORWARD, norm)
        self.inv = local_inverse or CudaLocal(self.dims, self.world, self.dtype, W.INVERSE, norm)

    def slab_shape(self):
        """Shape of this rank's x-slab (the spatial side)."""
        return (self.n0l, self.dims[1], self.dims[2])

    def spectral_shape(self):
        """Shape of this rank's y-slab (the spectral side)."""
        return (self.dims[0], self.n1l, self.dims[2])

    def _check(self, t: torch.Tensor, shape) -> None:
        want = shape[0] * shape[1] * shape[2]
        if not t.is_contiguous() or _elems(t) != want:
            raise ValueError(f"expected a contiguous tensor of {want} complex elements {shape}")

    # -- forward ---------------------------------------------------------------
    def forward_pack(self, x: torch.Tensor) -> torch.Tensor:
        """Steps 1-2: local z and y supersteps, then the regrouping by
        destination rank; returns the send buffer [G][n0/G][n1/G][n2]."""
        self._check(x, self.slab_shape())
        t = torch.empty_like(x)
        self.fwd.slab_2d(x, t)
        send = torch.empty_like(x)
        self.fwd.regroup(t, send, self.n0l, self.world, self.n1l * self.dims[2])
        return _view(send, self.spectral_shape())

    def forward_finish(self, recv: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Step 4 on the received y-slab [n0][n1/G][n2]: the x superstep."""
        self._check(recv, self.spectral_shape())
        recv = _view(recv, self.spectral_shape())
        out = recv if out is None else out
        self.fwd.axis0(recv, out)
        return out

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self.forward_finish(self.exchange(self.forward_pack(x)), out)

    # -- inverse ---------------------------------------------------------------
    def inverse_pack(self, y: torch.Tensor) -> torch.Tensor:
        """The x superstep of this rank's y-slab; its rows are already
        grouped by destination (x-slab d is rows d*n0/G ..)."""
        self._check(y, self.spectral_shape())
        send = torch.empty_like(y)
        self.inv.axis0(y, send)
        return _view(send, self.slab_shape())

    def inverse_finish(self, recv: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """After the exchange: regroup [G][n0/G][n1/G * n2] into row order
        [n0/G][G][n1/G * n2] = [n0/G][n1][n2], then the y and z supersteps."""
        self._check(recv, self.slab_shape())
        recv = _view(recv, self.slab_shape())
        u = torch.empty_like(recv)
        self.inv.regroup(recv, u, self.world, self.n0l, self.n1l * self.dims[2])
        out = u if out is None else out
        self.inv.slab_2d(u, out)
        return out

    def inverse(self, y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self.inverse_finish(self.exchange(self.inverse_pack(y)), out)

    # -- the exchange ----------------------------------------------------------
    def exchange(self, send: torch.Tensor) -> torch.Tensor:
        """Step 3: block d of `send` goes to rank d; block s of the result came
        from rank s (torch.distributed.all_to_all_single, equal blocks)."""
        import torch.distributed as dist
        if self.world == 1 and not (dist.is_available() and dist.is_initialized()):
            return send  # one rank without a process group: the exchange is the identity
        recv = torch.empty_like(send)
        dist.all_to_all_single(recv, send, group=self.group)
        return recv

    def close(self) -> None:
        for loc in (self.fwd, self.inv):
            c = getattr(loc, "close", None)
            if c:
                c()
