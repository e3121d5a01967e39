"""Local steps of the slab-distributed transform on CPU tensors, with
numpy's FFT (pocketfft, the paper's own validator) and numpy transposes:
a stand-in for the GPU kernels so that the partitioning and the exchange of
paper_2209_15040_gb300.distributed run under gloo without a GPU.  Test
infrastructure only."""
import numpy as np
import torch


class NumpyLocal:
    def __init__(self, direction: int):
        self.direction = direction

    def _fft(self, a, axes):
        # forward unscaled, inverse 1/n per axis: the paper's normalisation
        return np.fft.fftn(a, axes=axes) if self.direction < 0 else np.fft.ifftn(a, axes=axes)

    def slab_2d(self, x: torch.Tensor, out: torch.Tensor) -> None:
        a = x.numpy()
        out.copy_(torch.from_numpy(self._fft(a, axes=(1, 2)).astype(a.dtype)))

    def axis0(self, x: torch.Tensor, out: torch.Tensor) -> None:
        a = x.numpy()
        out.copy_(torch.from_numpy(self._fft(a, axes=(0,)).astype(a.dtype)))

    def regroup(self, x: torch.Tensor, out: torch.Tensor, a: int, b: int, c: int) -> None:
        v = x.reshape(a, b, c).numpy()
        out.copy_(torch.from_numpy(np.ascontiguousarray(v.transpose(1, 0, 2))).reshape(out.shape))
