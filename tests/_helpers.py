"""Shared helpers for the GPU parity tests: run the CUDA path through the C
ABI on seeded inputs and bring results back as complex128 for comparison
with the oracle."""
import numpy as np
import torch

from paper_2209_15040_gb300 import inputs
from paper_2209_15040_gb300 import wsfft as W

DT = {"c32": W.C32, "c16f": W.C16F, "c16bf": W.C16BF}
# relative-L2 bars vs the FP64 oracle, per storage type
TOL = {"c32": 5e-6, "c16f": 3e-3, "c16bf": 2e-2}


def to_device(x_storage: np.ndarray, dtype: str) -> torch.Tensor:
    if dtype == "c32":
        return torch.from_numpy(np.ascontiguousarray(x_storage)).cuda()
    if dtype == "c16f":
        return torch.from_numpy(np.ascontiguousarray(x_storage)).cuda()
    # bfloat16 bit patterns
    t = torch.from_numpy(np.ascontiguousarray(x_storage).view(np.int16))
    return t.view(torch.bfloat16).cuda()


def to_host_c128(t: torch.Tensor, dtype: str) -> np.ndarray:
    t = t.detach().cpu()
    if dtype == "c32":
        return t.numpy().astype(np.complex128)
    if dtype == "c16f":
        return inputs.storage_to_c128(t.numpy(), dtype)
    return inputs.storage_to_c128(t.view(torch.int16).numpy().view(np.uint16), dtype)


def run_plan(x_dev: torch.Tensor, dims, dtype: str, direction: int, batch: int, norm=None,
             inplace: bool = False) -> torch.Tensor:
    plan = W.Plan(dims, DT[dtype], direction, batch, norm)
    out = x_dev if inplace else torch.empty_like(x_dev)
    plan.execute(x_dev.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    return out


def seeded(shape, seed, dist, dtype):
    xs = inputs.complex_input(shape, seed, dist, dtype)
    return xs, inputs.storage_to_c128(xs, dtype)
