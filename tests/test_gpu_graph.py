"""Plans executed inside a captured CUDA graph.

wsfft_execute enqueues kernel launches (and, for the persistent schedules, a
counter reset) on the caller's stream and allocates nothing: tables and
workspaces are made when the schedule is built.  So a forward and an inverse
execute can be captured once and replayed on new data.  Each case captures
forward (x -> y) and inverse (y -> z) on a side stream after one warm
execute, replays the graph twice with fresh inputs copied into x, and checks
y against the FP64 oracle's DFT (in the plan's spectral layout) and z
against x (the round trip of Section 4.2's inverse).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build, inputs
from paper_2209_15040_gb300 import wsfft as W
from tests._helpers import DT, TOL, to_device, to_host_c128

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()
    torch.cuda.init()


def _stored(spec, layout):
    """Natural [..., n0, n1, n2] spectrum in the order a layout stores it."""
    if layout == W.LAYOUT_SWAPPED:
        return np.swapaxes(spec, -1, -2)
    if layout == W.LAYOUT_WAFER:
        return np.moveaxis(spec, -1, -3)
    return spec


CASES = [
    # dims, batch, dtype, layout, schedule
    ((64, 64, 64), 1, "c32", W.LAYOUT_NATURAL, None),  # one launch per superstep, PDL between them
    ((64, 64, 64), 2, "c16f", W.LAYOUT_NATURAL, None),
    ((2, 256, 256), 1, "c32", W.LAYOUT_NATURAL, 4),  # cluster-fused z and y
    ((2, 256, 256), 1, "c32", W.LAYOUT_NATURAL, 1),  # persistent: counter reset + launch
    ((2, 128, 256), 1, "c16bf", W.LAYOUT_SWAPPED, None),  # transposing store into the workspace
    ((64, 128, 256), 1, "c32", W.LAYOUT_WAFER, None),
    ((1 << 16,), 4, "c32", W.LAYOUT_NATURAL, None),  # four-step: workspace and inter-step twiddle
]


@pytest.mark.parametrize("dims,batch,dtype,layout,engine", CASES)
def test_forward_inverse_replayed(dims, batch, dtype, layout, engine):
    rank = len(dims)
    shape = (batch,) + dims
    dist = "normal" if dtype == "c32" else "uniform"
    plans = []
    for direction in (W.FORWARD, W.INVERSE):
        p = W.Plan(dims, DT[dtype], direction, batch)
        if layout != W.LAYOUT_NATURAL:
            p.set_layout(layout)
        if engine is not None:
            p.set_engine(engine)
            assert p.passes()[0] == 2  # the fused schedule, not the fallback
        plans.append(p)
    fwd, inv = plans
    xs0 = inputs.complex_input(shape, 70, dist, dtype)
    x = to_device(xs0, dtype)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fwd.execute(x.data_ptr(), y.data_ptr(), s)
        inv.execute(y.data_ptr(), z.data_ptr(), s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fwd.execute(x.data_ptr(), y.data_ptr())
        inv.execute(y.data_ptr(), z.data_ptr())
    norm = oracle.NORM_PAPER if dtype == "c32" else oracle.NORM_ORTHO
    for rep in range(2):
        xs = inputs.complex_input(shape, 71 + rep, dist, dtype)
        x.copy_(to_device(xs, dtype))
        y.zero_()
        z.zero_()
        graph.replay()
        torch.cuda.synchronize()
        xc = inputs.storage_to_c128(xs, dtype)
        ref = _stored(oracle.fftn(xc, rank=rank, norm=norm), layout)
        got = to_host_c128(y, dtype).reshape(ref.shape)
        err = oracle.rel_l2(got, ref)
        back = oracle.rel_l2(to_host_c128(z, dtype).reshape(xc.shape), xc)
        print(f"{dims} x{batch} {dtype} layout {layout} schedule {engine} replay {rep}: "
              f"rel_l2 {err:.2e}, round trip {back:.2e}")
        assert err < TOL[dtype]
        assert back < 2 * TOL[dtype]
    assert fwd.sync_status() == W.SUCCESS and inv.sync_status() == W.SUCCESS
    del graph
    for p in plans:
        p.close()
