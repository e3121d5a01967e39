"""GPU parity of the ragged batch: uneven 3D shapes in one persistent launch
(the ragged configuration: 256 shapes with axes drawn from {32, 64, 128, 256}
by seed 4), every instance against the FP64 oracle, in every storage type,
plus replay under a captured CUDA graph."""
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


def make_inputs(shapes, dtype, seed0):
    xs = [inputs.complex_input(tuple(s), seed0 + i, "normal", dtype) for i, s in enumerate(shapes)]
    return xs, [to_device(x, dtype) for x in xs]


@pytest.mark.parametrize("dtype", ["c32", "c16f", "c16bf"])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
def test_small_ragged_vs_oracle(dtype, direction):
    rng = np.random.default_rng(7)
    shapes = rng.choice([32, 64, 128], size=(12, 3))
    xs, xd = make_inputs(shapes, dtype, 100)
    outs = [torch.empty_like(x) for x in xd]
    plan = W.RaggedPlan(shapes, DT[dtype], direction)
    plan.execute([x.data_ptr() for x in xd], [y.data_ptr() for y in outs])
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    norm = oracle.NORM_PAPER if dtype == "c32" else oracle.NORM_ORTHO
    for x, y in zip(xs, outs):
        ref = oracle.fftn(inputs.storage_to_c128(x, dtype), sign=direction, norm=norm)
        assert oracle.rel_l2(to_host_c128(y, dtype), ref) < TOL[dtype]
    plan.close()


def test_ragged_in_place():
    shapes = np.array([[64, 32, 128], [32, 256, 32], [128, 64, 64]])
    xs, xd = make_inputs(shapes, "c32", 200)
    plan = W.RaggedPlan(shapes, W.C32, W.FORWARD)
    plan.execute([x.data_ptr() for x in xd], [x.data_ptr() for x in xd])
    torch.cuda.synchronize()
    for x, y in zip(xs, xd):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < TOL["c32"]
    plan.close()


def test_ragged_256_shapes_seed4():
    # the full ragged configuration; data generated on the device (seeded per
    # instance), every instance checked element by element against the FP64
    # oracle
    shapes = inputs.ragged_shapes(256, 4)
    g = torch.Generator(device="cuda")
    xd, outs = [], []
    for i, s in enumerate(shapes):
        g.manual_seed(1000 + i)
        xd.append(torch.view_as_complex(torch.randn(tuple(int(v) for v in s) + (2,), generator=g,
                                                    device="cuda")).contiguous())
        outs.append(torch.empty_like(xd[-1]))
    plan = W.RaggedPlan(shapes, W.C32, W.FORWARD)
    plan.execute([x.data_ptr() for x in xd], [y.data_ptr() for y in outs])
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    worst = 0.0
    for i, (x, y) in enumerate(zip(xd, outs)):
        ref = oracle.fftn(x.cpu().numpy().astype(np.complex128))
        err = oracle.rel_l2(y.cpu().numpy(), ref)
        worst = max(worst, err)
        assert err < TOL["c32"], (i, shapes[i], err)
    print(f"ragged 256 vs oracle: worst rel_l2 {worst:.2e}")


@pytest.mark.parametrize("dtype", ["c16f", "c16bf"])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
def test_ragged_half_storage_256_axes(dtype, direction):
    # 16-bit storage with 256-point axes in every position (the longest
    # ragged axis), against the oracle under the orthonormal scaling
    shapes = np.array([[256, 32, 64], [32, 256, 128], [64, 128, 256], [256, 256, 32], [32, 64, 256]])
    xs, xd = make_inputs(shapes, dtype, 400)
    outs = [torch.empty_like(x) for x in xd]
    plan = W.RaggedPlan(shapes, DT[dtype], direction)
    plan.execute([x.data_ptr() for x in xd], [y.data_ptr() for y in outs])
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    for s, x, y in zip(shapes, xs, outs):
        ref = oracle.fftn(inputs.storage_to_c128(x, dtype), sign=direction, norm=oracle.NORM_ORTHO)
        err = oracle.rel_l2(to_host_c128(y, dtype), ref)
        print(f"ragged {dtype} {tuple(s)} dir {direction}: rel_l2 {err:.2e}")
        assert err < TOL[dtype]
    plan.close()


def test_ragged_under_cuda_graph():
    shapes = inputs.ragged_shapes(16, 4)
    xs, xd = make_inputs(shapes, "c32", 300)
    outs = [torch.empty_like(x) for x in xd]
    plan = W.RaggedPlan(shapes, W.C32, W.FORWARD)
    ins, ous = [x.data_ptr() for x in xd], [y.data_ptr() for y in outs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.execute(ins, ous, s)  # first call uploads the pointer table
    torch.cuda.synchronize()
    for y in outs:
        y.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.execute(ins, ous, torch.cuda.current_stream())
    for _ in range(2):
        for y in outs:
            y.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for x, y in zip(xs, outs):
            assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < TOL["c32"]
    assert plan.sync_status() == W.SUCCESS
    plan.close()


def _run_variant(shapes, xs, xd, dtype, direction, sel, lag):
    outs = [torch.empty_like(x) for x in xd]
    plan = W.RaggedPlan(shapes, DT[dtype], direction)
    plan.set_variant(sel, lag)
    plan.execute([x.data_ptr() for x in xd], [y.data_ptr() for y in outs])
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    norm = oracle.NORM_PAPER if dtype == "c32" else oracle.NORM_ORTHO
    worst = 0.0
    for x, y in zip(xs, outs):
        ref = oracle.fftn(inputs.storage_to_c128(x, dtype), sign=direction, norm=norm)
        worst = max(worst, oracle.rel_l2(to_host_c128(y, dtype), ref))
    return worst


def test_ragged_every_tile_shape_selection():
    # all 16 selections of the second tile shape per axis length, on shapes
    # that use every length 32..256 on every axis
    shapes = np.array([[32, 64, 128], [256, 32, 64], [128, 256, 32], [64, 128, 256], [32, 32, 256],
                       [256, 64, 32]])
    xs, xd = make_inputs(shapes, "c32", 500)
    for sel in range(16):
        err = _run_variant(shapes, xs, xd, "c32", W.FORWARD if sel % 2 else W.INVERSE, sel, 1)
        assert err < TOL["c32"], (sel, err)


@pytest.mark.parametrize("dtype,sel,lag", [("c32", 15, 2), ("c32", 5, 4), ("c32", 0, 7), ("c16f", 15, 3),
                                           ("c16bf", 10, 2)])
def test_ragged_queue_lag(dtype, sel, lag):
    shapes = inputs.ragged_shapes(20, 9)
    xs, xd = make_inputs(shapes, dtype, 600)
    err = _run_variant(shapes, xs, xd, dtype, W.FORWARD, sel, lag)
    assert err < TOL[dtype], err


def test_ragged_variant_rejections():
    plan = W.RaggedPlan(np.array([[32, 32, 32]]), W.C32, W.FORWARD)
    with pytest.raises(RuntimeError):
        plan.set_variant(16, 1)
    with pytest.raises(RuntimeError):
        plan.set_variant(0, 0)
    plan.close()
    p = W.Plan((32, 32, 32), W.C32, W.FORWARD, 1)
    assert W.lib().wsfft_plan_set_ragged_variant(p.handle, 0, 1) == W.ERR_UNSUPPORTED
    p.close()
