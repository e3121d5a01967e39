"""Seeded random plans against the FP64 oracle.

The hand-written parity tests pick their shapes per kernel and per schedule;
this file draws whole plans at random from one seed so that combinations of
the plan builder's branches are checked together: rank 1-3, power-of-two axes
(1D up to 2^20, through the four-step), batch, storage type, direction, every
normalisation, the natural / swapped / wafer spectral layouts, the fused
schedules of n0 x n x n cubes, in place or out of place, device or pinned host
buffers.  Every result is compared element by element (relative L2 over the
whole output) with the oracle's DFT (Section 2, Eq. 1, over each axis) of the
same storage-rounded input.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build, inputs
from paper_2209_15040_gb300 import wsfft as W
from tests._helpers import DT, TOL, to_device, to_host_c128

pytestmark = pytest.mark.gpu

SEED = 2209
CASES = 64
MAX_ELEMS = 1 << 21  # per case (batch included): the oracle finishes each in well under a second


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()
    torch.cuda.init()


def _pow2(rng, lo, hi):
    return 1 << int(rng.integers(lo, hi + 1))


def draw(i):
    """Case i of the sequence: a dict describing one plan and its call."""
    rng = np.random.default_rng([SEED, i])
    rank = int(rng.choice([1, 2, 3], p=[0.3, 0.3, 0.4]))
    if rank == 1:
        dims = (_pow2(rng, 0, 20),)
    elif rank == 2:
        dims = (_pow2(rng, 0, 12), _pow2(rng, 0, 12))
    elif rng.random() < 0.5:
        m = _pow2(rng, 7, 9)  # n0 x n x n with n in {128, 256, 512}: the fused schedules apply
        dims = (_pow2(rng, 0, 9), m, m)
    else:
        dims = tuple(_pow2(rng, 0, 9) for _ in range(3))
    while int(np.prod(dims)) > MAX_ELEMS:
        dims = (dims[0] // 2,) + dims[1:] if dims[0] > 1 else dims[:-1] + (dims[-1] // 2,)
    n = int(np.prod(dims))
    batch = int(rng.integers(1, 6))
    while batch > 1 and batch * n > MAX_ELEMS:
        batch -= 1
    dtype = str(rng.choice(["c32", "c16f", "c16bf"], p=[0.5, 0.25, 0.25]))
    direction = int(rng.choice([W.FORWARD, W.INVERSE]))
    norms = [W.NORM_PAPER, W.NORM_NONE, W.NORM_ORTHO, W.NORM_FORWARD]
    if dtype != "c32" and n > 4096:
        norms = [W.NORM_ORTHO]  # unscaled 16-bit spectra of long transforms can leave FP16's range
    norm = int(rng.choice(norms))
    layouts = [W.LAYOUT_NATURAL]
    if rank >= 2 and all(64 <= d <= 4096 for d in dims[-2:]):
        layouts.append(W.LAYOUT_SWAPPED)
    if rank == 3 and all(64 <= d <= 4096 for d in dims):
        layouts.append(W.LAYOUT_WAFER)
    layout = int(rng.choice(layouts))
    engine = None
    if layout == W.LAYOUT_NATURAL and rank == 3 and dims[1] == dims[2] and dims[1] in (128, 256, 512):
        engine = int(rng.integers(0, 5))
    inplace = bool(rng.integers(0, 2))
    host = bool(rng.random() < 0.15) and not inplace
    return dict(dims=dims, batch=batch, dtype=dtype, direction=direction, norm=norm, layout=layout,
                engine=engine, inplace=inplace, host=host, seed=1000 + i)


def _scale(n, direction, norm):
    """Factor on the unnormalised DFT (Section 2's sums) for one normalisation."""
    if norm == W.NORM_NONE:
        return 1.0
    if norm == W.NORM_ORTHO:
        return 1.0 / np.sqrt(n)
    if norm == W.NORM_PAPER:
        return 1.0 / n if direction == W.INVERSE else 1.0
    return 1.0 / n if direction == W.FORWARD else 1.0  # NORM_FORWARD


def _logical(a, rank, layout):
    """The array a layout stores, as the natural [..., n0, n1, n2] it represents."""
    if layout == W.LAYOUT_SWAPPED:
        return np.swapaxes(a, -1, -2)
    if layout == W.LAYOUT_WAFER:  # stored [k2][k0][k1]
        return np.moveaxis(a, -3, -1)
    return a


def _stored_shape(dims, layout):
    if layout == W.LAYOUT_SWAPPED:
        return tuple(dims[:-2]) + (dims[-1], dims[-2])
    if layout == W.LAYOUT_WAFER:
        return (dims[2], dims[0], dims[1])
    return tuple(dims)


def expected(xc, c):
    """Oracle result for the call described by c, in the layout the plan writes."""
    dims, rank = c["dims"], len(c["dims"])
    n = int(np.prod(dims))
    sign = -1 if c["direction"] == W.FORWARD else +1
    if c["direction"] == W.FORWARD:
        spec = oracle.fftn(xc.reshape((c["batch"],) + dims), rank=rank, sign=sign, norm=oracle.NORM_NONE)
        spec = spec * _scale(n, c["direction"], c["norm"])
        out = spec  # natural -> stored
        if c["layout"] == W.LAYOUT_SWAPPED:
            out = np.swapaxes(spec, -1, -2)
        elif c["layout"] == W.LAYOUT_WAFER:
            out = np.moveaxis(spec, -1, -3)
        return out.reshape(-1)
    # inverse: the input is a spectrum stored in the layout
    stored = xc.reshape((c["batch"],) + _stored_shape(dims, c["layout"]))
    spec = np.ascontiguousarray(_logical(stored, rank, c["layout"]))
    back = oracle.fftn(spec, rank=rank, sign=sign, norm=oracle.NORM_NONE)
    return (back * _scale(n, c["direction"], c["norm"])).reshape(-1)


def _host_tensor(xs, dtype):
    if dtype == "c32":
        t = torch.from_numpy(np.ascontiguousarray(xs))
    elif dtype == "c16f":
        t = torch.from_numpy(np.ascontiguousarray(xs))
    else:
        t = torch.from_numpy(np.ascontiguousarray(xs).view(np.int16)).view(torch.bfloat16)
    return t.pin_memory()


def run_case(c):
    dims, rank = c["dims"], len(c["dims"])
    shape = (c["batch"],) + dims
    dist = "normal" if c["dtype"] == "c32" else "uniform"
    xs = inputs.complex_input(shape, c["seed"], dist, c["dtype"])
    xc = inputs.storage_to_c128(xs, c["dtype"]).reshape(-1)
    plan = W.Plan(dims, DT[c["dtype"]], c["direction"], c["batch"], c["norm"])
    try:
        if c["layout"] != W.LAYOUT_NATURAL:
            plan.set_layout(c["layout"])
        if c["engine"] is not None:
            plan.set_engine(c["engine"])
        if c["host"]:
            hx = _host_tensor(xs, c["dtype"])
            hy = torch.empty_like(hx).pin_memory()
            plan.execute_host(hx.data_ptr(), hy.data_ptr())
            assert plan.sync_status() == W.SUCCESS
            got = to_host_c128(hy, c["dtype"]).reshape(-1)
        else:
            x = to_device(xs, c["dtype"])
            out = x if c["inplace"] else torch.empty_like(x)
            plan.execute(x.data_ptr(), out.data_ptr())
            torch.cuda.synchronize()
            assert plan.sync_status() == W.SUCCESS
            got = to_host_c128(out, c["dtype"]).reshape(-1)
    finally:
        plan.close()
    ref = expected(xc, c)
    return oracle.rel_l2(got, ref), oracle.max_abs(got, ref)


def test_draws_cover_the_branches():
    # the sequence reaches every storage type, direction, normalisation and
    # layout, the four-step, a fused schedule, in-place and host calls
    cs = [draw(i) for i in range(CASES)]
    assert {c["dtype"] for c in cs} == {"c32", "c16f", "c16bf"}
    assert {c["direction"] for c in cs} == {W.FORWARD, W.INVERSE}
    assert {c["norm"] for c in cs} == {W.NORM_PAPER, W.NORM_NONE, W.NORM_ORTHO, W.NORM_FORWARD}
    assert {c["layout"] for c in cs} == {W.LAYOUT_NATURAL, W.LAYOUT_SWAPPED, W.LAYOUT_WAFER}
    assert any(len(c["dims"]) == 1 and c["dims"][0] > 4096 for c in cs)
    assert {c["engine"] for c in cs} >= {1, 2, 3, 4}
    assert any(c["inplace"] for c in cs) and any(c["host"] for c in cs)


@pytest.mark.parametrize("i", range(CASES))
def test_random_plan(i):
    c = draw(i)
    err, mx = run_case(c)
    print(f"case {i}: {c}: rel_l2 {err:.2e} max_abs {mx:.2e}")
    assert err < TOL[c["dtype"]], (c, err)
