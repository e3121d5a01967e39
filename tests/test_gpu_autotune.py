"""GPU checks of wsfft_autotune: it picks a schedule and kernel shapes by
timing them, the result stays a correct transform, and the choice is
remembered in the WSFFT_TUNE_CACHE file and reused by later plans."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build, inputs
from paper_2209_15040_gb300 import wsfft as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()


def test_autotune_cube_and_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("WSFFT_TUNE_CACHE", str(cache))
    n = 128
    xs = inputs.complex_input((n, n, n), 1, "normal", "c32")
    x = torch.from_numpy(xs).cuda()
    y = torch.empty_like(x)
    plan = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    plan.autotune()
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert entry["mode"] in (0, 1, 2, 3, 4) and entry["us"] > 0
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    ref = oracle.fftn(xs.astype(np.complex128))
    assert oracle.rel_l2(y.cpu().numpy(), ref) < 5e-6
    npass = plan.passes()[0]
    plan.close()
    # a new plan for the same key takes the remembered schedule without timing
    plan2 = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    assert plan2.passes()[0] == npass
    plan2.autotune()
    assert len(cache.read_text().strip().splitlines()) == 1
    y.zero_()
    plan2.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy(), ref) < 5e-6
    plan2.close()


@pytest.mark.parametrize("bad", [
    {"mode": 99, "variants": []},                      # no such schedule
    {"mode": 0, "variants": [[0, 0, 8]]},              # zero values per thread
    {"mode": 0, "variants": [[0, 16, 12345]]},         # a tile no kernel is instantiated for
    {"mode": 0, "variants": [[2, 64, 16]]},            # more values per thread than a pencil holds
    {"mode": 0, "variants": [[7, 16, 8]]},             # a pass the plan does not have
])
def test_cache_entries_that_do_not_hold_are_ignored(tmp_path, monkeypatch, bad):
    # the cache file is outside the library's control (stale from another
    # build, edited, corrupted): an entry that does not describe a launchable
    # schedule leaves the plan on its default schedule, which still computes
    # the transform
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("WSFFT_TUNE_CACHE", str(cache))
    n = 64
    plan = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    npass = plan.passes()[0]
    plan.autotune()
    plan.close()
    key = json.loads(cache.read_text().strip().splitlines()[0])["key"]
    entry = {"key": key, "mode": bad["mode"], "variants": bad["variants"], "us": 1.0}
    cache.write_text(json.dumps(entry) + "\n")
    xs = inputs.complex_input((n, n, n), 2, "normal", "c32")
    x = torch.from_numpy(xs).cuda()
    y = torch.empty_like(x)
    plan = W.Plan((n, n, n), W.C32, W.FORWARD, 1)
    assert plan.passes()[0] == npass
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(xs.astype(np.complex128))) < 5e-6
    plan.autotune()  # the bad entry is not taken: autotune times and appends a good one
    assert len(cache.read_text().strip().splitlines()) == 2
    plan.close()


def test_autotune_2d_without_cache(monkeypatch):
    monkeypatch.delenv("WSFFT_TUNE_CACHE", raising=False)
    xs = inputs.complex_input((2, 512, 256), 3, "normal", "c32")
    x = torch.from_numpy(xs).cuda()
    y = torch.empty_like(x)
    plan = W.Plan((512, 256), W.C32, W.INVERSE, 2)
    plan.autotune()
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    ref = oracle.fftn(xs.astype(np.complex128), rank=2, sign=+1)
    assert oracle.rel_l2(y.cpu().numpy(), ref) < 5e-6
    plan.close()


@pytest.mark.parametrize("dtype,code", [("c16f", W.C16F), ("c16bf", W.C16BF)])
def test_autotune_half_storage_512(monkeypatch, dtype, code):
    # the 16-bit candidates include the tensor-core contiguous superstep; the
    # tuned plan must stay within the storage type's error bar either way
    monkeypatch.delenv("WSFFT_TUNE_CACHE", raising=False)
    shape = (8, 64, 512)
    xs = inputs.complex_input(shape, 5, "uniform", dtype)
    xc = inputs.storage_to_c128(xs, dtype)
    if dtype == "c16f":
        x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    else:
        x = torch.from_numpy(np.ascontiguousarray(xs).view(np.int16)).view(torch.bfloat16).cuda()
    y = torch.empty_like(x)
    plan = W.Plan(shape, code, W.FORWARD, 1, W.NORM_ORTHO)
    plan.autotune()
    plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    got = y.cpu()
    got = inputs.storage_to_c128(got.numpy() if dtype == "c16f" else got.view(torch.int16).numpy().view(np.uint16),
                                 dtype)
    ref = oracle.fftn(xc, rank=3, norm=W.NORM_ORTHO)
    tol = 3e-3 if dtype == "c16f" else 2e-2
    assert oracle.rel_l2(got, ref) < tol
    plan.close()


def test_autotune_ragged_caches_a_choice(tmp_path, monkeypatch):
    # the ragged plan's tile shapes per axis length and its queue lag are
    # timed, the choice is cached under the shape multiset, the tuned plan
    # matches the oracle, and a plan created later for the same shapes (in
    # another order) finds the cached entry instead of timing again
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("WSFFT_TUNE_CACHE", str(cache))
    shapes = inputs.ragged_shapes(24, 4)
    xs = [inputs.complex_input(tuple(int(v) for v in s), 700 + i, "normal", "c32") for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty_like(x) for x in xd]
    plan = W.RaggedPlan(shapes, W.C32, W.FORWARD)
    plan.autotune()
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert "ragged24" in entry["key"] and entry["us"] > 0
    assert 1 <= entry["mode"] <= 4 and entry["variants"][0][0] == -1 and 0 <= entry["variants"][0][1] <= 15
    plan.execute([x.data_ptr() for x in xd], [y.data_ptr() for y in outs])
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    for x, y in zip(xs, outs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < 5e-6
    plan2 = W.RaggedPlan(shapes[::-1], W.C32, W.FORWARD)
    plan2.autotune()
    assert len(cache.read_text().strip().splitlines()) == 1
    for y in outs:
        y.zero_()
    plan2.execute([x.data_ptr() for x in xd[::-1]], [y.data_ptr() for y in outs[::-1]])
    torch.cuda.synchronize()
    plan2.close()
    for x, y in zip(xs, outs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < 5e-6
