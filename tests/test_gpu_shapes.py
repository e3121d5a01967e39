"""GPU parity of every kernel shape the library instantiates besides the
defaults: each (values per thread, pencils per block) shape of the
contiguous-axis and strided-axis superstep kernels, including the
pencil-pair, split-form pencil-pair and the 32-values-per-thread (radix-32)
shapes, selected with
wsfft_plan_set_pass_variant and compared with the FP64 oracle, for every
storage type, on full tiles and on ragged tails (pencil counts that are not a
multiple of the tile)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_15040_gb300 import build
from paper_2209_15040_gb300 import wsfft as W
from tests._helpers import DT, TOL, seeded, to_device, to_host_c128

pytestmark = pytest.mark.gpu

PAIR = 1000  # tile codes from PAIR_TILE on select the pencil-pair kernel
TC = 2000    # tile code of the tensor-core contiguous superstep (16-bit storage, 512)
SPLIT = 3000  # tile codes from SPLIT_TILE on select the split-form (packed FP32x2) pair kernel

# (values per thread, tile) shapes per axis length
CONTIG = {512: [(32, 16), (32, 8), (32, 32), (16, 8), (8, 8)], 256: [(8, 8)], 1024: [(32, 8)]}
STRIDED = {512: [(32, 16), (32, 8), (32, 32), (16, 16), (8, 8), (16, 8), (16, 32)],
           256: [(16, 32), (8, 16)], 1024: [(16, 8), (32, 8), (32, 16)]}
PAIRS = {512: [(8, PAIR + 16), (8, PAIR + 32), (8, PAIR + 8), (16, PAIR + 16), (16, PAIR + 32)],
         256: [(8, PAIR + 16)]}
SPLITS = {512: [(16, SPLIT + 16), (16, SPLIT + 32), (8, SPLIT + 16), (8, SPLIT + 32)]}
CONTIG_SPLITS = {512: [(16, SPLIT + 16), (16, SPLIT + 8), (8, SPLIT + 8)]}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    W.lib()
    torch.cuda.init()


_cache = {}


def _case(shape_full, rank, dtype, seed, direction=W.FORWARD):
    key = (shape_full, rank, dtype, seed, direction)
    if key not in _cache:
        xs, xc = seeded(shape_full, seed, "uniform", dtype)
        norm = W.NORM_PAPER if dtype == "c32" else W.NORM_ORTHO
        _cache[key] = (to_device(xs, dtype), oracle.fftn(xc, rank=rank, sign=direction, norm=norm),
                       norm)
    return _cache[key]


def run_variant(shape_full, rank, dtype, settings, seed=5, direction=W.FORWARD, inplace=False):
    x, ref, norm = _case(shape_full, rank, dtype, seed, direction)
    dims = shape_full[len(shape_full) - rank:]
    batch = int(np.prod(shape_full[:len(shape_full) - rank], dtype=np.int64))
    plan = W.Plan(dims, DT[dtype], direction, batch, norm)
    for pass_index, e, tile in settings:
        plan.set_pass_variant(pass_index, e, tile)
    out = x.clone() if inplace else torch.empty_like(x)
    plan.execute(out.data_ptr() if inplace else x.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert plan.sync_status() == W.SUCCESS
    plan.close()
    y = to_host_c128(out, dtype)
    err = oracle.rel_l2(y, ref)
    print(f"{shape_full} {dtype} {settings}: rel_l2={err:.3e} max_abs={oracle.max_abs(y, ref):.3e}")
    assert err < TOL[dtype], err


DTYPES = ["c32", "c16f", "c16bf"]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", CONTIG[512] + CONTIG_SPLITS[512])
def test_contig_512(dtype, shape):
    # pass 0 is the contiguous superstep of length 512 (8*512 = 4096 pencils)
    run_variant((64, 8, 512), 3, dtype, [(0, *shape)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", CONTIG[512] + CONTIG_SPLITS[512])
def test_contig_512_ragged(dtype, shape):
    # 37 pencils: the last tile of every shape is partial (and, for the
    # split-form pairs, the last pair has one pencil)
    run_variant((37, 512), 1, dtype, [(0, *shape)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", STRIDED[512] + PAIRS[512] + SPLITS[512])
def test_strided_512(dtype, shape):
    # pass 2 is the superstep along the outer axis (512, stride 8*64 elements)
    # and pass 1 the one along the middle axis (8)
    run_variant((512, 8, 64), 3, dtype, [(2, *shape)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", STRIDED[512])
def test_strided_512_ragged(dtype, shape):
    # batch 3 of 512 x 2: 6 strided pencils of 512, stride 2, in one partial tile
    run_variant((3, 512, 2), 2, dtype, [(1, *shape)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SPLITS[512])
def test_split_pairs_512_inverse_in_place(dtype, shape):
    # the inverse conjugates on load and scales on store (packed multiplies
    # in the split form); both strided supersteps of a 3D transform (strides
    # 32 and 512*32 elements), in place
    run_variant((512, 512, 32), 3, dtype, [(1, *shape), (2, *shape)], direction=W.INVERSE, inplace=True)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", CONTIG_SPLITS[512])
def test_contig_split_512_inverse_in_place(dtype, shape):
    # conjugate on load and scale on store in the split form, 2D 16 x 512
    run_variant((3, 16, 512), 2, dtype, [(0, *shape)], direction=W.INVERSE, inplace=True)


@pytest.mark.parametrize("dtype", DTYPES)
def test_pair_rejects_ragged(dtype):
    # the pencil-pair kernel wants whole tiles: the plan accepts the shape
    # (it exists) but the execute reports an error instead of running
    x, _, norm = _case((3, 512, 2), 2, dtype, 5)
    plan = W.Plan((512, 2), DT[dtype], W.FORWARD, 3, norm)
    plan.set_pass_variant(1, 8, PAIR + 16)
    out = torch.empty_like(x)
    with pytest.raises(RuntimeError):
        plan.execute(x.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_256_shapes(dtype):
    for sh in CONTIG[256]:
        run_variant((16, 8, 256), 3, dtype, [(0, *sh)])
    for sh in STRIDED[256] + PAIRS[256]:
        run_variant((256, 4, 32), 3, dtype, [(2, *sh)])


@pytest.mark.parametrize("dtype", DTYPES)
def test_1024_split_pairs(dtype):
    # split-form pencil pairs at 1024 points, 8 pencils per block: the default
    # strided shape below strides of 2^17 elements, selected explicitly and
    # reached by default plans (inner 64, 256, 1024), both directions
    run_variant((1024, 4, 16), 3, dtype, [(2, 16, SPLIT + 8)])
    run_variant((2, 1024, 64), 3, dtype, [(1, 16, SPLIT + 8)], direction=W.INVERSE)
    for shape, rank in (((2, 1024, 64), 3), ((1024, 256), 2), ((64, 1024, 1024), 3)):
        run_variant(shape, rank, dtype, [])
        run_variant(shape, rank, dtype, [], direction=W.INVERSE)


@pytest.mark.parametrize("dtype", ["c32", "c16f", "c16bf"])
def test_1024_shapes(dtype):
    for sh in CONTIG[1024]:
        run_variant((4, 8, 1024), 3, dtype, [(0, *sh)])
        run_variant((5, 1024), 1, dtype, [(0, *sh)])  # ragged: 5 pencils
    for sh in STRIDED[1024]:
        run_variant((1024, 4, 16), 3, dtype, [(2, *sh)])
        run_variant((3, 1024, 2), 2, dtype, [(1, *sh)])  # ragged: 6 pencils


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,settings", [
    (1 << 21, [(0, 32, 8)]),               # 2048 x 1024: 1024-point strided superstep, 8 pencils per block
    (1 << 21, [(0, 32, 16)]),              # the same, 16 pencils per block
    (1 << 19, [(1, 32, 8)]),               # 1024 x 512: 1024-point contiguous superstep, transposed store
    (1 << 19, [(0, 32, 16), (1, 32, 8)]),  # and the 512-point strided one, 32 values per thread
    (1 << 20, [(0, 32, 16)]),              # complex64 2048 x 512, 16-bit storage 1024 x 1024
    (1 << 18, []),                         # 512 x 512: 512-point contiguous superstep, 32 values x 16 pencils
    (1 << 18, [(1, 8, 0)]),                # the same with the general 8 values x 16 pencils
])
def test_four_step_shapes(dtype, n, settings):
    # 1D four-step split n = n1 (contiguous) x n2 (strided): pass 0 strided
    # with the inter-step twiddle, pass 1 contiguous with the transposed store
    run_variant((2, n), 1, dtype, settings)
    run_variant((1, n), 1, dtype, settings, direction=W.INVERSE)



# -- tensor-core contiguous superstep (DFT-16 on tcgen05, DFT-32 in registers)

@pytest.mark.parametrize("dtype", ["c16f", "c16bf"])
@pytest.mark.parametrize("direction", [W.FORWARD, W.INVERSE])
@pytest.mark.parametrize("shape_full,rank", [((64, 8, 512), 3), ((37, 512), 1), ((3, 16, 512), 2),
                                             ((1, 512), 1)])
def test_tensor_core_contig_512(dtype, direction, shape_full, rank):
    # 37 and 3*16 = 48 pencils: partial last tiles (the TMA box reads zeros past the end)
    run_variant(shape_full, rank, dtype, [(0, 16, TC)], direction=direction)


@pytest.mark.parametrize("dtype", ["c16f", "c16bf"])
def test_tensor_core_contig_512_in_place(dtype):
    run_variant((16, 16, 512), 3, dtype, [(0, 16, TC)], direction=W.INVERSE, inplace=True)


def test_tensor_core_contig_rejects_complex64():
    plan = W.Plan((8, 512), W.C32, W.FORWARD, 1)
    with pytest.raises(RuntimeError):
        plan.set_pass_variant(0, 16, TC)
    plan.close()
