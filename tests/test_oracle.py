"""Pins of the FP64 oracle against things other than itself.

Every check here is CPU-only.  The oracle (``oracle/``) evaluates the DFT of
the paper's Section 1 as one radix-2 superstep per axis; it is pinned by

* hand-worked DFTs (tests/golden/closed_forms.txt),
* the brute-force O(N^2) definition on tiny inputs,
* numpy's pocketfft -- the validator the paper itself used (Section 4.1),
* closed forms (delta, shifted delta, single exponential, constant),
* invariants (Parseval, linearity, shift theorem, conjugate symmetry,
  forward/inverse round trips, adjoint identity),
* finite differences for the loss gradient,
* and mutation checks: planted mistakes in a wrapper of the oracle must trip
  at least one of the pins above.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2209_15040_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")
TOL = 1e-13


def _parse_pairs(s):
    vals = []
    for tok in s.split():
        re, im = tok.split(",")
        vals.append(complex(float(re), float(im)))
    return np.array(vals, dtype=np.complex128)


def _golden_cases():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, dims, xin, xout = [p.strip() for p in line.split("|")]
            shape = tuple(int(d) for d in dims.split(","))
            cases.append((name, shape, _parse_pairs(xin).reshape(shape),
                          _parse_pairs(xout).reshape(shape)))
    return cases


def rand_c(shape, seed=0):
    p = inputs.draw(shape, seed, "normal")
    return p[..., 0] + 1j * p[..., 1]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_golden_hand_worked(case):
    _, shape, x, y = case
    np.testing.assert_allclose(oracle.fftn(x), y, atol=1e-14)
    np.testing.assert_allclose(oracle.dft_brute(x), y, atol=1e-14)


def test_unit_root_quadrants():
    # exp(-2 pi i m / n) at the exact points of the unit circle and one octant point
    for n in (1, 2, 4, 8, 16, 4096, 1 << 20):
        assert abs(oracle.unit_root(0, n) - 1) < 1e-16
        if n % 4 == 0:
            assert abs(oracle.unit_root(n // 4, n) - (-1j)) < 1e-16
            assert abs(oracle.unit_root(n // 2, n) - (-1)) < 1e-16
            assert abs(oracle.unit_root(3 * n // 4, n) - 1j) < 1e-16
        if n % 8 == 0:
            h = np.sqrt(0.5)
            assert abs(oracle.unit_root(n // 8, n) - complex(h, -h)) < 2.5e-16
            assert abs(oracle.unit_root(3 * n // 8, n, sign=+1) - complex(-h, h)) < 2.5e-16
    # against 30-digit arithmetic: within a couple of ulp
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(2 ** rng.integers(1, 24))
        m = int(rng.integers(-3 * n, 3 * n))
        want = complex(mpmath.exp(-2j * mpmath.pi * mpmath.mpf(m % n) / n))
        assert abs(oracle.unit_root(m, n) - want) < 2.5e-16


@pytest.mark.parametrize("shape", [(8, 8, 8), (4, 4, 4), (2, 4, 8), (64, 64), (1, 16),
                                   (2,), (4,), (8,), (32,), (256,), (1024,), (4096,)])
def test_fft_matches_brute_force(shape):
    x = rand_c(shape, seed=1)
    for sign in (-1, +1):
        got = oracle.fftn(x, sign=sign, norm=oracle.NORM_NONE)
        ref = oracle.dft_brute(x, sign=sign)
        assert oracle.rel_l2(got, ref) < TOL


def test_brute_force_batch_matches_loop():
    x = rand_c((3, 4, 8), seed=2)
    b = oracle.dft_brute(x, rank=2)
    for i in range(3):
        assert oracle.rel_l2(b[i], oracle.dft_brute(x[i])) < 1e-15


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 64, 8), (128, 128), (1 << 14,),
                                   (2, 8, 16, 32)])
def test_fft_matches_numpy(shape):
    x = rand_c(shape, seed=3)
    assert oracle.rel_l2(oracle.fftn(x), np.fft.fftn(x)) < TOL
    assert oracle.rel_l2(oracle.ifftn(x), np.fft.ifftn(x)) < TOL
    assert oracle.rel_l2(oracle.fftn(x, norm=oracle.NORM_ORTHO),
                         np.fft.fftn(x, norm="ortho")) < TOL


def test_batched_rank_matches_numpy_axes():
    x = rand_c((5, 16, 32), seed=4)
    got = oracle.fftn(x, rank=2)
    ref = np.fft.fftn(x, axes=(1, 2))
    assert oracle.rel_l2(got, ref) < TOL


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_superstep_matches_numpy(axis):
    x = rand_c((8, 16, 32), seed=6)
    got = oracle.fft_axis(x, axis, sign=-1)
    assert oracle.rel_l2(got, np.fft.fft(x, axis=axis)) < TOL
    got = oracle.fft_axis(x, axis, sign=+1, scale=1.0 / x.shape[axis])
    assert oracle.rel_l2(got, np.fft.ifft(x, axis=axis)) < TOL


def test_supersteps_compose_to_fftn():
    x = rand_c((2, 8, 4, 16), seed=7)
    y = x
    for axis in (1, 0, 2):  # any order (Section 1)
        y = oracle.fft_axis(y, axis, rank=3)
    assert oracle.rel_l2(y, oracle.fftn(x, rank=3)) < TOL


@pytest.mark.parametrize("shape", [(16,), (8, 4), (4, 8, 16)])
def test_closed_forms(shape):
    N = int(np.prod(shape))
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    # delta at the origin -> all ones
    x = np.zeros(shape, complex)
    x[(0,) * len(shape)] = 1
    assert np.max(np.abs(oracle.fftn(x) - 1)) < 1e-15
    # delta at a -> exp(-2 pi i sum a_d k_d / n_d)
    a = tuple(n // 3 + 1 if n > 1 else 0 for n in shape)
    a = tuple(ai % n for ai, n in zip(a, shape))
    x = np.zeros(shape, complex)
    x[a] = 1
    phase = sum(ai * g / n for ai, g, n in zip(a, grids, shape))
    assert np.max(np.abs(oracle.fftn(x) - np.exp(-2j * np.pi * phase))) < 1e-14
    # single exponential exp(+2 pi i sum a_d j_d / n_d) -> N delta_{k,a}
    x = np.exp(2j * np.pi * phase)
    want = np.zeros(shape, complex)
    want[a] = N
    assert np.max(np.abs(oracle.fftn(x) - want)) < 1e-12 * N
    # constant -> N delta_{k,0}
    want = np.zeros(shape, complex)
    want[(0,) * len(shape)] = 3.5 * N
    assert np.max(np.abs(oracle.fftn(np.full(shape, 3.5 + 0j)) - want)) < 1e-12 * N


def test_parseval_linearity_shift_symmetry():
    shape = (16, 8, 32)
    N = int(np.prod(shape))
    x = rand_c(shape, 8)
    y = rand_c(shape, 9)
    X = oracle.fftn(x)
    # Parseval: sum |X|^2 = N sum |x|^2
    assert abs(np.sum(abs(X) ** 2) - N * np.sum(abs(x) ** 2)) < 1e-12 * N * np.sum(abs(x) ** 2)
    # linearity
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    assert oracle.rel_l2(oracle.fftn(a * x + b * y), a * X + b * oracle.fftn(y)) < TOL
    # shift theorem: x[j - s] -> X[k] exp(-2 pi i sum s_d k_d / n_d)
    s = (3, 5, 7)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ramp = np.exp(-2j * np.pi * sum(si * g / n for si, g, n in zip(s, grids, shape)))
    assert oracle.rel_l2(oracle.fftn(np.roll(x, s, axis=(0, 1, 2))), X * ramp) < TOL
    # real input -> conjugate-symmetric output X[k] = conj(X[-k])
    R = oracle.fftn(x.real)
    flip = np.roll(np.flip(R, axis=(0, 1, 2)), 1, axis=(0, 1, 2))
    assert oracle.rel_l2(R, np.conj(flip)) < TOL


def test_round_trips():
    shape = (4, 16, 32)
    N = int(np.prod(shape))
    x = rand_c(shape, 10)
    # paper normalisation: inverse of forward is the identity (Section 4.2)
    assert oracle.rel_l2(oracle.ifftn(oracle.fftn(x)), x) < TOL
    # unnormalised: forward then inverse is N times the identity
    y = oracle.fftn(oracle.fftn(x, norm=oracle.NORM_NONE), sign=+1, norm=oracle.NORM_NONE)
    assert oracle.rel_l2(y, N * x) < TOL
    # per-axis 1/sqrt(n) both ways: unitary
    y = oracle.fftn(x, norm=oracle.NORM_ORTHO)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert oracle.rel_l2(oracle.ifftn(y, norm=oracle.NORM_ORTHO), x) < TOL


def test_adjoint_identity():
    shape = (8, 16, 4)
    x = rand_c(shape, 11)
    y = rand_c(shape, 12)
    Fx = oracle.fftn(x, norm=oracle.NORM_NONE)
    FHy = oracle.fftn(y, sign=+1, norm=oracle.NORM_NONE)
    lhs = np.vdot(y, Fx)  # <F x, y> = y^H F x
    rhs = np.vdot(FHy, x)  # <x, F^H y>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_loss_grad_finite_differences():
    # 16^3 instance; FP64 central differences on 80 sampled coordinates (re
    # and im parts).  L is quadratic in x, so a central difference has no
    # truncation error at any h; h = 1e-3 keeps the rounding error
    # (~ eps * L / h ~ 6e-7 here) well under the tolerance.
    shape = (16, 16, 16)
    x = rand_c(shape, 13)
    w = inputs.loss_weights(shape, 14).astype(np.float64)
    g = oracle.loss_grad(x, w)
    rng = np.random.default_rng(15)
    idx = rng.integers(0, x.size, size=40)
    h = 1e-3
    xf = x.ravel()
    for i in idx:
        for part in (1.0, 1j):
            xp = xf.copy()
            xm = xf.copy()
            xp[i] += h * part
            xm[i] -= h * part
            fd = (oracle.loss(xp.reshape(shape), w) - oracle.loss(xm.reshape(shape), w)) / (2 * h)
            an = g.ravel()[i].real if part == 1.0 else g.ravel()[i].imag
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an)) + 1e-5, (i, part, fd, an)


def test_dft_points_matches_fft():
    x = rand_c((8, 16, 32), 16)
    X = oracle.fftn(x)
    k = np.array([0, 1, 17, 511, 2048, 4095])
    got = oracle.dft_points(x, k)
    assert np.max(np.abs(got - X.ravel()[k])) < 1e-11


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fftn(np.zeros((6,), complex))
    with pytest.raises(ValueError):
        oracle.fftn(np.zeros((4, 12), complex))


# ---------------------------------------------------------------------------
# Mutation checks: each planted mistake, applied to the oracle's output or to
# its call, must be caught by a pin above.  The mistakes live only here.


def _pins_pass(fft):
    """Brute force, numpy and the delta closed form, on small shapes."""
    ok = True
    for shape in [(8, 4, 16), (32,)]:
        x = rand_c(shape, 20)
        ok &= oracle.rel_l2(fft(x), oracle.dft_brute(x)) < TOL
        ok &= oracle.rel_l2(fft(x), np.fft.fftn(x)) < TOL
    return bool(ok)


def test_pins_catch_planted_mistakes():
    assert _pins_pass(lambda x: oracle.fftn(x))
    mutants = {
        "wrong sign": lambda x: oracle.fftn(x, sign=+1, norm=oracle.NORM_NONE),
        "dropped term": lambda x: oracle.fftn(np.where(np.arange(x.size).reshape(x.shape) == 1, 0, x)),
        "transposed operand": lambda x: oracle.fftn(x.T.copy()).T if x.ndim > 1 else oracle.fftn(x[::-1]),
        "missing axis": lambda x: oracle.fft_axis(x, x.ndim - 1) if x.ndim > 1 else oracle.fftn(x) * 1.0001,
        "scaled": lambda x: oracle.fftn(x, norm=oracle.NORM_ORTHO),
    }
    for name, f in mutants.items():
        assert not _pins_pass(f), name
