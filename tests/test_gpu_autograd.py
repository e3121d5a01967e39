"""GPU checks of the hand-written adjoint behind torch.autograd.Function.

For Y = F x (unnormalised forward), the gradient of a real loss L is
F^H dL/dY*, and F^H is the inverse transform with conjugated roots and no
scaling (Section 4.2 describes the conjugated-roots inverse).  The loss of
the differentiable configuration is L = sum |W * F x|^2 with W real."""
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


def gpu_grad(xs, w, norm="none", inverse=False):
    x = torch.from_numpy(xs).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    f = W.ifftn if inverse else W.fftn
    loss = (wt * f(x, rank=3, norm=norm)).abs().pow(2).sum()
    loss.backward()
    return x.grad.cpu().numpy().astype(np.complex128), float(loss.item())


def test_grad_16cubed_vs_oracle_and_finite_differences():
    shape = (16, 16, 16)
    xs = inputs.complex_input(shape, 1, "normal", "c32")
    w = inputs.loss_weights(shape, 2)
    g, _ = gpu_grad(xs, w)
    x64 = xs.astype(np.complex128)
    w64 = w.astype(np.float64)
    g_ref = oracle.loss_grad(x64, w64)
    assert oracle.rel_l2(g, g_ref) < 5e-6
    # FP64 central differences on 64 sampled coordinates (L is quadratic, so
    # the difference has no truncation error; h keeps rounding small)
    rng = np.random.default_rng(3)
    h = 1e-3
    xf = x64.ravel()
    errs = []
    for i in rng.integers(0, xf.size, size=32):
        for part in (1.0, 1j):
            xp, xm = xf.copy(), xf.copy()
            xp[i] += h * part
            xm[i] -= h * part
            fd = (oracle.loss(xp.reshape(shape), w64) - oracle.loss(xm.reshape(shape), w64)) / (2 * h)
            an = g.ravel()[i].real if part == 1.0 else g.ravel()[i].imag
            errs.append(abs(fd - an))
    # pointwise error against the gradient's RMS: FP32 rounding of the GPU
    # path is ~1e-7 of that scale, the FD rounding ~eps*L/h smaller still
    rms = float(np.sqrt(np.mean(np.abs(g_ref) ** 2)))
    assert max(errs) < 1e-5 * rms, (max(errs), rms)


def test_grad_batch8_128cubed():
    # the differentiable configuration: batch of 8 fields 128^3, W ~ U[0,1)
    shape = (8, 128, 128, 128)
    xs = inputs.complex_input(shape, 1, "normal", "c32")
    w = inputs.loss_weights(shape, 2)
    g, loss = gpu_grad(xs, w)
    g_ref = oracle.loss_grad(xs.astype(np.complex128), w.astype(np.float64), rank=3)
    err = oracle.rel_l2(g, g_ref)
    print(f"batch 8 x 128^3 grad rel_l2 {err:.3e}")
    assert err < 5e-6
    l_ref = oracle.loss(xs.astype(np.complex128), w.astype(np.float64), rank=3)
    assert abs(loss - l_ref) / l_ref < 1e-5


@pytest.mark.parametrize("norm", ["paper", "ortho", "forward"])
@pytest.mark.parametrize("inverse", [False, True])
def test_grad_every_normalisation(norm, inverse):
    shape = (8, 32, 16)
    xs = inputs.complex_input(shape, 5, "normal", "c32")
    w = inputs.loss_weights(shape, 6)
    g, _ = gpu_grad(xs, w, norm=norm, inverse=inverse)
    # the map G as a scalar multiple of F or F^H: L = sum |w G x|^2, grad = 2 G^H (w^2 G x)
    N = float(np.prod(shape))
    sign = +1 if inverse else -1
    s = {("paper", False): 1.0, ("paper", True): 1.0 / N, ("ortho", False): N ** -0.5,
         ("ortho", True): N ** -0.5, ("forward", False): 1.0 / N, ("forward", True): 1.0}[(norm, inverse)]
    x64 = xs.astype(np.complex128)
    gx = s * oracle.fftn(x64, sign=sign, norm=oracle.NORM_NONE)
    ref = 2 * s * oracle.fftn(w.astype(np.float64) ** 2 * gx, sign=-sign, norm=oracle.NORM_NONE)
    assert oracle.rel_l2(g, ref) < 5e-6


def test_adjoint_dot_product_identity():
    shape = (64, 32, 128)
    x = torch.from_numpy(inputs.complex_input(shape, 7, "normal", "c32")).cuda()
    y = torch.from_numpy(inputs.complex_input(shape, 8, "normal", "c32")).cuda()
    Fx = W.fftn(x, norm="none")
    FHy = W.ifftn(y, norm="none")
    lhs = torch.vdot(y.ravel().to(torch.complex128), Fx.ravel().to(torch.complex128))
    rhs = torch.vdot(FHy.ravel().to(torch.complex128), x.ravel().to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))
