"""Differentiation pattern: the forward projection as a torch.autograd.Function
whose backward is the hand-written BP kernel. Checked by central finite
differences of the loss 1/2 ||y - A x||^2 (reduced in FP64) on seeded voxels,
by the adjoint dot-product test, and against the FP64 oracle's gradient."""
import numpy as np
import pytest

from helpers import gpu_geom, oracle_geom, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import projector as OP  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402
from paper_1903_11874_gb300.autograd import Projector  # noqa: E402

DEV = "cuda:0"

# differentiation workload: 128^3 volumes of 1 mm, 180 views over 360 deg,
# 192 x 192 detector of 1.6 mm, DSO 500 / DSD 1000
CFG4 = dict(kind="cone3d", nx=128, ny=128, nz=128, dx=1.0, dy=1.0, dz=1.0, n_views=180,
            nu=192, nv=192, du=1.6, dv=1.6, dso=500.0, dsd=1000.0, M=1, N=1)
SMALL = dict(kind="cone3d", nx=24, ny=20, nz=16, dx=1.0, dy=1.0, dz=1.0, n_views=12,
             nu=30, nv=22, du=1.6, dv=1.6, dso=80.0, dsd=160.0, M=1, N=1,
             angles=0.03 + np.arange(12) * (2 * np.pi / 12))


def _loss64(y, target):
    return 0.5 * ((y.double() - target.double()) ** 2).sum()


def test_gradient_matches_oracle_small():
    gg, og = gpu_geom(SMALL), oracle_geom(SMALL)
    xt = synth.ellipsoid_phantom(24, 20, 16, 4, seed=1).astype(np.float64)
    target = OP.fp(og, xt.reshape(-1))
    x0 = xt + 0.05 * synth.normal_array(xt.shape, 2)
    x = torch.tensor(x0, dtype=torch.float32, device=DEV, requires_grad=True)
    y = Projector.apply(x, gg)
    _loss64(y, torch.tensor(target, device=DEV)).backward()
    x0f = x0.astype(np.float32).astype(np.float64).reshape(-1)
    ref = OP.bp(og, OP.fp(og, x0f).reshape(-1) - target.reshape(-1)).reshape(-1)
    assert rel_l2(x.grad.cpu().double().numpy().reshape(-1), ref) < 1e-4


def test_finite_differences_and_adjoint_batch16():
    """Batch of 16 seeded 128^3 volumes through the autograd.Function: the
    gradient of 1/2 ||y - A x||^2 matches central differences (eps = 1e-3) on
    64 seeded voxels, and <A x, r> = <x, A^T r> holds to 1e-6."""
    gg = gpu_geom(CFG4)
    Bn = 16
    vols = np.stack([synth.ellipsoid_phantom(128, 128, 128, 10, seed=s) for s in range(Bn)])
    xt = torch.tensor(vols, dtype=torch.float32, device=DEV)
    with torch.no_grad():
        target = Projector.apply(xt, gg)
    pert = torch.tensor(0.05 * synth.normal_array(vols.shape, 99), dtype=torch.float32, device=DEV)
    x = (xt + pert).requires_grad_(True)
    _loss64(Projector.apply(x, gg), target).backward()
    grad = x.grad.detach()
    rng = np.random.default_rng(4)
    eps = 1e-3
    flat = x.detach().reshape(-1)
    idx = rng.choice(flat.numel(), 64, replace=False)
    errs = []
    for k in idx:
        xp = flat.clone()
        xm = flat.clone()
        xp[k] += eps
        xm[k] -= eps
        with torch.no_grad():
            lp = _loss64(Projector.apply(xp.view_as(x), gg), target)
            lm = _loss64(Projector.apply(xm.view_as(x), gg), target)
        fd = float((lp - lm) / (xp[k].double() - xm[k].double()))
        g = float(grad.reshape(-1)[k])
        errs.append(abs(fd - g) / max(abs(g), 1e-3 * float(grad.abs().max())))
    # The loss is quadratic, so the central difference has no truncation error;
    # what remains is the FP32 rounding of the ~2 x 180 ray sums through the
    # voxel (a few ulps of |y| ~ 1e2 each), divided by 2 eps: ~1e-3 relative in
    # the worst voxel, far less in most.
    assert max(errs) < 5e-3, max(errs)
    assert float(np.median(errs)) < 1e-4, float(np.median(errs))
    # adjoint dot-product test on the same operator, batched
    r = torch.tensor(synth.normal_array((Bn,) + tuple(gg.sino_shape), 5), dtype=torch.float32,
                     device=DEV)
    with torch.no_grad():
        ax = Projector.apply(xt, gg)
    xr = xt.clone().requires_grad_(True)
    (Projector.apply(xr, gg) * r).sum().backward()
    lhs = float((ax.double() * r.double()).sum())
    rhs = float((xt.double() * xr.grad.double()).sum())
    scale = float((ax.double().abs() * r.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale
