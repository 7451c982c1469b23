"""Differentiable forward projection.

Projector.apply(x, geom) computes y = A x with the library's Siddon FP kernel
(Sec. 1: FP and BP are computed on the fly); its backward is the matched BP
kernel, grad_x = A^T grad_y, the exact transpose of the forward operator. Both
run through the C ABI (bsgd_forward_project / bsgd_back_project); torch only
supplies the tensors and the stream.
"""
import torch

from . import binding as B


def _batched(t, inner_dim):
    return t if t.dim() == inner_dim + 1 else t.unsqueeze(0)


class Projector(torch.autograd.Function):
    """x: [B, nz, ny, nx] or [nz, ny, nx] float32 CUDA tensor -> y: [B, n_views,
    nv, nu] (or unbatched)."""

    @staticmethod
    def forward(ctx, x, geom):
        if x.dtype != torch.float32:
            raise B.BSGDError(1, "Projector expects float32 volumes")
        unbatched = x.dim() == 3
        xb = _batched(x, 3).contiguous()
        batch = xb.shape[0]
        if tuple(xb.shape[1:]) != tuple(geom.vol_shape):
            raise B.BSGDError(1, "volume shape %s does not match the geometry %s"
                              % (tuple(xb.shape[1:]), geom.vol_shape))
        y = torch.empty((batch,) + tuple(geom.sino_shape), device=x.device, dtype=torch.float32)
        B.bsgd_forward_project(geom, xb, y, batch=batch)
        ctx.geom = geom
        ctx.unbatched = unbatched
        return y[0] if unbatched else y

    @staticmethod
    def backward(ctx, gy):
        geom = ctx.geom
        gyb = _batched(gy, 3).contiguous().float()
        batch = gyb.shape[0]
        gx = torch.empty((batch,) + tuple(geom.vol_shape), device=gy.device, dtype=torch.float32)
        B.bsgd_back_project(geom, gyb, gx, batch=batch)
        return (gx[0] if ctx.unbatched else gx), None


def project(x, geom):
    return Projector.apply(x, geom)
