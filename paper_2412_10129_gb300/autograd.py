"""The projector pair as differentiable PyTorch operators (TIGRE v3, Sec. 2.8:
PyTorch operator wrappers), device resident.

``project(x, geo)`` is A x (interpolated projector) and its backward is the
matched backprojection A^T; ``backproject(y, geo)`` is A^T y with backward
A.  Both run on libtg through the C ABI, on the caller's CUDA stream, for a
single volume [nz, ny, nx] or a batch [B, nz, ny, nx] in one launch.  The
paper's wrapper copies through NumPy on every call; here nothing
leaves the GPU.

``unrolled_gd`` is the gradient step of Eq. 4,
x_{k+1} = x_k - eta A^T (A x_k - b), unrolled for a fixed number of steps,
with eta = 1 / ||A||^2 from a seeded power iteration and optional per-step
activation checkpointing (each step's intermediate projections are
recomputed in the backward pass instead of stored).
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as _ckpt

from . import tg


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, geo):
        ctx.geo = geo
        return tg.forward(geo, x.contiguous(), "interp")

    @staticmethod
    def backward(ctx, g):
        return tg.backproject(ctx.geo, g.contiguous(), "matched"), None


class _BackProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, geo):
        ctx.geo = geo
        return tg.backproject(geo, y.contiguous(), "matched")

    @staticmethod
    def backward(ctx, g):
        return tg.forward(ctx.geo, g.contiguous(), "interp"), None


def project(x: torch.Tensor, geo) -> torch.Tensor:
    """A x, differentiable (backward = matched A^T)."""
    _check(x)
    return _Project.apply(x, geo)


def backproject(y: torch.Tensor, geo) -> torch.Tensor:
    """A^T y, differentiable (backward = A)."""
    _check(y)
    return _BackProject.apply(y, geo)


class ProjOp(torch.nn.Module):
    """A as a module: ``ProjOp(geo)(x)`` = A x; ``.T(y)`` = A^T y."""

    def __init__(self, geo):
        super().__init__()
        self.geo = geo

    def forward(self, x):
        return project(x, self.geo)

    def T(self, y):
        return backproject(y, self.geo)


def _check(t):
    if not (t.is_cuda and t.dtype == torch.float32):
        raise ValueError("expected a float32 CUDA tensor")


def operator_norm_sq(geo, iters: int = 20, seed: int = 0, device="cuda") -> float:
    """||A||^2 (largest eigenvalue of A^T A) by power iteration from a seeded
    random start."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.rand(geo.vol_shape, generator=gen).to(device)
    lam = 0.0
    for _ in range(iters):
        v = v / torch.linalg.vector_norm(v)
        w = tg.backproject(geo, tg.forward(geo, v, "interp"), "matched")
        lam = float(torch.sum(v.double() * w.double()))
        v = w
    return lam


def gd_step(x: torch.Tensor, b: torch.Tensor, geo, eta: float) -> torch.Tensor:
    """One step of Eq. 4: x - eta A^T (A x - b)."""
    return x - eta * backproject(project(x, geo) - b, geo)


def unrolled_gd(x0: torch.Tensor, b: torch.Tensor, geo, steps: int = 10, eta: float | None = None,
                checkpoint: bool = True) -> torch.Tensor:
    """`steps` unrolled gradient steps; differentiable in x0 and b."""
    if eta is None:
        eta = 1.0 / operator_norm_sq(geo, device=x0.device)
    x = x0
    for _ in range(steps):
        if checkpoint and torch.is_grad_enabled():
            x = _ckpt.checkpoint(gd_step, x, b, geo, eta, use_reentrant=False)
        else:
            x = gd_step(x, b, geo, eta)
    return x
