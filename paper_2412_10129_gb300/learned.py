"""Learned-gradient reconstruction on libtg's kernels.

The paper adds PyTorch operator wrappers (Sec. 2.8) so that data-driven
reconstructions can put the projectors inside a network; learned primal-dual
is the example it names.  This module is that use, GPU resident: the
unrolled learned-gradient scheme

    x_{k+1} = x_k + Gamma_theta(x_k, A^T (A x_k - b)),   k = 0 .. K-1,

with A the interpolated projector, A^T the matched backprojector and Gamma a
3-D CNN shared by all K steps: five 3x3x3 convolutions with zero padding,
2 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU after the first four, BF16
weights and activations with FP32 accumulation.  The two input channels are
padded to 16 and the output channel to 8 (the tensor-core tiles' widths);
the padding carries zeros.

Every step -- the data-fit gradient (tg_gradient), the packing of the
network input, the convolutions, their backward passes and the update --
runs in libtg's kernels through the C ABI.  PyTorch holds the parameters and
the activations, computes the training loss and applies the optimiser step
(a few hundred thousand parameters).

Scaling.  The network sees sx x and sx eta A^T(Ax - b) with sx = 1 / mu_ref
(mu_ref = 0.05 /mm, the top of the phantoms' attenuation range) and
eta = 1 / ||A||^2, and its output is multiplied by 1 / sx.  With
``gd_init`` the weights start as one gradient step, Gamma = -eta A^T(Ax - b)
(channels 0 and 1 carry relu(c) and relu(-c) of the gradient channel c
through the hidden layers), with the other channels random and the last
layer reading only the first two, so training starts from plain gradient
descent and can only improve on it.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch
import torch.utils.checkpoint

from . import inputs, tg
from .autograd import operator_norm_sq

# (cin, cout, relu) of the five layers; cin of the first and cout of the last are padded
LAYERS = ((16, 32, True), (32, 32, True), (32, 32, True), (32, 32, True), (32, 8, False))
IN_CH, OUT_CH = 16, 8
MU_REF = 0.05  # /mm


def _centre(w: torch.Tensor) -> torch.Tensor:
    """The [cout, cin] weight matrix of the centre tap (offset (0, 0, 0))."""
    return w[13]


class LearnedGradient(torch.nn.Module):
    """Gamma_theta and the unrolled scheme around it."""

    def __init__(self, seed: int = 0, gd_init: bool = True, init_scale: float = 0.5, step: float = 1.0):
        super().__init__()
        gen = torch.Generator().manual_seed(seed)
        ws, bs = [], []
        for li, (cin, cout, _) in enumerate(LAYERS):
            fan_in = 27 * (2 if li == 0 else cin)
            w = torch.randn((27, cout, cin), generator=gen) * (init_scale * math.sqrt(2.0 / fan_in))
            if li == 0:
                w[:, :, 2:] = 0.0  # padded input channels
            if gd_init:
                if li == 0:
                    w[:, 0:2, :] = 0.0
                    _centre(w)[0, 1] = 1.0
                    _centre(w)[1, 1] = -1.0
                elif li < len(LAYERS) - 1:
                    w[:, 0:2, :] = 0.0
                    _centre(w)[0, 0] = 1.0
                    _centre(w)[1, 1] = 1.0
                else:
                    w.zero_()
                    _centre(w)[0, 0] = -step
                    _centre(w)[0, 1] = step
            if li == len(LAYERS) - 1:
                w[:, 1:, :] = 0.0  # padded output channels
            ws.append(torch.nn.Parameter(w))
            bs.append(torch.nn.Parameter(torch.zeros(cout)))
        self.weights = torch.nn.ParameterList(ws)
        self.biases = torch.nn.ParameterList(bs)

    def params(self):
        return list(self.weights) + list(self.biases)

    def step(self, x, b, geo, eta: float):
        """One learned-gradient step on a batch x [B, nz, ny, nx] (FP32, CUDA)."""
        sx = 1.0 / MU_REF
        cfg = (geo, sx, sx * eta, 1.0 / sx)
        if not torch.is_grad_enabled():
            return _lg_step_infer(x, b, cfg, self.weights, self.biases)
        return _LGStep.apply(x, b, cfg, *self.params())

    def forward(self, x0, b, geo, steps: int = 10, eta: float | None = None, checkpoint: bool = False):
        """x_K of the unrolled scheme from x0 [(B,) nz, ny, nx] and data b [(B,) nA, nv, nu]."""
        if eta is None:
            eta = 1.0 / operator_norm_sq(geo, device=x0.device)
        single = x0.ndim == 3
        x = x0[None] if single else x0
        bb = b[None] if single else b
        for _ in range(steps):
            if checkpoint and torch.is_grad_enabled():
                x = torch.utils.checkpoint.checkpoint(self.step, x, bb, geo, eta, use_reentrant=False)
            else:
                x = self.step(x, bb, geo, eta)
        return x[0] if single else x


def _conv_stack(inp, ws, bs, keep: bool):
    """The five convolutions; returns the FP32 output and (when ``keep``) the
    activations the backward pass needs (the input of every layer)."""
    acts = [inp]
    h = inp
    for li, (_, _, relu) in enumerate(LAYERS[:-1]):
        h = tg.conv3d(h, ws[li], bs[li], relu=relu)
        if keep:
            acts.append(h)
    out = tg.conv3d(h, ws[-1], bs[-1], relu=False, out_f32=True)
    return out, acts


def _lg_step_infer(x, b, cfg, ws, bs):
    """The step without autograd: no activation is kept."""
    geo, sx, sg, so = cfg
    x = x.contiguous()
    grad = tg.gradient(geo, x, b.contiguous())
    inp = tg.lg_pack(x, grad, IN_CH, sx, sg)
    del grad
    out, _ = _conv_stack(inp, [w.detach() for w in ws], [c.detach() for c in bs], keep=False)
    return tg.lg_update(x, out, so)


class _LGStep(torch.autograd.Function):
    """x -> x + so * Gamma(sx x, sg A^T(A x - b)) with a hand-written backward:
    the convolutions' transposes and weight gradients, then
    dL/dx = g + sx c0 + A^T A (sg c1), where (c0, c1) is the gradient in the
    network's two input channels (A^T(Ax - b) depends on x through A^T A)."""

    @staticmethod
    def forward(ctx, x, b, cfg, *params):
        geo, sx, sg, so = cfg
        ws, bs = params[:5], params[5:]
        x = x.contiguous()
        grad = tg.gradient(geo, x, b.contiguous())
        inp = tg.lg_pack(x, grad, IN_CH, sx, sg)
        out, acts = _conv_stack(inp, [w.detach() for w in ws], [c.detach() for c in bs], keep=True)
        xn = tg.lg_update(x, out, so)
        ctx.save_for_backward(*acts, *[w.detach() for w in ws])
        ctx.cfg = cfg
        return xn

    @staticmethod
    def backward(ctx, gxn):
        geo, sx, sg, so = ctx.cfg
        saved = ctx.saved_tensors
        acts, ws = saved[:5], saved[5:]
        gxn = gxn.contiguous()
        # Every layer gradient travels as a BF16 pair hi + lo (FP32 precision
        # on the BF16 tensor cores); activations and weights stay BF16.
        hi, lo = tg.lg_pack_split(gxn, OUT_CH, so)
        dws, dbs = [None] * 5, [None] * 5
        gin = None
        for li in range(4, -1, -1):
            dws[li] = tg.conv3d_backward_weight_split(acts[li], hi, lo)
            dbs[li] = tg.conv3d_backward_bias_split(hi, lo)
            gin = tg.conv3d_backward_data_split(hi, lo, ws[li])
            if li > 0:
                hi, lo = tg.grad_split(gin, acts[li])
                del gin
        del hi, lo
        gx = gxn.clone()
        gg = torch.empty_like(gxn)
        tg.lg_unpack_f32(gin, gx, gg, sx, sg, accumulate=True)
        tg.gradient(geo, gg, None, out=gx, accumulate=True)
        return (gx, None, None, *dws, *dbs)


# ---------------------------------------------------------------------------
# Batched inference over volumes of different sizes.
# ---------------------------------------------------------------------------

@torch.no_grad()
def infer_ragged(net: LearnedGradient, geos, bs, x0s, steps: int = 10, etas=None):
    """The unrolled scheme on volumes of different sizes at once: each step
    takes every volume's data-fit gradient with one launch of each
    projector for all geometries (tg_gradient_batched), packs all inputs
    into one buffer, runs each convolution over all volumes in a single
    launch (the per-volume tile table of tg_conv3d_forward_ragged) and
    updates all iterates in one launch.  Returns the reconstructions (views
    into one packed FP32 buffer)."""
    dev = x0s[0].device
    dims = [tuple(g.vol_shape) for g in geos]
    counts = [int(np.prod(d)) for d in dims]
    offs = np.concatenate([[0], np.cumsum(counts)])
    tot = int(offs[-1])
    if etas is None:
        etas = [1.0 / operator_norm_sq(g, device=dev) for g in geos]
    sx = 1.0 / MU_REF
    x = torch.empty(tot, dtype=torch.float32, device=dev)
    grad = torch.empty(tot, dtype=torch.float32, device=dev)
    bpk = torch.cat([b.reshape(-1) for b in bs]).contiguous()
    inp = torch.empty((tot, IN_CH), dtype=torch.bfloat16, device=dev)
    ha = torch.empty((tot, 32), dtype=torch.bfloat16, device=dev)
    hb = torch.empty((tot, 32), dtype=torch.bfloat16, device=dev)
    out = torch.empty((tot, OUT_CH), dtype=torch.float32, device=dev)
    xs = [x[offs[k]:offs[k + 1]].view(dims[k]) for k in range(len(geos))]
    gs = [grad[offs[k]:offs[k + 1]].view(dims[k]) for k in range(len(geos))]
    for k, x0 in enumerate(x0s):
        xs[k].copy_(x0)
    ws = [w.detach().contiguous() for w in net.weights]
    cb = [c.detach().contiguous() for c in net.biases]
    for _ in range(steps):
        tg.gradient_batched(geos, x, bpk, out=grad)
        for k in range(len(geos)):
            tg.lg_pack(xs[k], gs[k], IN_CH, sx, sx * etas[k], out=inp[offs[k]:offs[k + 1]])
        h = inp
        for li, (_, _, relu) in enumerate(LAYERS[:-1]):
            dst = ha if li % 2 == 0 else hb
            tg.conv3d_ragged(h, dims, ws[li], cb[li], relu=relu, out=dst)
            h = dst
        tg.conv3d_ragged(h, dims, ws[-1], cb[-1], relu=False, out_f32=True, out=out)
        tg.lg_update(x, out, 1.0 / sx, out=x)
    return xs


# ---------------------------------------------------------------------------
# Training data and training loop.
# ---------------------------------------------------------------------------

def make_sample(geo, seed: int, I0: float = 1e4, device="cuda", phantom=None):
    """(b, x0, x_true) for one seeded phantom: b = noisy line integrals
    (Siddon projection of the voxelised phantom, Poisson noise at I0 drawn on
    the device), x0 = FDK of b, x_true the phantom.  ``phantom`` may hold the
    voxelised phantom already (e.g. from a prefetching thread)."""
    if phantom is None:
        phantom = inputs.learned_phantom(geo, seed)
    gt = torch.from_numpy(phantom).to(device)
    b = inputs.poisson_noise_device(tg.forward(geo, gt, "siddon"), I0, seed + 1_000_003)
    x0 = tg.fdk(geo, b)
    return b, x0, gt


def samples(geo, seeds, I0: float = 1e4, device="cuda", prefetch: int = 4):
    """make_sample over ``seeds``, voxelising the next phantoms on host
    threads while the GPU works on the current one."""
    from concurrent.futures import ThreadPoolExecutor
    seeds = list(seeds)
    with ThreadPoolExecutor(max_workers=2) as pool:
        futs = [pool.submit(inputs.learned_phantom, geo, s) for s in seeds[:prefetch]]
        for i, s in enumerate(seeds):
            ph = futs[i].result()
            if i + prefetch < len(seeds):
                futs.append(pool.submit(inputs.learned_phantom, geo, seeds[i + prefetch]))
            yield make_sample(geo, s, I0, device, phantom=ph)


def psnr(x: torch.Tensor, gt: torch.Tensor) -> float:
    """10 log10(max(gt)^2 / MSE) over the whole volume."""
    mse = float(torch.mean((x.double() - gt.double()) ** 2))
    peak = float(gt.max())
    return 10.0 * math.log10(peak * peak / mse) if mse > 0 else float("inf")


def train(net: LearnedGradient, geo, seeds, steps: int = 10, batch: int = 2, lr: float = 1e-3,
          epochs: int = 1, I0: float = 1e4, checkpoint: bool = False, device="cuda", log=None):
    """Adam on the mean relative squared error ||x_K - x_true||^2 / ||x_true||^2
    over mini-batches of seeded phantoms; returns the per-batch losses."""
    eta = 1.0 / operator_norm_sq(geo, device=device)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    losses = []
    seeds = list(seeds)
    nb = len(seeds) // batch
    for _ in range(epochs):
        it = samples(geo, seeds[:nb * batch], I0, device)
        for _ in range(nb):
            smp = [next(it) for _ in range(batch)]
            b = torch.stack([s[0] for s in smp])
            x0 = torch.stack([s[1] for s in smp])
            gt = torch.stack([s[2] for s in smp])
            x = net(x0, b, geo, steps=steps, eta=eta, checkpoint=checkpoint)
            err = torch.sum((x - gt) ** 2, dim=(1, 2, 3)) / torch.sum(gt ** 2, dim=(1, 2, 3))
            loss = err.mean()
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            losses.append(float(loss.detach()))
            if log is not None:
                log(len(losses), losses[-1])
    return losses


def cgls_best(geo, b, gt, max_iter: int = 60):
    """Plain CGLS from zero: (best PSNR, iterations that reach it)."""
    best, best_k = -float("inf"), 0
    for k in range(1, max_iter + 1):
        p = psnr(tg.cgls(geo, b, k), gt)
        if p > best:
            best, best_k = p, k
    return best, best_k


def timed(fn, reps: int = 3):
    """Median wall time of fn() (seconds), synchronised on both sides."""
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def conv_benchmark(n: int = 256, reps: int = 5, layers=((32, 32), (16, 32), (32, 8))):
    """Device time of each convolution kernel on an n^3 volume (CUDA events):
    forward, input gradient and weight gradient per (cin, cout) pair, with
    their FLOP rates (2 * 27 * cin * cout per voxel)."""
    out = []
    for cin, cout in layers:
        gen = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn((1, n, n, n, cin), device="cuda", generator=gen).to(torch.bfloat16)
        gy = torch.randn((1, n, n, n, cout), device="cuda", generator=gen).to(torch.bfloat16)
        w = torch.randn((27, cout, cin), device="cuda", generator=gen) * 0.05
        ops = (("forward", lambda: tg.conv3d(x, w, None, relu=True)),
               ("backward_data", lambda: tg.conv3d_backward_data(gy, w)),
               ("backward_weight", lambda: tg.conv3d_backward_weight(x, gy)))
        for name, fn in ops:
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out.append({"cin": cin, "cout": cout, "op": name, "ms": ms,
                        "tflops": 2 * 27 * cin * cout * n ** 3 / ms / 1e9})
        tg.device_status()
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="learned-gradient kernels: convolution timings")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    from . import build
    build.build()
    for row in conv_benchmark(a.n, a.reps):
        print(json.dumps(row), flush=True)
