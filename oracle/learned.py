"""FP64 oracle of one learned-gradient step and of its gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The step is the
learned-gradient update that the paper's PyTorch wrappers (Sec. 2.8) are
meant to make possible:

    x' = x + so * Gamma(P(x))[..., 0],
    P(x) = (sx x, sg A^T (A x - b), 0, ..., 0)     (cin channels),

A the interpolated projector and A^T the matched backprojector of this
oracle (Eq. 1 and Eq. 4's gradient), Gamma a stack of 3x3x3 convolutions
(oracle.conv) with a ReLU after every layer but the last.  Weights are
W[kz, ky, kx, c_in, c_out] as in oracle.conv.

``step_backward`` is the chain rule written out for L = <gbar, x'>: the
layers' transposes from the last to the first, ReLU masks from the saved
activations, and the input channels mapped back to x through
d/dx A^T(A x - b) = A^T A.
"""
from __future__ import annotations

import numpy as np

from . import backproject, conv, forward


def _data_gradient(geo, x, b):
    """A^T (A x - b) (b may be None: A^T A x)."""
    r = forward(geo, x, "interp")
    if b is not None:
        r = r - np.asarray(b, np.float64)
    return backproject(geo, r, "matched")


def step(geo, x, b, Ws, Bs, sx, sg, so, round_act=None):
    """x' and the activations (input of every layer).  ``round_act`` (e.g.
    conv.bf16_round) is applied to the network input and every hidden
    activation when given, to mirror a reduced-precision implementation."""
    x = np.asarray(x, np.float64)
    cin = Ws[0].shape[3]
    inp = np.zeros(x.shape + (cin,))
    inp[..., 0] = sx * x
    inp[..., 1] = sg * _data_gradient(geo, x, b)
    rnd = (lambda a: a) if round_act is None else (lambda a: np.asarray(round_act(a), np.float64))
    h = rnd(inp)[None]
    acts = [h]
    for li, (W, B) in enumerate(zip(Ws, Bs)):
        last = li == len(Ws) - 1
        h = conv.conv3d(h, W, B, relu=not last)
        if not last:
            h = rnd(h)
            acts.append(h)
    return x + so * h[0, ..., 0], acts


def step_backward(geo, x, b, Ws, Bs, sx, sg, so, gbar, round_act=None):
    """Gradients of L = <gbar, x'> in x, in every W and in every bias, in
    FP64.  ``round_act`` (e.g. conv.bf16_round) rounds the network input and
    the hidden activations of the forward pass as in ``step`` -- the
    precision the learned network's definition fixes for its activations --
    so the gradient is the exact chain rule of that network; the gradients
    themselves are never rounded."""
    _, acts = step(geo, x, b, Ws, Bs, sx, sg, so, round_act=round_act)
    gbar = np.asarray(gbar, np.float64)
    gy = np.zeros(acts[-1].shape[:4] + (Ws[-1].shape[4],))
    gy[0, ..., 0] = so * gbar
    dWs, dBs = [None] * len(Ws), [None] * len(Ws)
    for li in range(len(Ws) - 1, -1, -1):
        dWs[li] = conv.conv3d_backward_weight(acts[li], gy)
        dBs[li] = gy.sum(axis=(0, 1, 2, 3))
        g_in = conv.conv3d_backward_data(gy, Ws[li])
        if li > 0:
            g_in = g_in * (acts[li] > 0)
        gy = g_in
    gx = gbar + sx * gy[0, ..., 0] + _data_gradient(geo, sg * gy[0, ..., 1], None)
    return gx, dWs, dBs
