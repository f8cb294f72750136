"""FP64 oracle of the learned part's 3-D convolutions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The learned-gradient
network (a learned-primal-dual style correction, the use case the paper's
PyTorch wrappers are motivated by, Sec. 2.8) is a stack of 3x3x3
convolutions with zero padding.  Layouts are channels-last:
activations x[n, z, y, x, c], weights W[kz, ky, kx, c_in, c_out].

Each function is the plain definition: a sum over the 27 kernel offsets of a
shifted copy of the input times the offset's weight matrix (numpy einsum as
the per-offset step)."""
from __future__ import annotations

import numpy as np


def _shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """s[n, z, y, x, :] = x[n, z + dz, y + dy, x + dx, :], zero outside."""
    n, Z, Y, X, c = x.shape
    out = np.zeros_like(x)
    zs = slice(max(0, -dz), min(Z, Z - dz))
    ys = slice(max(0, -dy), min(Y, Y - dy))
    xs = slice(max(0, -dx), min(X, X - dx))
    zt = slice(max(0, dz), min(Z, Z + dz))
    yt = slice(max(0, dy), min(Y, Y + dy))
    xt = slice(max(0, dx), min(X, X + dx))
    out[:, zs, ys, xs, :] = x[:, zt, yt, xt, :]
    return out


def conv3d(x, W, bias=None, relu: bool = False) -> np.ndarray:
    """y[v, o] = bias[o] + sum_{d in {-1,0,1}^3} sum_i x[v + d, i] W[d + 1, i, o]."""
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    y = np.zeros(x.shape[:4] + (W.shape[4],))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                y += np.einsum("nzyxi,io->nzyxo", _shift(x, kz - 1, ky - 1, kx - 1), W[kz, ky, kx])
    if bias is not None:
        y += np.asarray(bias, np.float64)
    if relu:
        y = np.maximum(y, 0.0)
    return y


def conv3d_backward_data(gy, W) -> np.ndarray:
    """The transpose of conv3d in its input: scatter of gy through each offset,
    gx[v + d, i] += gy[v, o] W[d + 1, i, o]."""
    gy = np.asarray(gy, np.float64)
    W = np.asarray(W, np.float64)
    gx = np.zeros(gy.shape[:4] + (W.shape[3],))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                t = np.einsum("nzyxo,io->nzyxi", gy, W[kz, ky, kx])
                gx += _shift(t, -(kz - 1), -(ky - 1), -(kx - 1))
    return gx


def conv3d_backward_weight(x, gy) -> np.ndarray:
    """dW[d + 1, i, o] = sum_v x[v + d, i] gy[v, o]."""
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    dW = np.zeros((3, 3, 3, x.shape[4], gy.shape[4]))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                dW[kz, ky, kx] = np.einsum("nzyxi,nzyxo->io", _shift(x, kz - 1, ky - 1, kx - 1), gy)
    return dW


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(a.shape)


def learned_net(x_in, weights, biases) -> np.ndarray:
    """Gamma(x, g): conv3d stack with ReLU after every layer but the last;
    x_in[n, z, y, x, 2] holds (x_k, gradient)."""
    h = np.asarray(x_in, np.float64)
    for li, (W, b) in enumerate(zip(weights, biases)):
        h = conv3d(h, W, b, relu=li < len(weights) - 1)
    return h
