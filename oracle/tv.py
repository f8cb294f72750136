"""Total-variation pieces of the POCS algorithms (Sec. 2.1, POCS methods;
Sec. 2.2 algorithm features: adaptive-weighted TV), in FP64 numpy.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``).  It shares no
code with the CUDA library.

Definitions (the paper prints AwTV for 2-D images; the readings extend it to
volumes [nz, ny, nx]):

* Backward differences d_a(v) = x(v) - x(v - e_a) along a = x, y, z, and 0
  where v - e_a lies outside the volume.
* Weights w_a(v) = exp(-(d_a(v) / delta)^2) (AwTV, Liu et al. 2012); delta =
  inf gives w = 1, plain TV.
* AwTV(x) = sum_v sqrt(w_x d_x^2 + w_y d_y^2 + w_z d_z^2 + eps), eps > 0 a
  smoothing constant that keeps the square root differentiable.
* Its gradient takes the weights as constants (they are recomputed from the
  current image at every gradient evaluation, as in Liu et al.):
      g(v) = sum_a w_a(v) d_a(v) / n(v) - sum_a w_a(v + e_a) d_a(v + e_a) / n(v + e_a),
  n(v) = sqrt(w_x d_x^2 + w_y d_y^2 + w_z d_z^2 + eps), the second sum over
  the neighbours inside the volume.

ASD-POCS (Sidky and Pan 2008) alternates a data step with TV steepest
descent, written out in ``asd_pocs`` in the order of that paper.
"""
from __future__ import annotations

import math

import numpy as np

from . import _f64, forward, ossart

AXES = (2, 1, 0)  # x, y, z of a [nz, ny, nx] array


def differences(x: np.ndarray):
    """Backward differences (d_x, d_y, d_z), 0 across the lower faces."""
    x = _f64(x)
    out = []
    for ax in AXES:
        d = np.zeros_like(x)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        d[tuple(sl_hi)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
        out.append(d)
    return out


def weights(ds, delta: float):
    if math.isinf(delta):
        return [np.ones_like(d) for d in ds]
    return [np.exp(-(d / delta) ** 2) for d in ds]


def awtv(x, delta: float = math.inf, eps: float = 1e-8, w=None) -> float:
    """AwTV(x); ``w`` overrides the weights (frozen weights)."""
    ds = differences(x)
    ws = weights(ds, delta) if w is None else w
    return float(np.sum(np.sqrt(sum(wa * d * d for wa, d in zip(ws, ds)) + eps)))


def awtv_gradient(x, delta: float = math.inf, eps: float = 1e-8) -> np.ndarray:
    """The gradient of AwTV with the weights of x held constant."""
    ds = differences(x)
    ws = weights(ds, delta)
    n = np.sqrt(sum(wa * d * d for wa, d in zip(ws, ds)) + eps)
    g = np.zeros_like(n)
    for ax, wa, d in zip(AXES, ws, ds):
        t = wa * d / n
        g += t
        # the neighbour ahead along ax holds -x(v) in its difference
        sl_v = [slice(None)] * 3
        sl_n = [slice(None)] * 3
        sl_v[ax] = slice(0, -1)
        sl_n[ax] = slice(1, None)
        g[tuple(sl_v)] -= t[tuple(sl_n)]
    return g


def tv_descent(x, steps: int, step: float, delta: float = math.inf, eps: float = 1e-8) -> np.ndarray:
    """``steps`` normalised steepest-descent steps x <- x - step g / ||g||."""
    x = _f64(x).copy()
    for _ in range(steps):
        g = awtv_gradient(x, delta, eps)
        nrm = float(np.linalg.norm(g))
        if nrm > 0:
            x = x - step * g / nrm
    return x


def asd_pocs(geo, b, niter: int, blocksize: int = 1, tv_steps: int = 20, alpha: float = 0.002,
             alpha_red: float = 0.95, r_max: float = 0.95, beta: float = 1.0, beta_red: float = 0.995,
             delta: float = math.inf, eps: float = 1e-8, data_tol: float = 0.0, x0=None):
    """ASD-POCS (Sidky and Pan 2008), OS-ASD-POCS for blocksize > 1:

        for each iteration:
            x_prev = x
            x = OS-SART sweep of x with relaxation beta, then x = max(x, 0)
            dd = ||A x - b||;  dp = ||x - x_prev||
            on the first iteration: dtvg = alpha * dp
            x_data = x
            tv_steps times: x = x - dtvg * g(x) / ||g(x)||   (g: AwTV gradient)
            dg = ||x - x_data||
            if dg > r_max * dp and dd > data_tol: dtvg = dtvg * alpha_red
            beta = beta * beta_red

    Defaults: Sidky and Pan's alpha_red 0.95, r_max 0.95, beta 1, beta_red
    0.995 and 20 TV steps; alpha 0.002 (their 0.2 makes the 20 normalised
    steps travel four times the first data step, from x0 = 0, and the TV
    descent overshoots).  Returns (x, dd after each iteration)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    b = _f64(b)
    hist = []
    dtvg = None
    for it in range(niter):
        x_prev = x
        x, _ = ossart(geo, b, 1, blocksize, lam=beta, nonneg=True, x0=x)
        dd = float(np.linalg.norm(forward(geo, x) - b))
        dp = float(np.linalg.norm(x - x_prev))
        if it == 0:
            dtvg = alpha * dp
        x_data = x
        x = tv_descent(x, tv_steps, dtvg, delta, eps)
        dg = float(np.linalg.norm(x - x_data))
        if dg > r_max * dp and dd > data_tol:
            dtvg *= alpha_red
        beta *= beta_red
        hist.append(dd)
    return x, np.array(hist)
