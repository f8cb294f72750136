"""FDK variants (Sec. 2.1, direct methods): filter windows, Parker short-scan
weights and Wang offset-detector weights, in FP64 numpy.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``).  It shares no
code with the CUDA library.

Sec. 2.1 lists FDK "with various filter types" and with Wang weights (detector
displacement) and Parker weights (angular range) without formulas, and the
experiments of Sec. 3 use the ramp, Hamming and Shepp-Logan filters.  The
definitions written out here are the published methods they name:

* Row filter.  The discrete band-limited ramp (Ram-Lak) kernel h of the
  spatial FDK filter (h[0] = 1/4, h[k odd] = -1/(pi k)^2, h[k even] = 0, in
  units of the isocentre pitch tau), made N-periodic for N the smallest power
  of two >= max(64, 2 nu) (|k| < N/2), has the real DFT R[m].  A window
  W(f) multiplies it at frequency f = m/N cycles per sample folded into
  [0, 1/2]:
      ram-lak      1
      shepp-logan  sin(pi f) / (pi f)       (Shepp and Logan 1974)
      cosine       cos(pi f)
      hamming      0.54 + 0.46 cos(2 pi f)
      hann         0.5 + 0.5 cos(2 pi f)
  A row of nu samples, zero padded to N, is multiplied by R W in the
  frequency domain; the first nu outputs, divided by tau, are the filtered
  row.  N >= 2 nu makes this a linear (non-circular) convolution, so for
  ram-lak it equals the spatial filter of ``oracle.fdk_filter``.
* Parker weights (Parker 1982, as generalised to over-scans by Wesarg et al.
  2002).  A circular orbit of increasing angle covers beta in [0, beta_max],
  beta = theta_a - theta_0 of the first Euler angle, with beta_max = pi + 2
  Delta.  A ray of fan angle gamma (measured towards +e_u) has its conjugate
  at (beta + pi - 2 gamma, -gamma) in this geometry; with g = -gamma the
  weight is
      sin^2(pi/4 beta / (Delta - g))              0 <= beta < 2 Delta - 2 g
      1                                           up to pi - 2 g
      sin^2(pi/4 (pi + 2 Delta - beta) / (Delta + g))   up to pi + 2 Delta
  so the two measurements of every line sum to 1.  The backprojection then
  uses the angle weight beta_max / (nAngles - 1) instead of pi / nAngles.
* Wang weights (Wang 2002, displaced detector, full orbit).  u is the
  detector coordinate along e_u measured from the foot of the perpendicular
  from the source; the detector covers [u_lo, u_hi]; u0 = min(-u_lo, u_hi)
  is the half-width of the region seen from both sides and s the sign of
  the longer side.  With t = s u the weight is 0 for t <= -u0,
  1 + sin(pi/2 t/u0) in between and 2 for t >= u0, so conjugate rays sum to
  2 (the full-orbit FDK angle weight pi / nAngles halves every line).

The fan angle is gamma = atan2((P - S).e_u, |(P - S).n|) for pixel centre P.

Parallel beam (geo.parallel): no cosine pre-weight and the pitch du (parallel
FBP); Parker and Wang weights are not defined for it here.
"""
from __future__ import annotations

import math

import numpy as np

from . import backproject, fdk_filter as _fdk_ramlak_spatial, frames, pixel_centres

WINDOWS = ("ram-lak", "shepp-logan", "cosine", "hamming", "hann")


def window(name: str, f) -> np.ndarray:
    """The filter window at |f| cycles per sample (0 <= |f| <= 1/2)."""
    f = np.abs(np.asarray(f, dtype=np.float64))
    if name == "ram-lak":
        return np.ones_like(f)
    if name == "shepp-logan":
        return np.sinc(f)  # numpy's sinc is sin(pi f) / (pi f)
    if name == "cosine":
        return np.cos(math.pi * f)
    if name == "hamming":
        return 0.54 + 0.46 * np.cos(2 * math.pi * f)
    if name == "hann":
        return 0.5 + 0.5 * np.cos(2 * math.pi * f)
    raise ValueError(f"unknown filter {name!r}")


def fft_length(nu: int) -> int:
    """N: the smallest power of two >= max(64, 2 nu)."""
    N = 64
    while N < 2 * nu:
        N *= 2
    return N


def ramlak_periodic(N: int) -> np.ndarray:
    """The Ram-Lak kernel at unit pitch on an N-periodic grid (|k| < N/2)."""
    h = np.zeros(N)
    h[0] = 0.25
    k = np.arange(1, N // 2, 2)
    h[k] = -1.0 / (math.pi * k) ** 2
    h[N - k] = h[k]
    return h


def filter_response(nu: int, name: str) -> np.ndarray:
    """R[m] W(m/N), m = 0..N-1, for rows of nu samples (unit pitch)."""
    N = fft_length(nu)
    R = np.fft.fft(ramlak_periodic(N)).real
    m = np.arange(N)
    f = np.minimum(m, N - m) / N
    return R * window(name, f)


def filter_rows(rows: np.ndarray, tau, name: str) -> np.ndarray:
    """Filters the last axis of ``rows`` (nu samples) with window ``name``;
    ``tau`` broadcasts against rows[..., 0] (the isocentre pitch)."""
    rows = np.asarray(rows, dtype=np.float64)
    nu = rows.shape[-1]
    N = fft_length(nu)
    H = filter_response(nu, name)
    spec = np.fft.fft(rows, n=N, axis=-1) * H
    out = np.fft.ifft(spec, axis=-1).real[..., :nu]
    return out / np.asarray(tau, dtype=np.float64)[..., None]


def ray_coordinates(geo, a: int):
    """(u, depth) of every pixel of projection a: u = (P - S).e_u and
    depth = |(P - S).n|, both [nv, nu] (mm)."""
    f = frames(geo)
    d = pixel_centres(geo, a) - f["S"][a]
    return d @ f["eu"][a], np.abs(d @ f["n"][a]), np.linalg.norm(d, axis=-1)


def parker_weight(beta, gamma, Delta: float) -> np.ndarray:
    """Parker weight of a ray at orbit position beta and fan angle gamma
    (towards +e_u) for a scan of pi + 2 Delta."""
    beta = np.asarray(beta, dtype=np.float64)
    g = -np.asarray(gamma, dtype=np.float64)
    beta, g = np.broadcast_arrays(beta, g)
    w = np.zeros(beta.shape)
    end = math.pi + 2 * Delta
    r1 = (beta >= 0) & (beta < 2 * Delta - 2 * g)
    r2 = (beta >= 2 * Delta - 2 * g) & (beta <= math.pi - 2 * g)
    r3 = (beta > math.pi - 2 * g) & (beta <= end)
    with np.errstate(divide="ignore", invalid="ignore"):
        w[r1] = np.sin(math.pi / 4 * beta[r1] / (Delta - g[r1])) ** 2
        w[r3] = np.sin(math.pi / 4 * (end - beta[r3]) / (Delta + g[r3])) ** 2
    w[r2] = 1.0
    return w


def parker_scan(geo):
    """(beta per angle, beta_max, Delta) of a circular orbit of increasing
    first Euler angle."""
    th = np.asarray(geo.angles, dtype=np.float64).reshape(-1, 3)[:, 0]
    beta = th - th[0]
    bmax = float(beta[-1])
    if len(th) < 2 or bmax <= math.pi or np.any(np.diff(th) <= 0):
        raise ValueError("Parker weights need increasing angles spanning more than pi")
    return beta, bmax, 0.5 * (bmax - math.pi)


def wang_weight(u, u0: float, side: float) -> np.ndarray:
    t = side * np.asarray(u, dtype=np.float64)
    w = 1.0 + np.sin(0.5 * math.pi * np.clip(t, -u0, u0) / u0)
    return w


def wang_overlap(geo, a: int):
    """(u0, side) of projection a: half-width of the doubly seen region and
    the sign of the longer detector side."""
    f = frames(geo)
    nu = int(geo.nDetector[0])
    uc = float((f["D"][a] - f["S"][a]) @ f["eu"][a])
    u_lo = uc - 0.5 * nu * geo.dDetector[0]
    u_hi = uc + 0.5 * nu * geo.dDetector[0]
    u0 = min(-u_lo, u_hi)
    if u0 <= 0:
        raise ValueError("the detector does not reach across the central ray")
    return u0, (1.0 if u_hi >= -u_lo else -1.0)


def pre_weights(geo, parker: bool = False, wang: bool = False) -> np.ndarray:
    """Cosine weight |(P-S).n|/|P-S| times the optional Parker and Wang
    weights, [nAngles, nv, nu]."""
    n = int(geo.nAngles)
    nu, nv = (int(v) for v in geo.nDetector)
    if getattr(geo, "parallel", False):
        if parker or wang:
            raise ValueError("Parker and Wang weights are defined for cone beams only")
        return np.ones((n, nv, nu))
    out = np.zeros((n, nv, nu))
    if parker:
        beta, _, Delta = parker_scan(geo)
    for a in range(n):
        u, depth, dist = ray_coordinates(geo, a)
        w = depth / dist
        if parker:
            w = w * parker_weight(beta[a], np.arctan2(u, depth), Delta)
        if wang:
            u0, side = wang_overlap(geo, a)
            w = w * wang_weight(u, u0, side)
        out[a] = w
    return out


def fdk_filter(geo, proj, filter: str = "ram-lak", parker: bool = False, wang: bool = False) -> np.ndarray:
    """Pre-weighted, row-filtered projections [nAngles, nv, nu]."""
    p = np.asarray(proj, dtype=np.float64).reshape(geo.proj_shape)
    if parker and wang:
        raise ValueError("Parker and Wang weights are not combined")
    if getattr(geo, "parallel", False):
        tau = np.full(int(geo.nAngles), float(geo.dDetector[0]))
    else:
        tau = np.asarray(geo.dDetector[0] * np.asarray(geo.DSO, np.float64).reshape(-1)
                         / np.asarray(geo.DSD, np.float64).reshape(-1))
    rows = p * pre_weights(geo, parker, wang)
    return filter_rows(rows, tau[:, None], filter)


def angle_weight(geo, parker: bool = False) -> float:
    """The backprojection's angle weight: beta_max / (nAngles - 1) for a
    Parker short scan, else pi / nAngles (full orbit, every line twice)."""
    if parker:
        _, bmax, _ = parker_scan(geo)
        return bmax / (int(geo.nAngles) - 1)
    return math.pi / int(geo.nAngles)


def fdk(geo, proj, filter: str = "ram-lak", parker: bool = False, wang: bool = False) -> np.ndarray:
    """FDK with a filter window and optional Parker or Wang weights."""
    q = fdk_filter(geo, proj, filter, parker, wang)
    # oracle.backproject(fdk) applies pi / nAngles; rescale to the angle weight
    return backproject(geo, q, "fdk") * (angle_weight(geo, parker) * int(geo.nAngles) / math.pi)


def ramlak_spatial(geo, proj) -> np.ndarray:
    """The C oracle's spatial cosine-weighted Ram-Lak filter (for comparison
    with the frequency-domain path)."""
    return _fdk_ramlak_spatial(geo, proj)
