"""FP64 CPU oracle for the cone-beam CT hot path (TIGRE v3, Biguri et al.).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the projectors live in
``oracle.c`` (plain C, FP64) and the iterative solvers below are written out in
numpy FP64 in the order the textbook algorithms state them.

Parity pins live in ``tests/test_oracle_*.py``.  Functions and the passage they
follow:

* ``frames`` -- geometry of Sec. 2.4 and the Appendix B parameter table.
* ``forward(method="interp")`` -- Eq. 1, ray-driven trilinear sampling reading.
* ``forward(method="siddon")`` -- Eq. 1 with exact intersection lengths.
* ``backproject(method="matched")`` -- A^T of the interpolated projector
  (Eq. 4 uses A^T), scatter form.
* ``backproject(method="siddon")`` -- A^T of the Siddon projector.
* ``fdk_filter``, ``backproject(method="fdk")``, ``fdk`` -- FDK (Sec. 2.1,
  direct methods).
* ``fdk_variants`` -- FDK filter windows (ram-lak, shepp-logan, cosine,
  hamming, hann) in the frequency domain, Parker short-scan and Wang
  displaced-detector weights (Sec. 2.1, direct methods).
* ``sirt``, ``ossart`` -- Kaczmarz-type methods (Sec. 2.1) with the ordered
  subsets update (Sec. 2.2.2, Eq. 6).
* ``cgls`` -- CGLS (Sec. 2.1, Krylov methods; Hestenes and Stiefel).
* ``tv`` -- AwTV (the adaptive-weighted TV of Sec. 2.2's algorithm features,
  extended to volumes), its gradient, TV steepest descent and ASD-POCS /
  OS-ASD-POCS (Sec. 2.1, POCS methods; Sidky and Pan).
* ``lsqr`` -- LSQR (Sec. 2.1, Krylov methods; Paige and Saunders 1982).
* ``lsmr`` -- LSMR (Sec. 2.1, Krylov methods; Fong and Saunders 2011).
* ``mlem``, ``osem`` -- MLEM (Sec. 2.1, Eq. 5) and its ordered-subsets form
  (statistical methods; Hudson and Larkin), with either projector pair.
* ``conv`` -- the 3x3x3 convolutions of the learned-gradient network and
  their transposes (the learned use of the PyTorch wrappers, Sec. 2.8).
* ``learned`` -- one learned-gradient step x + Gamma(x, A^T(Ax - b)) and its
  gradient by the chain rule.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_DEFAULT_SOURCE",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geo(ctypes.Structure):
    _fields_ = [
        ("nVoxel", ctypes.c_int32 * 3),
        ("dVoxel", ctypes.c_double * 3),
        ("nDetector", ctypes.c_int32 * 2),
        ("dDetector", ctypes.c_double * 2),
        ("accuracy", ctypes.c_double),
        ("nAngles", ctypes.c_int32),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("DSO", ctypes.POINTER(ctypes.c_double)),
        ("DSD", ctypes.POINTER(ctypes.c_double)),
        ("offOrigin", ctypes.POINTER(ctypes.c_double)),
        ("offDetector", ctypes.POINTER(ctypes.c_double)),
        ("rotDetector", ctypes.POINTER(ctypes.c_double)),
        ("COR", ctypes.POINTER(ctypes.c_double)),
        ("parallel", ctypes.c_int32),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = ctypes.POINTER(_Geo)
            for name, args in {
                "or_frames": [G, _DP],
                "or_forward_interp": [G, _DP, _DP],
                "or_forward_interp_rays": [G, _DP, ctypes.c_long, _IP, _DP],
                "or_forward_siddon": [G, _DP, _DP],
                "or_forward_siddon_rays": [G, _DP, ctypes.c_long, _IP, _DP],
                "or_backproject_matched": [G, _DP, _DP],
                "or_backproject_matched_voxels": [G, _DP, ctypes.c_long, _IP, _DP],
                "or_backproject_siddon": [G, _DP, _DP],
                "or_fdk_filter": [G, _DP, _DP],
                "or_backproject_fdk": [G, _DP, _DP],
                "or_backproject_fdk_voxels": [G, _DP, ctypes.c_long, _IP, _DP],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.or_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().or_num_threads())


class _GeoHolder:
    """Keeps the FP64 per-angle arrays alive while C holds pointers to them."""

    def __init__(self, geo):
        n = int(geo.nAngles)
        self.arrays = {
            "angles": np.ascontiguousarray(np.asarray(geo.angles, np.float64).reshape(n, 3)),
            "DSO": np.ascontiguousarray(np.asarray(geo.DSO, np.float64).reshape(n)),
            "DSD": np.ascontiguousarray(np.asarray(geo.DSD, np.float64).reshape(n)),
            "offOrigin": np.ascontiguousarray(np.asarray(geo.offOrigin, np.float64).reshape(n, 3)),
            "offDetector": np.ascontiguousarray(np.asarray(geo.offDetector, np.float64).reshape(n, 2)),
            "rotDetector": np.ascontiguousarray(np.asarray(geo.rotDetector, np.float64).reshape(n, 3)),
            "COR": np.ascontiguousarray(np.asarray(geo.COR, np.float64).reshape(n)),
        }
        g = _Geo()
        g.nVoxel[:] = [int(v) for v in geo.nVoxel]
        g.dVoxel[:] = [float(v) for v in geo.dVoxel]
        g.nDetector[:] = [int(v) for v in geo.nDetector]
        g.dDetector[:] = [float(v) for v in geo.dDetector]
        g.accuracy = float(geo.accuracy)
        g.nAngles = n
        g.parallel = 1 if getattr(geo, "parallel", False) else 0
        for k, arr in self.arrays.items():
            setattr(g, k, arr.ctypes.data_as(_DP))
        self.g = g
        self.nx, self.ny, self.nz = (int(v) for v in geo.nVoxel)
        self.nu, self.nv = (int(v) for v in geo.nDetector)
        self.n = n

    @property
    def ref(self):
        return ctypes.byref(self.g)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def frames(geo) -> dict:
    """Per-angle source S, detector centre D, pixel axes eu, ev, normal n (mm,
    volume-centred frame), each of shape [nAngles, 3]."""
    h = _GeoHolder(geo)
    out = np.zeros((h.n, 15))
    _load().or_frames(h.ref, _dp(out))
    return {"S": out[:, 0:3], "D": out[:, 3:6], "eu": out[:, 6:9], "ev": out[:, 9:12], "n": out[:, 12:15]}


def pixel_centres(geo, a: int) -> np.ndarray:
    """Centres [nv, nu, 3] of the detector pixels of projection ``a``."""
    f = frames(geo)
    nu, nv = (int(v) for v in geo.nDetector)
    su = ((np.arange(nu) + 0.5) - 0.5 * nu) * geo.dDetector[0]
    sv = ((np.arange(nv) + 0.5) - 0.5 * nv) * geo.dDetector[1]
    return (f["D"][a][None, None, :] + su[None, :, None] * f["eu"][a][None, None, :]
            + sv[:, None, None] * f["ev"][a][None, None, :])


def forward(geo, vol, method: str = "interp") -> np.ndarray:
    """A x for the whole geometry: vol [nz, ny, nx] -> proj [nAngles, nv, nu]."""
    h = _GeoHolder(geo)
    v = _f64(vol).reshape(h.nz, h.ny, h.nx)
    out = np.zeros((h.n, h.nv, h.nu))
    fn = {"interp": _load().or_forward_interp, "siddon": _load().or_forward_siddon}[method]
    if h.n:
        fn(h.ref, _dp(v), _dp(out))
    return out


def forward_rays(geo, vol, rays, method: str = "interp") -> np.ndarray:
    """A x on selected rays only; ``rays`` is an int array [m, 3] of (angle, iv, iu)."""
    h = _GeoHolder(geo)
    v = _f64(vol).reshape(h.nz, h.ny, h.nx)
    r = np.ascontiguousarray(np.asarray(rays, np.int32).reshape(-1, 3))
    out = np.zeros(len(r))
    fn = {"interp": _load().or_forward_interp_rays, "siddon": _load().or_forward_siddon_rays}[method]
    fn(h.ref, _dp(v), len(r), r.ctypes.data_as(_IP), _dp(out))
    return out


def backproject(geo, proj, method: str = "matched") -> np.ndarray:
    """proj [nAngles, nv, nu] -> vol [nz, ny, nx].

    ``matched``: A^T of the interpolated projector; ``siddon``: A^T of the
    Siddon projector; ``fdk``: the FDK distance-weighted backprojection (the
    input is expected to be already filtered)."""
    h = _GeoHolder(geo)
    p = _f64(proj).reshape(h.n, h.nv, h.nu)
    out = np.zeros((h.nz, h.ny, h.nx))
    fn = {"matched": _load().or_backproject_matched, "siddon": _load().or_backproject_siddon,
          "fdk": _load().or_backproject_fdk}[method]
    if h.n:
        fn(h.ref, _dp(p), _dp(out))
    return out


def backproject_voxels(geo, proj, voxels, method: str = "matched") -> np.ndarray:
    """The backprojection at selected voxels only; ``voxels`` is [m, 3] of (ix, iy, iz)."""
    h = _GeoHolder(geo)
    p = _f64(proj).reshape(h.n, h.nv, h.nu)
    vx = np.ascontiguousarray(np.asarray(voxels, np.int32).reshape(-1, 3))
    out = np.zeros(len(vx))
    fn = {"matched": _load().or_backproject_matched_voxels, "fdk": _load().or_backproject_fdk_voxels}[method]
    fn(h.ref, _dp(p), len(vx), vx.ctypes.data_as(_IP), _dp(out))
    return out


def fdk_filter(geo, proj) -> np.ndarray:
    """Cosine pre-weight and Ram-Lak row filter of every projection."""
    h = _GeoHolder(geo)
    p = _f64(proj).reshape(h.n, h.nv, h.nu)
    out = np.zeros_like(p)
    if h.n:
        _load().or_fdk_filter(h.ref, _dp(p), _dp(out))
    return out


def fdk(geo, proj) -> np.ndarray:
    """FDK reconstruction: filter, then distance-weighted backprojection."""
    return backproject(geo, fdk_filter(geo, proj), "fdk")


# ---------------------------------------------------------------------------
# Iterative solvers (numpy FP64 over the C projectors).
# ---------------------------------------------------------------------------

def _safe_inv(a: np.ndarray) -> np.ndarray:
    out = np.zeros_like(a)
    nz = a != 0
    out[nz] = 1.0 / a[nz]
    return out


# A voxel whose column sum A^T 1 (over the angles of a block) is below this
# fraction of one full-weight sample's (delta = accuracy * min(dVoxel)) counts
# as unseen by the block: V = 0 for SIRT / OS-SART, and it keeps its value in
# MLEM / OS-EM.  Below it V A^T r is a 0/0 limit that the position rounding of
# any FP32 implementation decides (the reading of the column normalisation of
# the Kaczmarz-type and statistical methods, Sec. 2.1).
COVERAGE_MIN = 1e-3


def coverage_floor(geo) -> float:
    """COVERAGE_MIN times the interpolated projector's sample step (mm)."""
    acc = float(geo.accuracy) if geo.accuracy > 0 else 0.5
    return COVERAGE_MIN * acc * float(min(geo.dVoxel))


def _column_inv(a: np.ndarray, floor: float) -> np.ndarray:
    """1 / a where a >= floor, else 0."""
    out = np.zeros_like(a)
    seen = a >= floor
    out[seen] = 1.0 / a[seen]
    return out


def sirt_weights(geo):
    """W = 1/(A 1) per ray (0 where the sum is 0) and V = 1/(A^T 1) per
    voxel (0 where the sum is below coverage_floor)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    nu, nv = (int(v) for v in geo.nDetector)
    W = _safe_inv(forward(geo, np.ones((nz, ny, nx))))
    V = _column_inv(backproject(geo, np.ones((geo.nAngles, nv, nu)), "matched"), coverage_floor(geo))
    return W, V


def sirt(geo, b, niter: int, lam: float = 1.0, nonneg: bool = True, x0=None):
    """SIRT: x <- P(x + lam * V A^T W (b - A x)), P = clamp at 0 when
    ``nonneg`` (ART with non-negativity, Sec. 2.1).  Returns (x, residual
    norms ||A x_k - b|| after each iteration)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    W, V = sirt_weights(geo)
    hist = []
    for _ in range(niter):
        r = W * (b - forward(geo, x))
        x = x + lam * V * backproject(geo, r, "matched")
        if nonneg:
            x = np.maximum(x, 0.0)
        hist.append(float(np.linalg.norm(forward(geo, x) - b)))
    return x, np.array(hist)


_MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One step of SplitMix64 (Steele, Lea and Flood 2014): returns (new
    state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def block_orders(n_blocks: int, niter: int, order: str = "sequential", seed: int = 0):
    """The block order of every iteration: acquisition order, or (random)
    a Fisher-Yates shuffle from the last position down, position k - 1
    swapped with j = (next SplitMix64 output) mod k, one stream seeded once
    for the whole run (Sec. 2.2.2 lists random orders; this is the reading)."""
    state = int(seed) & _MASK64
    out = []
    for _ in range(niter):
        perm = list(range(n_blocks))
        if order == "random":
            for k in range(n_blocks, 1, -1):
                state, r = splitmix64(state)
                j = r % k
                perm[k - 1], perm[j] = perm[j], perm[k - 1]
        elif order != "sequential":
            raise ValueError(order)
        out.append(perm)
    return out


def subsets(n_angles: int, blocksize: int):
    """Contiguous angle blocks of ``blocksize`` in acquisition order; the last
    block holds the remainder."""
    return [np.arange(s, min(s + blocksize, n_angles)) for s in range(0, n_angles, blocksize)]


def ossart(geo, b, niter: int, blocksize: int, lam: float = 1.0, nonneg: bool = True, x0=None,
           order: str = "sequential", seed: int = 0):
    """OS-SART: for each block s in order, x <- P(x + lam V_s A_s^T W_s (b_s
    - A_s x)) (Sec. 2.2.2, Eq. 6 with the SART row/column weights).  One
    iteration visits every block once, in acquisition order or in the
    seeded random order of ``block_orders``.  Returns (x, residual
    history)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    blocks = subsets(geo.nAngles, blocksize)
    sub = [geo.subset(idx) for idx in blocks]
    weights = [sirt_weights(g) for g in sub]
    hist = []
    for perm in block_orders(len(blocks), niter, order, seed):
        for q in perm:
            idx, g, (W, V) = blocks[q], sub[q], weights[q]
            r = W * (b[idx] - forward(g, x))
            x = x + lam * V * backproject(g, r, "matched")
            if nonneg:
                x = np.maximum(x, 0.0)
        hist.append(float(np.linalg.norm(forward(geo, x) - b)))
    return x, np.array(hist)


def cgls(geo, b, niter: int, x0=None):
    """CGLS on min ||A x - b|| (Hestenes-Stiefel, applied to the normal
    equations without forming them):
        r = b - A x, s = A^T r, p = s, gamma = ||s||^2
        repeat: q = A p; alpha = gamma / ||q||^2; x += alpha p; r -= alpha q
                s = A^T r; gamma' = ||s||^2; p = s + (gamma'/gamma) p
    Returns (x, ||r_k|| after each iteration)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    r = b - forward(geo, x)
    s = backproject(geo, r, "matched")
    p = s.copy()
    gamma = float(np.sum(s * s))
    hist = []
    for _ in range(niter):
        q = forward(geo, p)
        qq = float(np.sum(q * q))
        if qq == 0.0 or gamma == 0.0:
            hist.append(float(np.linalg.norm(r)))
            continue
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = backproject(geo, r, "matched")
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        hist.append(float(np.linalg.norm(r)))
    return x, np.array(hist)


# ---------------------------------------------------------------------------
# Statistical methods (Sec. 2.1): MLEM (Eq. 5) and OS-EM.
# ---------------------------------------------------------------------------

_EM_PAIRS = {"interp": ("interp", "matched"), "siddon": ("siddon", "siddon")}


def _safe_div(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    out = np.zeros_like(num)
    nz = den != 0
    out[nz] = num[nz] / den[nz]
    return out


def osem(geo, b, niter: int, blocksize: int, x0=None, method: str = "interp", order: str = "sequential",
         seed: int = 0):
    """OS-EM (Hudson and Larkin 1994): for each block s of consecutive angles
    in acquisition order,
        x <- x / (A_s^T 1) * A_s^T (b_s / (A_s x)),
    the MLEM update of Eq. 5 restricted to the block (Eq. 5's normalisation
    is the backprojection of ones, the sensitivity of each voxel).  A ray
    with A_s x = 0 contributes 0; a voxel the block does not see (A_s^T 1
    below coverage_floor) keeps its value.  x0 = 1 unless given.  ``method``
    picks the pair (A, A^T): interpolated + matched, or Siddon + its
    transpose.  Returns (x, ||A x_k - b|| after each iteration)."""
    fp, bp = _EM_PAIRS[method]
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b).reshape(geo.proj_shape)
    x = np.ones((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    blocks = subsets(geo.nAngles, blocksize)
    sub = [geo.subset(idx) for idx in blocks]
    sens = [backproject(g, np.ones(g.proj_shape), bp) for g in sub]
    floor = coverage_floor(geo)
    hist = []
    for perm in block_orders(len(blocks), niter, order, seed):
        for q in perm:
            idx, g, sv = blocks[q], sub[q], sens[q]
            ratio = _safe_div(b[idx], forward(g, x, fp))
            x = np.where(sv >= floor, x * _column_inv(sv, floor) * backproject(g, ratio, bp), x)
        hist.append(float(np.linalg.norm(forward(geo, x, fp) - b)))
    return x, np.array(hist)


def mlem(geo, b, niter: int, x0=None, method: str = "interp"):
    """MLEM (Eq. 5): OS-EM with one block holding every angle."""
    return osem(geo, b, niter, max(int(geo.nAngles), 1), x0, method)


def poisson_loglik(geo, x, b, method: str = "interp") -> float:
    """sum_i b_i log (A x)_i - (A x)_i over rays with (A x)_i > 0 (the
    objective MLEM increases; constant terms dropped)."""
    y = forward(geo, x, _EM_PAIRS[method][0])
    b = _f64(b).reshape(y.shape)
    m = y > 0
    return float(np.sum(b[m] * np.log(y[m]) - y[m]))


# ---------------------------------------------------------------------------
# LSQR (Sec. 2.1, Krylov methods; Paige and Saunders 1982).
# ---------------------------------------------------------------------------

def lsqr(geo, b, niter: int, x0=None):
    """LSQR on min ||A x - b|| (A interpolated, A^T matched), the steps of
    Paige and Saunders' algorithm:
        beta u = r0 = b - A x0,  alpha v = A^T u,  w = v,
        phibar = beta,  rhobar = alpha
        repeat: beta u = A v - alpha u;   alpha v = A^T u - beta v
                rho = sqrt(rhobar^2 + beta^2); c = rhobar/rho; s = beta/rho
                theta = s alpha; rhobar = -c alpha; phi = c phibar; phibar = s phibar
                x += (phi/rho) w;  w = v - (theta/rho) w
    A zero beta or alpha ends the recurrence (x is then exact).  Returns (x,
    phibar after each iteration, which equals ||b - A x_k||)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    u = b - forward(geo, x)
    beta = float(np.linalg.norm(u))
    u = u / beta if beta > 0 else u
    v = backproject(geo, u, "matched")
    alpha = float(np.linalg.norm(v))
    v = v / alpha if alpha > 0 else v
    w = v.copy()
    phibar, rhobar = beta, alpha
    hist = []
    for _ in range(niter):
        if beta == 0.0 or alpha == 0.0:
            hist.append(phibar)
            continue
        u = forward(geo, v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0:
            u = u / beta
        v = backproject(geo, u, "matched") - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0:
            v = v / alpha
        rho = math.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        hist.append(phibar)
    return x, np.array(hist)


def lsmr(geo, b, niter: int, x0=None):
    """LSMR on min ||A x - b|| without damping, the steps of Fong and
    Saunders' algorithm (the same bidiagonalisation as LSQR, then two plane
    rotations per iteration so that ||A^T r_k|| is minimised over the
    Krylov space):
        beta u = b - A x0, alpha v = A^T u; alphabar = alpha, zetabar = alpha beta,
        rho = 1, rhobar = 1, cbar = 1, sbar = 0, h = v, hbar = 0
        repeat: beta u = A v - alpha u;  alpha' v = A^T u - beta v
                rho_old = rho; rho = sqrt(alphabar^2 + beta^2)
                c = alphabar/rho; s = beta/rho; theta = s alpha'; alphabar = c alpha'
                rhobar_old = rhobar; thetabar = sbar rho
                rhobar = sqrt((cbar rho)^2 + theta^2)
                cbar = cbar rho / rhobar; sbar = theta / rhobar
                zeta = cbar zetabar; zetabar = -sbar zetabar
                hbar = h - (thetabar rho / (rho_old rhobar_old)) hbar
                x += (zeta / (rho rhobar)) hbar
                h = v - (theta / rho) h;  alpha = alpha'
    Returns (x, ||b - A x_k|| after each iteration, computed with one
    extra projection)."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    b = _f64(b)
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0).copy()
    u = b - forward(geo, x)
    beta = float(np.linalg.norm(u))
    u = u / beta if beta > 0 else u
    v = backproject(geo, u, "matched")
    alpha = float(np.linalg.norm(v))
    v = v / alpha if alpha > 0 else v
    alphabar, zetabar = alpha, alpha * beta
    rho, rhobar, cbar, sbar = 1.0, 1.0, 1.0, 0.0
    h = v.copy()
    hbar = np.zeros_like(x)
    hist = []
    for _ in range(niter):
        if alpha * beta == 0.0:
            hist.append(float(np.linalg.norm(b - forward(geo, x))))
            continue
        u = forward(geo, v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0:
            u = u / beta
        v = backproject(geo, u, "matched") - beta * v
        alpha_new = float(np.linalg.norm(v))
        if alpha_new > 0:
            v = v / alpha_new
        rho_old = rho
        rho = math.hypot(alphabar, beta)
        c, s = alphabar / rho, beta / rho
        theta = s * alpha_new
        alphabar = c * alpha_new
        rhobar_old = rhobar
        thetabar = sbar * rho
        rhobar = math.hypot(cbar * rho, theta)
        cbar, sbar = cbar * rho / rhobar, theta / rhobar
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar
        hbar = h - (thetabar * rho / (rho_old * rhobar_old)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta / rho) * h
        alpha = alpha_new
        hist.append(float(np.linalg.norm(b - forward(geo, x))))
    return x, np.array(hist)
