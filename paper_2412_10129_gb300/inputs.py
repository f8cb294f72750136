"""Seeded synthetic inputs: geometries, phantoms, noise.

This module holds none of the reconstruction arithmetic.  It describes a
scan with the parameters of the TIGRE geometry table (Appendix B: DSD, DSO,
nVoxel, dVoxel, offOrigin, COR, ZYZ angles, nDetector, dDetector,
offDetector, rotDetector), expanded to one value per projection because
every parameter except the sizes may vary per projection (Sec. 2.4), and it
draws seeded phantoms and noise.  Both the CUDA path and the CPU oracle take
their inputs from here; neither imports the other.

Phantom recipe (ellipsoids of the synthetic workloads):
  * centres uniform in a ball of radius 0.8 R, R = half the smallest
    in-plane volume extent;
  * semi-axes uniform in a range (4-24 mm for the 64^3 case, 2-12 % of R
    for the larger volumes);
  * orientation from a uniform random unit quaternion (Shoemake 1992);
  * attenuation uniform in [0.01, 0.05] /mm, additive where ellipsoids overlap;
  * voxelised by point sampling at voxel centres.
Noise: counts ~ Poisson(I0 exp(-b)), b_noisy = -ln(max(counts, 1) / I0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Geometry:
    """Cone-beam scan description.  Sizes are fixed; the rest is per angle."""

    nVoxel: tuple  # (nx, ny, nz)
    dVoxel: tuple  # mm (dx, dy, dz)
    nDetector: tuple  # (nu columns, nv rows)
    dDetector: tuple  # mm (du, dv)
    angles: np.ndarray  # [nA, 3] ZYZ Euler (z1, y1, z2), rad
    DSO: np.ndarray  # [nA] mm
    DSD: np.ndarray  # [nA] mm
    offOrigin: np.ndarray  # [nA, 3] mm
    offDetector: np.ndarray  # [nA, 2] mm (u, v)
    rotDetector: np.ndarray  # [nA, 3] rad (phi, theta, psi)
    COR: np.ndarray  # [nA] mm
    accuracy: float = 0.5  # interpolated-projector step, in units of min(dVoxel)
    parallel: bool = False  # parallel beam: every ray along D - S, through its own pixel

    @property
    def nAngles(self) -> int:
        return int(np.asarray(self.angles).shape[0])

    @property
    def vol_shape(self) -> tuple:
        nx, ny, nz = self.nVoxel
        return (int(nz), int(ny), int(nx))

    @property
    def proj_shape(self) -> tuple:
        nu, nv = self.nDetector
        return (self.nAngles, int(nv), int(nu))

    def subset(self, idx) -> "Geometry":
        idx = np.asarray(idx, dtype=np.int64)
        return dataclasses.replace(
            self,
            angles=np.asarray(self.angles)[idx], DSO=np.asarray(self.DSO)[idx],
            DSD=np.asarray(self.DSD)[idx], offOrigin=np.asarray(self.offOrigin)[idx],
            offDetector=np.asarray(self.offDetector)[idx],
            rotDetector=np.asarray(self.rotDetector)[idx], COR=np.asarray(self.COR)[idx])

    def with_volume(self, nVoxel, dVoxel) -> "Geometry":
        return dataclasses.replace(self, nVoxel=tuple(int(v) for v in nVoxel),
                                   dVoxel=tuple(float(v) for v in dVoxel))


def circular_geometry(nVoxel, dVoxel, nDetector, dDetector, n_angles: int, DSO: float, DSD: float,
                      arc: float = 2 * math.pi, accuracy: float = 0.5, start: float = 0.0) -> Geometry:
    """Circular orbit: angles (start + a * arc / nA, 0, 0), no offsets."""
    n = int(n_angles)
    ang = np.zeros((n, 3))
    ang[:, 0] = start + np.arange(n) * (arc / max(n, 1))
    return Geometry(
        nVoxel=tuple(int(v) for v in nVoxel), dVoxel=tuple(float(v) for v in dVoxel),
        nDetector=tuple(int(v) for v in nDetector), dDetector=tuple(float(v) for v in dDetector),
        angles=ang, DSO=np.full(n, float(DSO)), DSD=np.full(n, float(DSD)),
        offOrigin=np.zeros((n, 3)), offDetector=np.zeros((n, 2)), rotDetector=np.zeros((n, 3)),
        COR=np.zeros(n), accuracy=float(accuracy))


def parallel_geometry(nVoxel, dVoxel, nDetector, dDetector, n_angles: int, arc: float = math.pi,
                      DSO: float = 1000.0, DSD: float = 1536.0) -> Geometry:
    """Parallel-beam scan (synchrotron shapes): angles start + a * arc / nA;
    DSO and DSD only place the plane the rays start from and the detector."""
    g = circular_geometry(nVoxel, dVoxel, nDetector, dDetector, n_angles, DSO, DSD, arc=arc)
    return dataclasses.replace(g, parallel=True)


def jitter_geometry(geo: Geometry, seed: int, det_offset_px: float = 2.0, tilt_deg: float = 0.5,
                    source_mm: float = 0.5) -> Geometry:
    """Per-angle perturbations of the micro-CT workload: detector offset
    uniform in +-det_offset_px pixels (u and v), in-plane detector tilt (psi)
    uniform in +-tilt_deg, and source jitter uniform in +-source_mm along the
    source-axis line (DSO and DSD change together, so only the source moves)."""
    rng = np.random.default_rng(seed)
    n = geo.nAngles
    off = rng.uniform(-det_offset_px, det_offset_px, size=(n, 2)) * np.asarray(geo.dDetector)[None, :]
    rot = np.zeros((n, 3))
    rot[:, 2] = np.deg2rad(rng.uniform(-tilt_deg, tilt_deg, size=n))
    ds = rng.uniform(-source_mm, source_mm, size=n)
    return dataclasses.replace(geo, offDetector=off, rotDetector=rot,
                               DSO=np.asarray(geo.DSO) + ds, DSD=np.asarray(geo.DSD) + ds)


def random_geometry(nVoxel, dVoxel, nDetector, dDetector, n_angles: int, seed: int,
                    DSO: float = 1000.0, DSD: float = 1536.0) -> Geometry:
    """Arbitrary per-angle geometry for edge-case tests: ZYZ angles, origin
    and detector offsets, detector rotations and COR all drawn per angle."""
    rng = np.random.default_rng(seed)
    n = int(n_angles)
    g = circular_geometry(nVoxel, dVoxel, nDetector, dDetector, n, DSO, DSD)
    ext = np.asarray(nVoxel) * np.asarray(dVoxel)
    g.angles = np.stack([rng.uniform(0, 2 * math.pi, n), rng.uniform(-0.3, 0.3, n),
                         rng.uniform(-0.5, 0.5, n)], axis=1)
    g.offOrigin = rng.uniform(-0.05, 0.05, size=(n, 3)) * ext[None, :]
    g.offDetector = rng.uniform(-3, 3, size=(n, 2)) * np.asarray(dDetector)[None, :]
    g.rotDetector = rng.uniform(-0.05, 0.05, size=(n, 3))
    g.COR = rng.uniform(-1.0, 1.0, size=n)
    g.DSO = DSO + rng.uniform(-5, 5, size=n)
    g.DSD = DSD + rng.uniform(-5, 5, size=n)
    return g


# ---------------------------------------------------------------------------
# Workloads (sizes of the synthetic configurations).
# ---------------------------------------------------------------------------

def config_small() -> Geometry:
    """64^3 at 1 mm, DSO 1000, DSD 1536, 128x128 detector at 0.8 mm, 100 angles over 2 pi."""
    return circular_geometry((64, 64, 64), (1.0, 1.0, 1.0), (128, 128), (0.8, 0.8), 100, 1000.0, 1536.0)


def config_clinical() -> Geometry:
    """512^3 at 0.5 mm, 720 angles over 2 pi, 768 rows x 1024 columns at 0.4 mm."""
    return circular_geometry((512, 512, 512), (0.5, 0.5, 0.5), (1024, 768), (0.4, 0.4), 720, 1000.0, 1536.0)


def config_micro(seed: int = 3) -> Geometry:
    """1024^3 at 0.125 mm, 1600 angles, 1024^2 detector at 0.2 mm, per-angle jitter."""
    g = circular_geometry((1024, 1024, 1024), (0.125,) * 3, (1024, 1024), (0.2, 0.2), 1600, 1000.0, 1536.0)
    return jitter_geometry(g, seed)


def config_autograd() -> Geometry:
    """128^3 at 1 mm, 180 angles, 192^2 detector at 1.2 mm (used with a batch of 16)."""
    return circular_geometry((128, 128, 128), (1.0,) * 3, (192, 192), (1.2, 1.2), 180, 1000.0, 1536.0)


def config_learned(n: int = 256, n_angles: int = 60) -> Geometry:
    """Sparse-view learned-reconstruction workload: a 256 mm cube as n^3
    voxels (1 mm at n = 256), 60 angles over 2 pi, a (2n)^2 detector whose
    pixels (0.8 mm at n = 256) scale with the voxels, so that smaller n is the
    same scan at a coarser grid."""
    s = 256.0 / n
    return circular_geometry((n, n, n), (s,) * 3, (2 * n, 2 * n), (0.8 * s, 0.8 * s), n_angles, 1000.0, 1536.0)


# ---------------------------------------------------------------------------
# Phantoms.
# ---------------------------------------------------------------------------

def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake 1992), [n, 4] as (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    return np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                     a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)


def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_ellipsoids(geo: Geometry, n: int, seed: int, semi_axes=None, mu=(0.01, 0.05)) -> np.ndarray:
    """[n, 16] rows: centre (3, mm), semi-axes (3, mm), rotation matrix (9,
    row-major, columns = ellipsoid axes in the volume frame), attenuation."""
    rng = np.random.default_rng(seed)
    ext = np.asarray(geo.nVoxel, float) * np.asarray(geo.dVoxel, float)
    R = 0.5 * min(ext[0], ext[1])
    if semi_axes is None:
        semi_axes = (4.0, 24.0) if R <= 40 else (0.02 * R, 0.12 * R)
    # uniform in a ball of radius 0.8 R (direction x radius^(1/3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = 0.8 * R * rng.random(n) ** (1.0 / 3.0)
    centres = d * rad[:, None]
    centres[:, 2] = np.clip(centres[:, 2], -0.5 * ext[2], 0.5 * ext[2])
    axes = rng.uniform(semi_axes[0], semi_axes[1], size=(n, 3))
    quats = random_quaternions(rng, n)
    mus = rng.uniform(mu[0], mu[1], size=n)
    out = np.zeros((n, 16))
    out[:, 0:3] = centres
    out[:, 3:6] = axes
    for i in range(n):
        out[i, 6:15] = quat_to_matrix(quats[i]).reshape(-1)
    out[:, 15] = mus
    return out


def voxel_centres_1d(n: int, d: float) -> np.ndarray:
    return ((np.arange(n) + 0.5) - 0.5 * n) * d


def voxelize_ellipsoids(geo: Geometry, ell: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Point-sample the additive ellipsoid phantom at the voxel centres."""
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    dx, dy, dz = (float(v) for v in geo.dVoxel)
    cx, cy, cz = voxel_centres_1d(nx, dx), voxel_centres_1d(ny, dy), voxel_centres_1d(nz, dz)
    vol = np.zeros((nz, ny, nx), dtype=np.float32)
    for e in ell:
        c, a, Rm, mu = e[0:3], e[3:6], e[6:15].reshape(3, 3), e[15]
        r = float(a.max())
        sl = []
        for centres, ci in ((cx, c[0]), (cy, c[1]), (cz, c[2])):
            lo = np.searchsorted(centres, ci - r, side="left")
            hi = np.searchsorted(centres, ci + r, side="right")
            sl.append((lo, hi))
        (x0, x1), (y0, y1), (z0, z1) = sl
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        X = cx[x0:x1][None, None, :] - c[0]
        Y = cy[y0:y1][None, :, None] - c[1]
        Z = cz[z0:z1][:, None, None] - c[2]
        # coordinates in the ellipsoid frame: R^T (p - c)
        q0 = Rm[0, 0] * X + Rm[1, 0] * Y + Rm[2, 0] * Z
        q1 = Rm[0, 1] * X + Rm[1, 1] * Y + Rm[2, 1] * Z
        q2 = Rm[0, 2] * X + Rm[1, 2] * Y + Rm[2, 2] * Z
        inside = (q0 / a[0]) ** 2 + (q1 / a[1]) ** 2 + (q2 / a[2]) ** 2 <= 1.0
        vol[z0:z1, y0:y1, x0:x1] += (mu * inside).astype(np.float32)
    return vol.astype(dtype, copy=False)


def ellipsoid_phantom(geo: Geometry, n: int, seed: int, **kw) -> np.ndarray:
    return voxelize_ellipsoids(geo, random_ellipsoids(geo, n, seed, **kw))


def learned_phantom(geo: Geometry, seed: int, n: int = 20) -> np.ndarray:
    """Phantom of the learned-reconstruction workload: n ellipsoids with
    semi-axes 5-30 % of R (large enough to stay several voxels wide on the
    coarse training grids), otherwise the recipe above."""
    ext = np.asarray(geo.nVoxel, float) * np.asarray(geo.dVoxel, float)
    R = 0.5 * min(ext[0], ext[1])
    return voxelize_ellipsoids(geo, random_ellipsoids(geo, n, seed, semi_axes=(0.05 * R, 0.3 * R)))


def porous_cylinder(geo: Geometry, seed: int, n_pores: int = 500, mu: float = 0.03) -> np.ndarray:
    """Cylinder along z (radius 0.45 R, height 0.8 of the z extent) minus
    seeded spherical pores (radius 1-3 % of R) set to zero."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in geo.nVoxel)
    dx, dy, dz = (float(v) for v in geo.dVoxel)
    R = 0.5 * min(nx * dx, ny * dy)
    H = 0.8 * nz * dz
    cx, cy, cz = voxel_centres_1d(nx, dx), voxel_centres_1d(ny, dy), voxel_centres_1d(nz, dz)
    disk = (cx[None, :] ** 2 + cy[:, None] ** 2) <= (0.45 * R) ** 2
    slab = np.abs(cz) <= 0.5 * H
    vol = (slab[:, None, None] & disk[None, :, :]).astype(np.float32) * mu
    rr = 0.45 * R * np.sqrt(rng.random(n_pores))
    th = rng.uniform(0, 2 * np.pi, n_pores)
    pz = rng.uniform(-0.5 * H, 0.5 * H, n_pores)
    prad = rng.uniform(0.01 * R, 0.03 * R, n_pores)
    for x, y, z, r in zip(rr * np.cos(th), rr * np.sin(th), pz, prad):
        xs = slice(np.searchsorted(cx, x - r), np.searchsorted(cx, x + r, side="right"))
        ys = slice(np.searchsorted(cy, y - r), np.searchsorted(cy, y + r, side="right"))
        zs = slice(np.searchsorted(cz, z - r), np.searchsorted(cz, z + r, side="right"))
        m = ((cx[xs][None, None, :] - x) ** 2 + (cy[ys][None, :, None] - y) ** 2
             + (cz[zs][:, None, None] - z) ** 2) <= r * r
        sub = vol[zs, ys, xs]
        sub[m] = 0.0
    return vol


def micro_phantom(geo: Geometry, seed: int, n_ellipsoids: int = 200) -> np.ndarray:
    """Phantom of the micro-CT workload: n seeded ellipsoids (the recipe
    above) added to a porous cylinder drawn from the next seed."""
    vol = ellipsoid_phantom(geo, n_ellipsoids, seed)
    vol += porous_cylinder(geo, seed + 1)
    return vol


def random_volume(geo: Geometry, seed: int, dtype=np.float32) -> np.ndarray:
    """Uniform [0, 1) voxel values (white-noise volume for operator checks)."""
    return np.random.default_rng(seed).random(geo.vol_shape).astype(dtype)


def random_projections(geo: Geometry, seed: int, dtype=np.float32) -> np.ndarray:
    """Uniform [0, 1) projection values."""
    return np.random.default_rng(seed).random(geo.proj_shape).astype(dtype)


def poisson_noise_device(b, I0: float, seed: int):
    """poisson_noise for a torch tensor on its own device (a seeded torch
    generator there; a different stream of numbers than the numpy version)."""
    import torch
    gen = torch.Generator(device=b.device).manual_seed(int(seed))
    counts = torch.poisson(I0 * torch.exp(-b.double()), generator=gen)
    return (-torch.log(torch.clamp(counts, min=1.0) / I0)).to(b.dtype)


def poisson_noise(b: np.ndarray, I0: float, seed: int) -> np.ndarray:
    """Transmission noise on line integrals b: counts ~ Poisson(I0 e^-b),
    returned as -ln(max(counts, 1) / I0)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(I0 * np.exp(-np.asarray(b, np.float64)))
    return (-np.log(np.maximum(counts, 1) / I0)).astype(np.asarray(b).dtype)
