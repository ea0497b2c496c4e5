"""Seeded synthetic inputs for FB-LISA workloads: geometries, phantoms, noise.

This module is the one place both the FP64 oracle (``oracle/``) and the CUDA
library's callers (tests, ``bench.py``) draw their inputs from.  It holds none
of the method's arithmetic: no projector, no objective, no line search, no
batch sampling.  Everything here is a description of an input (a geometry) or
a seeded random draw (phantom, noise); the method's own random numbers (the
mini-batch permutations) are generated inside each implementation.

Shapes follow the paper's regime (Sec. 3): circular cone-beam orbit, uniform
angles over [0, 2*pi), whole 2D projections as the batch unit, attenuation
values in [0, 1].  The paper's walnut data (Sec. 3, "Dataset") is not
available; seeded ellipsoid phantoms stand in for it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

__all__ = [
    "Geometry", "Workload", "WORKLOADS", "ellipsoids", "phantom", "gaussian_noise",
    "poisson_log_data", "small_geometry",
]


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Circular cone-beam geometry; lengths in mm, volume centred on the axis.

    Volume ``nx*ny*nz`` voxels of size ``vx, vy, vz``; ``n_views`` views at
    ``angles`` (None: 2*pi*i/n_views); source-to-origin ``sod``;
    source-to-detector ``sdd``; flat detector of ``nu*nv`` pixels of size
    ``du*dv``.
    """
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    n_views: int
    sod: float
    sdd: float
    nu: int
    nv: int
    du: float
    dv: float
    angles: Optional[Tuple[float, ...]] = None

    @property
    def vol_shape(self) -> Tuple[int, int, int]:
        return (self.nz, self.ny, self.nx)

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def view_shape(self) -> Tuple[int, int]:
        return (self.nv, self.nu)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: geometry, phantom recipe, noise, run plan."""
    name: str
    geom: Geometry
    n_ellipsoids: int
    inclusions: int
    texture_std: float
    noise: str            # "gaussian" (sigma = rel * max) or "poisson"
    noise_rel: float
    I0: float
    N0: int
    epochs: int
    seed_phantom: int
    seed_noise: int
    seed_batches: int
    mu: float = 1.0


def _cube(n: int, n_views: int, det: int, voxel: float = 1.0) -> Geometry:
    return Geometry(nx=n, ny=n, nz=n, vx=voxel, vy=voxel, vz=voxel, n_views=n_views,
                    sod=1000.0, sdd=1500.0, nu=det, nv=det, du=1.5 * voxel, dv=1.5 * voxel)


# The five synthetic workloads.  Detector pixels are 1.5 mm and SDD/SOD = 1.5,
# so the detector (in pixels) is 1.5x the volume edge (in voxels).
WORKLOADS: Dict[str, Workload] = {
    "c1_64": Workload("c1_64", _cube(64, 90, 96), 10, 0, 0.0, "gaussian", 0.01, 0.0,
                      N0=10, epochs=5, seed_phantom=1001, seed_noise=2001, seed_batches=3001),
    "c2_256": Workload("c2_256", _cube(256, 360, 384), 40, 8, 0.0, "poisson", 0.0, 1e4,
                       N0=20, epochs=20, seed_phantom=1002, seed_noise=2002, seed_batches=3002),
    "c3_512": Workload("c3_512", _cube(512, 720, 768), 100, 0, 0.02, "gaussian", 0.01, 0.0,
                       N0=40, epochs=10, seed_phantom=1003, seed_noise=2003, seed_batches=3003),
    # the paper's three walnut cases (Sec. 3) in shape only: 560^3, 36 / 36 / 72
    # views, N_0 = 8, mu = 2 / 1 / 1, case 1 noise-free and cases 2-3 with
    # Gaussian noise of 2% of the maximum (the paper's "2% variance" read as that)
    "case1_560": Workload("case1_560", _cube(560, 36, 840), 60, 0, 0.02, "gaussian", 0.0, 0.0,
                          N0=8, epochs=0, seed_phantom=1301, seed_noise=2301, seed_batches=3301, mu=2.0),
    "case2_560": Workload("case2_560", _cube(560, 36, 840), 60, 0, 0.02, "gaussian", 0.02, 0.0,
                          N0=8, epochs=0, seed_phantom=1302, seed_noise=2302, seed_batches=3302, mu=1.0),
    "case3_560": Workload("case3_560", _cube(560, 72, 840), 60, 0, 0.02, "gaussian", 0.02, 0.0,
                          N0=8, epochs=0, seed_phantom=1303, seed_noise=2303, seed_batches=3303, mu=1.0),
    # a profiling-sized case: volume larger than L2, a few GB on the device in all
    "p384": Workload("p384", _cube(384, 120, 576), 40, 0, 0.0, "gaussian", 0.01, 0.0,
                     N0=20, epochs=2, seed_phantom=1009, seed_noise=2009, seed_batches=3009),
    # 1024 voxels of 1 mm would not fit between source and detector (circumradius
    # 724 mm > SDD - SOD = 500 mm): the 512^3 geometry at twice the resolution
    "c5b_1024": Workload("c5b_1024", _cube(1024, 1440, 1536, voxel=0.5), 100, 0, 0.0, "gaussian", 0.01,
                         0.0, N0=60, epochs=10, seed_phantom=1005, seed_noise=2005,
                         seed_batches=3005),
}


def batched_small_workloads() -> List[Workload]:
    """16 small uneven volumes, the batched workload scaled down by 4 in edge
    (N_i = round(24 + 56 i/15), 30 + 6 i views, detector ceil(1.5 N_i)^2):
    the regime where one volume alone cannot fill the GPU."""
    out = []
    for i in range(16):
        n = int(round(24 + 56 * i / 15))
        views = 30 + 6 * i
        det = int(math.ceil(1.5 * n))
        out.append(Workload(f"c5s_{i}", _cube(n, views, det), 8, 0, 0.0, "gaussian", 0.01, 0.0,
                            N0=int(math.ceil(views / 12)), epochs=2, seed_phantom=1200 + i,
                            seed_noise=2200 + i, seed_batches=3200 + i))
    return out


def batched_workloads() -> List[Workload]:
    """The 16 uneven volumes of the batched workload: N_i = round(96 + 224 i/15),
    120 + 24 i views, detector ceil(1.5 N_i) square."""
    out = []
    for i in range(16):
        n = int(round(96 + 224 * i / 15))
        views = 120 + 24 * i
        det = int(math.ceil(1.5 * n))
        out.append(Workload(f"c5a_{i}", _cube(n, views, det), 20, 0, 0.0, "gaussian", 0.01, 0.0,
                            N0=int(math.ceil(views / 12)), epochs=2, seed_phantom=1100 + i,
                            seed_noise=2100 + i, seed_batches=3100 + i))
    return out


def small_geometry(nx=40, ny=36, nz=28, n_views=24, nu=70, nv=50, v=1.0, du=1.5, dv=1.5,
                   sod=1000.0, sdd=1500.0, angles=None) -> Geometry:
    """A small anisotropic geometry with ragged sizes for parity tests."""
    return Geometry(nx=nx, ny=ny, nz=nz, vx=v, vy=v, vz=v, n_views=n_views, sod=sod, sdd=sdd,
                    nu=nu, nv=nv, du=du, dv=dv,
                    angles=None if angles is None else tuple(float(a) for a in angles))


def _rot_zyz(a: float, b: float, c: float) -> np.ndarray:
    def rz(t):
        return np.array([[math.cos(t), -math.sin(t), 0.0], [math.sin(t), math.cos(t), 0.0],
                         [0.0, 0.0, 1.0]])

    def ry(t):
        return np.array([[math.cos(t), 0.0, math.sin(t)], [0.0, 1.0, 0.0],
                         [-math.sin(t), 0.0, math.cos(t)]])
    return rz(a) @ ry(b) @ rz(c)


def ellipsoids(geom: Geometry, n: int, seed: int, inclusions: int = 0):
    """Seeded ellipsoid list: (centre[3] mm, semi-axes[3] mm, R (3x3), value, mode).

    Ellipsoid 0 is the background (semi-axes 0.85 x half extent, value 0.5).
    The others have centres uniform in the ball of radius 0.5 x half extent,
    semi-axes uniform in [0.05, 0.35] x half extent, uniform ZYZ Euler angles
    and additive values uniform in [-0.3, 0.4].  ``inclusions`` extra small
    ellipsoids (semi-axes 1-3 voxels) set their voxels to 1.0 (mode "set").
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    half = np.array([geom.nx * geom.vx, geom.ny * geom.vy, geom.nz * geom.vz]) / 2.0
    h = float(half.min())
    out = [(np.zeros(3), 0.85 * half, np.eye(3), 0.5, "add")]
    for _ in range(max(0, n - 1)):
        while True:
            c = rng.uniform(-1.0, 1.0, 3)
            if np.dot(c, c) <= 1.0:
                break
        centre = 0.5 * h * c
        axes = rng.uniform(0.05, 0.35, 3) * h
        R = _rot_zyz(*rng.uniform(0.0, 2.0 * math.pi, 3))
        val = float(rng.uniform(-0.3, 0.4))
        out.append((centre, axes, R, val, "add"))
    vmin = min(geom.vx, geom.vy, geom.vz)
    for _ in range(inclusions):
        while True:
            c = rng.uniform(-1.0, 1.0, 3)
            if np.dot(c, c) <= 1.0:
                break
        centre = 0.6 * h * c
        axes = rng.uniform(1.0, 3.0, 3) * vmin
        R = _rot_zyz(*rng.uniform(0.0, 2.0 * math.pi, 3))
        out.append((centre, axes, R, 1.0, "set"))
    return out


def _voxel_axes(geom: Geometry):
    x = (np.arange(geom.nx) - 0.5 * (geom.nx - 1)) * geom.vx
    y = (np.arange(geom.ny) - 0.5 * (geom.ny - 1)) * geom.vy
    z = (np.arange(geom.nz) - 0.5 * (geom.nz - 1)) * geom.vz
    return x, y, z


def _box_blur(f: np.ndarray, radius: int) -> np.ndarray:
    """Separable box filter of width 2*radius+1, zero outside (cumulative sums)."""
    for ax in range(3):
        n = f.shape[ax]
        pad = [(0, 0)] * 3
        pad[ax] = (radius + 1, radius)
        c = np.cumsum(np.pad(f, pad), axis=ax)
        hi = np.take(c, np.arange(2 * radius + 1, 2 * radius + 1 + n), axis=ax)
        lo = np.take(c, np.arange(0, n), axis=ax)
        f = (hi - lo) / (2 * radius + 1)
    return f


def _texture(shape, seed: int, std: float, cell: int = 4) -> np.ndarray:
    """Smooth low-amplitude texture: a seeded N(0,1) field on a grid `cell`
    times coarser, box-blurred twice with radius 1, repeated up to the full
    grid and scaled to standard deviation `std`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    coarse = tuple(-(-n // cell) for n in shape)
    t = rng.standard_normal(coarse, dtype=np.float32)
    for _ in range(2):
        t = _box_blur(t, 1).astype(np.float32)
    for ax in range(3):
        t = np.repeat(t, cell, axis=ax)
    t = np.ascontiguousarray(t[:shape[0], :shape[1], :shape[2]])
    t *= np.float32(std / max(float(t.std()), 1e-30))
    return t


def phantom(geom: Geometry, n_ellipsoids: int, seed: int, inclusions: int = 0,
            texture_std: float = 0.0, dtype=np.float32) -> np.ndarray:
    """Point-sampled ellipsoid phantom [nz][ny][nx], clipped to [0, 1].

    The value of a voxel is the sum of the additive ellipsoids that contain
    its centre; "set" inclusions then overwrite with 1.0; an optional texture
    (see _texture) is added inside the background ellipsoid; finally the
    volume is clipped to [0, 1].  Each ellipsoid is evaluated in float64 over
    its bounding box only.
    """
    x, y, z = _voxel_axes(geom)
    vol = np.zeros(geom.vol_shape, dtype=np.float32)
    ells = ellipsoids(geom, n_ellipsoids, seed, inclusions)
    bg_mask = None
    for e, (c, a, R, val, mode) in enumerate(ells):
        ext = np.sqrt(((R * a[None, :]) ** 2).sum(axis=1))  # half extent along x, y, z
        lo = [int(np.searchsorted(ax, c[d] - ext[d], "left")) for d, ax in enumerate((x, y, z))]
        hi = [int(np.searchsorted(ax, c[d] + ext[d], "right")) for d, ax in enumerate((x, y, z))]
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        xs, ys = x[lo[0]:hi[0]] - c[0], y[lo[1]:hi[1]] - c[1]
        step = max(1, (1 << 22) // max(1, xs.size * ys.size))
        for z0 in range(lo[2], hi[2], step):
            zs = z[z0:min(hi[2], z0 + step)] - c[2]
            # coordinates in the ellipsoid's frame: q = R^T (p - c)
            r = 0.0
            for k in range(3):
                qk = (zs[:, None, None] * R[2, k] + ys[None, :, None] * R[1, k]
                      + xs[None, None, :] * R[0, k]) / a[k]
                r = r + qk * qk
            inside = r <= 1.0
            sl = (slice(z0, z0 + zs.size), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
            if mode == "add":
                vol[sl] += np.float32(val) * inside
            else:
                vol[sl][inside] = np.float32(val)
            if e == 0:
                if bg_mask is None:
                    bg_mask = np.zeros(geom.vol_shape, dtype=bool)
                bg_mask[sl] |= inside
    if texture_std > 0.0 and bg_mask is not None:
        vol += np.where(bg_mask, _texture(geom.vol_shape, seed + 777, texture_std), np.float32(0.0))
    np.clip(vol, 0.0, 1.0, out=vol)
    return vol.astype(dtype, copy=False)


def gaussian_noise(shape, sigma: float, seed: int, dtype=np.float32) -> np.ndarray:
    """sigma * N(0, 1) from a seeded PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.standard_normal(shape, dtype=np.float32 if dtype == np.float32 else np.float64)
    n *= sigma
    return n.astype(dtype, copy=False)


def poisson_log_data(clean: np.ndarray, I0: float, seed: int, dtype=np.float32) -> np.ndarray:
    """Log-transformed Poisson data: kappa = 3/max(clean),
    c ~ Poisson(I0 * exp(-kappa * clean)), b = -ln(max(c, 1)/I0)/kappa."""
    kappa = 3.0 / max(float(clean.max()), 1e-30)
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = I0 * np.exp(-kappa * clean.astype(np.float64))
    c = rng.poisson(lam)
    b = -np.log(np.maximum(c, 1) / I0) / kappa
    return b.astype(dtype)
