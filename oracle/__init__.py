"""FP64 CPU oracle for the FB-LISA hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; both sides take their inputs
from ``synth``.

Contents:
  * ``project`` / ``backproject`` / ``project_rays`` / ``backproject_voxels``
    -- the cone-beam operator A_S of eq. (2.5) and its exact transpose, in
    plain C double precision (``joseph.c``);
  * ``fblisa`` -- Algorithm 1 (FB-LISA) step by step in numpy float64;
  * ``fdk`` -- the FDK reconstruction (cosine weighting, Ram-Lak filter,
    weighted backprojection) in numpy float64;
  * ``tv`` -- other regularisers: the box-constrained l1 prox and the
    isotropic TV prox by FGP iterations on the dual, in numpy float64;
  * ``mlp`` -- the step-proposal network (forward, gradient, Adam) in FP64;
  * ``proposal`` -- the learned step proposal inside Algorithm 1 (features,
    network output, first grid index) driving ``fblisa.fb_step``.

Pins (checks against facts the paper and mathematics fix, not against this
code) live in ``tests/test_oracle_*.py``.  Parity unpinned against the paper
itself: the whole FB-LISA trajectory on the paper's walnut data (the data are
not available), pinned only through its parts, and the learned proposal, which
has no counterpart in the paper (pinned by the properties listed in
``proposal.py``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["project", "backproject", "project_rays", "backproject_voxels", "num_threads",
           "load"]

_lib = None


class _OrcGeom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
        ("n_views", ctypes.c_int32), ("angles", ctypes.POINTER(ctypes.c_double)),
        ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
        ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
    ]


def load():
    """Build (if stale) and load the oracle's C library."""
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        lib.orc_project.argtypes = [P(_OrcGeom), P(ctypes.c_double), P(ctypes.c_int32),
                                    ctypes.c_int, P(ctypes.c_double)]
        lib.orc_project.restype = None
        lib.orc_backproject.argtypes = [P(_OrcGeom), P(ctypes.c_double), P(ctypes.c_int32),
                                        ctypes.c_int, P(ctypes.c_double)]
        lib.orc_backproject.restype = ctypes.c_int
        lib.orc_project_ray.argtypes = [P(_OrcGeom), P(ctypes.c_double), ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int]
        lib.orc_project_ray.restype = ctypes.c_double
        lib.orc_backproject_voxels.argtypes = [P(_OrcGeom), P(ctypes.c_double),
                                               P(ctypes.c_int32), ctypes.c_int,
                                               P(ctypes.c_int64), ctypes.c_int,
                                               P(ctypes.c_double)]
        lib.orc_backproject_voxels.restype = None
        lib.orc_ray.argtypes = [P(_OrcGeom), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                P(ctypes.c_double), P(ctypes.c_double)]
        lib.orc_ray.restype = None
        lib.orc_dominant_axis.argtypes = [P(ctypes.c_double)]
        lib.orc_dominant_axis.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


class _Geom:
    """Keeps the ctypes struct and its angle array alive together."""

    def __init__(self, geom):
        self.angles = None
        if geom.angles is not None:
            self.angles = np.ascontiguousarray(np.asarray(geom.angles, dtype=np.float64))
            if self.angles.size != geom.n_views:
                raise ValueError("angles must have n_views entries")
        self.s = _OrcGeom(geom.nx, geom.ny, geom.nz, geom.vx, geom.vy, geom.vz, geom.n_views,
                          None if self.angles is None else
                          self.angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          geom.sod, geom.sdd, geom.nu, geom.nv, geom.du, geom.dv)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _views(geom, views):
    v = np.ascontiguousarray(np.asarray(views, dtype=np.int32).ravel())
    if v.size and (v.min() < 0 or v.max() >= geom.n_views):
        raise ValueError("view index out of range")
    return v


def num_threads() -> int:
    return int(load().orc_num_threads())


def project(geom, x, views):
    """A_S x in float64: x [nz][ny][nx] -> y [len(views)][nv][nu]."""
    lib = load()
    g = _Geom(geom)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(geom.vol_shape))
    v = _views(geom, views)
    y = np.zeros((v.size, geom.nv, geom.nu), dtype=np.float64)
    lib.orc_project(g.ref, _dp(x), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), v.size,
                    _dp(y))
    return y


def backproject(geom, y, views):
    """A_S^T y in float64 (ray-driven scatter): y [len(views)][nv][nu] -> x."""
    lib = load()
    g = _Geom(geom)
    v = _views(geom, views)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(v.size, geom.nv, geom.nu))
    x = np.zeros(geom.vol_shape, dtype=np.float64)
    rc = lib.orc_backproject(g.ref, _dp(y), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             v.size, _dp(x))
    if rc != 0:
        raise MemoryError("oracle backprojection could not allocate its buffers")
    return x


def project_rays(geom, x, rays):
    """(A x) for single rays given as (view, iu, iv) triples."""
    lib = load()
    g = _Geom(geom)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(geom.vol_shape))
    out = np.empty(len(rays), dtype=np.float64)
    for n, (v, iu, iv) in enumerate(rays):
        out[n] = lib.orc_project_ray(g.ref, _dp(x), int(v), int(iu), int(iv))
    return out


def backproject_voxels(geom, y, views, voxels):
    """(A_S^T y)_j for the listed (k, j, i) voxels, by brute force over all rays."""
    lib = load()
    g = _Geom(geom)
    v = _views(geom, views)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(v.size, geom.nv, geom.nu))
    vox = np.asarray(voxels, dtype=np.int64).reshape(-1, 3)
    lin = np.ascontiguousarray((vox[:, 0] * geom.ny + vox[:, 1]) * geom.nx + vox[:, 2])
    out = np.zeros(lin.size, dtype=np.float64)
    lib.orc_backproject_voxels(g.ref, _dp(y), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               v.size, lin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               lin.size, _dp(out))
    return out


def ray(geom, view, iu, iv):
    """Source point and direction d = P - s of one ray (float64)."""
    lib = load()
    g = _Geom(geom)
    s = np.zeros(3)
    d = np.zeros(3)
    lib.orc_ray(g.ref, int(view), int(iu), int(iv), _dp(s), _dp(d))
    return s, d


def dominant_axis(d) -> int:
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    return int(load().orc_dominant_axis(_dp(d)))
