"""The benchmark's work counts, checked on the CPU.

The roofline figures divide counted work by measured time. The projector's
count is the ray-plane samples whose crossing lies inside the volume, as
computed by `bench.active_samples`. Here that count is compared with a brute
force one: every ray from the source to a detector pixel, stepped plane by
plane along its dominant axis, with the inside test (-1, N_b) x (-1, N_z) on
the crossing. The quarter-turn shortcut for square volumes on uniform orbits
must agree with the explicit per-view count. The sweep's nominal units are
n_views·nu·nv·N for the forward half and n_views·N³ for the back half.
"""
import math
import os
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def brute_force_samples(g, views):
    V = (g.vx, g.vy, g.vz)
    N = (g.nx, g.ny, g.nz)
    c = [0.5 * (n - 1) for n in N]
    u = (np.arange(g.nu) - 0.5 * (g.nu - 1)) * g.du
    w = (np.arange(g.nv) - 0.5 * (g.nv - 1)) * g.dv
    total = 0
    for v in views:
        th = 2.0 * math.pi * v / g.n_views if g.angles is None else g.angles[v]
        S = np.array([g.sod * math.cos(th), g.sod * math.sin(th), 0.0])
        # detector pixel (iu, iv): centre of the detector plus u along the
        # in-plane axis and w along z
        D0 = -(g.sdd - g.sod) * np.array([math.cos(th), math.sin(th), 0.0])
        ax_u = np.array([-math.sin(th), math.cos(th), 0.0])
        P = D0[None, None] + u[None, :, None] * ax_u[None, None] + w[:, None, None] * np.array([0, 0, 1.0])
        d = P - S[None, None]                                   # [nv, nu, 3]
        dom = np.where(np.abs(d[..., 1]) > np.abs(d[..., 0]), 1, 0)
        for a in (0, 1):
            b = 1 - a
            sel = dom == a
            if not sel.any():
                continue
            da, db, dz = d[..., a][sel], d[..., b][sel], d[..., 2][sel]
            for m in range(N[a]):
                t = ((m - c[a]) * V[a] - S[a]) / da
                qb = (S[b] + t * db) / V[b] + c[b]
                qz = (t * dz) / V[2] + c[2]
                total += int(np.count_nonzero((qb > -1) & (qb < N[b]) & (qz > -1) & (qz < N[2])))
    return total


GEOMS = {
    "cube": synth.Geometry(nx=24, ny=24, nz=24, vx=1.0, vy=1.0, vz=1.0, n_views=8, sod=1000.0,
                           sdd=1500.0, nu=36, nv=36, du=1.5, dv=1.5),
    "ragged": synth.small_geometry(nx=20, ny=16, nz=12, n_views=6, nu=34, nv=22),
    "angles": synth.small_geometry(nx=18, ny=18, nz=10, n_views=3, nu=30, nv=16,
                                   angles=(0.1, 0.9, 2.4)),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_active_samples_equal_brute_force(name):
    g = GEOMS[name]
    views = list(range(g.n_views))
    assert bench.active_samples(g, views) == brute_force_samples(g, views)


def test_quarter_turn_shortcut_equals_explicit_count():
    g = GEOMS["cube"]
    explicit = sum(bench.active_samples(g, [v]) for v in range(g.n_views))
    assert bench.active_samples(g, list(range(g.n_views))) == explicit


def test_sweep_units():
    g = synth.WORKLOADS["c3_512"].geom
    fwd, back = bench.sweep_units(g)
    assert fwd == 720 * 768 * 768 * 512
    assert back == 720 * 512 ** 3
