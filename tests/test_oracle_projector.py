"""Pins of the oracle's operator A (and A^T) to facts outside the oracle.

* a uniform slab: the Joseph sum of a constant volume along a ray that stays
  inside the slab equals the physical chord length c * T * |d| / |d_a|;
* analytic chords through a uniform, rotated, off-centre ellipsoid: the
  projection of the point-sampled ellipsoid converges to c * chord length as
  the grid is refined (a wrong sign, axis or offset in the geometry would
  not converge);
* a single voxel projects onto the detector pixel predicted by the
  perspective map u = SDD * eta / (SOD - xi);
* the scatter adjoint equals the transpose of the explicit matrix of A on
  8^3 (columns of A from unit volumes, rows from unit sinograms);
* the dot test <A x, y> = <x, A^T y> on 32^3;
* the brute-force per-voxel adjoint equals the scatter adjoint.

The definitions under test are the problem's operator A of eq. (2.1) and its
restriction A_N of eq. (2.5); the discretisation is the one stated in
oracle/joseph.c (the paper delegates it to a library, Sec. 3).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    rz1 = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    rz2 = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1.0]])
    return rz1 @ ry @ rz2


def _chord(s, d, centre, axes, R):
    """Length of the segment of the line s + t d inside the ellipsoid (exact)."""
    p = (s - centre) @ R / axes
    q = d @ R / axes
    A = q @ q
    B = 2.0 * p @ q
    C = p @ p - 1.0
    disc = B * B - 4 * A * C
    if disc <= 0:
        return 0.0
    return math.sqrt(disc) / A * np.linalg.norm(d)


def test_uniform_slab_chord_length():
    # Thin slab along x (6 planes of 2 mm), wide in y and z; view 0 looks along -x,
    # so every ray is x-dominant and, with a small detector, stays inside on all planes.
    g = synth.Geometry(nx=6, ny=80, nz=80, vx=2.0, vy=1.0, vz=1.0, n_views=1, sod=500.0,
                       sdd=800.0, nu=21, nv=17, du=1.1, dv=1.3, angles=(0.0,))
    c = 0.7
    x = np.full(g.vol_shape, c)
    y = oracle.project(g, x, [0])[0]
    T = g.nx * g.vx
    for iv in range(g.nv):
        for iu in range(g.nu):
            s, d = oracle.ray(g, 0, iu, iv)
            assert oracle.dominant_axis(d) == 0
            expect = c * T * np.linalg.norm(d) / abs(d[0])
            assert y[iv, iu] == pytest.approx(expect, rel=1e-13)


def test_analytic_ellipsoid_chords_converge():
    centre = np.array([5.0, -8.0, 3.0])
    axes = np.array([20.0, 12.0, 15.0])
    R = _rot(0.4, 0.9, -0.3)
    L = 64.0
    angles = (0.3, 1.1, 2.5, 4.0)
    errs = []
    for n in (20, 40, 80):  # voxels of 3.2, 1.6, 0.8 mm: none of unit size
        v = L / n
        g = synth.Geometry(nx=n, ny=n, nz=n, vx=v, vy=v, vz=v, n_views=len(angles), sod=400.0,
                           sdd=600.0, nu=40, nv=36, du=3.0, dv=3.0, angles=angles)
        xs = (np.arange(n) - 0.5 * (n - 1)) * v
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        P = np.stack([X, Y, Z], axis=-1) - centre
        q = P @ R / axes
        vol = ((q ** 2).sum(-1) <= 1.0).astype(np.float64)
        y = oracle.project(g, vol, range(len(angles)))
        ref = np.zeros_like(y)
        for vi in range(len(angles)):
            for iv in range(g.nv):
                for iu in range(g.nu):
                    s, d = oracle.ray(g, vi, iu, iv)
                    ref[vi, iv, iu] = _chord(s, d, centre, axes, R)
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    # first-order convergence of the point-sampled discretisation
    assert errs[1] < 0.75 * errs[0]
    assert errs[2] < 0.75 * errs[1]
    assert errs[2] < 0.03


def test_single_voxel_lands_on_perspective_projection():
    # anisotropic voxels; the shadow's centroid (its taps are hat functions
    # centred on the voxel) is the perspective image of the voxel centre
    g = synth.Geometry(nx=24, ny=24, nz=24, vx=0.8, vy=1.25, vz=1.1, n_views=3, sod=300.0,
                       sdd=450.0, nu=81, nv=81, du=0.75, dv=0.75, angles=(0.2, 1.9, 3.7))
    i, j, k = 17, 6, 15
    x = np.zeros(g.vol_shape)
    x[k, j, i] = 1.0
    y = oracle.project(g, x, range(3))
    px = (i - 11.5) * g.vx
    py = (j - 11.5) * g.vy
    pz = (k - 11.5) * g.vz
    uu, vv = np.meshgrid(np.arange(g.nu), np.arange(g.nv))
    for vi, th in enumerate(g.angles):
        xi = px * math.cos(th) + py * math.sin(th)
        eta = -px * math.sin(th) + py * math.cos(th)
        mag = g.sdd / (g.sod - xi)
        iu = eta * mag / g.du + 0.5 * (g.nu - 1)
        iv = pz * mag / g.dv + 0.5 * (g.nv - 1)
        ivm, ium = np.unravel_index(np.argmax(y[vi]), y[vi].shape)
        assert abs(ium - iu) <= 1.0 and abs(ivm - iv) <= 1.0
        w = y[vi] / y[vi].sum()
        assert abs((w * uu).sum() - iu) <= 0.1 and abs((w * vv).sum() - iv) <= 0.1


def _tiny_geom():
    return synth.Geometry(nx=8, ny=8, nz=8, vx=1.0, vy=1.0, vz=1.0, n_views=5, sod=60.0,
                          sdd=90.0, nu=13, nv=11, du=1.5, dv=1.5)


def test_explicit_matrix_transpose_8cubed():
    g = _tiny_geom()
    views = list(range(g.n_views))
    nvox = g.n_vox
    nray = g.n_views * g.nu * g.nv
    A = np.zeros((nray, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = oracle.project(g, e.reshape(g.vol_shape), views).ravel()
    AT = np.zeros((nvox, nray))
    for r in range(nray):
        e = np.zeros(nray)
        e[r] = 1.0
        AT[:, r] = oracle.backproject(g, e.reshape(g.n_views, g.nv, g.nu), views).ravel()
    assert np.count_nonzero(A) > 1000
    assert np.max(np.abs(A - AT.T)) <= 1e-14 * np.max(np.abs(A))


def test_dot_product_32cubed():
    g = synth.Geometry(nx=32, ny=32, nz=32, vx=1.0, vy=1.0, vz=1.0, n_views=7, sod=200.0,
                       sdd=300.0, nu=50, nv=48, du=1.5, dv=1.5)
    rng = np.random.default_rng(5)
    views = [0, 2, 3, 6]
    x = rng.standard_normal(g.vol_shape)
    y = rng.standard_normal((len(views), g.nv, g.nu))
    lhs = float(np.dot(oracle.project(g, x, views).ravel(), y.ravel()))
    rhs = float(np.dot(x.ravel(), oracle.backproject(g, y, views).ravel()))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_brute_force_voxels_match_scatter():
    g = synth.small_geometry(nx=20, ny=18, nz=14, n_views=6, nu=36, nv=26)
    rng = np.random.default_rng(7)
    views = [1, 4, 5]
    y = rng.standard_normal((len(views), g.nv, g.nu))
    full = oracle.backproject(g, y, views)
    vox = [(0, 0, 0), (13, 17, 19), (7, 9, 10), (3, 1, 18), (10, 12, 2)]
    got = oracle.backproject_voxels(g, y, views, vox)
    want = np.array([full[k, j, i] for (k, j, i) in vox])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_all_three_families_present_and_z_family_handled():
    # A short source distance with a tall detector gives z-dominant rays.
    g = synth.Geometry(nx=10, ny=10, nz=10, vx=1.0, vy=1.0, vz=1.0, n_views=2, sod=30.0,
                       sdd=45.0, nu=9, nv=81, du=1.5, dv=1.5, angles=(0.0, math.pi / 4 + 0.1))
    fam = set()
    for v in range(2):
        for iu in range(g.nu):
            for iv in range(g.nv):
                _, d = oracle.ray(g, v, iu, iv)
                fam.add(oracle.dominant_axis(d))
    assert fam == {0, 1, 2}
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.vol_shape)
    y = rng.standard_normal((2, g.nv, g.nu))
    lhs = float(np.dot(oracle.project(g, x, [0, 1]).ravel(), y.ravel()))
    rhs = float(np.dot(x.ravel(), oracle.backproject(g, y, [0, 1]).ravel()))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
