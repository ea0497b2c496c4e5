"""Pins of the FDK oracle against facts that do not come from its code:

* the discrete Ram-Lak kernel is the band-limited ramp: its spectrum
  t * sum_k h(k t) cos(2 pi f k t) equals |f| on [0, 1/(2t)] up to the tail
  truncated at the detector width (at most 1/(pi^2 nu t) + a rounding term);
* the view weights cover the circle once (sum 2 pi), uniform angles give
  2 pi / n each;
* a uniform ball reconstructed from its analytic projections (exact chord
  lengths 2 sqrt(R^2 - d^2), no projector involved) comes out at its value in
  the interior of the central slice, and 0 well outside it;
* so do off-axis and off-plane balls in a strong cone with uneven view
  angles, at the right place (their centroids).
"""
import math

import numpy as np

from oracle import fdk
import synth


def test_ramp_kernel_spectrum_is_band_limited_ramp():
    for nu, t in ((64, 1.0), (301, 0.7)):
        h = fdk.ramp_kernel(nu, t)
        k = np.arange(-(nu - 1), nu)
        f = np.linspace(0.0, 0.5 / t, 97)
        R = t * (h[None, :] * np.cos(2 * math.pi * f[:, None] * k[None, :] * t)).sum(axis=1)
        assert np.max(np.abs(R - f)) <= 1.0 / (math.pi ** 2 * nu * t) * 1.05 + 1e-12
        assert h[nu - 1] == 1.0 / (4 * t * t) and h[nu] < 0 and h[nu + 1] == 0.0


def test_view_weights_cover_the_circle():
    w = fdk.view_weights(2 * math.pi * np.arange(12) / 12)
    assert np.allclose(w, 2 * math.pi / 12)
    ang = np.array([0.3, 1.0, 2.5, 4.0, 6.0])
    w = fdk.view_weights(ang)
    assert math.isclose(w.sum(), 2 * math.pi, rel_tol=1e-12)
    assert math.isclose(w[1], 0.5 * (2.5 - 0.3))                  # half the gaps to its neighbours
    assert math.isclose(w[0], 0.5 * (1.0 - (6.0 - 2 * math.pi)))   # across the 0 / 2 pi seam


def _ball_projections(g, R, value, centre=(0.0, 0.0, 0.0)):
    """Exact line integrals of a uniform ball (radius R) for every ray: the
    chord 2 sqrt(R^2 - d^2), d the distance of the centre from the ray."""
    th = np.asarray(g.angles) if g.angles is not None else 2 * math.pi * np.arange(g.n_views) / g.n_views
    c0 = np.asarray(centre, dtype=np.float64)
    cu, cv = (g.nu - 1) / 2.0, (g.nv - 1) / 2.0
    u = (np.arange(g.nu) - cu) * g.du
    v = (np.arange(g.nv) - cv) * g.dv
    y = np.zeros((g.n_views, g.nv, g.nu))
    for s, a in enumerate(th):
        c, sn = math.cos(a), math.sin(a)
        src = np.array([g.sod * c, g.sod * sn, 0.0])
        det = -(g.sdd - g.sod) * np.array([c, sn, 0.0])
        eu = np.array([-sn, c, 0.0])
        P = det[None, None, :] + u[None, :, None] * eu[None, None, :] + v[:, None, None] * np.array([0, 0, 1.0])
        d = P - src
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        cross = np.cross((c0 - src)[None, None, :], d)  # (centre - source) x direction
        dist2 = (cross ** 2).sum(axis=-1)
        y[s] = value * 2.0 * np.sqrt(np.maximum(R * R - dist2, 0.0))
    return y


def test_uniform_ball_from_exact_projections():
    g = synth.Geometry(nx=48, ny=48, nz=9, vx=1.0, vy=1.0, vz=1.0, n_views=180, sod=400.0, sdd=600.0,
                       nu=96, nv=40, du=1.5, dv=1.5)
    R, value = 15.0, 1.0
    y = _ball_projections(g, R, value)
    f = fdk.fdk(g, y, range(g.n_views))
    mid = f[g.nz // 2]
    jj, ii = np.meshgrid(np.arange(g.ny), np.arange(g.nx), indexing="ij")
    r = np.hypot((ii - (g.nx - 1) / 2.0) * g.vx, (jj - (g.ny - 1) / 2.0) * g.vy)
    inside = mid[r < 0.7 * R]
    outside = mid[r > 1.4 * R]
    assert abs(inside.mean() - value) <= 0.02 * value
    assert np.max(np.abs(inside - value)) <= 0.06 * value
    assert np.max(np.abs(outside)) <= 0.03 * value
    # the sampled-voxel form gives the same values
    vox = [(g.nz // 2, 24, 24), (g.nz // 2, 10, 30), (0, 5, 5)]
    assert np.allclose(fdk.fdk(g, y, range(g.n_views), voxels=vox), [f[v] for v in vox], rtol=0, atol=1e-12)


def test_off_axis_balls_strong_cone_uneven_angles():
    # Off-axis and off-plane balls in a strong cone (SOD 60 mm, the balls up to
    # 28 mm off the axis: U from 0.55 to 1.45), t = du m = 0.65, and twice as
    # many views on one half circle as on the other.  The reconstruction must
    # hold the ball's value inside, little outside, and the ball's centroid:
    # the view weights, the 1/U^2 weight, the U in the detector coordinates and
    # their orientation all show in one of these.
    ang = np.concatenate([math.pi * np.arange(120) / 120, math.pi + math.pi * np.arange(60) / 60])
    g = synth.Geometry(nx=56, ny=56, nz=24, vx=1.0, vy=1.0, vz=1.0, n_views=180, sod=60.0, sdd=120.0,
                       nu=400, nv=90, du=1.3, dv=1.3, angles=tuple(ang))
    k, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    P = np.stack([(i - (g.nx - 1) / 2.0) * g.vx, (j - (g.ny - 1) / 2.0) * g.vy, (k - (g.nz - 1) / 2.0) * g.vz])
    for centre, R in (((15.0, -10.0, 0.0), 8.0), ((12.0, 5.0, 6.0), 5.0)):
        f = fdk.fdk(g, _ball_projections(g, R, 1.0, centre), range(g.n_views))
        r = np.sqrt(((P - np.asarray(centre)[:, None, None, None]) ** 2).sum(axis=0))
        inside = f[r < 0.6 * R]
        # 1%: the discretisation (bilinear taps, 60-180 views) costs ~0.5% here
        assert abs(inside.mean() - 1.0) <= 0.01 and inside.min() >= 0.97
        assert np.abs(f[(r > 1.6 * R) & (r < 2.5 * R)]).mean() <= 0.03
        w = np.where(r < 1.3 * R, f, 0.0)
        cen = (P * w[None]).reshape(3, -1).sum(axis=1) / w.sum()
        assert np.abs(cen - np.asarray(centre)).max() <= 0.1


def test_filter_equals_direct_convolution():
    # the FFT form of step 2 against the convolution sum written out
    g = synth.Geometry(nx=8, ny=8, nz=8, vx=1.0, vy=1.0, vz=1.0, n_views=2, sod=300.0, sdd=450.0,
                       nu=37, nv=5, du=1.2, dv=1.1)
    rng = np.random.default_rng(3)
    y = rng.standard_normal((2, g.nv, g.nu))
    q = fdk.filtered(g, y, [0, 1])
    m = g.sod / g.sdd
    t = g.du * m
    h = fdk.ramp_kernel(g.nu, t)
    a = (np.arange(g.nu) - (g.nu - 1) / 2) * g.du * m
    b = (np.arange(g.nv) - (g.nv - 1) / 2) * g.dv * m
    for s in range(2):
        for r in range(g.nv):
            pw = y[s, r] * g.sod / np.sqrt(g.sod ** 2 + a ** 2 + b[r] ** 2)
            direct = [t * sum(h[(i - n) + g.nu - 1] * pw[n] for n in range(g.nu)) for i in range(g.nu)]
            assert np.allclose(q[s, r], direct, rtol=1e-12, atol=1e-12 * np.abs(direct).max())
