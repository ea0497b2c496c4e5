"""FDK (Feldkamp-Davis-Kress) reconstruction in numpy float64: the analytic
baseline the paper compares against and uses for its reference volumes
(Sec. 3, "Dataset" and the comparison methods).

TEST INFRASTRUCTURE: see ``oracle/__init__.py``.

The paper names the method and takes it from a library; these are the
textbook steps for a circular orbit and a flat detector, written on the
virtual detector through the rotation axis (scale m = SOD/SDD):

  1. cosine weighting  p_w(a, b) = p(a, b) * SOD / sqrt(SOD^2 + a^2 + b^2),
     with a = u m, b = v m the virtual-detector coordinates of a pixel centre;
  2. ramp filtering along each detector row with the spatial Ram-Lak kernel
     of spacing t = du m:  h(0) = 1/(4 t^2), h(k t) = -1/(pi^2 k^2 t^2) for odd
     k, 0 for even k != 0;  q(a_i) = t * sum_n h(a_i - a_n) p_w(a_n)  (the row
     is zero outside the detector);
  3. weighted backprojection  f(x) = sum_views (dtheta/2) * q(a(x), b(x)) / U^2
     with U = (SOD - xi)/SOD, xi = x cos(theta) + y sin(theta),
     a(x) = eta / U, b(x) = z / U, eta = -x sin(theta) + y cos(theta), q
     interpolated bilinearly (zero outside the detector), and dtheta the
     angular interval a view stands for (half the gaps to its neighbours over
     the full circle; 2 pi / n for uniform angles).

Geometry conventions are those of the projector (source at SOD (cos, sin, 0),
detector e_u = (-sin, cos, 0), pixel (iu, iv) at ((iu - cu) du, (iv - cv) dv),
voxel centres at ((i - (N-1)/2) v, ...)).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np


def _angles(geom) -> np.ndarray:
    if geom.angles is not None:
        return np.asarray(geom.angles, dtype=np.float64)
    return 2.0 * math.pi * np.arange(geom.n_views, dtype=np.float64) / geom.n_views


def view_weights(angles: np.ndarray) -> np.ndarray:
    """dtheta of each view: half the circular gaps to its two neighbours."""
    a = np.mod(np.asarray(angles, dtype=np.float64), 2.0 * math.pi)
    order = np.argsort(a)
    s = a[order]
    n = s.size
    if n == 1:
        return np.array([2.0 * math.pi])
    nxt = np.roll(s, -1)
    nxt[-1] += 2.0 * math.pi
    prv = np.roll(s, 1)
    prv[0] -= 2.0 * math.pi
    w_sorted = 0.5 * (nxt - prv)
    w = np.empty(n)
    w[order] = w_sorted
    return w


def ramp_kernel(nu: int, t: float) -> np.ndarray:
    """Ram-Lak taps h(k t) for k = -(nu-1) .. nu-1."""
    k = np.arange(-(nu - 1), nu, dtype=np.float64)
    h = np.zeros_like(k)
    h[k == 0] = 1.0 / (4.0 * t * t)
    odd = (np.abs(k) % 2) == 1
    h[odd] = -1.0 / (math.pi ** 2 * k[odd] ** 2 * t * t)
    return h


def filtered(geom, y: np.ndarray, views: Sequence[int]) -> np.ndarray:
    """Steps 1-2: weighted, ramp-filtered projections q[s][iv][iu]."""
    m = geom.sod / geom.sdd
    cu, cv = (geom.nu - 1) / 2.0, (geom.nv - 1) / 2.0
    a = (np.arange(geom.nu) - cu) * geom.du * m
    b = (np.arange(geom.nv) - cv) * geom.dv * m
    W = geom.sod / np.sqrt(geom.sod ** 2 + a[None, :] ** 2 + b[:, None] ** 2)
    t = geom.du * m
    nu = geom.nu
    h = ramp_kernel(nu, t)  # h(k t), k = -(nu-1) .. nu-1
    # q_i = t sum_n h(i - n) p_n as a circular convolution of length 2 nu: the
    # kernel's negative offsets sit at the end of the period, and for outputs
    # 0 <= i < nu no product wraps onto another (|i - n| <= nu - 1 < nu + 1)
    L = 2 * nu
    hc = np.zeros(L)
    hc[:nu] = h[nu - 1:]            # k = 0 .. nu-1
    hc[L - (nu - 1):] = h[:nu - 1]  # k = -(nu-1) .. -1
    Hf = np.fft.rfft(hc)
    y = np.asarray(y, dtype=np.float64).reshape(len(views), geom.nv, nu)
    q = np.empty_like(y)
    for s in range(len(views)):
        pw = y[s] * W
        q[s] = t * np.fft.irfft(np.fft.rfft(pw, n=L, axis=1) * Hf[None, :], n=L, axis=1)[:, :nu]
    return q


def _bilinear(q2: np.ndarray, fv: np.ndarray, fu: np.ndarray) -> np.ndarray:
    nv, nu = q2.shape
    iv0 = np.floor(fv).astype(np.int64)
    iu0 = np.floor(fu).astype(np.int64)
    tv = fv - iv0
    tu = fu - iu0

    def at(iv, iu):
        ok = (iv >= 0) & (iv < nv) & (iu >= 0) & (iu < nu)
        out = np.zeros(iv.shape)
        out[ok] = q2[iv[ok], iu[ok]]
        return out

    return ((1 - tv) * ((1 - tu) * at(iv0, iu0) + tu * at(iv0, iu0 + 1))
            + tv * ((1 - tu) * at(iv0 + 1, iu0) + tu * at(iv0 + 1, iu0 + 1)))


def fdk(geom, y: np.ndarray, views: Sequence[int], voxels: Optional[np.ndarray] = None) -> np.ndarray:
    """FDK of the projections y[len(views)][nv][nu] taken at the listed views.
    Returns the volume [nz][ny][nx], or the values at voxels (k, j, i) rows."""
    views = list(views)
    ang = _angles(geom)[views]
    dth = view_weights(ang)
    q = filtered(geom, y, views)
    m = geom.sod / geom.sdd
    cu, cv = (geom.nu - 1) / 2.0, (geom.nv - 1) / 2.0
    if voxels is None:
        k, j, i = np.meshgrid(np.arange(geom.nz), np.arange(geom.ny), np.arange(geom.nx), indexing="ij")
    else:
        vox = np.asarray(voxels, dtype=np.int64).reshape(-1, 3)
        k, j, i = vox[:, 0], vox[:, 1], vox[:, 2]
    x = (i - (geom.nx - 1) / 2.0) * geom.vx
    yy = (j - (geom.ny - 1) / 2.0) * geom.vy
    z = (k - (geom.nz - 1) / 2.0) * geom.vz
    f = np.zeros(x.shape)
    for s, th in enumerate(ang):
        c, sn = math.cos(th), math.sin(th)
        xi = x * c + yy * sn
        eta = -x * sn + yy * c
        U = (geom.sod - xi) / geom.sod
        fu = (eta / U) / (geom.du * m) + cu
        fv = (z / U) / (geom.dv * m) + cv
        f += 0.5 * dth[s] * _bilinear(q[s], fv, fu) / (U * U)
    return f
