"""Shared helpers for the GPU parity tests (inputs come from synth; expected
values from the oracle only)."""
import numpy as np

import oracle
import synth


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def problem(geom, n_ell=6, seed=0, noise_rel=0.01):
    """Phantom x_true, data b = A x_true (oracle) + Gaussian noise, all views."""
    xt = synth.phantom(geom, n_ell, 1000 + seed).astype(np.float64)
    clean = oracle.project(geom, xt, range(geom.n_views))
    sigma = noise_rel * float(clean.max())
    b = clean + synth.gaussian_noise(clean.shape, sigma, 2000 + seed, dtype=np.float64)
    return xt, b


def cuda(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def host(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()


GEOMS = {
    # ragged, anisotropic, several tiles in every direction
    "ragged": synth.small_geometry(nx=40, ny=36, nz=28, n_views=24, nu=70, nv=50),
    # views exactly on the 45-degree family boundaries, odd detector
    "diag": synth.Geometry(nx=33, ny=30, nz=21, vx=1.0, vy=1.2, vz=0.9, n_views=8, sod=400.0,
                           sdd=700.0, nu=61, nv=37, du=1.3, dv=1.1),
    # non-uniform angles, small detector that clips the volume
    "angles": synth.small_geometry(nx=24, ny=24, nz=24, n_views=5, nu=19, nv=23,
                                   angles=(0.05, 0.8, 2.2, 3.9, 5.5)),
}
