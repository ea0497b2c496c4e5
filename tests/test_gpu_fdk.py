"""FDK on the GPU against the FP64 oracle (oracle/fdk.py, pinned by the ramp
spectrum and an analytic ball): full volumes on small geometries (ragged
sizes, anisotropic voxels and 45-degree views, non-uniform angles and a
clipping detector), a subset of views (the angular weights), host buffers,
no views, and sampled voxels at the full 512^3 / 720-view workload.

Tolerance 1e-5 relative L2 (FP32 filtering and interpolation, FP64 detector
coordinates per voxel column), as for the other FP32 operators; 2e-5 on the
sampled voxels of the 720-view volume, whose values are FP32 sums of 720
terms of both signs."""
import numpy as np
import pytest

import oracle
from oracle import fdk as ofdk
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_fdk_matches_oracle(name):
    import paper_2605_12085_gb300 as fbl
    g = GEOMS[name]
    xt, b = problem(g, seed=71)
    y = b.astype(np.float32)
    views = list(range(g.n_views))
    G = fbl.geometry_create(g)
    x = host(fbl.fdk(G, cuda(y), views))
    ref = ofdk.fdk(g, y.astype(np.float64), views)
    assert rel_l2(x, ref) <= TOL


def test_fdk_random_data_view_subset_and_host_buffers():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    rng = np.random.default_rng(72)
    views = list(range(0, g.n_views, 3)) + [1, 5]
    y = rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32)
    G = fbl.geometry_create(g)
    ref = ofdk.fdk(g, y.astype(np.float64), views)
    assert rel_l2(host(fbl.fdk(G, cuda(y), views)), ref) <= TOL
    xh = np.zeros(g.vol_shape, np.float32)
    fbl.fdk(G, y, views, x=xh)  # host input and output
    assert rel_l2(xh, ref) <= TOL
    z = host(fbl.fdk(G, cuda(np.zeros((0, g.nv, g.nu), np.float32)), []))
    assert not z.any()


def test_fdk_reconstructs_the_c1_phantom():
    # a quality check, not parity: 90 views of a 64^3 phantom with 1% noise
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["c1_64"]
    g = wl.geom
    xt, b = problem(g, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    G = fbl.geometry_create(g)
    x = host(fbl.fdk(G, cuda(b.astype(np.float32)), range(g.n_views)))
    assert rel_l2(x, xt) <= 0.35


def test_fdk_fullsize_sampled_voxels():
    import torch
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["c3_512"]
    g = wl.geom
    G = fbl.geometry_create(g)
    gen = torch.Generator(device="cuda").manual_seed(73)
    xs = torch.rand(g.vol_shape, device="cuda", generator=gen)
    views = list(range(g.n_views))
    y = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32, device="cuda")
    for v0 in range(0, g.n_views, 120):
        fbl.project(G, xs, views[v0:v0 + 120], y=y[v0:v0 + 120])
    x = fbl.fdk(G, y, views)
    rng = np.random.default_rng(74)
    vox = [tuple(int(t) for t in rng.integers(0, 512, 3)) for _ in range(40)]
    vox += [(0, 0, 0), (511, 511, 511), (256, 255, 256)]
    got = np.array([float(x[k, j, i]) for (k, j, i) in vox])
    ref = ofdk.fdk(g, host(y), views, voxels=vox)
    assert np.linalg.norm(got - ref) <= 2 * TOL * np.linalg.norm(ref)
