"""Parity at the full 512^3 / 720-view / 768^2 workload, in the launch
configuration the benchmark times (one 40-view mini-batch per call):

* the projector on sampled rays, each recomputed by the FP64 oracle;
* the backprojector on sampled voxels, each recomputed by the oracle's
  brute-force per-voxel transpose;
* the dot test of the two GPU operators at full size;
* one FB-LISA iteration: the mini-batch equals the oracle's and the accepted
  step satisfies F_N(x_bar) <= F_N(x) - ||d||^2/(2 alpha) (from (2.3) and the
  prox optimality (A3));
* the sums the line search decides on, in the autotuned launch configuration:
  rho0 = ||A_N x - b_N||^2 from the residual projection (Step 2b) and rho1 from
  the trial-objective projection (Step 2c), against the oracle's FP64 sums
  (relative 2e-5), at this workload and at the paper-shaped 560^3 / 840^2 /
  36-view geometry (Sec. 3, cases 1-2).
"""
import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth
from gpu_common import cuda, host

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["c3_512"]
G3 = WL.geom


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2605_12085_gb300 as fbl
    x = synth.phantom(G3, WL.n_ellipsoids, WL.seed_phantom, texture_std=WL.texture_std)
    G = fbl.geometry_create(G3)
    views = fbl.fbl_epoch_batches(WL.seed_batches, 1, G3.n_views, WL.N0)[0]
    assert views == fblisa.epoch_batches(WL.seed_batches, 1, G3.n_views, WL.N0)[0]
    yield fbl, G, x, torch.from_numpy(x).cuda(), views


def _sample_rays(rng, n_sel, n):
    s = rng.integers(0, n_sel, n)
    iu = rng.integers(0, G3.nu, n)
    iv = rng.integers(0, G3.nv, n)
    edges = [(0, 0, 0), (n_sel - 1, G3.nu - 1, G3.nv - 1), (0, G3.nu // 2, G3.nv // 2),
             (1, G3.nu // 2 - 1, 0), (2, 0, G3.nv // 2)]
    return [(int(a), int(b), int(c)) for a, b, c in zip(s, iu, iv)] + edges


def test_fullsize_project_sampled_rays(setup):
    fbl, G, x, xd, views = setup
    y = fbl.project(G, xd, views)
    rng = np.random.default_rng(11)
    rays = _sample_rays(rng, len(views), 400)
    got = np.array([float(y[s, iv, iu]) for (s, iu, iv) in rays])
    ref = oracle.project_rays(G3, x, [(views[s], iu, iv) for (s, iu, iv) in rays])
    scale = float(np.abs(ref).max())
    assert scale > 10.0
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= 2e-5 * scale


def test_fullsize_backproject_sampled_voxels(setup):
    fbl, G, x, xd, views = setup
    import torch
    gen = torch.Generator(device="cuda").manual_seed(5)
    y = torch.randn((len(views), G3.nv, G3.nu), device="cuda", generator=gen)
    xb = fbl.backproject(G, y, views)
    rng = np.random.default_rng(12)
    vox = [tuple(int(t) for t in rng.integers(0, 512, 3)) for _ in range(28)]
    vox += [(0, 0, 0), (511, 511, 511), (256, 255, 256), (100, 400, 5)]
    got = np.array([float(xb[k, j, i]) for (k, j, i) in vox])
    ref = oracle.backproject_voxels(G3, host(y), views, vox)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_fullsize_dot_test(setup):
    fbl, G, x, xd, views = setup
    import torch
    gen = torch.Generator(device="cuda").manual_seed(6)
    y = torch.randn((len(views), G3.nv, G3.nu), device="cuda", generator=gen)
    Ax = fbl.project(G, xd, views)
    ATy = fbl.backproject(G, y, views)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((xd.double() * ATy.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_fullsize_step_decrease_property(setup):
    fbl, G, x, xd, views = setup
    import torch
    b = fbl.project(G, xd, range(G3.n_views))
    gen = torch.Generator(device="cuda").manual_seed(7)
    b += 0.01 * float(b.max()) * torch.randn(b.shape, device="cuda", generator=gen)
    S = fbl.fblisa_create(G, fbl.params_default(N0=WL.N0, seed=WL.seed_batches, mu=WL.mu))
    xs = torch.zeros_like(xd)
    prev_l1 = 0.0
    for it in range(2):
        st = S.step(xs, b)
        assert S.last_batch() == fblisa.epoch_batches(WL.seed_batches, 1, G3.n_views, WL.N0)[it]
        l1 = float(xs.double().sum())
        assert float(xs.min()) >= 0.0
        lhs = st["f_xbar"] + WL.mu * l1
        rhs = st["f_x"] + WL.mu * prev_l1 - st["dnorm2"] / (2 * st["alpha"])
        assert lhs <= rhs + 1e-6 * abs(rhs)
        assert st["margin"] >= 0
        prev_l1 = l1


def _scalar_parity(fbl, wl, x_true, seed):
    """rho0 of the solver's first iteration and rho1 of residual_norm, both on
    x0 = x_true/2 with data b = A x_true + 1% noise on the first mini-batch
    (the oracle's projection; the other views are never read), against the
    oracle's FP64 sum; the launch configuration is the autotuner's."""
    import torch
    g = wl.geom
    G = fbl.geometry_create(g)
    tune = fbl.geometry_autotune(G, fbl.F32, wl.N0)
    views = fblisa.epoch_batches(wl.seed_batches, 1, g.n_views, wl.N0)[0]
    clean = oracle.project(g, x_true.astype(np.float64), views)
    noise = synth.gaussian_noise(clean.shape, 0.01 * float(clean.max()), seed, dtype=np.float64)
    b = np.zeros((g.n_views, g.nv, g.nu), np.float32)
    b[views] = (clean + noise).astype(np.float32)
    x0 = (0.5 * x_true).astype(np.float32)
    r = oracle.project(g, x0.astype(np.float64), views) - b[views].astype(np.float64)
    rho_ref = float(np.dot(r.ravel(), r.ravel()))
    bd = torch.from_numpy(b).cuda()
    S = fbl.fblisa_create(G, fbl.params_default(N0=wl.N0, seed=wl.seed_batches, mu=wl.mu))
    st = S.step(torch.from_numpy(x0).cuda(), bd)
    assert S.last_batch() == list(views)
    rho1 = fbl.residual_norm(G, torch.from_numpy(x0).cuda(), views, bd)
    return tune, st["rho0"], rho1, rho_ref


def test_fullsize_line_search_sums_match_oracle(setup):
    fbl, G, x, xd, views = setup
    tune, rho0, rho1, ref = _scalar_parity(fbl, WL, x, 2101)
    assert rho0 == pytest.approx(ref, rel=2e-5), tune
    assert rho1 == pytest.approx(ref, rel=2e-5), tune


def test_paper_case_geometry_line_search_sums_match_oracle():
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["case2_560"]
    x = synth.phantom(wl.geom, wl.n_ellipsoids, wl.seed_phantom, texture_std=wl.texture_std)
    tune, rho0, rho1, ref = _scalar_parity(fbl, wl, x, 2102)
    assert rho0 == pytest.approx(ref, rel=2e-5), tune
    assert rho1 == pytest.approx(ref, rel=2e-5), tune
