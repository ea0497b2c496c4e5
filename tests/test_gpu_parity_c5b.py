"""Parity at the large configuration: a 1024^3 volume, 1440 views, 1536^2
detector, FP16 storage with FP32 accumulation, 60-view mini-batches, learned
step proposal -- in the launch configuration its solver uses:

* the projector on sampled rays of one mini-batch, each recomputed by the FP64
  oracle on the FP16-stored volume (FP32 arithmetic on rounded storage: 1e-5);
* the backprojector on sampled voxels (oracle brute-force transpose);
* one FB-LISA iteration with FP16 storage and the learned proposal: the
  mini-batch is the oracle's, the first trial lies on the plain rule's grid,
  and the accepted step satisfies F_N(x_bar) <= F_N(x) - ||d||^2/(2 alpha)
  (from (2.3) and the prox optimality (A3)).
"""
import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth
from gpu_common import host

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["c5b_1024"]
GB = WL.geom


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2605_12085_gb300 as fbl
    gen = torch.Generator(device="cuda").manual_seed(1005)
    xd = torch.rand(GB.vol_shape, device="cuda", generator=gen).to(torch.float16)
    G = fbl.geometry_create(GB)
    views = fbl.fbl_epoch_batches(WL.seed_batches, 1, GB.n_views, WL.N0)[0]
    assert views == fblisa.epoch_batches(WL.seed_batches, 1, GB.n_views, WL.N0)[0]
    yield fbl, G, xd, views


def test_c5b_project_sampled_rays_fp16_storage(setup):
    fbl, G, xd, views = setup
    import torch
    y = fbl.project(G, xd, views)
    x64 = xd.cpu().numpy().astype(np.float64)  # the stored FP16 values, exactly
    rng = np.random.default_rng(21)
    n = 120
    rays = [(int(s), int(iu), int(iv)) for s, iu, iv in
            zip(rng.integers(0, len(views), n), rng.integers(0, GB.nu, n), rng.integers(0, GB.nv, n))]
    rays += [(0, 0, 0), (len(views) - 1, GB.nu - 1, GB.nv - 1), (3, GB.nu // 2, GB.nv // 2)]
    got = np.array([float(y[s, iv, iu]) for (s, iu, iv) in rays])
    ref = oracle.project_rays(GB, x64, [(views[s], iu, iv) for (s, iu, iv) in rays])
    del x64
    assert float(np.abs(ref).max()) > 100.0
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    assert y.dtype == torch.float32


def test_c5b_backproject_sampled_voxels(setup):
    fbl, G, xd, views = setup
    import torch
    gen = torch.Generator(device="cuda").manual_seed(22)
    y = torch.randn((len(views), GB.nv, GB.nu), device="cuda", generator=gen)
    xb = fbl.backproject(G, y, views)
    rng = np.random.default_rng(23)
    vox = [tuple(int(t) for t in rng.integers(0, 1024, 3)) for _ in range(8)]
    vox += [(0, 0, 0), (1023, 1023, 1023), (512, 511, 512), (200, 900, 17)]
    got = np.array([float(xb[k, j, i]) for (k, j, i) in vox])
    ref = oracle.backproject_voxels(GB, host(y), views, vox)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_c5b_fp16_learned_step(setup):
    fbl, G, xd, views = setup
    import torch
    from paper_2605_12085_gb300 import proposal
    net, _ = proposal.load()
    b = torch.empty((GB.n_views, GB.nv, GB.nu), dtype=torch.float16, device="cuda")
    for v0 in range(0, GB.n_views, 120):
        vs = list(range(v0, min(GB.n_views, v0 + 120)))
        b[v0:v0 + len(vs)] = fbl.project(G, xd, vs).to(torch.float16)
    p = fbl.params_default(N0=WL.N0, seed=WL.seed_batches, mu=WL.mu, alpha0=1e-3,
                           x_dtype=fbl.F16, b_dtype=fbl.F16, use_graph=1)
    S = fbl.fblisa_create(G, p)
    S.set_proposal(net)
    xs = torch.zeros(GB.vol_shape, dtype=torch.float16, device="cuda")
    prev_l1 = 0.0
    for it in range(2):
        st = S.step(xs, b)
        assert S.last_batch() == fblisa.epoch_batches(WL.seed_batches, 1, GB.n_views, WL.N0)[it]
        assert st["alpha_init"] == 1e-3 * 0.5 ** st["j_start"]
        assert st["alpha"] == 1e-3 * 0.5 ** (st["j_start"] + st["backtracks"])
        l1 = float(xs.double().sum())
        assert float(xs.min()) >= 0.0
        # (2.3) holds exactly on the stored point; the prox optimality (A3)
        # holds for the exact prox point p, and the stored x_bar = p + e with
        # |e| <= 2^-11 |p| (FP16) changes mu*||x||_1 + the quadratic model by
        # at most about mu * ||e||_1 <= 2^-11 mu ||x_bar||_1
        lhs = st["f_xbar"] + WL.mu * l1
        rhs = st["f_x"] + WL.mu * prev_l1 - st["dnorm2"] / (2 * st["alpha"])
        assert st["margin"] >= 0
        assert lhs <= rhs + 1e-6 * abs(rhs) + 2.0 ** -10 * WL.mu * l1
        assert lhs <= st["f_x"] + WL.mu * prev_l1
        prev_l1 = l1
