"""The paper's comparators on the same kernels (Sec. 3): the deterministic
forward-backward method with a constant step and no line search
(fbl_params.fixed_step, N0 = n_max = n_views), and FB-LISA with the full batch
(a proximal gradient method with backtracking, so F decreases monotonically).
"""
import math

import numpy as np
import pytest

from oracle import fblisa
import synth
from gpu_common import cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["c1_64"]
G1 = WL.geom


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2605_12085_gb300 as fbl
    xt, b = problem(G1, n_ell=WL.n_ellipsoids, seed=WL.seed_phantom, noise_rel=WL.noise_rel)
    b32 = b.astype(np.float32)
    G = fbl.geometry_create(G1)
    # L = ||A||^2 of the full-batch fidelity 1/2 ||A x - b||^2, by power iteration
    views = list(range(G1.n_views))
    v = torch.ones(G1.vol_shape, dtype=torch.float32, device="cuda")
    lam = 0.0
    for _ in range(30):
        w = fbl.backproject(G, fbl.project(G, v, views), views)
        lam = float(torch.linalg.vector_norm(w) / torch.linalg.vector_norm(v))
        v = w / torch.linalg.vector_norm(w)
    yield fbl, G, b32, lam * 1.02  # a little above the estimate (power iteration approaches from below)


@pytest.mark.parametrize("N0", [90, 10])
def test_fixed_step_fb_matches_oracle(setup, N0):
    fbl, G, b32, L = setup
    alpha = 0.9 / L * (N0 / G1.n_views)  # conservative for the mini-batch fidelity too
    p = fblisa.Params(alpha0=alpha, mu=WL.mu, N0=N0, seed=WL.seed_batches, fixed_step=True)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=alpha, mu=WL.mu, N0=N0, seed=WL.seed_batches,
                                                fixed_step=1))
    x = cuda(np.zeros(G1.vol_shape, np.float32))
    n_it = 6
    bd = cuda(b32)
    st = [S.step(x, bd) for _ in range(n_it)]
    assert all(s["backtracks"] == 0 and s["alpha"] == alpha for s in st)
    assert all(math.isnan(s["f_xbar"]) and math.isnan(s["margin"]) for s in st)
    xo, recs = fblisa.run(G1, b32.astype(np.float64), np.zeros(G1.vol_shape), p,
                          epochs=1 if N0 < G1.n_views else n_it, max_iters=n_it)
    assert len(recs) == n_it
    assert [s["f_x"] for s in st] == pytest.approx([r.f_x for r in recs], rel=2e-5)
    assert rel_l2(host(x), xo) <= 1e-4


def test_fixed_step_full_batch_decreases_F(setup):
    fbl, G, b32, L = setup
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=0.9 / L, mu=WL.mu, N0=G1.n_views, fixed_step=1))
    x = cuda(np.zeros(G1.vol_shape, np.float32))
    bd = cuda(b32)
    F = [fbl.evaluate(G, x, bd, WL.mu)[0]]
    for _ in range(8):
        S.step(x, bd)
        F.append(fbl.evaluate(G, x, bd, WL.mu)[0])
    assert all(F[i + 1] <= F[i] * (1 + 1e-6) for i in range(len(F) - 1))
    assert F[-1] < 0.5 * F[0]


def test_full_batch_fblisa_is_monotone(setup):
    fbl, G, b32, L = setup
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=1e-2, mu=WL.mu, N0=G1.n_views, seed=3))
    x = cuda(np.zeros(G1.vol_shape, np.float32))
    bd = cuda(b32)
    F = [fbl.evaluate(G, x, bd, WL.mu)[0]]
    for _ in range(8):
        st = S.step(x, bd)
        assert st["N_t"] == G1.n_views
        F.append(fbl.evaluate(G, x, bd, WL.mu)[0])
    assert all(F[i + 1] <= F[i] * (1 + 1e-6) for i in range(len(F) - 1))


def test_batch_rejects_fixed_step():
    import paper_2605_12085_gb300 as fbl
    G = fbl.geometry_create(G1)
    with pytest.raises(fbl.FblError):
        fbl.fblisa_batch_create([G], [fbl.params_default(N0=10, fixed_step=1)])
