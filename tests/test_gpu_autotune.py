"""Autotuner and launch configurations (batched/tuned execution, A10).

Every launch configuration the autotuner may pick gives the projector and
backprojector parity with the FP64 oracle, and a tuned solver takes the same
FB-LISA steps as an untuned one."""
import itertools

import numpy as np
import pytest

import oracle
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cols,split,vpl", list(itertools.product((4, 8), (0, 1, 2), (2, 4, 8, 16, 24, 28))))
def test_every_launch_configuration_matches_oracle(cols, split, vpl):
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    G = fbl.geometry_create(g)
    fbl.geometry_set_launch(G, cols, split, vpl)
    rng = np.random.default_rng(cols + 10 * split + 100 * vpl)
    views = [0, 3, 9, 14, 22]
    x = rng.uniform(0, 1, g.vol_shape).astype(np.float32)
    y = rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32)
    assert rel_l2(host(fbl.project(G, cuda(x), views)), oracle.project(g, x.astype(np.float64), views)) <= 1e-5
    assert rel_l2(host(fbl.backproject(G, cuda(y), views)),
                  oracle.backproject(g, y.astype(np.float64), views)) <= 1e-5


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_group_backprojection_equals_single_column_bit_for_bit(name):
    # a 2x2 group of voxel columns per warp forms each column's z-profile once
    # for both in-plane neighbours: every voxel gets the same terms in the same
    # order as with one voxel column per warp, so the results are identical
    # (odd sizes leave partial groups; 45-degree views mix the two ray families)
    import torch
    import paper_2605_12085_gb300 as fbl
    g = GEOMS[name]
    G = fbl.geometry_create(g)
    rng = np.random.default_rng(5)
    views = list(range(g.n_views))
    y = cuda(rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32))
    for vpl in (4, 8):
        fbl.geometry_set_launch(G, 8, 1, vpl)
        one = fbl.backproject(G, y, views)
        fbl.geometry_set_launch(G, 8, 1, 20 + vpl)
        grp = fbl.backproject(G, y, views)
        torch.cuda.synchronize()
        assert torch.equal(one, grp)


def test_set_launch_rejects_bad_values():
    import paper_2605_12085_gb300 as fbl
    G = fbl.geometry_create(GEOMS["ragged"])
    with pytest.raises(fbl.FblError):
        fbl.geometry_set_launch(G, 16, 0, 4)


def test_autotuned_solver_takes_the_same_steps():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=3)
    bd = cuda(b.astype(np.float32))
    G = fbl.geometry_create(g)
    rep = fbl.geometry_autotune(G, n_sel=6)
    assert rep["k1_cols"] in (4, 8) and rep["k1_split"] in (0, 1, 2) and rep["k2_vpl"] in (2, 4, 8, 16, 24, 28)
    assert all(t > 0 for t in rep["k1_ms"]) and all(t > 0 for t in rep["k2_ms"])
    runs = []
    for tune in (0, 1):
        S = fbl.fblisa_create(G, fbl.params_default(N0=6, mu=0.5, alpha0=1e-2, seed=4, autotune=tune))
        x = cuda(np.zeros(g.vol_shape, np.float32))
        tr = S.run(x, bd, 2)
        runs.append((host(x), [t["alpha"] for t in tr]))
    assert runs[0][1] == runs[1][1]
    assert rel_l2(runs[0][0], runs[1][0]) <= 1e-6
