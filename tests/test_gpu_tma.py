"""The TMA-staged projector (launch configuration k1_split = 2): the volume
reaches each block as shared-memory bricks copied by cp.async.bulk.tensor.

It walks the same planes of the same rays in the same order, with the same
accumulation, as the masked plane loop (k1_split = 0) with 8 columns per
block, and only the source of each voxel value changes (brick or global
copy), so its results must be bit-identical to that configuration -- which
checks every brick origin and index; it must also match the FP64 oracle.
Covered: ragged sizes, views on the 45-degree family boundary (blocks with
two families), a detector that clips the volume, the three storage types,
the residual and objective epilogues, and a solver run.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

TMA = (8, 2, 4)
MASKED8 = (8, 0, 4)


def _pair(fbl, g):
    Gt = fbl.geometry_create(g)
    fbl.geometry_set_launch(Gt, *TMA)
    Gm = fbl.geometry_create(g)
    fbl.geometry_set_launch(Gm, *MASKED8)
    return Gt, Gm


@pytest.mark.parametrize("name", sorted(GEOMS) + ["wide"])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_tma_projection_bit_identical_to_masked_loop(name, dtype):
    import torch
    import paper_2605_12085_gb300 as fbl
    # "wide": a strong cone and thin voxels along z, so 32 detector rows span
    # more z than a brick holds and every chunk takes the global-read path
    g = GEOMS.get(name) or synth.Geometry(nx=72, ny=64, nz=80, vx=1.0, vy=1.0, vz=0.4, n_views=16,
                                          sod=300.0, sdd=600.0, nu=150, nv=48, du=1.0, dv=1.5)
    td = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 1.0, g.vol_shape).astype(np.float32)
    views = list(range(g.n_views))
    Gt, Gm = _pair(fbl, g)
    xd = cuda(x, td)
    yt = host(fbl.project(Gt, xd, views))
    ym = host(fbl.project(Gm, xd, views))
    assert np.array_equal(yt, ym)
    ref = oracle.project(g, host(xd), views)
    assert rel_l2(yt, ref) <= 1e-5


def test_tma_residual_and_objective_epilogues():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=61)
    rng = np.random.default_rng(61)
    x = rng.uniform(0, 1, g.vol_shape).astype(np.float32)
    views = [1, 4, 9, 16, 23]
    Gt, Gm = _pair(fbl, g)
    bd = cuda(b.astype(np.float32))
    rt = fbl.residual_norm(Gt, cuda(x), views, bd)
    rm = fbl.residual_norm(Gm, cuda(x), views, bd)
    assert rt == rm
    F_t = fbl.evaluate(Gt, cuda(x), bd, 0.5)
    F_m = fbl.evaluate(Gm, cuda(x), bd, 0.5)
    assert F_t == F_m


def test_tma_solver_matches_masked_solver():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=62)
    bd = cuda(b.astype(np.float32))
    Gt, Gm = _pair(fbl, g)
    out = []
    for G in (Gt, Gm):
        for graph in (0, 1):
            S = fbl.fblisa_create(G, fbl.params_default(N0=6, mu=0.5, alpha0=1e-2, seed=4,
                                                        use_graph=graph))
            x = cuda(np.zeros(g.vol_shape, np.float32))
            tr = S.run(x, bd, 2)
            out.append((host(x), [t["alpha"] for t in tr]))
    for xo, al in out[1:]:
        assert al == out[0][1]
        assert np.array_equal(xo, out[0][0])
