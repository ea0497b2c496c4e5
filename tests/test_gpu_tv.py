"""Other regularisers on the GPU against the FP64 oracle (oracle/tv.py,
pinned by closed forms, the adjoint and the duality gap):

* prox_tv (FGP on the dual, FP32) on ragged, thin and one-voxel volumes, with
  and without an upper bound, from zero and from a given dual (device and host
  buffers), lambda = 0 and zero iterations; tv_norm;
* the solver with R = mu TV + box (reg = FBL_REG_TV, the dual carried from one
  prox to the next): its steps equal the free-running oracle's and its
  iterate matches;
* the solver with R = mu ||x||_1 + box (finite x_max): host loop against the
  oracle, the graph-captured iteration and the batched launch bit for bit
  against the host loop, and the bound holds;
* the combinations the library refuses.

Tolerances: 1e-5 relative L2 on prox_tv's volume (FP32 arithmetic through 20
iterations of a nonexpansive map), 1e-4 on its dual (components on the unit
sphere are decided by FP32 projections) and on iterates after several solver
steps, as for the other solver tests.
"""
import math

import numpy as np
import pytest

from oracle import fblisa
from oracle import tv as otv
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
SHAPES = [(19, 23, 37), (3, 5, 300), (8, 1, 1), (40, 48, 64)]  # [nz][ny][nx]


def _vol(shape, seed):
    rng = np.random.default_rng(seed)
    base = np.zeros(shape)
    nz, ny, nx = shape
    base[:, : ny // 2, : nx // 3] = 0.8                          # a block with edges
    return (base + 0.3 * rng.uniform(0, 1, shape)).astype(np.float32)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lam,x_max", [(0.05, math.inf), (0.2, 0.7)])
def test_prox_tv_matches_oracle(shape, lam, x_max):
    import torch
    import paper_2605_12085_gb300 as fbl
    v = _vol(shape, 11)
    q = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    x = host(fbl.prox_tv(cuda(v), lam, 20, x_max, q=q))
    xo, qo = otv.prox_tv(v.astype(np.float64), lam, 20, x_max)
    assert rel_l2(x, xo) <= TOL
    assert rel_l2(host(q), qo) <= 1e-4
    assert x.min() >= 0.0 and x.max() <= np.float32(x_max)


def test_prox_tv_warm_start_host_buffers_and_edges():
    import paper_2605_12085_gb300 as fbl
    shape = (9, 14, 33)
    v = _vol(shape, 12)
    v64 = v.astype(np.float64)
    _, q0 = otv.prox_tv(v64, 0.1, 40)
    q0 = q0.astype(np.float32)
    q0[0, :, :, -1] = 5.0  # components without a difference are ignored (zeroed)
    qh = q0.copy()
    xh = np.zeros(shape, np.float32)
    fbl.prox_tv(v, 0.1, 6, q=qh, q_in=True, x=xh)  # host v, q, x
    xo, qo = otv.prox_tv(v64, 0.1, 6, q0=q0.astype(np.float64))
    assert rel_l2(xh, xo) <= TOL
    assert rel_l2(qh, qo) <= 1e-4 and not qh[0, :, :, -1].any()
    # lambda = 0 and zero iterations: the box projection of v (resp. of v - lam K^T q0)
    w = (v - 0.5).astype(np.float32)
    assert np.array_equal(host(fbl.prox_tv(cuda(w), 0.0, 10, 0.3)), np.clip(w, 0, np.float32(0.3)))
    x0 = host(fbl.prox_tv(cuda(v), 0.1, 0, q=cuda(q0), q_in=True))
    xo0, _ = otv.prox_tv(v64, 0.1, 0, q0=q0.astype(np.float64))
    assert rel_l2(x0, xo0) <= TOL
    one = np.array([[[1.7]]], np.float32)
    assert float(host(fbl.prox_tv(cuda(one), 0.5, 20, 1.0)).ravel()[0]) == 1.0


@pytest.mark.parametrize("shape", SHAPES)
def test_tv_norm_matches_oracle(shape):
    import paper_2605_12085_gb300 as fbl
    v = _vol(shape, 13)
    assert fbl.tv_norm(cuda(v)) == pytest.approx(otv.tv(v.astype(np.float64)), rel=1e-6)
    assert fbl.tv_norm(v) == pytest.approx(otv.tv(v.astype(np.float64)), rel=1e-6)


def _wl():
    wl = synth.WORKLOADS["c1_64"]
    xt, b = problem(wl.geom, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    return wl, xt, b.astype(np.float32)


def test_solver_tv_matches_oracle():
    import paper_2605_12085_gb300 as fbl
    wl, xt, b32 = _wl()
    g = wl.geom
    kw = dict(alpha0=1e-3, beta=0.5, mu=20.0, N0=wl.N0, seed=wl.seed_batches)
    p = fblisa.Params(reg="tv", tv_iters=10, **kw)
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(reg=fbl.REG_TV, tv_iters=10, **kw))
    x = cuda(np.zeros(g.vol_shape, np.float32))
    bd = cuda(b32)
    n_it = 6
    trace = [S.step(x, bd) for _ in range(n_it)]
    xo, recs = fblisa.run(g, b32.astype(np.float64), np.zeros(g.vol_shape), p, 1, max_iters=n_it)
    assert [t["alpha"] for t in trace] == [r.alpha for r in recs]
    assert [t["f_x"] for t in trace] == pytest.approx([r.f_x for r in recs], rel=2e-5)
    assert sum(t["backtracks"] for t in trace) > 0
    assert rel_l2(host(x), xo) <= 1e-4
    # TV lowered: against the same run with the l1 regulariser of the same weight
    S1 = fbl.fblisa_create(G, fbl.params_default(**kw))
    x1 = cuda(np.zeros(g.vol_shape, np.float32))
    for _ in range(n_it):
        S1.step(x1, bd)
    assert fbl.tv_norm(x) < fbl.tv_norm(x1)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_solver_tv_low_precision_storage(dtype):
    # the storage types of the iterate (FP32 arithmetic): the same steps as the
    # FP32 TV solver and iterates within the storage rounding
    import torch
    import paper_2605_12085_gb300 as fbl
    wl, xt, b32 = _wl()
    g = wl.geom
    code, td = {"bf16": (fbl.BF16, torch.bfloat16), "f16": (fbl.F16, torch.float16)}[dtype]
    kw = dict(alpha0=1e-3, beta=0.5, mu=20.0, N0=wl.N0, seed=wl.seed_batches, reg=fbl.REG_TV, tv_iters=10,
              x_max=0.8)
    G = fbl.geometry_create(g)
    n_it = 4
    S32 = fbl.fblisa_create(G, fbl.params_default(**kw))
    x32 = cuda(np.zeros(g.vol_shape, np.float32))
    tr32 = [S32.step(x32, cuda(b32)) for _ in range(n_it)]
    S = fbl.fblisa_create(G, fbl.params_default(x_dtype=code, b_dtype=code, **kw))
    x = cuda(np.zeros(g.vol_shape, np.float32), td)
    tr = [S.step(x, cuda(b32, td)) for _ in range(n_it)]
    assert [t["alpha"] for t in tr] == [t["alpha"] for t in tr32]
    xh = host(x)
    assert np.isfinite(xh).all() and xh.min() >= 0.0 and xh.max() <= 0.8
    assert rel_l2(xh, host(x32)) <= 1e-2


def test_solver_l1_box_host_graph_and_oracle():
    import paper_2605_12085_gb300 as fbl
    wl, xt, b32 = _wl()
    g = wl.geom
    kw = dict(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    G = fbl.geometry_create(g)
    bd = cuda(b32)
    n_it = 12
    # a bound the iterate reaches: half the largest value of the unbounded run
    S0 = fbl.fblisa_create(G, fbl.params_default(**kw))
    x0 = cuda(np.zeros(g.vol_shape, np.float32))
    for _ in range(n_it):
        S0.step(x0, bd)
    x_max = 0.5 * float(host(x0).max())
    out = []
    for graph in (0, 1):
        S = fbl.fblisa_create(G, fbl.params_default(x_max=x_max, use_graph=graph, **kw))
        x = cuda(np.zeros(g.vol_shape, np.float32))
        tr = [S.step(x, bd) for _ in range(n_it)]
        out.append((host(x), [t["alpha"] for t in tr]))
    assert out[0][1] == out[1][1] and np.array_equal(out[0][0], out[1][0])
    xg = out[0][0]
    assert xg.max() <= np.float32(x_max) and (xg == np.float32(x_max)).sum() > 0
    p = fblisa.Params(x_max=x_max, **kw)
    xo, recs = fblisa.run(g, b32.astype(np.float64), np.zeros(g.vol_shape), p, 2, max_iters=n_it)
    assert [r.alpha for r in recs] == out[0][1]
    assert rel_l2(xg, xo) <= 1e-4


def test_batch_with_box_matches_single_solvers():
    import paper_2605_12085_gb300 as fbl
    vols = [GEOMS["ragged"], GEOMS["diag"]]
    kws = [dict(N0=6, mu=0.5, alpha0=1e-2, seed=4), dict(N0=3, mu=0.2, alpha0=2e-2, seed=11)]
    data = [problem(g, seed=60 + q)[1].astype(np.float32) for q, g in enumerate(vols)]
    Gs = [fbl.geometry_create(g) for g in vols]
    for G in Gs:
        fbl.geometry_set_launch(G, 8, 1, 4)
    iters = 6
    for G, g, b, kw in zip(Gs, vols, data, kws):  # bounds the iterates reach
        S = fbl.fblisa_create(G, fbl.params_default(**kw))
        x = cuda(np.zeros(g.vol_shape, np.float32))
        for _ in range(iters):
            S.step(x, cuda(b))
        kw["x_max"] = 0.5 * float(host(x).max())
    ref = []
    for G, g, b, kw in zip(Gs, vols, data, kws):
        S = fbl.fblisa_create(G, fbl.params_default(**kw))
        x = cuda(np.zeros(g.vol_shape, np.float32))
        tr = [S.step(x, cuda(b)) for _ in range(iters)]
        ref.append((host(x), [t["alpha"] for t in tr]))
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in kws])
    xs = [cuda(np.zeros(g.vol_shape, np.float32)) for g in vols]
    steps = [B.step(xs, [cuda(b) for b in data]) for _ in range(iters)]
    for v in range(2):
        assert [st[v]["alpha"] for st in steps] == ref[v][1]
        assert np.array_equal(host(xs[v]), ref[v][0])
        assert ref[v][0].max() <= np.float32(kws[v]["x_max"])
        assert (ref[v][0] == np.float32(kws[v]["x_max"])).sum() > 0


def test_refused_combinations():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    G = fbl.geometry_create(g)
    with pytest.raises(RuntimeError, match="host-loop"):
        fbl.fblisa_create(G, fbl.params_default(reg=fbl.REG_TV, use_graph=1))
    with pytest.raises(RuntimeError, match="x_max"):
        fbl.fblisa_create(G, fbl.params_default(x_max=0.0))
    with pytest.raises(RuntimeError, match="reg"):
        fbl.fblisa_create(G, fbl.params_default(reg=7))
    with pytest.raises(RuntimeError, match="l1 prox"):
        fbl.fblisa_batch_create([G], [fbl.params_default(reg=fbl.REG_TV)])
    with pytest.raises(RuntimeError):
        fbl.prox_tv(cuda(np.zeros((2, 2, 2), np.float32)), -1.0, 5)
