"""Batched FB-LISA over several uneven volumes (A10): every phase of an
iteration of all volumes runs as one persistent launch, and the whole
iteration (every volume's backtracking included) as one graph.

Each volume runs its own Algorithm 1, so its iterates, steps and mini-batches
must be bit-identical to a single-volume solver with the same geometry,
parameters and launch configuration; one volume is also checked against the
FP64 oracle (replaying the GPU's accepted steps).
"""
import numpy as np
import pytest

from oracle import fblisa
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

VOLS = [
    GEOMS["ragged"],                                   # 40 x 36 x 28, 24 views
    GEOMS["diag"],                                     # anisotropic voxels, 45-degree views
    GEOMS["angles"],                                   # non-uniform angles, clipping detector
    synth.small_geometry(nx=20, ny=28, nz=36, n_views=12, nu=44, nv=60),
]
PARAMS = [dict(N0=6, mu=0.5, alpha0=1e-2, seed=4), dict(N0=3, mu=0.2, alpha0=2e-2, seed=11),
          dict(N0=2, mu=1.0, alpha0=1e-2, seed=5), dict(N0=4, mu=0.3, alpha0=5e-2, seed=8)]


def _data():
    out = []
    for q, g in enumerate(VOLS):
        xt, b = problem(g, seed=40 + q)
        out.append(b.astype(np.float32))
    return out


@pytest.fixture(scope="module")
def data():
    return _data()


def _geoms(fbl, cfg):
    """Geometries with launch configurations: one (cols, split, vpl) for all,
    or a list of one per volume."""
    Gs = [fbl.geometry_create(g) for g in VOLS]
    cfgs = cfg if isinstance(cfg, list) else [cfg] * len(Gs)
    for G, c in zip(Gs, cfgs):
        fbl.geometry_set_launch(G, *c)
    return Gs


# per-volume plane-loop form and voxels per lane (the block width is common)
MIXED = [(8, 1, 4), (8, 0, 8), (8, 1, 16), (8, 0, 2)]


def _singles(fbl, Gs, bs, iters, dtype, torch_dtype, proposal=None, **extra):
    xs, traces = [], []
    for G, g, b, kw in zip(Gs, VOLS, bs, PARAMS):
        S = fbl.fblisa_create(G, fbl.params_default(x_dtype=dtype, b_dtype=dtype, **kw, **extra))
        if proposal is not None:
            S.set_proposal(proposal)
        x = cuda(np.zeros(g.vol_shape, np.float32), torch_dtype)
        bd = cuda(b, torch_dtype)
        tr = [S.step(x, bd) for _ in range(iters)]
        xs.append(host(x))
        traces.append(tr)
    return xs, traces


@pytest.mark.parametrize("cfg", [(8, 1, 4), (4, 0, 8), MIXED, [(8, 1, 24), (8, 0, 28), (8, 1, 8), (8, 0, 24)]])
def test_batch_is_bit_identical_to_single_volume_solvers(data, cfg):
    import torch
    import paper_2605_12085_gb300 as fbl
    Gs = _geoms(fbl, cfg)
    iters = 8  # crosses epoch boundaries of every volume
    ref_x, ref_tr = _singles(fbl, Gs, data, iters, fbl.F32, torch.float32)
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in PARAMS])
    info = B.info()
    big = max(range(len(VOLS)), key=lambda q: VOLS[q].n_vox)
    want = cfg[big] if isinstance(cfg, list) else cfg
    assert (info["k1_cols"], info["k1_split"], info["k2_vpl"]) == want
    xs = [cuda(np.zeros(g.vol_shape, np.float32)) for g in VOLS]
    bs = [cuda(b) for b in data]
    steps = [B.step(xs, bs) for _ in range(iters)]
    for v in range(len(VOLS)):
        got = [st[v] for st in steps]
        assert [t["alpha"] for t in got] == [t["alpha"] for t in ref_tr[v]]
        assert [t["backtracks"] for t in got] == [t["backtracks"] for t in ref_tr[v]]
        assert [t["N_t"] for t in got] == [t["N_t"] for t in ref_tr[v]]
        assert [t["f_x"] for t in got] == [t["f_x"] for t in ref_tr[v]]
        assert np.array_equal(host(xs[v]), ref_x[v])
    assert any(st[v]["backtracks"] > 0 for st in steps for v in range(len(VOLS)))
    assert info["launches"] == 0 and B.info()["launches"] > 0


def test_batch_mini_batches_follow_each_volumes_schedule(data):
    import paper_2605_12085_gb300 as fbl
    Gs = _geoms(fbl, (8, 1, 4))
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in PARAMS])
    xs = [cuda(np.zeros(g.vol_shape, np.float32)) for g in VOLS]
    bs = [cuda(b) for b in data]
    B.step(xs, bs)
    for v, (g, kw) in enumerate(zip(VOLS, PARAMS)):
        assert B.last_batch(v) == fblisa.epoch_batches(kw["seed"], 1, g.n_views, kw["N0"])[0]


def test_batch_volume_matches_fp64_oracle(data):
    import paper_2605_12085_gb300 as fbl
    Gs = _geoms(fbl, (8, 1, 4))
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in PARAMS])
    xs = [cuda(np.zeros(g.vol_shape, np.float32)) for g in VOLS]
    bs = [cuda(b) for b in data]
    steps = B.run(xs, bs, 8)
    g, kw = VOLS[0], PARAMS[0]
    p = fblisa.Params(alpha0=kw["alpha0"], beta=0.5, mu=kw["mu"], N0=kw["N0"], seed=kw["seed"])
    alphas = [st[0]["alpha"] for st in steps]
    b64 = data[0].astype(np.float64)
    # 8 iterations of volume 0 = 2 epochs of 4 batches of 6 views
    xo, recs = fblisa.run(g, b64, np.zeros(g.vol_shape), p, 2, replay=alphas)
    assert len(recs) == 8
    assert rel_l2(host(xs[0]), xo) <= 1e-4


def test_batch_with_learned_proposal_matches_single_solvers(data):
    import torch
    import paper_2605_12085_gb300 as fbl
    from paper_2605_12085_gb300 import proposal
    net, _ = proposal.load()
    Gs = _geoms(fbl, (8, 1, 8))
    ref_x, ref_tr = _singles(fbl, Gs, data, 6, fbl.F32, torch.float32, proposal=net)
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in PARAMS])
    B.set_proposal(net)
    xs = [cuda(np.zeros(g.vol_shape, np.float32)) for g in VOLS]
    bs = [cuda(b) for b in data]
    steps = [B.step(xs, bs) for _ in range(6)]
    for v in range(len(VOLS)):
        assert [st[v]["j_start"] for st in steps] == [t["j_start"] for t in ref_tr[v]]
        assert [st[v]["alpha"] for st in steps] == [t["alpha"] for t in ref_tr[v]]
        assert np.array_equal(host(xs[v]), ref_x[v])
    assert any(st[v]["j_start"] > 0 for st in steps for v in range(len(VOLS)))


def test_batch_bf16_and_host_buffers(data):
    import torch
    import paper_2605_12085_gb300 as fbl
    Gs = _geoms(fbl, (8, 1, 4))
    ref_x, ref_tr = _singles(fbl, Gs, data, 4, fbl.BF16, torch.bfloat16)
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(x_dtype=fbl.BF16, b_dtype=fbl.BF16, **kw)
                                     for kw in PARAMS])
    xs = [cuda(np.zeros(g.vol_shape, np.float32), torch.bfloat16) for g in VOLS]
    bs = [cuda(b, torch.bfloat16) for b in data]
    # host (CPU) buffers for half of the volumes
    xs[1], bs[1] = xs[1].cpu(), bs[1].cpu()
    xs[2] = xs[2].cpu()
    for _ in range(4):
        B.step(xs, bs)
    for v in range(len(VOLS)):
        assert np.array_equal(host(xs[v]), ref_x[v])


def test_batch_failing_volume_is_isolated(data):
    import paper_2605_12085_gb300 as fbl
    Gs = _geoms(fbl, (8, 1, 4))
    params = [dict(kw) for kw in PARAMS]
    params[2].update(force_reject=1, max_backtracks=3)
    B = fbl.fblisa_batch_create(Gs, [fbl.params_default(**kw) for kw in params])
    x0 = [np.full(g.vol_shape, 0.1, np.float32) for g in VOLS]
    xs = [cuda(x) for x in x0]
    bs = [cuda(b) for b in data]
    rc, st = B.step_raw(xs, bs)
    assert rc == 5
    assert st[2]["status"] == 5 and st[2]["backtracks"] == 3
    assert np.array_equal(host(xs[2]), x0[2].astype(np.float64))
    for v in (0, 1, 3):
        assert st[v]["status"] == 0
        assert not np.array_equal(host(xs[v]), x0[v].astype(np.float64))
    # the failed volume's schedule did not advance: its next batch is the same
    first = B.last_batch(2)
    B.step_raw(xs, bs)
    assert B.last_batch(2) == first


def test_batch_rejects_mixed_dtypes():
    import paper_2605_12085_gb300 as fbl
    Gs = [fbl.geometry_create(g) for g in VOLS[:2]]
    with pytest.raises(fbl.FblError):
        fbl.fblisa_batch_create(Gs, [fbl.params_default(N0=2),
                                     fbl.params_default(N0=2, x_dtype=fbl.BF16, b_dtype=fbl.BF16)])
    with pytest.raises(fbl.FblError):
        fbl.fblisa_batch_create(Gs, [fbl.params_default(N0=2, b_dtype=fbl.BF16),
                                     fbl.params_default(N0=2, b_dtype=fbl.BF16)])
