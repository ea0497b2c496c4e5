"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: relative L2 <= 1e-5 for FP32 projections, adjoints and trial
objectives; relative <= 1e-6 on the FP64 line-search reductions; iterates
after 10 epochs <= 1e-4.  Mini-batch indices are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fbl():
    import paper_2605_12085_gb300 as m
    return m


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_project_matches_oracle(fbl, name):
    g = GEOMS[name]
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 1.0, g.vol_shape).astype(np.float32)
    views = list(rng.permutation(g.n_views)[: max(1, g.n_views // 2)])
    G = fbl.geometry_create(g)
    y = host(fbl.project(G, cuda(x), views))
    ref = oracle.project(g, x.astype(np.float64), views)
    assert rel_l2(y, ref) <= TOL
    # every ray individually close (no missing planes at the edges)
    assert np.max(np.abs(y - ref)) <= 5e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_backproject_matches_oracle(fbl, name):
    g = GEOMS[name]
    rng = np.random.default_rng(2)
    views = list(rng.permutation(g.n_views)[: max(1, (g.n_views + 1) // 2)])
    y = rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32)
    G = fbl.geometry_create(g)
    x = host(fbl.backproject(G, cuda(y), views))
    ref = oracle.backproject(g, y.astype(np.float64), views)
    assert rel_l2(x, ref) <= TOL


def test_fine_detector_rows_take_the_row_by_row_taps(fbl):
    # rows at 0.5 mm under 1 mm voxels: five or more taps per voxel and column,
    # so the backprojector reads the residual row by row (no quad-row copy);
    # the operator and one solver step still match the oracle
    g = synth.small_geometry(nx=24, ny=22, nz=20, n_views=6, nu=40, nv=100, du=1.5, dv=0.5)
    G = fbl.geometry_create(g)
    B = fbl.fblisa_batch_create([G], [fbl.params_default(N0=3)])
    assert B.info()["ntap"] > 4
    rng = np.random.default_rng(8)
    views = [0, 2, 3, 5]
    y = rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32)
    x = host(fbl.backproject(G, cuda(y), views))
    assert rel_l2(x, oracle.backproject(g, y.astype(np.float64), views)) <= TOL
    xt, b = problem(g, seed=13)
    p = fblisa.Params(alpha0=1e-2, beta=0.5, mu=0.3, N0=3, seed=6)
    S = fbl.fblisa_create(G, _params(fbl, p))
    x0 = (0.5 * xt).astype(np.float32)
    xd = cuda(x0)
    st = S.step(xd, cuda(b.astype(np.float32)))
    xr, rec = fblisa.fb_step(g, x0.astype(np.float64), b.astype(np.float32).astype(np.float64),
                             S.last_batch(), p)
    assert st["backtracks"] == rec.backtracks
    assert rel_l2(host(xd), xr) <= TOL


def test_gpu_operators_are_adjoint(fbl):
    g = GEOMS["ragged"]
    rng = np.random.default_rng(3)
    views = [0, 5, 6, 11, 17, 23]
    x = rng.standard_normal(g.vol_shape).astype(np.float32)
    y = rng.standard_normal((len(views), g.nv, g.nu)).astype(np.float32)
    G = fbl.geometry_create(g)
    Ax = host(fbl.project(G, cuda(x), views))
    ATy = host(fbl.backproject(G, cuda(y), views))
    lhs = float(np.dot(Ax.ravel(), y.ravel().astype(np.float64)))
    rhs = float(np.dot(x.ravel().astype(np.float64), ATy.ravel()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_backproject_accumulate_and_host_buffers(fbl):
    g = GEOMS["angles"]
    rng = np.random.default_rng(4)
    views = [1, 3]
    y = rng.standard_normal((2, g.nv, g.nu)).astype(np.float32)
    G = fbl.geometry_create(g)
    x0 = rng.standard_normal(g.vol_shape).astype(np.float32)
    xd = cuda(x0)
    fbl.backproject(G, cuda(y), views, x=xd, accumulate=True)
    ref = x0 + oracle.backproject(g, y.astype(np.float64), views)
    assert rel_l2(host(xd), ref) <= TOL
    # host (numpy) buffers through the same entry points
    xh = np.zeros(g.vol_shape, dtype=np.float32)
    fbl.backproject(G, y, views, x=xh)
    assert rel_l2(xh, ref - x0) <= TOL
    yh = np.zeros((2, g.nv, g.nu), dtype=np.float32)
    fbl.project(G, x0, views, y=yh)
    assert rel_l2(yh, oracle.project(g, x0.astype(np.float64), views)) <= TOL


def test_empty_and_single_view(fbl):
    g = GEOMS["ragged"]
    G = fbl.geometry_create(g)
    x = np.ones(g.vol_shape, dtype=np.float32)
    y = fbl.project(G, cuda(x), [])
    assert tuple(y.shape) == (0, g.nv, g.nu)
    xb = fbl.backproject(G, cuda(np.zeros((0, g.nv, g.nu), np.float32)), [])
    assert float(host(xb).max()) == 0.0 and float(host(xb).min()) == 0.0
    y1 = host(fbl.project(G, cuda(x), [g.n_views - 1]))
    assert rel_l2(y1, oracle.project(g, x.astype(np.float64), [g.n_views - 1])) <= TOL


def test_invalid_views_rejected(fbl):
    g = GEOMS["ragged"]
    G = fbl.geometry_create(g)
    x = cuda(np.zeros(g.vol_shape, np.float32))
    with pytest.raises(fbl.FblError) as e:
        fbl.project(G, x, [0, g.n_views])
    assert e.value.status == 1


def test_residual_norm_matches_oracle(fbl):
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=5)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, g.vol_shape).astype(np.float32)
    views = [2, 7, 19]
    G = fbl.geometry_create(g)
    rho = fbl.residual_norm(G, cuda(x), views, cuda(b.astype(np.float32)))
    r = oracle.project(g, x.astype(np.float64), views) - b.astype(np.float32).astype(np.float64)[views]
    ref = float(np.dot(r.ravel(), r.ravel()))
    assert rho == pytest.approx(ref, rel=2 * TOL)
    rho_h = fbl.residual_norm(G, x, views, b.astype(np.float32))  # host buffers
    assert rho_h == pytest.approx(rho, rel=1e-12)


def test_prox_reduce_matches_definition(fbl):
    rng = np.random.default_rng(6)
    n = 1_000_003
    x = np.maximum(rng.standard_normal(n), 0).astype(np.float32)
    gr = (rng.standard_normal(n) * 3).astype(np.float32)
    alpha, mu = 0.013, 0.7
    xb, (gTd, dd, l1) = fbl.prox_reduce(cuda(x), cuda(gr), alpha, mu)
    xb = host(xb)
    ref = fblisa.prox(x.astype(np.float64) - alpha * gr.astype(np.float64), alpha, mu)
    assert np.max(np.abs(xb - ref)) <= 1e-6 * max(1.0, np.abs(ref).max())
    d = xb - x.astype(np.float64)
    assert gTd == pytest.approx(float(np.dot(gr.astype(np.float64), d)), rel=1e-6)
    assert dd == pytest.approx(float(np.dot(d, d)), rel=1e-6)
    assert l1 == pytest.approx(float(xb.sum()), rel=1e-6)


def _params(fbl, p: fblisa.Params, **kw):
    return fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, C=p.C, eps_base=p.eps_base,
                              N0=p.N0, n_max=p.n_max, max_backtracks=p.max_backtracks,
                              seed=p.seed, **kw)


def test_single_step_matches_oracle(fbl):
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=7)
    p = fblisa.Params(alpha0=1e-2, beta=0.5, mu=0.5, N0=6, seed=99)
    rng = np.random.default_rng(7)
    x0 = (0.5 * xt + 0.1 * rng.uniform(0, 1, g.vol_shape)).astype(np.float32)
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, _params(fbl, p))
    xd = cuda(x0)
    st = S.step(xd, cuda(b.astype(np.float32)))
    views = S.last_batch()
    assert views == fblisa.epoch_batches(p.seed, 1, g.n_views, 6)[0]
    xr, rec = fblisa.fb_step(g, x0.astype(np.float64), b.astype(np.float32).astype(np.float64),
                             views, p)
    assert st["backtracks"] == rec.backtracks
    assert st["alpha"] == rec.alpha
    assert st["f_x"] == pytest.approx(rec.f_x, rel=2e-5)
    assert st["f_xbar"] == pytest.approx(rec.trials[-1].f_xbar, rel=2e-5)
    assert st["dnorm2"] == pytest.approx(rec.trials[-1].dnorm2, rel=1e-4)
    assert rel_l2(host(xd), xr) <= TOL


def _run_pair(fbl, wl_geom, b, p, epochs):
    G = fbl.geometry_create(wl_geom)
    S = fbl.fblisa_create(G, _params(fbl, p))
    x = cuda(np.zeros(wl_geom.vol_shape, np.float32))
    trace = S.run(x, cuda(b.astype(np.float32)), epochs)
    return host(x), trace


def test_run_c1_matches_oracle_10_epochs(fbl):
    wl = synth.WORKLOADS["c1_64"]
    g = wl.geom
    xt, b = problem(g, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    b32 = b.astype(np.float32).astype(np.float64)
    p = fblisa.Params(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    xg, trace = _run_pair(fbl, g, b32, p, 10)
    alphas = [t["alpha"] for t in trace]
    # the oracle replays the GPU's accepted steps (decisions compared below)
    xo, recs = fblisa.run(g, b32, np.zeros(g.vol_shape), p, 10, replay=alphas)
    assert len(recs) == len(trace) == 90
    assert [r.views for r in recs][:1] == [fblisa.epoch_batches(p.seed, 1, 90, 10)[0]]
    flips = sum(1 for r in recs if r.trials[-1].rhs - r.trials[-1].f_xbar < 0)
    assert flips == 0, "oracle rejects %d of the GPU's accepted steps" % flips
    assert rel_l2(xg, xo) <= 1e-4
    # free-running oracle takes the same decisions
    xf, recf = fblisa.run(g, b32, np.zeros(g.vol_shape), p, 10)
    assert [r.alpha for r in recf] == alphas
    assert rel_l2(xg, xf) <= 1e-4


def test_forced_reject_hits_cap_and_leaves_x(fbl):
    g = GEOMS["angles"]
    xt, b = problem(g, seed=9)
    G = fbl.geometry_create(g)
    p = fbl.params_default(N0=2, max_backtracks=3, force_reject=1, mu=0.1)
    S = fbl.fblisa_create(G, p)
    x0 = np.full(g.vol_shape, 0.25, np.float32)
    xd = cuda(x0)
    rc, st = S.step_raw(xd, cuda(b.astype(np.float32)))
    assert rc == 5 and st["status"] == 5 and st["backtracks"] == 3
    assert np.array_equal(host(xd), x0.astype(np.float64))


def test_nonfinite_data_reported(fbl):
    g = GEOMS["angles"]
    xt, b = problem(g, seed=10)
    b = b.astype(np.float32)
    b[:, 3, 4] = np.nan
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(N0=5, mu=0.1))
    xd = cuda(np.zeros(g.vol_shape, np.float32))
    rc, st = S.step_raw(xd, cuda(b))
    assert rc == 6


def test_evaluate_full_objective_and_relative_error(fbl):
    g = synth.WORKLOADS["c1_64"].geom
    xt, b = problem(g, seed=12)
    rng = np.random.default_rng(12)
    x = np.maximum(xt + 0.05 * rng.standard_normal(g.vol_shape), 0).astype(np.float32)
    G = fbl.geometry_create(g)
    b32 = b.astype(np.float32)
    F, fid, re = fbl.evaluate(G, cuda(x), cuda(b32), 0.7, x_true=cuda(xt.astype(np.float32)))
    Fo = fblisa.full_objective(g, x.astype(np.float64), b32.astype(np.float64), 0.7)
    assert F == pytest.approx(Fo, rel=2e-5)
    xt32 = xt.astype(np.float32).astype(np.float64)
    assert re == pytest.approx(np.linalg.norm(x - xt32) / np.linalg.norm(xt32), rel=1e-5)
    Fh, fidh, reh = fbl.evaluate(G, x, b32, 0.7)  # host buffers, no reference volume
    assert Fh == pytest.approx(F, rel=1e-12) and reh == 0.0
