"""Graph-captured FB-LISA iterations (A10): the whole iteration, backtracking
included, as one CUDA graph whose WHILE node runs trials until the device-side
test of (2.3) accepts.  The decisions are the host loop's, so the iterates must
be bit-identical to the host-driven solver, and failure modes must be the
same."""
import numpy as np
import pytest

from oracle import fblisa
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu


def _solver(fbl, G, graph, **kw):
    base = dict(N0=6, mu=0.5, alpha0=1e-2, seed=4)
    base.update(kw)
    return fbl.fblisa_create(G, fbl.params_default(use_graph=graph, **base))


def test_graph_mode_is_bit_identical_to_host_loop():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=21)
    bd = cuda(b.astype(np.float32))
    G = fbl.geometry_create(g)
    out = []
    for graph in (0, 1):
        S = _solver(fbl, G, graph)
        x = cuda(np.zeros(g.vol_shape, np.float32))
        tr = S.run(x, bd, 3)
        out.append((host(x), tr))
    (x0, t0), (x1, t1) = out
    assert [t["alpha"] for t in t0] == [t["alpha"] for t in t1]
    assert [t["backtracks"] for t in t0] == [t["backtracks"] for t in t1]
    assert any(t["backtracks"] > 0 for t in t1)
    assert np.array_equal(x0, x1)
    for a, c in zip(t0, t1):
        assert a["f_x"] == c["f_x"] and a["f_xbar"] == c["f_xbar"] and a["margin"] == c["margin"]


def test_graph_mode_host_data_and_oracle():
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["c1_64"]
    g = wl.geom
    xt, b = problem(g, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    b32 = b.astype(np.float32)
    p = fblisa.Params(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, N0=p.N0,
                                                seed=p.seed, use_graph=1))
    x = np.zeros(g.vol_shape, np.float32)  # host iterate and host data through the graph path
    tr = S.run(x, b32, 3)
    xo, recs = fblisa.run(g, b32.astype(np.float64), np.zeros(g.vol_shape), p, 3)
    assert [t["alpha"] for t in tr] == [r.alpha for r in recs]
    assert rel_l2(x, xo) <= 1e-4


def test_graph_mode_backtrack_cap_and_nonfinite():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["angles"]
    xt, b = problem(g, seed=22)
    G = fbl.geometry_create(g)
    S = _solver(fbl, G, 1, N0=2, max_backtracks=4, force_reject=1)
    x0 = np.full(g.vol_shape, 0.25, np.float32)
    xd = cuda(x0)
    rc, st = S.step_raw(xd, cuda(b.astype(np.float32)))
    assert rc == 5 and st["backtracks"] == 4
    assert np.array_equal(host(xd), x0.astype(np.float64))
    bn = b.astype(np.float32)
    bn[:, 2, 3] = np.nan
    S2 = _solver(fbl, G, 1, N0=5)
    rc, st = S2.step_raw(cuda(np.zeros(g.vol_shape, np.float32)), cuda(bn))
    assert rc == 6
