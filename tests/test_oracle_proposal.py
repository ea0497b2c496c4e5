"""Pins of the step-proposal oracle (oracle/proposal.py) to facts outside it.

The proposal has no counterpart in the paper (which restarts every line
search at alpha_0, Step 2d), so these pins come from the method and the
mathematics of the fidelity:

* without a network the proposal run is the plain method's run, iterate for
  iterate and step for step (oracle/fblisa.run);
* a predictor that returns exactly the change of the plain rule's accepted
  grid index makes every first trial the plain rule's accepted step: the run
  equals the plain run with no backtrack at all, for any margin in [0, 1/2)
  (pins the grid alpha_0 beta^j, the base j_prev and the rounding);
* every feature uses the data only through ratios: scaling x0, b and mu by s
  scales every iterate by s and leaves every feature and decision unchanged;
* f_N is the quadratic n_theta/(2N_t) ||A_N x - b_N||^2, so ||grad f_N||^2 <=
  2 L_N f_N with L_N = (n_theta/N_t) ||A_N||^2: the curvature index never
  exceeds log2(alpha_0 L_N), and with data along the top right singular
  vector of A_N it equals it at x = 0 (L_N from a dense SVD).
"""
import math

import numpy as np

import oracle
from oracle import fblisa, mlp
from oracle import proposal as prop
import synth


def _geom(n=8, views=6, det=13):
    return synth.Geometry(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, n_views=views, sod=60.0,
                          sdd=90.0, nu=det, nv=det - 2, du=1.5, dv=1.5)


def _problem(seed=0, g=None):
    g = g or _geom()
    rng = np.random.default_rng(seed)
    xt = synth.phantom(g, 4, 100 + seed).astype(np.float64)
    b = oracle.project(g, xt, range(g.n_views)) + 0.05 * rng.standard_normal((g.n_views, g.nv, g.nu))
    return g, xt, b


def _dense_A(g, views):
    cols = []
    for j in range(g.n_vox):
        e = np.zeros(g.n_vox)
        e[j] = 1.0
        cols.append(oracle.project(g, e.reshape(g.vol_shape), views).ravel())
    return np.stack(cols, axis=1)


def _params(**kw):
    base = dict(alpha0=0.02, beta=0.5, mu=0.3, N0=2, seed=11)
    base.update(kw)
    return fblisa.Params(**base)


def test_without_network_is_the_plain_method():
    g, xt, b = _problem(3)
    p = _params()
    x_plain, recs = fblisa.run(g, b, np.zeros(g.vol_shape), p, 2)
    x_prop, precs = prop.run(g, b, np.zeros(g.vol_shape), p, 2, predict=None)
    assert np.array_equal(x_plain, x_prop)
    assert [r.alpha for r in recs] == [q.step.alpha for q in precs]
    assert [r.backtracks for r in recs] == [q.step.backtracks for q in precs]
    assert all(q.j_start == 0 and q.step.alpha_init == p.alpha0 for q in precs)


def test_exact_predictor_reproduces_the_plain_run_without_backtracks():
    g, xt, b = _problem(4)
    p = _params(alpha0=0.05)
    x_plain, recs = fblisa.run(g, b, np.zeros(g.vol_shape), p, 3)
    # accepted grid index of the plain rule at every iteration (beta = 1/2: exact)
    jstar = [int(round(math.log2(p.alpha0 / r.alpha))) for r in recs]
    assert [p.alpha0 * 0.5 ** j for j in jstar] == [r.alpha for r in recs]
    assert max(jstar) >= 2 and len(set(jstar)) >= 2  # the plain rule backtracks, by varying amounts
    for margin in (0.0, 0.25, 0.49):
        calls = []

        def predict(feat):
            k = len(calls)
            calls.append(feat)
            return float(jstar[k] - (jstar[k - 1] if k else 0))

        x, precs = prop.run(g, b, np.zeros(g.vol_shape), p, 3, predict=predict, margin=margin)
        assert np.array_equal(x, x_plain)
        assert [q.j_start for q in precs] == jstar
        assert all(q.step.backtracks == 0 for q in precs)
        assert [q.step.alpha for q in precs] == [r.alpha for r in recs]
    # the features along that run, from the plain run's own records
    n = g.n_views
    for k, q in enumerate(precs):
        f, g2 = recs[k].f_x, recs[k].grad_norm2
        assert q.features[4] == recs[k].N_t / n
        assert math.isclose(q.features[5], 0.1 * math.log(1 + k), rel_tol=1e-12, abs_tol=1e-15)
        if k == 0:
            assert q.features[6] == 0 and q.features[1] == q.features[2] == q.features[3] == 0
            assert math.isclose(q.features[0], 0.1 * math.log2(p.alpha0 * g2 / (2 * f)), rel_tol=1e-12)
        else:
            fp, g2p = recs[k - 1].f_x, recs[k - 1].grad_norm2
            assert q.features[6] == 1 and q.features[0] == 0
            assert math.isclose(q.features[1], math.log(f / fp), rel_tol=1e-10, abs_tol=1e-13)
            assert math.isclose(q.features[2], math.log(math.sqrt(g2) / math.sqrt(g2p)), rel_tol=1e-10,
                                abs_tol=1e-13)
        assert q.features[7] == (0.25 * (jstar[k - 1] - jstar[k - 2]) if k >= 2 else 0.0)


def test_features_and_decisions_are_invariant_under_scaling():
    g, xt, b = _problem(5)
    p = _params(alpha0=0.05)
    net = prop.network(mlp.init(7))
    s = 3.7
    x1, r1 = prop.run(g, b, np.zeros(g.vol_shape) + 0.1, p, 2, predict=net)
    ps = _params(alpha0=0.05, mu=p.mu * s)
    x2, r2 = prop.run(g, s * b, s * (np.zeros(g.vol_shape) + 0.1), ps, 2, predict=net)
    assert len(r1) == len(r2) >= 6
    for a, c in zip(r1, r2):
        assert np.allclose(a.features, c.features, rtol=1e-9, atol=1e-11)
        assert a.j_start == c.j_start and a.step.backtracks == c.step.backtracks
        assert a.step.alpha == c.step.alpha
    assert np.allclose(x2, s * x1, rtol=1e-10, atol=1e-12)
    assert any(q.j_start > 0 for q in r1)  # the network moved the first trial


def test_curvature_index_is_bounded_by_the_lipschitz_constant():
    g, xt, b = _problem(6)
    p = _params(alpha0=0.05)
    x, recs = prop.run(g, b, np.zeros(g.vol_shape), p, 2, predict=prop.network(mlp.init(9)))
    c = 0.0
    for k, q in enumerate(recs):
        views = q.step.views
        L = (g.n_views / len(views)) * np.linalg.norm(_dense_A(g, views), 2) ** 2
        # c_k from the features alone: 10 * feature 0 at k = 0, plus 10 * feature 3 after
        c = 10.0 * q.features[0] if k == 0 else c + 10.0 * q.features[3]
        assert c <= math.log2(p.alpha0 * L) + 1e-9
        assert c >= math.log2(p.alpha0 * L) - 12.0  # not vacuous


def test_curvature_index_equals_the_bound_along_the_top_singular_vector():
    g = _geom(views=6)
    p = _params(alpha0=0.01, N0=2)
    views = fblisa.epoch_batches(p.seed, 1, g.n_views, 2)[0]
    A = _dense_A(g, views)
    U, sv, Vt = np.linalg.svd(A, full_matrices=False)
    u = Vt[0].reshape(g.vol_shape)
    b = oracle.project(g, u, range(g.n_views))
    x, recs = prop.run(g, b, np.zeros(g.vol_shape), p, 1, predict=None, max_iters=1)
    L = (g.n_views / len(views)) * sv[0] ** 2
    assert recs[0].step.views == list(views)
    assert math.isclose(recs[0].features[0], 0.1 * math.log2(p.alpha0 * L), rel_tol=1e-9)
