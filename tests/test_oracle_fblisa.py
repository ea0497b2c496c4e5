"""Pins of the oracle's Algorithm 1 (FB-LISA) to facts outside the oracle.

* prox (Sec. 2.2's prox_{alpha R}, R = mu||.||_1 + indicator{x >= 0}) against a
  brute-force 1-D minimisation of its defining problem;
* grad f_N against central differences of f_N (exact for a quadratic);
* unbiasedness: the mean of f_N over every mini-batch of size N_t equals the
  fidelity 1/2||Ax - b||^2 of eq. (2.1) -- this pins the n_theta/N_t factor of
  eq. (2.5);
* the Lemma of the appendix: any alpha <= 1/L passes (2.3) at once, and the
  accepted alpha exceeds beta/L, with L the Lipschitz constant of grad f_N
  from a dense SVD;
* (2.3) plus the prox optimality (A3) give F_N(x_bar) <= F_N(x) - ||d||^2/(2 alpha)
  on every accepted step;
* with N_0 = n_max = n_theta the method is deterministic proximal gradient with
  backtracking, so the full objective F never increases;
* Step 1's schedule: N_t stays at N_0 = 8 until ceil(0.99^-K) first exceeds 8,
  which the closed form puts at K = 207 (epoch 23 for n_theta = 72), and the
  batch grows from 8 to 13 without reaching full batch within ~250
  iterations, as Sec. 3 reports for Case 3 (Fig. 2 discussion);
* the per-epoch permutations are permutations with uniform marginals;
* SplitMix64's first outputs equal the published reference outputs for three
  starting states (tests/golden/splitmix64.txt).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth


def _geom(n=8, views=6, det=13):
    return synth.Geometry(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, n_views=views, sod=60.0,
                          sdd=90.0, nu=det, nv=det - 2, du=1.5, dv=1.5)


def _dense_A(g, views):
    cols = []
    for j in range(g.n_vox):
        e = np.zeros(g.n_vox)
        e[j] = 1.0
        cols.append(oracle.project(g, e.reshape(g.vol_shape), views).ravel())
    return np.stack(cols, axis=1)


def _problem(seed=0, g=None):
    g = g or _geom()
    rng = np.random.default_rng(seed)
    xt = synth.phantom(g, 4, 100 + seed).astype(np.float64)
    b = oracle.project(g, xt, range(g.n_views)) + 0.05 * rng.standard_normal((g.n_views, g.nv, g.nu))
    return g, xt, b


def test_prox_matches_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(50):
        v = float(rng.uniform(-2, 2))
        alpha = float(rng.uniform(0.01, 1.0))
        mu = float(rng.uniform(0.0, 3.0))
        z = np.linspace(0.0, 4.0, 400001)          # the feasible set z >= 0
        obj = 0.5 * (z - v) ** 2 + alpha * mu * np.abs(z)
        zbest = z[np.argmin(obj)]
        got = float(fblisa.prox(np.array([v]), alpha, mu)[0])
        assert abs(got - zbest) <= 2e-5


def test_gradient_is_derivative_of_f_N():
    g, xt, b = _problem(1)
    views = [0, 3, 4]
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, g.vol_shape)
    scale = g.n_views / len(views)

    def f_N(z):
        r = oracle.project(g, z, views) - b[views]
        return 0.5 * scale * float(np.dot(r.ravel(), r.ravel()))

    r = oracle.project(g, x, views) - b[views]
    grad = scale * oracle.backproject(g, r, views)
    for _ in range(5):
        e = rng.standard_normal(g.vol_shape)
        h = 1e-3
        fd = (f_N(x + h * e) - f_N(x - h * e)) / (2 * h)
        assert fd == pytest.approx(float(np.dot(grad.ravel(), e.ravel())), rel=1e-8)


def test_minibatch_objective_is_unbiased():
    g, xt, b = _problem(2, _geom(views=6))
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, g.vol_shape)
    r_all = oracle.project(g, x, range(g.n_views)) - b
    full = 0.5 * float(np.dot(r_all.ravel(), r_all.ravel()))
    for N_t in (1, 2, 4):
        vals = []
        for S in itertools.combinations(range(g.n_views), N_t):
            r = r_all[list(S)]
            vals.append(g.n_views / (2 * N_t) * float(np.dot(r.ravel(), r.ravel())))
        assert np.mean(vals) == pytest.approx(full, rel=1e-12)


def test_fb_step_quantities_are_unbiased_and_consistent():
    # eq. (2.5) through fb_step itself: over all C(6, 2) mini-batches the mean
    # of f_N(x) is 1/2 ||A x - b||^2 and the mean stochastic gradient is
    # A^T (A x - b) from the explicit matrix.  The gradient is read off
    # x_bar = x - alpha g (mu = 0 and x large, so nothing is clipped); each
    # trial's f_N(x_bar) equals f_N at x_bar from a second step.
    g, xt, b = _problem(8, _geom(views=6))
    A = _dense_A(g, range(g.n_views))
    x = 5.0 + np.random.default_rng(8).uniform(0, 1, g.vol_shape)
    r_all = A @ x.ravel() - b.ravel()
    alpha = 1e-4
    p = fblisa.Params(alpha0=alpha, beta=0.5, mu=0.0)
    fs, gs = [], []
    for S in itertools.combinations(range(g.n_views), 2):
        xb, rec = fblisa.fb_step(g, x, b, list(S), p, replay_alpha=alpha)
        assert (xb > 0).all()
        fs.append(rec.f_x)
        gs.append(((x - xb) / alpha).ravel())
        _, rec2 = fblisa.fb_step(g, xb, b, list(S), p, replay_alpha=alpha)
        assert rec.trials[-1].f_xbar == pytest.approx(rec2.f_x, rel=1e-12)
    assert np.mean(fs) == pytest.approx(0.5 * float(r_all @ r_all), rel=1e-12)
    full_g = A.T @ r_all
    assert np.abs(np.mean(gs, axis=0) - full_g).max() <= 1e-6 * np.abs(full_g).max()


def test_sufficient_decrease_test_has_its_half():
    # (2.3) on a quadratic: f(x_bar) = f(x) + g^T d + 1/2 d^T H d, so with d
    # along the top eigenvector of H = A^T A (eigenvalue L) the test holds iff
    # alpha <= 1/L: 0.9/L passes and 1.5/L fails (||d||^2/alpha in place of
    # ||d||^2/(2 alpha) would pass both).
    g, xt, b0 = _problem(9, _geom(views=6))
    views = list(range(g.n_views))  # full batch
    A = _dense_A(g, views)
    _, sv, Vt = np.linalg.svd(A, full_matrices=False)
    L = sv[0] ** 2
    v = Vt[0]
    x = np.full(g.vol_shape, 10.0)
    b = (A @ x.ravel() - A @ v).reshape(b0.shape)  # A x - b = A v: g = L v
    p = fblisa.Params(alpha0=1.0, beta=0.5, mu=0.0)
    for a, want in ((0.9 / L, True), (1.5 / L, False)):
        xb, rec = fblisa.fb_step(g, x, b, views, p, replay_alpha=a)
        assert (xb > 0).all()
        assert bool(rec.trials[-1].accepted) == want


def _lipschitz(g, views):
    A = _dense_A(g, views)
    return g.n_views / len(views) * np.linalg.norm(A, 2) ** 2


def test_lemma_small_steps_never_backtrack():
    g, xt, b = _problem(4)
    views = [1, 2, 5]
    L = _lipschitz(g, views)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, g.vol_shape)
    p = fblisa.Params(alpha0=0.99 / L, beta=0.5, mu=0.3)
    _, rec = fblisa.fb_step(g, x, b, views, p)
    assert rec.backtracks == 0


def test_lemma_accepted_step_exceeds_beta_over_L():
    g, xt, b = _problem(5)
    rng = np.random.default_rng(5)
    for views in ([0, 1], [2, 3, 4, 5], [0, 2, 4]):
        L = _lipschitz(g, views)
        x = rng.uniform(0, 1, g.vol_shape)
        for beta in (0.5, 0.3):
            p = fblisa.Params(alpha0=50.0 / L, beta=beta, mu=0.5)
            _, rec = fblisa.fb_step(g, x, b, views, p)
            assert rec.backtracks >= 1
            assert rec.alpha > beta / L
            assert all(not t.accepted for t in rec.trials[:-1]) and rec.trials[-1].accepted


def test_accepted_steps_decrease_F_N():
    g, xt, b = _problem(6)
    p = fblisa.Params(alpha0=1e-2, beta=0.5, mu=0.2, N0=2, seed=11)
    x = np.zeros(g.vol_shape)
    n = 0
    for t, (N_t, _) in enumerate(fblisa.schedule(g.n_views, p.N0, g.n_views, p.C, p.eps_base, 3), 1):
        for views in fblisa.epoch_batches(p.seed, t, g.n_views, N_t):
            xn, rec = fblisa.fb_step(g, x, b, views, p)
            tr = rec.trials[-1]
            F_x = rec.f_x + p.mu * np.abs(x).sum()
            F_xbar = tr.f_xbar + p.mu * np.abs(xn).sum()
            assert F_xbar <= F_x - tr.dnorm2 / (2 * tr.alpha) + 1e-9 * abs(F_x)
            assert np.all(xn >= 0)
            x = xn
            n += 1
    assert n >= 6


def test_full_batch_is_monotone_proximal_gradient():
    g, xt, b = _problem(7)
    p = fblisa.Params(alpha0=1.0, beta=0.5, mu=0.1, N0=g.n_views, n_max=g.n_views, seed=3)
    x0 = np.zeros(g.vol_shape)
    x, recs = fblisa.run(g, b, x0, p, epochs=12)
    assert all(r.N_t == g.n_views for r in recs)
    Fs = [fblisa.full_objective(g, x0, b, p.mu)]
    xk = x0
    for r in recs:
        xk, _ = fblisa.fb_step(g, xk, b, r.views, p, replay_alpha=r.alpha)
        Fs.append(fblisa.full_objective(g, xk, b, p.mu))
    assert np.allclose(xk, x)
    assert all(Fs[i + 1] <= Fs[i] * (1 + 1e-12) for i in range(len(Fs) - 1))
    assert Fs[-1] < 0.5 * Fs[0]


def test_full_batch_tv_and_box_are_monotone():
    # any convex R with an exact prox: (2.3) and the prox inequality give
    # F(x_bar) <= F(x) - ||x_bar - x||^2 / (2 alpha) in full batch; the TV prox
    # runs to a duality gap far below the decrease (300 FGP iterations)
    from oracle import tv
    g, xt, b = _problem(7)
    for reg, kw in (("tv", dict(tv_iters=300, tv_warm=False)), ("l1", dict(x_max=0.05))):
        p = fblisa.Params(alpha0=1.0, beta=0.5, mu=0.1, N0=g.n_views, n_max=g.n_views, seed=3, reg=reg, **kw)
        x, recs = fblisa.run(g, b, np.zeros(g.vol_shape), p, epochs=8)

        def F(z):
            fid = fblisa.full_objective(g, z, b, 0.0)
            return fid + p.mu * (tv.tv(z) if reg == "tv" else float(np.abs(z).sum()))

        xs = [np.zeros(g.vol_shape)]
        st = fblisa.TVState()
        for r in recs:
            xn, _ = fblisa.fb_step(g, xs[-1], b, r.views, p, replay_alpha=r.alpha, tv_state=st)
            xs.append(xn)
        assert np.allclose(xs[-1], x)
        Fs = [F(z) for z in xs]
        assert all(Fs[i + 1] <= Fs[i] * (1 + 1e-9) for i in range(len(Fs) - 1))
        assert Fs[-1] < 0.9 * Fs[0]
        if reg == "l1":
            assert x.max() <= 0.05 and (x == 0.05).any()


def test_schedule_case3_closed_form_and_paper_growth():
    # Case 3: n_theta = 72 views, N_0 = 8, M = C = 1, eps_k = 0.99^k (Sec. 3).
    sched = fblisa.schedule(72, 8, 72, 1.0, 0.99, 40)
    # Closed form: ceil(0.99^-K) > 8  <=>  K > ln 8 / -ln 0.99 = 206.9..., and
    # with N = 8 the epochs are 9 iterations long, so K = 9 t first reaches 207 at t = 23.
    K_first = math.ceil(math.log(8.0) / -math.log(0.99))
    assert K_first == 207
    assert all(N == 8 and it == 9 for N, it in sched[:22])
    assert sched[22][0] == 9
    # Sec. 3: the batch grows from 8 to 13 within the 240 s run and never reaches
    # full batch; under this reading 13 first applies at iteration 242 and 14 at 254.
    k = 0
    first = {}
    for N, it in sched:
        first.setdefault(N, k)
        k += it
    assert first[13] == 242 and first[14] == 254
    assert max(N for N, _ in sched[:30]) == 13


def test_schedule_bounds_and_iteration_counts():
    for n_theta, N0, n_max in ((90, 10, 90), (360, 20, 360), (720, 40, 720), (36, 8, 20)):
        sched = fblisa.schedule(n_theta, N0, n_max, 1.0, 0.99, 60)
        prev = N0
        for N, it in sched:
            assert N0 <= N <= n_max and N >= prev
            assert it == -(-n_theta // N)
            prev = N


def test_epoch_permutations_are_uniform():
    n = 12
    counts = np.zeros((n, n))
    for t in range(1, 3001):
        perm = fblisa.epoch_permutation(12345, t, n)
        assert sorted(perm) == list(range(n))
        for pos, v in enumerate(perm):
            counts[pos, v] += 1
    expect = 3000 / n
    chi2 = ((counts - expect) ** 2 / expect).sum()
    # 121 degrees of freedom; the 99.99% quantile is about 190
    assert chi2 < 190


def test_batches_cover_epoch_and_pad_from_front():
    for n_theta, N_t in ((90, 10), (90, 7), (20, 20), (13, 5)):
        batches = fblisa.epoch_batches(77, 3, n_theta, N_t)
        perm = fblisa.epoch_permutation(77, 3, n_theta)
        assert len(batches) == -(-n_theta // N_t)
        assert all(len(bt) == N_t and len(set(bt)) == N_t for bt in batches)
        assert sorted(set(itertools.chain(*batches))) == list(range(n_theta))
        r = n_theta % N_t
        if r:
            assert batches[-1] == perm[-r:] + perm[:N_t - r]


def test_splitmix64_matches_published_reference_outputs():
    # The mini-batch generator is SplitMix64 from its publication: its first
    # outputs from three starting states equal the published reference ones
    # (tests/golden/splitmix64.txt), so a wrong constant, shift or increment fails.
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.txt")
    rows = [[int(t) for t in ln.split()] for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for state, *outs in rows:
        assert [fblisa.splitmix64_draw(state, i) for i in range(len(outs))] == outs


def test_splitmix64_stream_properties():
    # Draws are distinct, and their top bits are close to fair coins.
    zs = [fblisa.splitmix64_draw(42, i) for i in range(4096)]
    assert len(set(zs)) == len(zs)
    bits = np.array([[(z >> s) & 1 for s in range(0, 64, 7)] for z in zs])
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.04)


def test_fixed_step_forward_backward_descent_lemma():
    # Constant-step FB on the full batch with alpha <= 1/L: the descent lemma and
    # the prox optimality give F(x+) <= F(x) - ||x+ - x||^2 / (2 alpha) (textbook
    # proximal gradient), so F decreases; a gradient of the wrong sign or a
    # missing prox shift breaks it.  Past 2/L the iteration diverges.
    g, xt, b = _problem(8)
    views = list(range(g.n_views))
    L = _lipschitz(g, views)
    x = np.zeros(g.vol_shape)
    p = fblisa.Params(alpha0=0.9 / L, mu=0.1, N0=g.n_views, fixed_step=True)
    F = fblisa.full_objective(g, x, b, p.mu)
    for _ in range(15):
        xn, rec = fblisa.fb_step(g, x, b, views, p)
        Fn = fblisa.full_objective(g, xn, b, p.mu)
        d2 = float(((xn - x) ** 2).sum())
        assert rec.backtracks == 0 and rec.alpha == p.alpha0
        assert Fn <= F - d2 / (2 * p.alpha0) + 1e-10 * abs(F)
        x, F = xn, Fn
    assert F < 0.5 * fblisa.full_objective(g, np.zeros(g.vol_shape), b, p.mu)
    # same point as the line search's first trial at the same step
    x0 = np.full(g.vol_shape, 0.2)
    a, _ = fblisa.fb_step(g, x0, b, views, p)
    c, _ = fblisa.fb_step(g, x0, b, views, fblisa.Params(alpha0=0.9 / L, mu=0.1, N0=g.n_views))
    assert np.array_equal(a, c)
    # far beyond 2/L the constant step does not converge
    q = fblisa.Params(alpha0=5.0 / L, mu=0.0, N0=g.n_views, fixed_step=True)
    y = np.full(g.vol_shape, 0.3)
    for _ in range(6):
        y, _ = fblisa.fb_step(g, y, b, views, q)
    assert fblisa.full_objective(g, y, b, 0.0) > fblisa.full_objective(g, np.full(g.vol_shape, 0.3), b, 0.0)
