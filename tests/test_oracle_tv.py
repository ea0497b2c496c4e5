"""Pins of the other-regulariser oracle (oracle/tv.py) against facts that do
not come from its code:

* K^T is the adjoint of K (dot test), and K itself gives the closed-form TV of
  a step edge (one jump per row) and of a linear ramp in two directions (the
  isotropic norm sqrt(a^2 + b^2) inside, |a| or |b| on two faces, 0 on an edge);
* the prox of lam |x2 - x1| on two voxels has a closed form (merge to the
  mean within 2 lam, else move each by lam);
* a constant volume and lam = 0 return the box projection;
* the duality gap of the FGP output goes to zero (an independent certificate:
  weak duality makes the gap >= 0 for any feasible pair, and 1/2||x - x*||^2
  <= gap), with and without an active upper bound, and is >= 0 for random
  feasible pairs;
* the box l1 prox equals a 1-D brute-force minimisation;
* the warm start: zero further iterations from a converged dual reproduce the
  converged volume;
* the FB-LISA oracle with reg "l1" and no bound is the paper's iteration.
"""
import math

import numpy as np
import pytest

from oracle import tv
from oracle import fblisa as ofb


def test_adjoint_dot_test():
    rng = np.random.default_rng(1)
    for shape in ((5, 4, 3), (1, 6, 7), (4, 1, 1), (3, 3, 1)):
        x = rng.standard_normal(shape)
        q = rng.standard_normal((3,) + shape)
        lhs = float((tv.grad(x) * q).sum())
        rhs = float((x * tv.grad_adjoint(q)).sum())
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_tv_of_step_edge_and_ramp():
    nz, ny, nx = 4, 5, 7
    x = np.zeros((nz, ny, nx))
    x[:, :, :3] = 2.5                       # a jump of 2.5 between x = 2 and x = 3
    assert math.isclose(tv.tv(x), 2.5 * ny * nz, rel_tol=1e-14)
    a, b = 0.7, -1.3
    ii = np.arange(nx)[None, None, :]
    jj = np.arange(ny)[None, :, None]
    x = a * ii + b * jj + np.zeros((nz, 1, 1))
    want = ((nx - 1) * (ny - 1) * nz * math.hypot(a, b) + (ny - 1) * nz * abs(b) + (nx - 1) * nz * abs(a))
    assert math.isclose(tv.tv(x), want, rel_tol=1e-13)
    # the z direction counts as well
    x = 0.4 * np.arange(nz)[:, None, None] + np.zeros((1, ny, nx))
    assert math.isclose(tv.tv(x), 0.4 * (nz - 1) * ny * nx, rel_tol=1e-13)


@pytest.mark.parametrize("b1,b2,lam", [(5.0, 5.3, 0.2), (5.0, 9.0, 0.5), (7.0, 3.0, 1.25), (4.0, 4.0, 0.3)])
def test_two_voxel_closed_form(b1, b2, lam):
    v = np.array([b1, b2]).reshape(1, 1, 2)
    x, q = tv.prox_tv(v, lam, 3000)
    if abs(b2 - b1) <= 2 * lam:
        want = [0.5 * (b1 + b2)] * 2
    else:
        s = math.copysign(lam, b2 - b1)
        want = [b1 + s, b2 - s]
    assert np.allclose(x.ravel(), want, rtol=0, atol=1e-8)


def test_constant_volume_and_zero_lambda():
    v = np.full((3, 4, 5), 0.8)
    x, _ = tv.prox_tv(v, 0.3, 25, x_max=0.5)
    assert np.allclose(x, 0.5)
    rng = np.random.default_rng(2)
    v = rng.uniform(-1, 2, (3, 4, 5))
    x, _ = tv.prox_tv(v, 0.0, 25, x_max=1.5)
    assert np.array_equal(x, np.clip(v, 0, 1.5))


@pytest.mark.parametrize("x_max", [math.inf, 0.6])
def test_duality_gap_vanishes(x_max):
    rng = np.random.default_rng(3)
    v = rng.uniform(0, 1, (5, 4, 6))
    lam = 0.08
    gaps = []
    for iters in (10, 100, 2000):
        x, q = tv.prox_tv(v, lam, iters, x_max=x_max)
        gaps.append(tv.duality_gap(v, lam, x, q, x_max))
    assert all(g >= -1e-12 for g in gaps)
    assert gaps[-1] <= 1e-9 * (0.5 * float((v * v).sum()))
    assert gaps[-1] < gaps[0]


def test_weak_duality_on_random_feasible_pairs():
    rng = np.random.default_rng(4)
    v = rng.uniform(-0.5, 1.5, (4, 3, 5))
    for _ in range(20):
        x = np.clip(rng.uniform(-1, 2, v.shape), 0, 1.2)
        q = rng.standard_normal((3,) + v.shape)
        q /= np.maximum(np.sqrt((q * q).sum(axis=0)), 1.0)[None]
        assert tv.duality_gap(v, 0.3, x, q, 1.2) >= -1e-12


def test_l1_box_prox_against_brute_force():
    grid = np.linspace(-1.0, 3.0, 40001)
    for v, a, mu, xmax in ((1.7, 0.5, 0.4, 1.0), (0.1, 0.5, 0.4, 1.0), (2.5, 0.1, 1.0, math.inf), (-0.3, 1, 1, 2)):
        obj = 0.5 * (grid - v) ** 2 + a * mu * np.abs(grid)
        obj[(grid < 0) | (grid > xmax)] = np.inf
        want = grid[np.argmin(obj)]
        got = float(tv.prox_l1_box(np.array([v]), a, mu, xmax)[0])
        assert abs(got - want) <= 1e-4


def test_warm_start_reproduces_converged_volume():
    rng = np.random.default_rng(5)
    v = rng.uniform(0, 1, (4, 4, 4))
    x1, q1 = tv.prox_tv(v, 0.05, 500)
    x2, q2 = tv.prox_tv(v, 0.05, 0, q0=q1)
    assert np.allclose(x1, x2, rtol=0, atol=1e-14)
    x3, _ = tv.prox_tv(v, 0.05, 5, q0=q1)   # a few more steps from there barely move
    assert np.abs(x3 - x1).max() <= 1e-4


def test_l1_default_is_the_papers_prox():
    rng = np.random.default_rng(6)
    v = rng.normal(0, 1, (3, 4, 5))
    p = ofb.Params(mu=0.7)
    assert np.array_equal(ofb.reg_prox(v, 0.3, p), ofb.prox(v, 0.3, 0.7))
