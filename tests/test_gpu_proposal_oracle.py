"""The learned step proposal inside the solver, with the trained network,
against the FP64 oracle of the proposal (oracle/proposal.py).

The proposal replaces Step 2d's restart at alpha_0 by a first trial
alpha_0 beta^j on the plain rule's grid; the kernels compute its eight
features from the iteration's f_N(x) and ||grad f_N(x)||^2, evaluate the
network (a second implementation of it, inside the line-search kernel) and
take j.  Checked at every iteration of two epochs, in the host-loop and the
graph-captured solver and for one volume of the batched solver:

* the features against the oracle's, which it computes from its own f_N(x)
  and ||grad f_N||^2 (absolute 2e-5 + relative 1e-5: FP32 features of FP64
  sums);
* the network output against oracle/mlp.forward of the same features
  (<= 1e-5);
* j_start exactly: the kernel's own rounding of its output in FP32, and the
  oracle's rule on the oracle's output wherever that lies farther than 1e-4
  from a rounding boundary (none may lie closer);
* backtracks and accepted steps equal to the oracle's, which runs with the
  GPU's first trials imposed, and the iterates within 1e-4 (relative L2).
"""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle import proposal as oprop
from oracle import fblisa
import synth
from gpu_common import GEOMS, cuda, host, problem, rel_l2

pytestmark = pytest.mark.gpu

MARGIN = 0.25


@pytest.fixture(scope="module")
def case():
    from paper_2605_12085_gb300 import proposal
    params, _ = proposal.load()
    wl = synth.WORKLOADS["c1_64"]
    g = wl.geom
    xt, b = problem(g, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    b32 = b.astype(np.float32)
    p = fblisa.Params(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    return params, g, b32, p


def _fp32_rule(j_prev, have_prev, pred, cap):
    """The first index as the kernel rounds it: FP32 additions, then floor."""
    f32 = np.float32
    base = f32(j_prev if have_prev else 0)
    arg = f32(f32(f32(base + f32(pred)) + f32(0.5)) - f32(MARGIN))
    return min(max(int(math.floor(arg)), 0), cap)


def _check_against_oracle(trace, params, g, b32, p, x_gpu, label):
    alpha_inits = [t["alpha_init"] for t in trace]
    xo, recs = oprop.run(g, b32.astype(np.float64), np.zeros(g.vol_shape), p, 99,
                         predict=oprop.network(params.astype(np.float64)), margin=MARGIN,
                         impose_alpha_init=alpha_inits, max_iters=len(trace))
    assert len(recs) == len(trace)
    P = params.astype(np.float64)
    j_prev, have = 0, False
    near = 0
    for k, (t, r) in enumerate(zip(trace, recs)):
        feat = np.asarray(t["features"], dtype=np.float64)
        assert np.allclose(feat, r.features, rtol=1e-5, atol=2e-5), (label, k, feat, r.features)
        y = float(mlp.forward(P, feat[None, :])[0][0])
        assert abs(t["pred"] - y) <= 1e-5 * max(1.0, abs(y)), (label, k, t["pred"], y)
        assert t["j_start"] == _fp32_rule(j_prev, have, t["pred"], p.max_backtracks), (label, k)
        arg = (j_prev if have else 0) + r.pred + 0.5 - MARGIN
        if abs(arg - round(arg)) > 1e-4:
            assert t["j_start"] == r.j_start, (label, k, t["j_start"], r.j_start)
        else:
            near += 1
        assert t["alpha_init"] == p.alpha0 * p.beta ** t["j_start"]
        assert t["backtracks"] == r.step.backtracks, (label, k)
        assert t["alpha"] == r.step.alpha
        assert t["margin"] >= 0.0
        j_prev, have = t["j_start"] + t["backtracks"], True
    assert near == 0, "%s: %d network outputs within 1e-4 of a rounding boundary" % (label, near)
    assert rel_l2(x_gpu, xo) <= 1e-4, label
    # the network moves the first trial (not a constant start)
    js = [t["j_start"] for t in trace]
    assert max(js) >= 1 and len(set(js)) >= 2, js


@pytest.mark.parametrize("graph", [0, 1])
def test_in_solver_proposal_matches_oracle(case, graph):
    import paper_2605_12085_gb300 as fbl
    params, g, b32, p = case
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, N0=p.N0,
                                                seed=p.seed, proposal=1, use_graph=graph))
    S.set_proposal(params, margin=MARGIN)
    x = cuda(np.zeros(g.vol_shape, np.float32))
    trace = S.run(x, cuda(b32), 2)
    assert len(trace) == 18
    _check_against_oracle(trace, params, g, b32, p, host(x), "graph=%d" % graph)


def test_batched_proposal_matches_oracle(case):
    import paper_2605_12085_gb300 as fbl
    params, g, b32, p = case
    other = GEOMS["ragged"]
    _, b_other = problem(other, seed=44)
    Gs = [fbl.geometry_create(g), fbl.geometry_create(other)]
    B = fbl.fblisa_batch_create(Gs, [
        fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, N0=p.N0, seed=p.seed, proposal=1),
        fbl.params_default(alpha0=1e-2, mu=0.5, N0=6, seed=4, proposal=1)])
    B.set_proposal(params, margin=MARGIN)
    xs = [cuda(np.zeros(g.vol_shape, np.float32)), cuda(np.zeros(other.vol_shape, np.float32))]
    steps = B.run(xs, [cuda(b32), cuda(b_other.astype(np.float32))], 12)
    trace = [st[0] for st in steps]
    _check_against_oracle(trace, params, g, b32, p, host(xs[0]), "batch")
