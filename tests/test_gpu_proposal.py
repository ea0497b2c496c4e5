"""The learned step proposal (no counterpart in the paper, which restarts every
line search from alpha_0, Step 2d).

* The first trial is always a point of the plain rule's grid alpha_0 * beta^j
  with j = clamp(floor(j_prev + pred + 1/2 - margin), 0, cap); acceptance
  (2.3) and backtracking are unchanged, so every accepted step still
  satisfies (2.3).
* Graph and host-loop modes take identical decisions with the proposal on.
* The trained network (package data, trained on traces of the plain method on
  seeded 128^3-256^3 phantoms) saves backtracks on a held-out problem of a size
  it has not seen, at a comparable objective after the same epochs.
"""
import math
import os

import numpy as np
import pytest

import synth
from gpu_common import GEOMS, cuda, host, problem

pytestmark = pytest.mark.gpu

NP = 4801


def _constant_net(c):
    p = np.zeros(NP, np.float32)
    p[-1] = c  # b3: the output is c whatever the input
    return p


def test_first_trial_is_on_the_plain_grid():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=31)
    bd = cuda(b.astype(np.float32))
    G = fbl.geometry_create(g)
    a0, beta = 1e-2, 0.5
    for c, margin, cap in ((3.2, 0.5, 60), (-0.7, 0.25, 60), (1000.0, 0.25, 7)):
        S = fbl.fblisa_create(G, fbl.params_default(N0=6, mu=0.5, alpha0=a0, beta=beta, seed=4,
                                                    proposal=1, max_backtracks=cap))
        S.set_proposal(_constant_net(c), margin=margin)
        x = cuda(np.zeros(g.vol_shape, np.float32))
        j_prev = 0
        for _ in range(3):
            rc, st = S.step_raw(x, bd)
            j = min(max(int(math.floor(j_prev + c + 0.5 - margin)), 0), cap)
            assert st["j_start"] == j
            assert st["alpha_init"] == a0 * beta ** j
            assert st["pred"] == pytest.approx(c)
            if rc == 0:
                assert st["alpha"] == a0 * beta ** (j + st["backtracks"])
                assert st["margin"] >= 0.0
                j_prev = j + st["backtracks"]


def test_proposal_requires_a_network():
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["angles"]
    xt, b = problem(g, seed=32)
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(N0=2, proposal=1))
    rc, _ = S.step_raw(cuda(np.zeros(g.vol_shape, np.float32)), cuda(b.astype(np.float32)))
    assert rc == 1


def _weights():
    from paper_2605_12085_gb300 import proposal
    return proposal.load()


def test_graph_and_host_modes_agree_with_proposal():
    import paper_2605_12085_gb300 as fbl
    params, _ = _weights()
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=33)
    bd = cuda(b.astype(np.float32))
    G = fbl.geometry_create(g)
    out = []
    for graph in (0, 1):
        S = fbl.fblisa_create(G, fbl.params_default(N0=6, mu=0.5, seed=4, proposal=1,
                                                    use_graph=graph))
        S.set_proposal(params)
        x = cuda(np.zeros(g.vol_shape, np.float32))
        tr = S.run(x, bd, 3)
        out.append((host(x), [(t["j_start"], t["backtracks"], t["alpha"]) for t in tr]))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_trained_proposal_saves_backtracks_on_a_held_out_problem():
    import torch
    import paper_2605_12085_gb300 as fbl
    params, meta = _weights()
    assert meta["traces"] >= 20000
    n, views, N0 = 112, 150, 12  # a size and view count not used for training
    det = int(math.ceil(1.5 * n))
    g = synth.Geometry(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, n_views=views, sod=1000.0,
                       sdd=1500.0, nu=det, nv=det, du=1.5, dv=1.5)
    xt = synth.phantom(g, 15, 9999)
    G = fbl.geometry_create(g)
    b = fbl.project(G, torch.from_numpy(xt).cuda(), range(views))
    b += torch.from_numpy(synth.gaussian_noise(tuple(b.shape), 0.01 * float(b.max()), 9998)).cuda()
    res = {}
    for prop in (0, 1):
        S = fbl.fblisa_create(G, fbl.params_default(N0=N0, mu=1.0, seed=77, proposal=prop))
        if prop:
            S.set_proposal(params)
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device="cuda")
        tr = S.run(x, b, 4)
        F, _, re = fbl.evaluate(G, x, b, 1.0, x_true=torch.from_numpy(xt).cuda())
        res[prop] = dict(bt=float(np.mean([t["backtracks"] for t in tr])),
                         trials=float(np.mean([t["backtracks"] + 1 for t in tr])), F=F, re=re,
                         margins=min(t["margin"] for t in tr), n=len(tr))
    print("plain: %.2f backtracks/iter, F=%.6g, RE=%.4f | learned: %.2f backtracks/iter, "
          "F=%.6g, RE=%.4f" % (res[0]["bt"], res[0]["F"], res[0]["re"], res[1]["bt"], res[1]["F"],
                               res[1]["re"]))
    assert res[0]["n"] == res[1]["n"]
    assert res[1]["margins"] >= 0.0
    assert res[1]["bt"] <= 0.5 * res[0]["bt"]          # at least half the backtracks saved
    assert res[1]["trials"] <= 0.6 * res[0]["trials"]  # at least 40% fewer trial evaluations
    assert res[1]["F"] <= 1.05 * res[0]["F"]
