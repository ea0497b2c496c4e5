"""Storage precision variants (BF16 / FP16 volume and data, FP32 arithmetic,
FP64 line-search sums) against the FP64 oracle.

Where only the storage is rounded, the arithmetic is still FP32 and must match
the oracle evaluated on the same rounded inputs to 1e-5.  For whole FB-LISA
runs the error against the FP64 oracle's own trajectory is measured and
stated (it comes from rounding every iterate to 8 or 11 significant bits);
the bounds below are the stated levels, with margin.
"""
import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth
from gpu_common import GEOMS, problem, rel_l2

pytestmark = pytest.mark.gpu

DT = {"bf16": (1, "bfloat16", 2.0 ** -8), "f16": (2, "float16", 2.0 ** -11)}


def _torch_dtype(name):
    import torch
    return getattr(torch, DT[name][1])


def _round(a, name):
    """Round float64 data to the storage type (through torch), back to float64."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(_torch_dtype(name)).to(
        torch.float64).numpy()


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_projector_fp32_arithmetic_on_rounded_storage(name):
    import torch
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, g.vol_shape)
    xs = torch.from_numpy(x.astype(np.float32)).to(_torch_dtype(name)).cuda()
    views = [1, 4, 8, 15]
    G = fbl.geometry_create(g)
    y = fbl.project(G, xs, views)  # FP32 output
    ref = oracle.project(g, _round(x, name), views)
    assert rel_l2(y.double().cpu().numpy(), ref) <= 1e-5
    # output stored in the low-precision type: within its rounding
    y2 = fbl.project(G, xs, views, y_dtype=DT[name][0])
    err = np.abs(y2.double().cpu().numpy() - ref) / np.maximum(np.abs(ref), 1e-3)
    assert float(err.max()) <= 1.01 * DT[name][2]


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_backprojector_reads_rounded_data(name):
    import torch
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["angles"]
    rng = np.random.default_rng(2)
    views = [0, 2, 4]
    y = rng.standard_normal((3, g.nv, g.nu))
    ys = torch.from_numpy(y.astype(np.float32)).to(_torch_dtype(name)).cuda()
    G = fbl.geometry_create(g)
    x = fbl.backproject(G, ys, views)
    assert rel_l2(x.double().cpu().numpy(), oracle.backproject(g, _round(y, name), views)) <= 1e-5


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_residual_norm_and_prox_rounded(name):
    import torch
    import paper_2605_12085_gb300 as fbl
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=4)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, g.vol_shape)
    td = _torch_dtype(name)
    xs = torch.from_numpy(x.astype(np.float32)).to(td).cuda()
    bs = torch.from_numpy(b.astype(np.float32)).to(td).cuda()
    views = [0, 7, 11]
    G = fbl.geometry_create(g)
    rho = fbl.residual_norm(G, xs, views, bs)
    r = oracle.project(g, _round(x, name), views) - _round(b, name)[views]
    assert rho == pytest.approx(float((r * r).sum()), rel=2e-5)
    # prox: x_bar is the FP32 prox rounded once to the storage type
    gr = rng.standard_normal(x.size).astype(np.float32)
    xb, (gTd, dd, l1) = fbl.prox_reduce(xs.reshape(-1), torch.from_numpy(gr).cuda(), 0.05, 0.3)
    want = fblisa.prox(_round(x, name).ravel() - 0.05 * gr.astype(np.float64), 0.05, 0.3)
    got = xb.double().cpu().numpy()
    assert np.all(np.abs(got - want) <= DT[name][2] * np.maximum(np.abs(want), 1e-30) + 1e-7)
    d = got - _round(x, name).ravel()
    assert gTd == pytest.approx(float(np.dot(gr.astype(np.float64), d)), rel=1e-5)
    assert dd == pytest.approx(float(np.dot(d, d)), rel=1e-5)


@pytest.mark.parametrize("name,replay_bound", [("bf16", 2e-2), ("f16", 3e-3)])
def test_run_error_against_fp64_oracle_is_stated(name, replay_bound):
    """10 epochs on the 64^3 workload with BF16/FP16 iterates and data.

    Two numbers are stated: (1) the rel-L2 error of x when the FP64 oracle
    replays the GPU's accepted step sizes -- the effect of storage rounding
    alone; (2) free-running, where the two may accept different (equally
    valid) steps, the rel-L2 difference of x and the relative gap of the full
    objective F.
    """
    import torch
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["c1_64"]
    g = wl.geom
    xt, b = problem(g, n_ell=wl.n_ellipsoids, seed=wl.seed_phantom, noise_rel=wl.noise_rel)
    b64 = _round(b, name)  # the oracle sees the same rounded data
    p = fblisa.Params(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    td = _torch_dtype(name)
    G = fbl.geometry_create(g)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, N0=p.N0,
                                                seed=p.seed, x_dtype=DT[name][0],
                                                b_dtype=DT[name][0]))
    x = torch.zeros(g.vol_shape, dtype=td, device="cuda")
    tr = S.run(x, torch.from_numpy(b.astype(np.float32)).to(td).cuda(), 10)
    xg = x.double().cpu().numpy()
    x_rep, _ = fblisa.run(g, b64, np.zeros(g.vol_shape), p, 10, replay=[t["alpha"] for t in tr])
    x_free, recs = fblisa.run(g, b64, np.zeros(g.vol_shape), p, 10)
    e_rep = rel_l2(xg, x_rep)
    e_free = rel_l2(xg, x_free)
    F_g = fblisa.full_objective(g, xg, b64, p.mu)
    F_o = fblisa.full_objective(g, x_free, b64, p.mu)
    agree = sum(1 for t, r in zip(tr, recs) if t["alpha"] == r.alpha)
    print("%s: replayed steps: rel-L2(x) = %.3e | free-running: rel-L2(x) = %.3e, "
          "|F_gpu - F_oracle|/F_oracle = %.3e, agreeing steps %d/%d"
          % (name, e_rep, e_free, abs(F_g - F_o) / F_o, agree, len(recs)))
    assert len(tr) == len(recs) == 90
    assert e_rep <= replay_bound
    assert e_free <= 5e-2
    assert abs(F_g - F_o) <= 5e-3 * F_o
    assert float(xg.min()) >= 0.0
