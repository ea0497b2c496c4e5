"""The 256^3 Poisson configuration (40-ellipsoid phantom with small
high-contrast inclusions, 360 views, 384x384 detector, log-Poisson data with
I_0 = 1e4, 20-view mini-batches) against the FP64 oracle: the data are the
oracle's projection of the phantom, log-Poisson sampled (synth), and the
first iterations of the GPU solver (FP32, autotuned launch configuration)
must take the oracle's mini-batches and steps, with f_N(x) within 2e-5 and
the iterate within 1e-4 (relative L2)."""
import numpy as np
import pytest

import oracle
from oracle import fblisa
import synth
from gpu_common import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


def test_c2_poisson_iterations_match_oracle():
    import paper_2605_12085_gb300 as fbl
    wl = synth.WORKLOADS["c2_256"]
    g = wl.geom
    xt = synth.phantom(g, wl.n_ellipsoids, wl.seed_phantom, inclusions=wl.inclusions)
    clean = oracle.project(g, xt.astype(np.float64), range(g.n_views))
    b = synth.poisson_log_data(clean, wl.I0, wl.seed_noise)
    assert np.isfinite(b).all() and b.dtype == np.float32
    G = fbl.geometry_create(g)
    fbl.geometry_autotune(G, fbl.F32, wl.N0)
    p = fblisa.Params(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=p.alpha0, beta=p.beta, mu=p.mu, N0=p.N0, seed=p.seed))
    x = cuda(np.zeros(g.vol_shape, np.float32))
    bd = cuda(b)
    iters = 3
    trace = [S.step(x, bd) for _ in range(iters)]
    xo, recs = fblisa.run(g, b.astype(np.float64), np.zeros(g.vol_shape), p, 1, max_iters=iters)
    assert [r.views for r in recs] == fblisa.epoch_batches(p.seed, 1, g.n_views, p.N0)[:iters]
    for t, r in zip(trace, recs):
        assert t["N_t"] == r.N_t == 20
        assert t["f_x"] == pytest.approx(r.f_x, rel=2e-5)
        assert t["backtracks"] == r.backtracks and t["alpha"] == r.alpha
    assert max(t["backtracks"] for t in trace) >= 1
    assert rel_l2(host(x), xo) <= 1e-4
