"""C-ABI checks that need no GPU: the library loads, exports every call that
include/fblisa.h declares, rejects bad arguments before touching the device,
and its host-side schedule (Alg. 1 Step 1) and mini-batch sampling (Step 2a)
reproduce the oracle's bit for bit."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fbl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_12085_gb300 as m
    return m


def _declared():
    names = []
    with open(os.path.join(ROOT, "include", "fblisa.h")) as f:
        for m in re.finditer(r"FBL_API\s+[\w\s\*]+?\b(\w+)\s*\(", f.read()):
            names.append(m.group(1))
    return names


def test_exports_every_declared_symbol(fbl):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(fbl.lib, n), n
    assert sorted(names) == sorted(fbl.EXPORTS)


def test_geometry_argument_validation(fbl):
    import synth
    bad = synth.Geometry(nx=0, ny=8, nz=8, vx=1, vy=1, vz=1, n_views=4, sod=100, sdd=150, nu=8,
                         nv=8, du=1, dv=1)
    with pytest.raises(fbl.FblError) as e:
        fbl.geometry_create(bad)
    assert e.value.status == 1
    bad2 = synth.Geometry(nx=8, ny=8, nz=8, vx=1, vy=1, vz=1, n_views=4, sod=100, sdd=90, nu=8,
                          nv=8, du=1, dv=1)
    with pytest.raises(fbl.FblError) as e:
        fbl.geometry_create(bad2)
    assert e.value.status == 1


def test_schedule_matches_oracle(fbl):
    from oracle import fblisa
    for args in ((90, 10, 90), (360, 20, 360), (720, 40, 720), (72, 8, 72), (36, 8, 20),
                 (1440, 60, 1440), (13, 5, 13)):
        n, N0, nmax = args
        assert fbl.fbl_schedule(n, N0, nmax, 1.0, 0.99, 50) == fblisa.schedule(n, N0, nmax, 1.0,
                                                                                 0.99, 50)


def test_batches_match_oracle_and_golden(fbl):
    from oracle import fblisa
    for seed in (0, 1, 3001, 2 ** 63 + 5):
        for (n, N_t, t) in ((90, 10, 1), (90, 7, 4), (720, 40, 2), (13, 13, 1), (1440, 60, 9)):
            assert fbl.fbl_epoch_batches(seed, t, n, N_t) == fblisa.epoch_batches(seed, t, n, N_t)
    with open(os.path.join(ROOT, "tests", "golden", "batches.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            head, views = line.split(":")
            seed, n, N0, t, k, N_t = map(int, head.split())
            got = fbl.fbl_epoch_batches(seed, t, n, N_t)
            assert [int(v) for v in views.split()] in got


def test_host_helpers_reject_bad_arguments(fbl):
    with pytest.raises(fbl.FblError):
        fbl.fbl_schedule(10, 0, 10, 1.0, 0.99, 3)
    with pytest.raises(fbl.FblError):
        fbl.fbl_schedule(10, 4, 10, 1.0, 1.5, 3)
    with pytest.raises(fbl.FblError):
        fbl.fbl_epoch_batches(1, 1, 10, 11)


def test_params_defaults_read_back(fbl):
    # the fields after fixed_step (reg, tv_iters, tv_warm, x_max) land where the C struct has them
    import math
    p = fbl.params_default()
    assert (p.alpha0, p.beta, p.mu, p.N0, p.max_backtracks) == (1e-3, 0.5, 1.0, 8, 60)
    assert (p.fixed_step, p.reg, p.tv_iters, p.tv_warm) == (0, fbl.REG_L1, 20, 1)
    assert math.isinf(p.x_max) and p.x_max > 0


def test_tv_calls_reject_bad_arguments(fbl):
    import numpy as np
    with pytest.raises(fbl.FblError) as e:
        fbl.prox_tv(np.zeros((0, 2, 2), np.float32), 0.1, 5)
    assert e.value.status == 1
    with pytest.raises(fbl.FblError) as e:
        fbl.prox_tv(np.zeros((2, 2, 2), np.float32), -0.1, 5)
    assert e.value.status == 1
    with pytest.raises(fbl.FblError) as e:
        fbl.prox_tv(np.zeros((2, 2, 2), np.float32), 0.1, 5, x_max=0.0)
    assert e.value.status == 1
    with pytest.raises(fbl.FblError) as e:
        fbl.tv_norm(np.zeros((2, 0, 2), np.float32))
    assert e.value.status == 1
    q = np.zeros((3, 2, 2, 2), np.float32)
    with pytest.raises(fbl.FblError) as e:
        fbl.prox_tv(np.zeros((2, 2, 2), np.float32), 0.1, 5, q=q, x=q[0])  # x aliases q
    assert e.value.status == 1
