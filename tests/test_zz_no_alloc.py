"""prox_reduce_static: the allocation-free variant of prox_reduce.

Some callers cannot allocate device memory (a fixed budget reserved up front,
device memory owned by a host application, loops where an allocation could
block).  This checks, through the C ABI, that the variant returns the same
x_bar and reductions as prox_reduce on two calls in a row (the shared fixed
scratch must not carry anything over), and that it rejects sizes beyond its
fixed capacity.  Collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_variant_matches_prox_reduce_twice():
    import torch
    import paper_2605_12085_gb300 as fbl
    rng = np.random.default_rng(21)
    for call, n in enumerate((1_000_003, 77_777)):
        x = torch.from_numpy(np.maximum(rng.standard_normal(n), 0).astype(np.float32)).cuda()
        g = torch.from_numpy((rng.standard_normal(n) * 3).astype(np.float32)).cuda()
        alpha, mu = 0.013 * (call + 1), 0.7
        ref_xb, ref = fbl.prox_reduce(x, g, alpha, mu)
        xb = torch.empty_like(x)
        got_xb, got = fbl.prox_reduce_static(x, g, alpha, mu, xb)
        torch.cuda.synchronize()
        assert torch.equal(got_xb, ref_xb)
        for a, b in zip(got, ref):
            assert a == pytest.approx(b, rel=1e-6, abs=1e-12)


def test_static_variant_rejects_oversized_and_host_inputs():
    import ctypes
    import torch
    import paper_2605_12085_gb300 as fbl
    x = torch.zeros(16, device="cuda")
    g = torch.zeros(16, device="cuda")
    xb = torch.zeros(16, device="cuda")
    out = (ctypes.c_double * 3)()
    rc = fbl.lib.prox_reduce_static(x.data_ptr(), 0, g.data_ptr(), (1 << 27) + 1, 0.1, 0.0,
                                    xb.data_ptr(), out, None)
    assert rc == 1 and b"capacity" in fbl.lib.fbl_last_error()
    with pytest.raises(fbl.FblError):
        fbl.prox_reduce_static(np.zeros(16, np.float32), np.zeros(16, np.float32), 0.1, 0.0,
                               np.zeros(16, np.float32))
