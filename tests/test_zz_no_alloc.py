"""prox_reduce_static: the allocation-free variant of prox_reduce.

Some callers cannot allocate device memory (a fixed budget reserved up front,
device memory owned by a host application, loops where an allocation could
block).  This checks, through the C ABI, that the variant returns the same
x_bar and reductions as prox_reduce on two calls in a row (the shared fixed
scratch must not carry anything over), in every storage type and for n = 0,
and that it rejects sizes beyond its fixed capacity, host buffers and
mismatched arguments.  Collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, n, dtype):
    import torch
    x = torch.from_numpy(np.maximum(rng.standard_normal(n), 0).astype(np.float32)).cuda().to(dtype)
    g = torch.from_numpy((rng.standard_normal(n) * 3).astype(np.float32)).cuda()
    return x, g


@pytest.mark.parametrize("dtype_name", ["float32", "bfloat16", "float16"])
def test_static_variant_matches_prox_reduce_twice(dtype_name):
    import torch
    import paper_2605_12085_gb300 as fbl
    dtype = getattr(torch, dtype_name)
    rng = np.random.default_rng(21)
    for call, n in enumerate((1_000_003, 77_777)):
        x, g = _inputs(rng, n, dtype)
        alpha, mu = 0.013 * (call + 1), 0.7
        ref_xb, ref = fbl.prox_reduce(x, g, alpha, mu)
        xb = torch.empty_like(x)
        got_xb, got = fbl.prox_reduce_static(x, g, alpha, mu, xb)
        torch.cuda.synchronize()
        assert torch.equal(got_xb, ref_xb)
        # same kernels, same grid, same fixed-order reduction: identical sums
        assert tuple(got) == tuple(ref)


def test_static_variant_empty_input():
    import torch
    import paper_2605_12085_gb300 as fbl
    x = torch.zeros(0, device="cuda")
    g = torch.zeros(0, device="cuda")
    xb = torch.zeros(0, device="cuda")
    _, got = fbl.prox_reduce_static(x, g, 0.1, 0.5, xb)
    assert tuple(got) == (0.0, 0.0, 0.0)


def test_static_variant_rejects_oversized_host_and_mismatched_inputs():
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
    hx = np.zeros(16, np.float32)
    rc = fbl.lib.prox_reduce_static(hx.ctypes.data, 0, g.data_ptr(), 16, 0.1, 0.0, xb.data_ptr(), out, None)
    assert rc == 1 and b"current device" in fbl.lib.fbl_last_error()
    with pytest.raises(TypeError):
        fbl.prox_reduce_static(np.zeros(16, np.float32), np.zeros(16, np.float32), 0.1, 0.0,
                               np.zeros(16, np.float32))
    with pytest.raises(TypeError):  # xbar narrower than x
        fbl.prox_reduce_static(x, g, 0.1, 0.0, torch.zeros(16, device="cuda", dtype=torch.bfloat16))
    with pytest.raises(ValueError):  # xbar shorter than x
        fbl.prox_reduce_static(x, g, 0.1, 0.0, torch.zeros(15, device="cuda"))
    with pytest.raises(TypeError):  # g not float32
        fbl.prox_reduce_static(x, g.to(torch.bfloat16), 0.1, 0.0, xb)
    with pytest.raises(ValueError):  # g shorter than x
        fbl.prox_reduce_static(x, g[:8], 0.1, 0.0, xb)
