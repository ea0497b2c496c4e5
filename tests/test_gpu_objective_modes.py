"""The residual pass and the trial-objective pass evaluate the same f_N.

Algorithm 1 compares f_N(x̄) with f_N(x) + <grad f_N(x), x̄ - x> + ||x̄ - x||^2 / (2 alpha)
(eq. (2.3)).  The library computes f_N(x) in the residual pass (K1, which also
stores the residual) and f_N(x̄) in the objective pass (K1 without the store).
When the trial point equals x, bit for bit, the right-hand side is f_N(x)
and the test accepts only if both passes give the same sum.  A difference in
the last bit would make the line search reject every small step and end at
its backtrack cap.  Here alpha_0 is tiny and mu large, so the prox leaves x
unchanged: voxels of x > 0 move by far less than half an ulp of their
storage, and voxels at 0 stay at 0.  The first trial must then pass with
f_N(x̄) == f_N(x) exactly.  This is checked for each storage type, for the
host loop and the graph-captured iteration, and for every projector launch
form.
"""
import numpy as np
import pytest

from gpu_common import GEOMS, cuda, problem

pytestmark = pytest.mark.gpu

DTYPES = ["f32", "bf16", "f16"]
LAUNCH = [(4, 0, 4), (4, 1, 8), (8, 0, 28), (8, 1, 24)]


@pytest.fixture(scope="module")
def data():
    g = GEOMS["ragged"]
    xt, b = problem(g, seed=11)
    return g, xt, b


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("launch", LAUNCH)
def test_unchanged_trial_point_passes_with_equal_objectives(data, dtype, graph, launch):
    import torch
    import paper_2605_12085_gb300 as fbl
    g, xt, b = data
    code = {"f32": fbl.F32, "bf16": fbl.BF16, "f16": fbl.F16}[dtype]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    G = fbl.geometry_create(g)
    fbl.geometry_set_launch(G, *launch)
    p = fbl.params_default(alpha0=1e-24, beta=0.5, mu=1e8, N0=6, seed=5, x_dtype=code, b_dtype=code,
                           use_graph=graph, max_backtracks=0)
    S = fbl.fblisa_create(G, p)
    x = cuda(xt.astype(np.float32)).to(tdt)
    x0 = x.clone()
    bb = cuda(b.astype(np.float32)).to(tdt)
    for _ in range(3):
        st = S.step(x, bb)
        assert st["status"] == 0 and st["backtracks"] == 0, st
        assert st["f_xbar"] == st["f_x"], (st["f_x"], st["f_xbar"])
        assert st["dnorm2"] == 0.0 and st["gTd"] == 0.0
    # the accepted point is x itself
    assert torch.equal(x, x0)
