"""The FP64 reference perceptron's gradient against central finite
differences of its loss (the network has no counterpart in the paper; this
pins the oracle used to check the GPU training kernels)."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init(7)
    p += 0.1 * rng.standard_normal(p.size)  # non-zero biases too
    X = rng.standard_normal((37, 8))
    t = rng.standard_normal(37)
    g = mlp.gradient(p, X, t)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros_like(p)
        e[q] = h
        fd = (mlp.loss(p + e, X, t) - mlp.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 + 1e-5 * abs(g[q])


def test_pack_layout_and_size():
    assert mlp.NPARAMS == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1 == 4801
    p = np.arange(mlp.NPARAMS, dtype=np.float64)
    d = mlp.unpack(p)
    assert d["W1"][1, 0] == 8 and d["b1"][0] == 512 and d["b3"][0] == 4800
    assert np.array_equal(mlp.pack(d), p)
