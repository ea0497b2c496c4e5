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


def test_adam_constant_gradient_closed_form():
    # With the same gradient g at every step the bias-corrected moments equal
    # g and g^2 exactly, so every step moves p by lr * g / (|g| + eps); a
    # missing bias correction or a swapped beta breaks this at steps 1-5.
    rng = np.random.default_rng(3)
    g = rng.standard_normal(50) * np.logspace(-6, 2, 50)
    p = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 2e-3, 1e-8
    for step in range(1, 6):
        p_new, m, v = mlp.adam_step(p, m, v, g, step, lr, eps=eps)
        assert np.allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
        p = p_new


def test_adam_first_moments_follow_the_gradient_sequence():
    # two different gradients: the step-2 update is the bias-corrected
    # exponential average (0.9*0.1*g1 + 0.1*g2) / 0.19 over the rms of the
    # second moments, written out from the definitions
    g1, g2 = np.array([1.0, -2.0, 0.5]), np.array([3.0, 1.0, -0.5])
    p1, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g1, 1, 0.1, eps=0.0)
    p2, m, v = mlp.adam_step(p1, m, v, g2, 2, 0.1, eps=0.0)
    m_hat = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    v_hat = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(p2 - p1, -0.1 * m_hat / np.sqrt(v_hat), rtol=1e-12)
