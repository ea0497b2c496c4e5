"""The step-proposal network's hand-written kernels against the FP64
reference perceptron (oracle/mlp.py): forward values, the full-batch
gradient, and that Adam training fits a smooth target."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_and_gradient_match_fp64_reference():
    import paper_2605_12085_gb300 as fbl
    rng = np.random.default_rng(1)
    p = mlp.init(3) + 0.05 * rng.standard_normal(mlp.NPARAMS)
    p32 = p.astype(np.float32).astype(np.float64)
    X = rng.standard_normal((1000, 8)).astype(np.float32).astype(np.float64)
    t = rng.standard_normal(1000).astype(np.float32).astype(np.float64)
    y = fbl.mlp_forward(_cuda(p32), _cuda(X)).double().cpu().numpy()
    yo, _ = mlp.forward(p32, X)
    assert np.max(np.abs(y - yo)) <= 1e-5 * (1 + np.abs(yo).max())
    g, loss = fbl.mlp_gradient(_cuda(p32), _cuda(X), _cuda(t))
    go = mlp.gradient(p32, X, t)
    g = g.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    assert loss == pytest.approx(mlp.loss(p32, X, t), rel=1e-5)


def test_training_fits_a_smooth_target():
    import paper_2605_12085_gb300 as fbl
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (4096, 8))
    t = np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3]
    P = _cuda(mlp.init(5))
    tr = fbl.MlpTrainer(P)
    Xd, td = _cuda(X), _cuda(t)
    _, l0 = fbl.mlp_gradient(P, Xd, td)
    tr.train(Xd, td, batch=128, epochs=60, lr=3e-3)
    _, l1 = fbl.mlp_gradient(P, Xd, td)
    assert l1 < 0.05 * l0
    assert int(tr.step.item()) == 60 * 32
    # the trained weights evaluate the same on the FP64 reference
    y = fbl.mlp_forward(P, Xd).double().cpu().numpy()
    yo, _ = mlp.forward(P.double().cpu().numpy(), X.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 1e-5 * (1 + np.abs(yo).max())


def test_two_adam_steps_match_fp64_reference():
    # full-batch minibatches: each kernel step uses the gradient at the current
    # parameters, so two steps of the kernel must equal two oracle steps
    import paper_2605_12085_gb300 as fbl
    rng = np.random.default_rng(4)
    n = 512
    X = rng.standard_normal((n, 8)).astype(np.float32).astype(np.float64)
    t = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    p0 = mlp.init(9).astype(np.float32).astype(np.float64)
    lr = 1e-3
    P = _cuda(p0)
    tr = fbl.MlpTrainer(P)
    tr.train(_cuda(X), _cuda(t), batch=n, epochs=2, lr=lr)
    assert int(tr.step.item()) == 2
    p_gpu = P.double().cpu().numpy()
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    p = p0
    grads = []
    for step in (1, 2):
        g = mlp.gradient(p, X, t)
        grads.append(g)
        p, m, v = mlp.adam_step(p, m, v, g, step, lr)
    # Adam moves a parameter by about lr whatever the size of its gradient, so a
    # gradient within FP32 rounding of zero may flip its step; compare the
    # parameters whose gradients are clearly non-zero in both steps
    scale = np.median(np.abs(grads[0]))
    keep = (np.abs(grads[0]) > 1e-3 * scale) & (np.abs(grads[1]) > 1e-3 * scale)
    assert keep.mean() > 0.95
    d_gpu, d_ref = (p_gpu - p0)[keep], (p - p0)[keep]
    assert np.linalg.norm(d_gpu - d_ref) <= 1e-3 * np.linalg.norm(d_ref)
    assert np.max(np.abs(p_gpu - p)) <= 2.5 * lr  # any flipped step stays a step
