"""FP64 reference of the step-proposal network (test infrastructure).

The paper has no learned component (it resets the step to alpha_0 at every
iteration, Step 2d); this is the textbook definition of the perceptron the
library uses, 8 -> 64 -> 64 -> 1 with tanh hidden units, and of its loss
1/(2n) sum (y - t)^2, with the gradient by the chain rule, and the Adam update
the training kernel takes.  Pinned by central finite differences of the loss
and by Adam's closed form under a constant gradient (tests/test_oracle_mlp.py).  Parameters are
packed as W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
import numpy as np

NI, NH = 8, 64
SIZES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)),
         ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init(seed):
    """Seeded Glorot-uniform weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            fan_out = shape[0] if len(shape) == 2 else 1
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            d[name] = rng.uniform(-lim, lim, shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ w["W1"].T + w["b1"])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"])
    return h2 @ w["W3"] + w["b3"][0], (h1, h2)


def loss(p, X, t):
    y, _ = forward(p, X)
    r = y - np.asarray(t, dtype=np.float64)
    return 0.5 * float(np.mean(r * r))


def gradient(p, X, t):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    y, (h1, h2) = forward(p, X)
    n = X.shape[0]
    dy = (y - np.asarray(t, dtype=np.float64)) / n
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, w["W3"]) * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def adam_step(p, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015, Algorithm 1): moment estimates
    m, v updated with the gradient g, bias-corrected by 1 - beta^step (step
    counts from 1), then p - lr * m_hat / (sqrt(v_hat) + eps).  Returns the new
    (p, m, v)."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return np.asarray(p, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
