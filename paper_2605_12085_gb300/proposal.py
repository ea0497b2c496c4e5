"""Training of the learned step proposal.

The plain method (Step 2d: every line search starts from alpha_0) is run on
seeded synthetic phantoms; each iteration gives one trace: the proposal's
eight input features (computed by the solver, fbl_step_stats.features) and
the grid index j = log_beta(alpha / alpha_0) of the step the plain rule
accepted.  The network (8 -> 64 -> 64 -> 1, tanh) is fitted, with the
library's own CUDA training kernels (mlp_train), to the change of j from the
previous iteration (to j itself at a run's first iteration): consecutive
iterations need similar steps, so the change transfers across problem sizes
where j does not.  The solver then starts each search at
alpha_0 * beta^floor(j_prev + prediction + 1/2 - margin), a point of the plain
rule's own grid; acceptance (2.3) and backtracking are unchanged.

    python -m paper_2605_12085_gb300.proposal --out PATH [--traces N]

writes the trained parameters and the training record as JSON.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "proposal_mlp.json")


def _glorot(seed: int) -> np.ndarray:
    """Seeded Glorot-uniform weights and zero biases in the packed layout
    W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def w(fan_out, fan_in):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, fan_out * fan_in)

    parts = [w(64, 8), np.zeros(64), w(64, 64), np.zeros(64), w(1, 64), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def trace_problems(n_problems: int, seed: int):
    """Seeded problem settings: cube edge 128..256 voxels, detector 1.5x, views
    and mini-batch size, mu and noise level drawn per problem."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n_problems):
        n = int(rng.choice([128, 144, 160, 192, 224, 256]))
        views = int(rng.choice([90, 120, 180, 240, 360]))
        N0 = int(rng.choice([8, 10, 16, 20, 40]))
        mu = float(rng.choice([0.25, 0.5, 1.0, 2.0]))
        noise = float(rng.choice([0.0, 0.005, 0.01, 0.02]))
        out.append(dict(n=n, views=views, N0=min(N0, views), mu=mu, noise=noise,
                        seed=5000 + seed * 1000 + q))
    return out


def make_problem(fbl, prob, device):
    """Phantom, geometry and data b = A x_true + noise for one trace problem."""
    import torch
    import synth
    n = prob["n"]
    det = int(math.ceil(1.5 * n))
    g = synth.Geometry(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, n_views=prob["views"],
                       sod=1000.0, sdd=1500.0, nu=det, nv=det, du=1.5, dv=1.5)
    xt = synth.phantom(g, 12, prob["seed"])
    G = fbl.geometry_create(g)
    xd = torch.from_numpy(xt).to(device)
    b = fbl.project(G, xd, range(g.n_views))
    if prob["noise"] > 0:
        sig = prob["noise"] * float(b.max())
        b += torch.from_numpy(synth.gaussian_noise(tuple(b.shape), sig, prob["seed"] + 1)).to(device)
    return g, G, b


def generate_traces(target: int, seed: int = 0, epochs: int = 12, use_graph: int = 1, log=print):
    """Run the plain method on seeded problems until `target` traces exist.
    Returns X [n][8] (float32), t [n] (float32 change of the accepted grid
    index), info."""
    import torch
    import paper_2605_12085_gb300 as fbl
    device = torch.device("cuda")
    X, T, info = [], [], []
    q = 0
    t0 = time.time()
    while sum(len(x) for x in X) < target:
        prob = trace_problems(q + 1, seed)[q]
        q += 1
        g, G, b = make_problem(fbl, prob, device)
        p = fbl.params_default(alpha0=1e-3, beta=0.5, mu=prob["mu"], N0=prob["N0"],
                               seed=prob["seed"], use_graph=use_graph)
        S = fbl.fblisa_create(G, p)
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device=device)
        tr = S.run(x, b, epochs)
        feats = np.array([t["features"] for t in tr], dtype=np.float32)
        j_acc = np.array([t["j_start"] + t["backtracks"] for t in tr], dtype=np.float32)
        j_prev = np.concatenate([[0.0], j_acc[:-1]])  # one uninterrupted run per problem
        X.append(feats)
        T.append((j_acc - j_prev).astype(np.float32))
        info.append(dict(prob, iterations=len(tr),
                         mean_backtracks=float(np.mean([t["backtracks"] for t in tr]))))
        log("problem %d: n=%d views=%d N0=%d mu=%g noise=%g -> %d traces, mean backtracks %.2f "
            "(%.0f s)" % (q, prob["n"], prob["views"], prob["N0"], prob["mu"], prob["noise"],
                          len(tr), info[-1]["mean_backtracks"], time.time() - t0))
        del S, G, b, x
    return np.concatenate(X), np.concatenate(T), info


def train(X, t, epochs: int = 200, batch: int = 256, lr: float = 2e-3, seed: int = 0,
          val_frac: float = 0.1, log=print):
    """Fit the network on (X, t) with the library's Adam kernel; returns the
    parameters (numpy float32) and a record of the training."""
    import torch
    import paper_2605_12085_gb300 as fbl
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(len(t))
    nval = max(1, int(val_frac * len(t)))
    vi, ti = perm[:nval], perm[nval:]
    Xt = torch.from_numpy(np.ascontiguousarray(X[ti])).cuda()
    tt = torch.from_numpy(np.ascontiguousarray(t[ti])).cuda()
    Xv = torch.from_numpy(np.ascontiguousarray(X[vi])).cuda()
    tv = torch.from_numpy(np.ascontiguousarray(t[vi])).cuda()
    P = torch.from_numpy(_glorot(seed)).cuda()
    tr = fbl.MlpTrainer(P)
    rec = []
    chunk = 20
    for e0 in range(0, epochs, chunk):
        # reshuffle the training set between chunks of epochs
        sh = torch.from_numpy(rng.permutation(len(ti))).cuda()
        Xs, ts = Xt[sh].contiguous(), tt[sh].contiguous()
        tr.train(Xs, ts, batch=batch, epochs=min(chunk, epochs - e0), lr=lr)
        _, lt = fbl.mlp_gradient(P, Xt, tt)
        _, lv = fbl.mlp_gradient(P, Xv, tv)
        pv = fbl.mlp_forward(P, Xv).cpu().numpy()
        acc = float(np.mean(np.abs(pv - t[vi]) < 0.5))
        rec.append(dict(epoch=e0 + min(chunk, epochs - e0), train_loss=lt, val_loss=lv,
                        val_within_half=acc))
        log("epoch %d: train loss %.4f, val loss %.4f, val |pred - t| < 0.5: %.3f"
            % (rec[-1]["epoch"], lt, lv, acc))
    return P.cpu().numpy(), rec


def save(path, params, meta):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(dict(meta, params=[float(v) for v in params]), f)


def load(path=DEFAULT_WEIGHTS):
    """The trained parameters (numpy float32, 4801 values) and their record."""
    with open(path) as f:
        d = json.load(f)
    p = np.asarray(d.pop("params"), dtype=np.float32)
    if p.size != 4801:
        raise ValueError("proposal weights must have 4801 values")
    return p, d


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--traces", type=int, default=50000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    t0 = time.time()
    X, t, info = generate_traces(args.traces, seed=args.seed)
    t1 = time.time()
    params, rec = train(X, t, epochs=args.epochs, seed=args.seed)
    np.savez(os.path.splitext(args.out)[0] + "_traces.npz", X=X, t=t)
    meta = dict(network="8-64-64-1 tanh",
                target="change of the plain rule's accepted grid index from the previous iteration",
                traces=int(len(t)), problems=info, training=rec,
                trace_seconds=t1 - t0, train_seconds=time.time() - t1,
                target_mean=float(t.mean()), target_std=float(t.std()))
    save(args.out, params, meta)
    print("wrote %s: %d traces, final val loss %.4f" % (args.out, len(t), rec[-1]["val_loss"]))
    return 0


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(HERE))
    sys.exit(main())
