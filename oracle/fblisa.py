"""FB-LISA (Algorithm 1) step by step in numpy float64.

TEST INFRASTRUCTURE: see ``oracle/__init__.py``.

Notation follows Sec. 2: x the volume, A_N the operator restricted to the
views of the mini-batch N_k (eq. (2.5)), f_N(x) = n_theta/(2 N_t) ||A_N x - b_N||^2,
R(x) = mu ||x||_1 + indicator{x >= 0} (eq. (2.1)), the forward-backward
update x_bar = prox_{alpha R}(x - alpha grad f_N(x)) and the sufficient-decrease
test (2.3).  Readings of points the paper leaves open (all listed in the
design notes):

  * eq. (2.4) as printed is off by n_theta; the consistent reading is
    f_i = (n_theta/2) ||A_i x - b_i||^2, so that (1/n_theta) sum_i f_i equals the
    fidelity of (2.1); this gives eq. (2.5) unchanged;
  * "n" in Step 1 and Step 2 is n_theta; C = M = 1; n_max = n_theta; eps_k = 0.99^k;
  * beta = 0.5 (the paper defers it to Deep-LISA); a cap of 60 backtracks;
  * a mini-batch is a slice of a per-epoch Fisher-Yates permutation drawn
    from SplitMix64; a short last slice is padded from the front of the
    same permutation;
  * the prox of mu||.||_1 + indicator{x >= 0} is max(v - alpha mu, 0).

Params.reg / x_max / tv_iters / tv_warm select the other regularisers of
oracle/tv.py (the box-constrained l1 and isotropic TV); the defaults are the
paper's R.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from . import backproject, project
from . import tv as tv_oracle

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15          # SplitMix64 increment (Steele, Lea & Flood, 2014)
EPOCH_KEY = 0xD1B54A32D192ED03      # odd constant that separates the epochs' streams


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output function (variant-13 finaliser), on 64-bit ints."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_draw(state: int, i: int) -> int:
    """Output number i (0-based) of a SplitMix64 generator started at ``state``."""
    return splitmix64_mix((state + (i + 1) * GAMMA) & MASK64)


def epoch_permutation(seed: int, epoch: int, n: int) -> List[int]:
    """Fisher-Yates permutation of 0..n-1 for epoch ``epoch`` (1-based).

    Draw i is u_i = (z >> 11) * 2^-53 with z = SplitMix64 output i of the
    stream started at seed XOR (epoch * EPOCH_KEY); swap entry i with entry
    i + floor(u_i * (n - i)).
    """
    state = (seed ^ ((epoch * EPOCH_KEY) & MASK64)) & MASK64
    perm = list(range(n))
    for i in range(n - 1):
        u = (splitmix64_draw(state, i) >> 11) * (1.0 / 9007199254740992.0)
        j = i + int(math.floor(u * (n - i)))
        j = min(j, n - 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def epoch_batches(seed: int, epoch: int, n_theta: int, N_t: int) -> List[List[int]]:
    """The ceil(n_theta/N_t) mini-batches N_k of one epoch (Alg. 1, Step 2a)."""
    perm = epoch_permutation(seed, epoch, n_theta)
    iters = -(-n_theta // N_t)
    out = []
    for j in range(iters):
        sl = perm[j * N_t:(j + 1) * N_t]
        if len(sl) < N_t:
            sl = sl + perm[:N_t - len(sl)]
        out.append(sl)
    return out


def schedule(n_theta: int, N0: int, n_max: int, C: float, eps_base: float, epochs: int):
    """Alg. 1 Step 1 for t = 1..epochs: list of (N_t, iterations in epoch t).

    N_t = min{n_max, max{ceil(C / eps_{k_hat + ceil(n/N_{t-1})}), N_0}} with
    eps_k = eps_base^k and N_{t-1} = N_0 at t = 1; the epoch then runs
    ceil(n/N_t) iterations and k_hat grows by that (Step 3).
    """
    k_hat = 0
    N_prev = N0
    out = []
    for _t in range(1, epochs + 1):
        K = k_hat + -(-n_theta // N_prev)
        N_t = min(n_max, max(int(math.ceil(C / (eps_base ** K))), N0))
        iters = -(-n_theta // N_t)
        out.append((N_t, iters))
        k_hat += iters
        N_prev = N_t
    return out


def prox(v: np.ndarray, alpha: float, mu: float) -> np.ndarray:
    """prox of alpha*(mu||.||_1 + indicator{x >= 0}): max(v - alpha mu, 0) elementwise."""
    return np.maximum(v - alpha * mu, 0.0)


@dataclasses.dataclass
class Params:
    alpha0: float = 1e-3
    beta: float = 0.5
    mu: float = 1.0
    C: float = 1.0
    eps_base: float = 0.99
    N0: int = 8
    n_max: int = 0            # 0 -> n_theta
    max_backtracks: int = 60
    seed: int = 0
    fixed_step: bool = False  # forward-backward with the constant step alpha0, no test (2.3)
    reg: str = "l1"           # "l1": mu||x||_1, "tv": mu TV(x); either with the box [0, x_max]
    x_max: float = math.inf
    tv_iters: int = 20        # FGP iterations per prox ("tv")
    tv_warm: bool = True      # each TV prox starts from the dual the previous one ended with


class TVState:
    """The dual field carried from one TV prox to the next (warm start)."""

    def __init__(self):
        self.q = None


def reg_prox(v: np.ndarray, alpha: float, p: Params, tv_state: Optional[TVState] = None) -> np.ndarray:
    """prox_{alpha R}(v) for the regulariser p.reg (oracle/tv.py)."""
    if p.reg == "l1":
        return tv_oracle.prox_l1_box(v, alpha, p.mu, p.x_max)
    if p.reg != "tv":
        raise ValueError("unknown regulariser %r" % p.reg)
    q0 = tv_state.q if (p.tv_warm and tv_state is not None) else None
    x, q = tv_oracle.prox_tv(v, alpha * p.mu, p.tv_iters, p.x_max, q0=q0)
    if p.tv_warm and tv_state is not None:
        tv_state.q = q
    return x


@dataclasses.dataclass
class Trial:
    alpha: float
    rho1: float
    gTd: float
    dnorm2: float
    f_xbar: float
    rhs: float
    accepted: bool


@dataclasses.dataclass
class StepRecord:
    k: int
    epoch: int
    N_t: int
    views: List[int]
    rho0: float
    f_x: float
    trials: List[Trial]
    alpha: float
    backtracks: int
    grad_norm2: float = float("nan")   # ||grad f_N(x)||^2
    alpha_init: float = float("nan")   # the first trial step

    @property
    def margin(self) -> float:
        t = self.trials[-1]
        return t.rhs - t.f_xbar


class LineSearchError(RuntimeError):
    pass


def fb_step(geom, x: np.ndarray, b: np.ndarray, views: Sequence[int], p: Params,
            alpha_init: Optional[float] = None, replay_alpha: Optional[float] = None,
            k: int = 0, epoch: int = 0, tv_state: Optional[TVState] = None,
            first_step=None):
    """One iteration of Alg. 1, Steps 2b-2d, on the mini-batch ``views``.

    Returns (x_next, StepRecord).  With ``replay_alpha`` the step size is
    imposed instead of searched (the test (2.3) is still evaluated and
    recorded, so a disagreement shows as a negative margin).  ``first_step``:
    a callable (f_N(x), ||grad f_N(x)||^2) -> first trial step, called after
    Step 2b (the learned proposal, oracle/proposal.py); else ``alpha_init``
    or alpha_0.
    """
    n_theta = geom.n_views
    N_t = len(views)
    scale = n_theta / N_t
    bS = np.asarray(b, dtype=np.float64)[list(views)]
    # Step 2b: f_N(x) and grad f_N(x) = (n_theta/N_t) A_N^T (A_N x - b_N)
    r = project(geom, x, views) - bS
    rho0 = float(np.dot(r.ravel(), r.ravel()))
    f_x = 0.5 * scale * rho0
    g = scale * backproject(geom, r, views)
    g2 = float(np.dot(g.ravel(), g.ravel()))
    alpha = p.alpha0 if alpha_init is None else alpha_init
    if first_step is not None:
        alpha = first_step(f_x, g2)
    if replay_alpha is not None:
        alpha = replay_alpha
    a_first = alpha
    if p.fixed_step:
        # the deterministic FB baseline of Sec. 3 (with the full batch): one
        # forward-backward step at the constant alpha_0, no sufficient-decrease test
        xbar = reg_prox(x - p.alpha0 * g, p.alpha0, p, tv_state)
        d = xbar - x
        t = Trial(p.alpha0, float("nan"), float(np.dot(g.ravel(), d.ravel())),
                  float(np.dot(d.ravel(), d.ravel())), float("nan"), float("nan"), True)
        return xbar, StepRecord(k, epoch, N_t, list(views), rho0, f_x, [t], p.alpha0, 0, g2, p.alpha0)
    trials = []
    for bt in range(p.max_backtracks + 1):
        # Step 2c: forward-backward point and the test (2.3)
        xbar = reg_prox(x - alpha * g, alpha, p, tv_state)
        d = xbar - x
        gTd = float(np.dot(g.ravel(), d.ravel()))
        dd = float(np.dot(d.ravel(), d.ravel()))
        r1 = project(geom, xbar, views) - bS
        rho1 = float(np.dot(r1.ravel(), r1.ravel()))
        f_xbar = 0.5 * scale * rho1
        rhs = f_x + gTd + dd / (2.0 * alpha)
        ok = f_xbar <= rhs
        trials.append(Trial(alpha, rho1, gTd, dd, f_xbar, rhs, ok))
        if ok or replay_alpha is not None:
            # Step 2d: x^(k+1) = x_bar; the next iteration restarts from alpha_0
            return xbar, StepRecord(k, epoch, N_t, list(views), rho0, f_x, trials, alpha, bt, g2, a_first)
        alpha *= p.beta
    raise LineSearchError("no step size passed (2.3) within %d backtracks" % p.max_backtracks)


def run(geom, b: np.ndarray, x0: np.ndarray, p: Params, epochs: int,
        replay: Optional[Sequence[float]] = None, max_iters: Optional[int] = None):
    """Alg. 1 for ``epochs`` epochs; returns (x, [StepRecord, ...]).

    ``replay``: accepted step sizes to impose, one per iteration.
    ``max_iters``: stop after that many iterations (for short checks).
    """
    n_theta = geom.n_views
    n_max = p.n_max if p.n_max > 0 else n_theta
    x = np.asarray(x0, dtype=np.float64).reshape(geom.vol_shape).copy()
    records = []
    k = 0
    tv_state = TVState()
    for t, (N_t, iters) in enumerate(schedule(n_theta, p.N0, n_max, p.C, p.eps_base, epochs),
                                     start=1):
        for views in epoch_batches(p.seed, t, n_theta, N_t):
            if max_iters is not None and k >= max_iters:
                return x, records
            ra = None if replay is None else replay[k]
            x, rec = fb_step(geom, x, b, views, p, replay_alpha=ra, k=k, epoch=t, tv_state=tv_state)
            records.append(rec)
            k += 1
    return x, records


def full_objective(geom, x: np.ndarray, b: np.ndarray, mu: float) -> float:
    """F(x) = 1/2 ||A x - b||^2 + mu ||x||_1 over all views (eq. (2.1); x >= 0)."""
    r = project(geom, x, range(geom.n_views)) - np.asarray(b, dtype=np.float64)
    return 0.5 * float(np.dot(r.ravel(), r.ravel())) + mu * float(np.abs(x).sum())
