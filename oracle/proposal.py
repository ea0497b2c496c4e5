"""FP64 reference of the learned step proposal (test infrastructure).

TEST INFRASTRUCTURE: see ``oracle/__init__.py``.

The paper restarts every line search at alpha_0 (Alg. 1, Step 2d).  The
library can instead start it at a point alpha_0 * beta^j of the plain rule's
own grid, j chosen by a small network from mini-batch statistics; the test
(2.3) and the backtracking stay as the paper defines them.  The paper has no
counterpart of the proposal, so this module follows its definition in the
library's interface (fblisa_set_proposal), written out step by step in FP64:

  * features of iteration k, from f = f_N(x), g2 = ||grad f_N(x)||^2 and the
    statistics of the previous accepted iterations, with the curvature index
    c = log2(alpha_0 g2 / (2 f)):
      0: c/10 at the first iteration, 0 afterwards
      1: log(f / f_prev)
      2: log(|g| / |g_prev|)
      3: (c - c_prev)/10
      4: N_t / n_theta
      5: log(1 + k)/10, k the number of accepted iterations so far
      6: 1 if there is a previous iteration, else 0
      7: (j_prev - j_prevprev)/4, the last change of the accepted grid index
    (features 1-3 and 7 are 0 while their inputs do not exist yet);
  * the network's output pred (oracle/mlp.forward of the features);
  * the first trial's grid index j = clamp(floor(j_prev + pred + 1/2 - margin),
    0, max_backtracks), j_prev the accepted index of the previous iteration
    (0 at the first), j = 0 when pred is not finite; the first trial step is
    alpha_0 multiplied j times by beta, the plain rule's j-th trial;
  * after an accepted step of index j_acc = j + backtracks the statistics
    move on: f_prev, g2_prev <- f, g2; the last change j_acc - j_prev; j_prev
    <- j_acc; k <- k + 1.

Parity against the paper: unpinned (no counterpart).  Pinned by facts outside
this module (tests/test_oracle_proposal.py): without a network the run is the
plain method's; an exact predictor of the plain rule's next index reproduces
the plain run with no backtrack at all; every feature is invariant under a
scaling of the problem; and with data along the top singular vector of the
first mini-batch's operator, feature 0 equals log2(alpha_0 L_N)/10.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

from . import fblisa, mlp


@dataclasses.dataclass
class PropState:
    """Statistics carried from one accepted iteration to the next."""
    f_prev: float = 0.0
    g2_prev: float = 0.0
    k: int = 0
    j_prev: int = 0
    have_prev: bool = False
    dj_prev: int = 0
    have_dj: bool = False


def _curvature_index(alpha0: float, g2: float, f: float) -> float:
    """c = log2(alpha_0 g2 / (2 f)); g2 / (2 f) <= L_N for the quadratic f_N."""
    return math.log2(max(alpha0 * g2 / max(2.0 * f, 1e-300), 1e-300))


def features(st: PropState, f: float, g2: float, alpha0: float, N_t: int, n_theta: int) -> np.ndarray:
    """The eight inputs of the proposal network at one iteration."""
    c = _curvature_index(alpha0, g2, f)
    out = np.zeros(8)
    if st.have_prev:
        c_prev = _curvature_index(alpha0, st.g2_prev, st.f_prev)
        out[1] = math.log(max(f, 1e-300) / max(st.f_prev, 1e-300))
        out[2] = 0.5 * math.log(max(g2, 1e-300) / max(st.g2_prev, 1e-300))
        out[3] = 0.1 * (c - c_prev)
        out[6] = 1.0
    else:
        out[0] = 0.1 * c
    out[4] = N_t / n_theta
    out[5] = 0.1 * math.log(1.0 + st.k)
    if st.have_dj:
        out[7] = 0.25 * st.dj_prev
    return out


def first_index(st: PropState, pred: float, margin: float, cap: int) -> int:
    """Grid index of the first trial: clamp(floor(j_prev + pred + 1/2 - margin), 0, cap)."""
    if not math.isfinite(pred):
        return 0
    base = st.j_prev if st.have_prev else 0
    return min(max(int(math.floor(base + pred + 0.5 - margin)), 0), cap)


def grid_step(alpha0: float, beta: float, j: int) -> float:
    """The plain rule's j-th trial: alpha_0 reduced j times by the factor beta."""
    a = alpha0
    for _ in range(j):
        a *= beta
    return a


def accept(st: PropState, f: float, g2: float, j_acc: int) -> None:
    """Move the statistics on after an accepted step of grid index j_acc."""
    st.f_prev = f
    st.g2_prev = g2
    st.dj_prev = j_acc - st.j_prev
    st.have_dj = st.have_prev
    st.j_prev = j_acc
    st.have_prev = True
    st.k += 1


@dataclasses.dataclass
class ProposalRecord:
    features: np.ndarray
    pred: float
    j_start: int
    step: fblisa.StepRecord


def network(params) -> Callable[[np.ndarray], float]:
    """The predictor of a parameter vector (oracle/mlp.forward)."""
    p = np.asarray(params, dtype=np.float64)
    return lambda feat: float(mlp.forward(p, feat[None, :])[0][0])


def run(geom, b: np.ndarray, x0: np.ndarray, p: fblisa.Params, epochs: int,
        predict: Optional[Callable[[np.ndarray], float]], margin: float = 0.25,
        impose_alpha_init: Optional[List[float]] = None, max_iters: Optional[int] = None):
    """Alg. 1 (oracle/fblisa.py) with the first trial of every line search
    taken from the proposal.  ``predict``: features -> pred (None: the plain
    rule, first trial alpha_0).  ``impose_alpha_init``: first trial steps to use
    instead of the proposal's, one per iteration (the proposal is still
    evaluated and recorded).  Returns (x, [ProposalRecord, ...])."""
    n_theta = geom.n_views
    n_max = p.n_max if p.n_max > 0 else n_theta
    x = np.asarray(x0, dtype=np.float64).reshape(geom.vol_shape).copy()
    st = PropState()
    out: List[ProposalRecord] = []
    k = 0
    for t, (N_t, _iters) in enumerate(fblisa.schedule(n_theta, p.N0, n_max, p.C, p.eps_base, epochs), start=1):
        for views in fblisa.epoch_batches(p.seed, t, n_theta, N_t):
            if max_iters is not None and k >= max_iters:
                return x, out
            seen = {}

            def first_step(f, g2, N_t=N_t, k=k, seen=seen):
                feat = features(st, f, g2, p.alpha0, N_t, n_theta)
                pred = predict(feat) if predict is not None else 0.0
                j = first_index(st, pred, margin, p.max_backtracks) if predict is not None else 0
                seen.update(feat=feat, pred=pred, j=j, f=f, g2=g2)
                if impose_alpha_init is not None:
                    return impose_alpha_init[k]
                return grid_step(p.alpha0, p.beta, j)

            x, rec = fblisa.fb_step(geom, x, b, views, p, k=k, epoch=t, first_step=first_step)
            j_first = seen["j"]
            if impose_alpha_init is not None:
                j_first = int(round(math.log(impose_alpha_init[k] / p.alpha0) / math.log(p.beta)))
            accept(st, seen["f"], seen["g2"], j_first + rec.backtracks)
            out.append(ProposalRecord(seen["feat"], seen["pred"], seen["j"], rec))
            k += 1
    return x, out
