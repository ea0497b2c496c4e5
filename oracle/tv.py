"""Other regularisers for FB-LISA in numpy float64: the box-constrained l1
prox and the prox of isotropic total variation by inner iterations.

TEST INFRASTRUCTURE: see ``oracle/__init__.py``.

FB-LISA allows any proper convex lower-semicontinuous R with a computable
prox (Sec. 2.1 and the conclusions); the paper only runs
R = mu ||x||_1 + indicator{x >= 0} (eq. (2.1)).  Two more choices here, each
with the box C = [0, x_max]:

* R = mu ||x||_1 + indicator_C:  prox_{a R}(v) = clip(v - a mu, 0, x_max)
  (a separable convex quadratic on an interval: the unconstrained minimiser
  v - a mu projected onto [0, x_max]);
* R = mu TV(x) + indicator_C, TV(x) = sum over voxels of ||(K x)_v||_2, K the
  forward differences along the three axes with a zero difference at each
  axis's last index (unit grid spacing).  Its prox has no closed form; it is
  computed by the fast gradient projection of Beck and Teboulle (2009, FGP)
  on the dual: with lambda = a mu and the unit-ball set Q,

      x(q) = P_C(v - lambda K^T q)                     (primal of a dual point)
      q_k  = P_Q(r_k + K x(r_k) / (12 lambda))         (12 >= ||K||^2 in 3D)
      t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  r_{k+1} = q_k + (t_k - 1)/t_{k+1} (q_k - q_{k-1})

  from r_1 = q_0 (zero, or the previous call's dual: a warm start) and t_1 = 1,
  for a fixed number of iterations; the result is x(q_last).

Arrays are [nz][ny][nx]; a dual field is q[3][nz][ny][nx] with components
along x, y, z.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

AXES = (2, 1, 0)  # numpy axis of the x, y, z differences of a [nz][ny][nx] array


def prox_l1_box(v: np.ndarray, a: float, mu: float, x_max: float = math.inf) -> np.ndarray:
    """prox of a*(mu ||.||_1 + indicator{0 <= x <= x_max})."""
    return np.clip(v - a * mu, 0.0, x_max)


def grad(x: np.ndarray) -> np.ndarray:
    """K x: forward differences along x, y, z; zero at each axis's last index."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((3,) + x.shape)
    for c, ax in enumerate(AXES):
        n = x.shape[ax]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        dst = [c] + lo
        out[tuple(dst)] = x[tuple(hi)] - x[tuple(lo)]
    return out


def grad_adjoint(q: np.ndarray) -> np.ndarray:
    """K^T q, written out from the definition of K: voxel v takes -q_c(v) from
    its own difference and +q_c(v - e_c) from its lower neighbour's, for the
    differences that exist (v_c < n_c - 1, resp. v_c >= 1)."""
    q = np.asarray(q, dtype=np.float64)
    shape = q.shape[1:]
    out = np.zeros(shape)
    for c, ax in enumerate(AXES):
        n = shape[ax]
        own = [slice(None)] * 3
        own[ax] = slice(0, n - 1)
        out[tuple(own)] -= q[c][tuple(own)]
        up = [slice(None)] * 3
        up[ax] = slice(1, n)
        out[tuple(up)] += q[c][tuple(own)]
    return out


def tv(x: np.ndarray) -> float:
    """Isotropic TV: sum over voxels of the Euclidean norm of K x."""
    g = grad(x)
    return float(np.sqrt((g * g).sum(axis=0)).sum())


def _proj_ball(q: np.ndarray) -> np.ndarray:
    nrm = np.sqrt((q * q).sum(axis=0))
    return q / np.maximum(nrm, 1.0)[None]


def prox_tv(v: np.ndarray, lam: float, iters: int, x_max: float = math.inf,
            q0: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """prox of lam TV + indicator{0 <= x <= x_max} at v by ``iters`` FGP
    iterations from the dual q0 (zero if None).  Returns (x, q)."""
    v = np.asarray(v, dtype=np.float64)
    q = np.zeros((3,) + v.shape) if q0 is None else np.array(q0, dtype=np.float64)
    # a dual component where its difference does not exist (the last index of
    # its axis) takes no part: it is zero, so the ball projection ignores it
    for c, ax in enumerate(AXES):
        last = [slice(None)] * 3
        last[ax] = slice(v.shape[ax] - 1, v.shape[ax])
        q[c][tuple(last)] = 0.0

    def primal(p):
        return np.clip(v - lam * grad_adjoint(p), 0.0, x_max)

    if lam <= 0.0:
        return np.clip(v, 0.0, x_max), q
    r = q.copy()
    t = 1.0
    for _ in range(iters):
        q_new = _proj_ball(r + grad(primal(r)) / (12.0 * lam))
        t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        r = q_new + ((t - 1.0) / t_new) * (q_new - q)
        q, t = q_new, t_new
    return primal(q), q


def duality_gap(v: np.ndarray, lam: float, x: np.ndarray, q: np.ndarray,
                x_max: float = math.inf) -> float:
    """P(x) - D(q) for min_{x in C} 1/2 ||x - v||^2 + lam TV(x): x in C, q in
    Q.  Weak duality makes it >= 0, and it bounds 1/2 ||x - x*||^2 from above
    (strong convexity), so a small gap certifies x without trusting the
    iteration that made it."""
    v = np.asarray(v, dtype=np.float64)
    P = 0.5 * float(((x - v) ** 2).sum()) + lam * tv(x)
    z = np.clip(v - lam * grad_adjoint(q), 0.0, x_max)
    D = 0.5 * float(((z - v) ** 2).sum()) + lam * float((grad_adjoint(q) * z).sum())
    return P - D
