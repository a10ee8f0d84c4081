"""The comparators of slimLS and its damping schedules, float64 (oracle side).

Test infrastructure only: nothing on the product path imports this module.

sg (Sec. 2): Eq. (ram) with B_k = alpha_k I, the stochastic (sampled)
gradient method
    x_k = x_{k-1} - alpha_k A_k^T (A_k x_{k-1} - b_k).

olbfgs (the comparator of Sec. 4.1, the online limited-memory BFGS method of
the paper's reference [mokhtari2015global], memory tau):
    g_k = A_k^T (A_k x_{k-1} - b_k)              the sampled gradient,
    x_k = x_{k-1} - alpha_k H_k g_k,
with H_k the L-BFGS approximation of the inverse Hessian built from the last
tau curvature pairs
    s_j = x_j - x_{j-1},   y_j = A_j^T A_j s_j,
y_j being the change of block j's sampled gradient between x_{j-1} and x_j
(the same sample at both points, so the data term cancels).  H_k is applied by
the two-loop recursion from H^0 = gamma_k I, gamma_k the mean of
s_j^T y_j / y_j^T y_j over the stored pairs (the averaged initial scaling of
the online method; H_k = I before the first pair).  A pair with s^T y <= 0 is
not stored (the curvature condition BFGS needs).

Step size: both comparators take alpha_k = 1/lambda_k, with lambda_k from the
damping schedule of slimLS, so one parameter sweeps the three methods over the
same range (Sec. 4.1 compares them at the same step sizes / damping factors).

Decaying damping (end of Sec. 3: a decaying damping parameter after a
constant one gives more accurate solutions): lambda_k = lambda for k <= K,
lambda_k = lambda k / K after (alpha_k = alpha K / k, a 1/k decay; the paper
names no law).  With the ramp of Sec. 4.2 as well, the ramp governs k <= r+1.
"""
from __future__ import annotations

import collections

import numpy as np


def damping(lam: float, k: int, r: int = 0, ramp: bool = False, decay_after: int = 0) -> float:
    """lambda_k: the ramp of Sec. 4.2 for k <= r+1, the 1/k decay after step
    `decay_after` (0: none), else lambda."""
    if ramp and k <= r + 1:
        return lam * (r + 1) / k
    if decay_after > 0 and k > decay_after:
        return lam * k / decay_after
    return lam


def step_sg(x_prev, A_k, b_k, alpha_k: float, eta: float = 1.0):
    """One sampled-gradient step.  Returns (x_k, r_k)."""
    r_k = A_k @ x_prev - b_k
    return x_prev - eta * alpha_k * (A_k.T @ r_k), r_k


def two_loop(g, pairs, gamma: float):
    """H g by the L-BFGS two-loop recursion over `pairs` (oldest first, each
    (s, y, rho) with rho = 1/(s^T y)) from H^0 = gamma I."""
    q = np.array(g, dtype=np.float64)
    a = []
    for s, y, rho in reversed(pairs):
        ai = rho * (s @ q)
        q = q - ai * y
        a.append(ai)
    q = gamma * q
    for (s, y, rho), ai in zip(pairs, reversed(a)):
        bi = rho * (y @ q)
        q = q + (ai - bi) * s
    return q


def initial_scaling(pairs) -> float:
    """gamma_k: mean of s^T y / y^T y over the stored pairs (1 if none)."""
    if not pairs:
        return 1.0
    return float(np.mean([(s @ y) / (y @ y) for s, y, _ in pairs]))


class Olbfgs:
    """State of the online L-BFGS comparator: the last `memory` pairs."""

    def __init__(self, memory: int = 10):
        self.pairs = collections.deque(maxlen=memory) if memory > 0 else None

    def step(self, x_prev, A_k, b_k, alpha_k: float, eta: float = 1.0):
        """One step.  Returns (x_k, r_k)."""
        r_k = A_k @ x_prev - b_k
        g = A_k.T @ r_k
        pairs = list(self.pairs) if self.pairs is not None else []
        d = two_loop(g, pairs, initial_scaling(pairs))
        s = -eta * alpha_k * d
        if self.pairs is not None:
            y = A_k.T @ (A_k @ s)
            sy = float(s @ y)
            if sy > 0.0:
                self.pairs.append((s, y, 1.0 / sy))
        return x_prev + s, r_k


def run(source, blocks, lam: float, method: str = "sg", memory: int = 10, x0=None,
        eta: float = 1.0, decay_after: int = 0):
    """sg or olbfgs over the given sequence of blocks (row ids of `source`, a
    slim.RowSource), alpha_k = 1/lambda_k.  Yields (k, x_k, r_k)."""
    x = np.zeros(source.n) if x0 is None else np.array(x0, dtype=np.float64)
    opt = Olbfgs(memory) if method == "olbfgs" else None
    for k, ids in enumerate(blocks, start=1):
        A_k = source.rows(ids)
        alpha_k = 1.0 / damping(lam, k, decay_after=decay_after)
        if opt is None:
            x, r_k = step_sg(x, A_k, source.rhs(ids), alpha_k, eta)
        else:
            x, r_k = opt.step(x, A_k, source.rhs(ids), alpha_k, eta)
        yield k, x, r_k
