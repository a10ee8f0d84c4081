"""One slimLS iteration and runs of it, float64 (the oracle of the method).

Eq. (ram):   x_k = x_{k-1} - B_k A_k^T (A_k x_{k-1} - b_k)
Eq. (B_k):   B_k = (alpha_k^{-1} C_k + M_k^T M_k)^{-1},  M_k = [A_{k-r}; ...; A_k]
with C_k = I and lambda_k = 1/alpha_k.  Blocks with index < 1 are empty, so M_k
holds min(k, r+1) blocks; a block drawn twice appears twice (M_k is indexed by
iteration).  An extra step size eta multiplies s_k (eta = 1 is Eq. (ram)).

Sec. 4.2 writes the step as x_k = x_{k-1} - s_k and notes that s_k solves a
stacked damped least-squares problem (Eq. slimLSstep).  Two exact forms of s_k:

  direct    s = (lambda_k I_n + M_k^T M_k)^{-1} A_k^T r_k           (n x n solve)
  Woodbury  s = M_k^T z,  (lambda_k I_p + M_k M_k^T) z = [0; ...; 0; r_k]

The Woodbury form (Sec. 2 names the Sherman-Woodbury identity) follows from
A_k^T r_k = M_k^T [0;...;0;r_k] (A_k is the last block of M_k) and
(lambda I + M^T M)^{-1} M^T = M^T (lambda I + M M^T)^{-1}.

Damping ramp (Sec. 4.2): alpha_k = k*alpha/(r+1) for the first r+1 iterations,
i.e. lambda_k = lambda*(r+1)/k for k <= r+1.
"""
from __future__ import annotations

import collections
from typing import Callable, Iterable

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import joseph, rng


def damping(lam: float, k: int, r: int, ramp: bool) -> float:
    """lambda_k: constant, or the ramp of Sec. 4.2 for k <= r+1."""
    if ramp and k <= r + 1:
        return lam * (r + 1) / k
    return lam


def _as_csr(Mrows) -> sp.csr_matrix:
    return Mrows if sp.issparse(Mrows) else sp.csr_matrix(np.asarray(Mrows))


def step_woodbury(x_prev, blocks, b_new, lam_k: float, eta: float = 1.0):
    """One step in Woodbury form.

    blocks: the row blocks of M_k, oldest first; the last one is A_k (its rows
    are the sampled rows of this step).  Returns (x_k, r_k, s_k, z).
    """
    M = sp.vstack([_as_csr(B) for B in blocks], format="csr")
    A_k = _as_csr(blocks[-1])
    ell = A_k.shape[0]
    p = M.shape[0]
    r_k = A_k @ x_prev - b_new
    G = (M @ M.T).toarray()
    K = lam_k * np.eye(p) + G
    rhs = np.zeros(p)
    rhs[p - ell:] = r_k
    z = sla.cho_solve(sla.cho_factor(K, lower=True), rhs)
    s = M.T @ z
    return x_prev - eta * s, r_k, s, z


def step_direct(x_prev, blocks, b_new, lam_k: float, eta: float = 1.0):
    """One step in direct form: dense n x n solve (small n only)."""
    M = sp.vstack([_as_csr(B) for B in blocks], format="csr")
    A_k = _as_csr(blocks[-1])
    r_k = A_k @ x_prev - b_new
    n = M.shape[1]
    H = lam_k * np.eye(n) + (M.T @ M).toarray()
    s = sla.cho_solve(sla.cho_factor(H, lower=True), A_k.T @ r_k)
    return x_prev - eta * s, r_k, s


class RowSource:
    """A matrix known only through its rows: rows(ids) -> csr, b(ids) -> vector."""

    def __init__(self, rows_fn: Callable, b: np.ndarray, n: int):
        self._rows = rows_fn
        self.b = np.asarray(b, dtype=np.float64)
        self.n = n

    def rows(self, ids):
        return self._rows(ids)

    def rhs(self, ids):
        return self.b[np.asarray(ids, dtype=np.int64)]


def dense_source(A: np.ndarray, b: np.ndarray) -> RowSource:
    A = np.asarray(A, dtype=np.float64)
    return RowSource(lambda ids: sp.csr_matrix(A[np.asarray(ids, dtype=np.int64)]), b, A.shape[1])


def tomo_source(g: joseph.Geometry, b: np.ndarray) -> RowSource:
    cache = {}

    def rows_fn(ids):
        ids = np.asarray(ids, dtype=np.int64)
        key = ids.tobytes()
        if key not in cache:
            if len(cache) > 4096:
                cache.clear()
            cache[key] = joseph.rows(g, ids)
        return cache[key]

    return RowSource(rows_fn, b, g.n)


def run(source: RowSource, blocks: Iterable, r: int, lam: float, x0=None, eta: float = 1.0,
        ramp: bool = False, form: str = "woodbury", callback=None):
    """Run slimLS over the given sequence of blocks (each an array of row ids).

    Yields (k, x_k, r_k) for k = 1, 2, ...  The memory S_k keeps the last r+1
    blocks, oldest first.
    """
    x = np.zeros(source.n) if x0 is None else np.array(x0, dtype=np.float64)
    mem = collections.deque(maxlen=r + 1)
    step = step_woodbury if form == "woodbury" else step_direct
    for k, ids in enumerate(blocks, start=1):
        mem.append(source.rows(ids))
        lam_k = damping(lam, k, r, ramp)
        out = step(x, list(mem), source.rhs(ids), lam_k, eta)
        x, r_k = out[0], out[1]
        yield k, x, r_k


# --------------------------------------------------------------------------
# Block schedules (the sampling of W_k, Sec. 1)
# --------------------------------------------------------------------------
def view_block_ids(g: joseph.Geometry, seed: int, k: int, cyclic: bool = False) -> np.ndarray:
    """Row ids of the block drawn at step k: one view, uniform with replacement
    (Sec. 1), or the view of step k in the random cyclic order (Sec. 4.3)."""
    view = (rng.cyclic_block(seed, k, g.n_views) if cyclic
            else rng.view_block(seed, k, g.n_views))
    return g.view_rays(view)


def view_schedule(g: joseph.Geometry, seed: int, steps: int, k0: int = 1, cyclic: bool = False):
    for k in range(k0, k0 + steps):
        yield view_block_ids(g, seed, k, cyclic)


def random_ray_schedule(seed: int, ell: int, n_avail: int, steps: int, k0: int = 1,
                        distinct: bool = False):
    """Random-ray blocks: ell ids drawn independently, or ell distinct ids (Floyd)."""
    draw = rng.distinct_rays if distinct else rng.random_rays
    for k in range(k0, k0 + steps):
        yield np.array(draw(seed, k, ell, n_avail), dtype=np.int64)


def streaming_ray_schedule(seed: int, ell: int, n_views: int, rays_per_view: int,
                           steps_per_view: int, steps: int, k0: int = 1, distinct: bool = False):
    """Streaming data (Sec. 4.3, 3D streaming): views arrive in angle order, view v
    from step steps_per_view * v + 1 on; step k draws ell rays uniformly from the
    views that have arrived (independently, or ell distinct ones by Floyd)."""
    draw = rng.distinct_rays if distinct else rng.random_rays
    for k in range(k0, k0 + steps):
        arrived = min(n_views, (k - 1) // steps_per_view + 1)
        yield np.array(draw(seed, k, ell, arrived * rays_per_view), dtype=np.int64)


def contiguous_block_ids(i: int, ell: int) -> np.ndarray:
    """Sec. 4.1's selectors W^(i): rows ell*i .. ell*i + ell - 1 (0-based i)."""
    return np.arange(ell * i, ell * (i + 1))
