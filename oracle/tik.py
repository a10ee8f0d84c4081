"""One slimTik iteration, float64 (the oracle of the Tikhonov form of slimLS).

Test infrastructure only: nothing on the product path imports this module.

Sec. 2 applies slimLS to the Tikhonov problem, Eq. (TLS1),

    x_tik = argmin_x ||A x - b||^2 + lam_tik^2 ||L x||^2,   L invertible,

by sampling the stacked rows [W_k^T A; M^{-1/2} lam_tik L] (the selector
W~_k), with C_k = L^T L in Eq. (B_k).  The iterate is Eq. (slimTik):

    x_k = x_{k-1} - (mu_k L^T L + M_k^T M_k)^{-1}
                    (A_k^T (A_k x_{k-1} - b_k) + beta L^T L x_{k-1}),
    beta = lam_tik^2 / M,   mu_k = alpha_k^{-1} + c_k beta,

M the number of blocks of the partition and alpha_k^{-1} = lambda_k the
damping of slimLS (constant or the ramp of Sec. 4.2).  c_k counts the blocks
whose Tikhonov rows the stacked M~_k holds.  The paper prints c_k = r.  slimLS
on the stacked problem, which is what Eq. (slimTik) is said to equal, gives
c_k = the number of blocks in M_k, min(k, r+1) (M_k = [A_{k-r}; ...; A_k], with
blocks of index < 1 empty): only that count makes the full-memory iterates
telescope to the Tikhonov solution.  Both readings are offered
(`reading="window"`, the default, or `"printed"`).

Two forms of the step s_k (x_k = x_{k-1} - eta s_k):

  direct     the n x n system above as written, any invertible L (small n);
  Woodbury   L = diag(l), P = L^T L, W = P^{-1} = diag(1/l^2) (step_woodbury;
             step_woodbury_general takes any invertible L, with W dense):
                 (mu_k I_p + M_k W M_k^T) z = c - (beta/mu_k) M_k x_{k-1},
                 s_k = (beta/mu_k) x_{k-1} + W M_k^T z,
             c = [0; ...; 0; r_k] (r_k = A_k x_{k-1} - b_k in the rows of the
             newest block).  Check: (mu P + M^T M) s = beta P x + M^T[(beta/mu) M x
             + (mu I + M W M^T) z] = beta P x + M^T c, the right-hand side of
             Eq. (slimTik), since A_k^T r_k = M_k^T c.
"""
from __future__ import annotations

import collections

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .slim import damping


def window_count(k: int, r: int, reading: str = "window") -> int:
    """c_k: blocks of M_k (min(k, r+1)), or r as printed in Eq. (slimTik)."""
    if reading == "window":
        return min(k, r + 1)
    if reading == "printed":
        return r
    raise ValueError(reading)


def shift(lam_k: float, lam_tik: float, n_blocks: int, count: int) -> float:
    """mu_k = alpha_k^{-1} + c_k lam_tik^2 / M."""
    return lam_k + count * lam_tik * lam_tik / n_blocks


def _stack(blocks):
    M = sp.vstack([B if sp.issparse(B) else sp.csr_matrix(np.asarray(B)) for B in blocks],
                  format="csr")
    A_k = blocks[-1] if sp.issparse(blocks[-1]) else sp.csr_matrix(np.asarray(blocks[-1]))
    return M, sp.csr_matrix(A_k)


def gradient(A_k, r_k, P, x_prev, beta):
    """Right-hand side of Eq. (slimTik): A_k^T r_k + beta L^T L x_{k-1}."""
    return A_k.T @ r_k + beta * (P @ x_prev)


def step_direct(x_prev, blocks, b_new, lam_k: float, lam_tik: float, n_blocks: int, count: int,
                L, eta: float = 1.0):
    """Eq. (slimTik) as written: dense n x n Cholesky of mu_k L^T L + M_k^T M_k.

    blocks: the row blocks of M_k, oldest first, the last one A_k; L: n x n
    (dense or sparse), invertible.  Returns (x_k, r_k, s_k)."""
    M, A_k = _stack(blocks)
    L = L.toarray() if sp.issparse(L) else np.asarray(L, dtype=np.float64)
    P = L.T @ L
    beta = lam_tik * lam_tik / n_blocks
    mu = shift(lam_k, lam_tik, n_blocks, count)
    r_k = A_k @ x_prev - b_new
    H = mu * P + (M.T @ M).toarray()
    s = sla.cho_solve(sla.cho_factor(H, lower=True), gradient(A_k, r_k, P, x_prev, beta))
    return x_prev - eta * s, r_k, s


def step_woodbury(x_prev, blocks, b_new, lam_k: float, lam_tik: float, n_blocks: int, count: int,
                  l=None, eta: float = 1.0):
    """The step in Woodbury form for L = diag(l) (l = None: L = I).

    Returns (x_k, r_k, s_k, z): z solves the p x p system in the order of
    `blocks`."""
    M, A_k = _stack(blocks)
    n = M.shape[1]
    Wd = np.ones(n) if l is None else 1.0 / np.square(np.asarray(l, dtype=np.float64))
    beta = lam_tik * lam_tik / n_blocks
    mu = shift(lam_k, lam_tik, n_blocks, count)
    ell, p = A_k.shape[0], M.shape[0]
    r_k = A_k @ x_prev - b_new
    c = np.zeros(p)
    c[p - ell:] = r_k
    MW = M @ sp.diags(Wd)
    K = mu * np.eye(p) + (MW @ M.T).toarray()
    z = sla.cho_solve(sla.cho_factor(K, lower=True), c - (beta / mu) * (M @ x_prev))
    s = (beta / mu) * x_prev + MW.T @ z
    return x_prev - eta * s, r_k, s, z


def bidiagonal(d0, d1) -> sp.csr_matrix:
    """L with (L x)_i = d0_i x_i + d1_i x_{i-1} (d1_0 unused): lower bidiagonal."""
    d0 = np.asarray(d0, dtype=np.float64)
    d1 = np.asarray(d1, dtype=np.float64)
    return sp.diags([d0, d1[1:]], [0, -1], format="csr")


def step_woodbury_general(x_prev, blocks, b_new, lam_k: float, lam_tik: float, n_blocks: int,
                          count: int, L, eta: float = 1.0):
    """The Woodbury form with any invertible L, W = (L^T L)^{-1} formed densely
    (small n): (mu I + M W M^T) z = c - (beta/mu) M x, s = (beta/mu) x + W M^T z.
    Returns (x_k, r_k, s_k, z)."""
    M, A_k = _stack(blocks)
    L = L.toarray() if sp.issparse(L) else np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    W = sla.cho_solve(sla.cho_factor(L.T @ L, lower=True), np.eye(n))
    beta = lam_tik * lam_tik / n_blocks
    mu = shift(lam_k, lam_tik, n_blocks, count)
    ell, p = A_k.shape[0], M.shape[0]
    r_k = A_k @ x_prev - b_new
    c = np.zeros(p)
    c[p - ell:] = r_k
    Md = M.toarray()
    K = mu * np.eye(p) + Md @ W @ Md.T
    z = sla.cho_solve(sla.cho_factor(K, lower=True), c - (beta / mu) * (Md @ x_prev))
    s = (beta / mu) * x_prev + W @ (Md.T @ z)
    return x_prev - eta * s, r_k, s, z


def run(source, blocks, r: int, lam: float, lam_tik: float, n_blocks: int, l=None, x0=None,
        eta: float = 1.0, ramp: bool = False, reading: str = "window", form: str = "woodbury",
        L=None):
    """slimTik over the given sequence of blocks (arrays of row ids of
    `source`, a slim.RowSource).  form "woodbury" takes L = diag(l); form
    "direct" takes L (n x n, default diag(l) or I).  Yields (k, x_k, r_k)."""
    n = source.n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if form == "direct" and L is None:
        L = np.diag(np.ones(n) if l is None else np.asarray(l, dtype=np.float64))
    mem = collections.deque(maxlen=r + 1)
    for k, ids in enumerate(blocks, start=1):
        mem.append(source.rows(ids))
        lam_k = damping(lam, k, r, ramp)
        cnt = window_count(k, r, reading)
        if form == "woodbury":
            out = step_woodbury(x, list(mem), source.rhs(ids), lam_k, lam_tik, n_blocks, cnt, l,
                                eta)
        else:
            out = step_direct(x, list(mem), source.rhs(ids), lam_k, lam_tik, n_blocks, cnt, L, eta)
        x, r_k = out[0], out[1]
        yield k, x, r_k
