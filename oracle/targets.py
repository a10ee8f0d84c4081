"""Reference solutions the iterates are measured against (oracle side).

x_LS   = argmin ||A x - b||_2^2 = (A^T A)^{-1} A^T b               (Eq. LS)
x_tik  = argmin ||A x - b||_2^2 + lam ||x||_2^2 = (A^T A + lam I)^{-1} A^T b

(x_tik uses the damping lam of the iteration with C_k = I: with memory holding
every block drawn so far, slimLS lands on it exactly after one pass over all
blocks; see Appendix A for the lam -> 0 statement.)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def x_ls_qr(A, b):
    """x_LS by Householder QR of a dense A (LAPACK geqrf)."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    Q, R = sla.qr(A, mode="economic")
    return sla.solve_triangular(R, Q.T @ b)


def x_ls_normal(A, b):
    """x_LS from the normal equations, for cross-checking x_ls_qr."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    return sla.solve(A.T @ A, A.T @ b, assume_a="pos")


def x_tik_dense(A, b, lam: float):
    """(A^T A + lam I)^{-1} A^T b by a dense Cholesky of the n x n normal matrix."""
    AtA = (A.T @ A).toarray() if sp.issparse(A) else np.asarray(A).T @ np.asarray(A)
    n = AtA.shape[0]
    return sla.cho_solve(sla.cho_factor(AtA + lam * np.eye(n), lower=True), A.T @ b)


def cgls(A, b, lam: float, tol: float = 1e-13, maxit: int = 100000, x0=None):
    """CGLS for min ||A x - b||^2 + lam ||x||^2 (Hestenes-Stiefel on the normal
    equations, Bjorck's formulation).  Stops when ||A^T(b - Ax) - lam x|| <= tol * ||A^T b||.
    Returns (x, iterations, relative normal-equation residual)."""
    n = A.shape[1]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    s = A.T @ r - lam * x
    p = s.copy()
    gamma = float(s @ s)
    norm0 = float(np.linalg.norm(A.T @ b))
    if norm0 == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit and np.sqrt(gamma) > tol * norm0:
        q = A @ p
        delta = float(q @ q) + lam * float(p @ p)
        alpha = gamma / delta
        x += alpha * p
        r -= alpha * q
        s = A.T @ r - lam * x
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        it += 1
    return x, it, np.sqrt(gamma) / norm0
