"""LSQR for the damped least-squares problem of one slimLS step, float64.

Test infrastructure only: the oracle of the matrix-free inner solver.

Sec. 4.2 writes the step as x_k = x_{k-1} - s_k with s_k the solution of the
stacked damped least-squares problem, Eq. (slimLSstep),

    s_k = argmin_s || [M_k; alpha_k^{-1/2} L_k] s - [0; ...; 0; r_k; 0] ||,

and solves it with LSQR for damped least squares (the paper's reference
[PaSa82b]; L_k = I here, so the damping is d = sqrt(lambda_k)).  This module
states that method from its mathematics:

Golub-Kahan bidiagonalisation of M started from the right-hand side c:
    beta_1 u_1 = c,                    alpha_1 v_1 = M^T u_1,
    beta_{i+1} u_{i+1} = M v_i - alpha_i u_i,
    alpha_{i+1} v_{i+1} = M^T u_{i+1} - beta_{i+1} v_i,
so that M V_i = U_{i+1} B_i with B_i lower bidiagonal (alphas on the diagonal,
betas below).  The iterate s_i = V_i y_i minimises
|| [B_i; d I] y - beta_1 e_1 || over y, i.e. the damped residual over the
Krylov space K_i(M^T M, M^T c).  Each step updates the QR factorisation of
[B_i; d I] with two plane rotations: one folds the damping row into the
diagonal (rho_bar -> hypot(rho_bar, d)), the next removes beta_{i+1}; the
iterate and the search direction w follow by recurrence.

The residual of the normal equations, || M^T(c - M s) - d^2 s ||, is available
from the scalars as |phi_bar_{i+1} c_i| alpha_{i+1}; the stopping rule used
here is that quantity falling to `tol` times its value at s = 0,
alpha_1 beta_1 = ||M^T c|| (tol = 0: exactly `max_iter` iterations).
"""
from __future__ import annotations

import math
from typing import Callable, NamedTuple

import numpy as np


class LsqrResult(NamedTuple):
    s: np.ndarray          # the iterate after `iters` steps
    iters: int             # iterations taken
    normal_res: float      # |phi_bar c| alpha of the last iteration (estimate of ||M^T r - d^2 s||)
    normal_res0: float     # alpha_1 beta_1 = ||M^T c||


def rotation(a: float, b: float):
    """Plane rotation [c s; -s c] with c a + s b = r >= 0 and -s a + c b = 0."""
    r = math.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def lsqr_damped(matvec: Callable, rmatvec: Callable, c: np.ndarray, n: int, damp: float,
                max_iter: int, tol: float = 0.0, trace: list | None = None) -> LsqrResult:
    """Minimise ||M s - c||^2 + damp^2 ||s||^2 with matvec(v) = M v (length of c)
    and rmatvec(u) = M^T u (length n).  `trace`, if given, receives s after each
    iteration."""
    c = np.asarray(c, dtype=np.float64)
    s = np.zeros(n)
    beta = float(np.linalg.norm(c))
    if beta == 0.0:
        return LsqrResult(s, 0, 0.0, 0.0)
    u = c / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LsqrResult(s, 0, 0.0, 0.0)
    v = v / alpha
    w = v.copy()
    rho_bar, phi_bar = alpha, beta
    res0 = alpha * beta
    res = res0
    it = 0
    while it < max_iter:
        it += 1
        # next bidiagonalisation step
        u = matvec(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        v = rmatvec(u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        # fold the damping row into the diagonal
        c1, s1, rho_hat = rotation(rho_bar, damp)
        phi_hat = c1 * phi_bar
        # remove the subdiagonal beta_{i+1}
        cr, sr, rho = rotation(rho_hat, beta)
        theta = sr * alpha
        rho_bar = -cr * alpha
        phi = cr * phi_hat
        phi_bar = sr * phi_hat
        # iterate and search direction
        s = s + (phi / rho) * w
        w = v - (theta / rho) * w
        if trace is not None:
            trace.append(s.copy())
        res = abs(phi_bar * cr) * alpha
        if tol > 0.0 and res <= tol * res0:
            break
    return LsqrResult(s, it, res, res0)


def step_lsqr(x_prev, blocks, b_new, lam_k: float, max_iter: int, tol: float = 0.0,
              eta: float = 1.0):
    """One slimLS step with s_k from LSQR on Eq. (slimLSstep), C_k = I.

    blocks: the row blocks of M_k, oldest first, the last one A_k (as for
    slim.step_woodbury).  Returns (x_k, r_k, LsqrResult)."""
    import scipy.sparse as sp
    M = sp.vstack([sp.csr_matrix(B) for B in blocks], format="csr")
    A_k = sp.csr_matrix(blocks[-1])
    ell, p = A_k.shape[0], M.shape[0]
    r_k = A_k @ x_prev - b_new
    c = np.zeros(p)
    c[p - ell:] = r_k
    res = lsqr_damped(lambda v: M @ v, lambda u: M.T @ u, c, M.shape[1], math.sqrt(lam_k),
                      max_iter, tol)
    return x_prev - eta * res.s, r_k, res


def step_tik_lsqr(x_prev, blocks, b_new, lam_k: float, lam_tik: float, n_blocks: int, count: int,
                  cdiag=None, max_iter: int = 1000, tol: float = 0.0, eta: float = 1.0):
    """One slimTik step (Eq. slimTik, C_k = diag(c), c = None: I) by LSQR.

    With W = C^{-1}, beta = lam_tik^2 / M and mu = lambda_k + count beta, the
    step s solves (mu C + M^T M) s = M^T c0 + beta C x (c0 = [0; ...; r_k]),
    i.e. s = (beta/mu) x + W^{1/2} y with
        y = argmin || M W^{1/2} y - (c0 - (beta/mu) M x) ||^2 + mu ||y||^2
    (substitute s = (beta/mu) x + W^{1/2} y in the normal equations), which is
    LSQR for damped least squares on the column-scaled window, damping
    sqrt(mu).  Returns (x_k, r_k, LsqrResult of y)."""
    import scipy.sparse as sp
    M = sp.vstack([sp.csr_matrix(B) for B in blocks], format="csr")
    A_k = sp.csr_matrix(blocks[-1])
    ell, p, n = A_k.shape[0], M.shape[0], M.shape[1]
    wh = np.ones(n) if cdiag is None else 1.0 / np.sqrt(np.asarray(cdiag, dtype=np.float64))
    beta = lam_tik * lam_tik / n_blocks
    mu = lam_k + count * beta
    r_k = A_k @ x_prev - b_new
    c = np.zeros(p)
    c[p - ell:] = r_k
    c = c - (beta / mu) * (M @ x_prev)
    MW = M @ sp.diags(wh)
    res = lsqr_damped(lambda v: MW @ v, lambda u: MW.T @ u, c, n, math.sqrt(mu), max_iter, tol)
    s = (beta / mu) * x_prev + wh * res.s
    return x_prev - eta * s, r_k, res
