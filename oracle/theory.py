"""Sec. 3 quantities for slimLS with r = 0, C_k = I and a fixed alpha (oracle side).

For M equally likely row blocks A_i = W^(i)T A (Sec. 1, beta = 1/M):

  B_i(alpha) = alpha (I + alpha A_i^T A_i)^{-1}
  Q          = E B_k/alpha = (1/M) sum_i (I + alpha A_i^T A_i)^{-1}     (rate matrix)
  B          = I - Q = E B_k A_k^T A_k
  x_hat      = B^{-1} E B_k A_k^T b_k                                    (Eq. xhat)

Theorem 3.1 (i): E x_k - x_hat = Q^k (x_0 - x_hat), so ||E x_k - x_hat|| <= rho^k ||x_0 - x_hat||
with rho = ||Q||_2 < 1.  (ii): E||x_k - x_hat||^2 <= (1-2c)^k ||x_0 - x_hat||^2 + alpha^2 sigma^2 / c,
c = lambda_min(B)/(1 + alpha A_max).

Readings where the text is ambiguous:
  * A_min, A_max: min / max over the M blocks of the eigenvalues of A_i^T A_i; A_min
    is taken over the *positive* eigenvalues (with ell < n every block is singular,
    so "lambda_min > 0" can only mean the smallest nonzero eigenvalue).
  * sigma^2 := E||A_k^T (A_k x_hat - b_k)||^2 (the proof of Thm 3.1(ii) uses the
    squared norm; the statement writes sigma = E||.||).
  * Lemma 3.2's constant C writes E||A_k^T W_k||, whose factors do not conform;
    read as E||A_k^T W_k^T||_2 = E||A_k||_2 for row selectors.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class R0Theory:
    def __init__(self, A: np.ndarray, b: np.ndarray, ell: int, alpha: float):
        A = np.asarray(A, dtype=np.float64)
        self.A, self.b, self.ell, self.alpha = A, np.asarray(b, dtype=np.float64), ell, alpha
        m, n = A.shape
        if m % ell:
            raise ValueError("m must be a multiple of ell")
        self.M = m // ell
        self.n = n
        I = np.eye(n)
        self.blocks = [A[i * ell:(i + 1) * ell] for i in range(self.M)]
        self.bblocks = [self.b[i * ell:(i + 1) * ell] for i in range(self.M)]
        self.inv = [sla.inv(I + alpha * Ai.T @ Ai) for Ai in self.blocks]   # B_i / alpha
        self.Q = sum(self.inv) / self.M
        self.Bmat = I - self.Q
        rhs = sum(alpha * Ji @ (Ai.T @ bi) for Ji, Ai, bi in zip(self.inv, self.blocks, self.bblocks)) / self.M
        self.x_hat = sla.solve(self.Bmat, rhs)
        eig = [np.linalg.eigvalsh(Ai.T @ Ai) for Ai in self.blocks]
        tol = 1e-10 * max(float(e.max()) for e in eig)
        self.A_max = max(float(e.max()) for e in eig)
        self.A_min = min(float(e[e > tol].min()) for e in eig)

    @property
    def rho(self) -> float:
        return float(np.linalg.norm(self.Q, 2))

    def mean_iterate(self, x0: np.ndarray, k: int) -> np.ndarray:
        """E x_k by Theorem 3.1(i): x_hat + Q^k (x0 - x_hat)."""
        return self.x_hat + np.linalg.matrix_power(self.Q, k) @ (x0 - self.x_hat)

    def step_matrix_norms(self) -> float:
        """max_i ||B_i A_i^T A_i||_2 (Lemma B.1(iii) bounds it by alpha A_max/(1+alpha A_max))."""
        return max(float(np.linalg.norm(self.alpha * Ji @ (Ai.T @ Ai), 2))
                   for Ji, Ai in zip(self.inv, self.blocks))

    def sigma2(self) -> float:
        return float(np.mean([np.linalg.norm(Ai.T @ (Ai @ self.x_hat - bi)) ** 2
                              for Ai, bi in zip(self.blocks, self.bblocks)]))

    def c_const(self) -> float:
        lmin = float(np.linalg.eigvalsh(self.Bmat).min())
        return lmin / (1.0 + self.alpha * self.A_max)

    def horizon_bound(self, x0: np.ndarray, k: int) -> float:
        """Right side of Eq. (horizon)."""
        c = self.c_const()
        return (1 - 2 * c) ** k * float(np.linalg.norm(x0 - self.x_hat)) ** 2 \
            + self.alpha ** 2 * self.sigma2() / c

    def bias_bound(self) -> float:
        """Lemma 3.2's bound on ||x_hat - x_LS||."""
        A, a, M = self.A, self.alpha, self.M
        AtA_inv = sla.inv(A.T @ A)
        Ak_norm = np.mean([np.linalg.norm(Ai, 2) for Ai in self.blocks])
        AtAk_norm = np.mean([np.linalg.norm(Ai.T @ Ai, 2) for Ai in self.blocks])
        C = Ak_norm + np.linalg.norm(AtA_inv, 2) * np.linalg.norm(A, 2) * AtAk_norm
        Q_A_b = self.b - A @ (AtA_inv @ (A.T @ self.b))
        fac = a * M * (1 + a * self.A_min) * self.A_max / ((1 + a * self.A_max) * self.A_min)
        return float(fac * C * np.linalg.norm(Q_A_b))
