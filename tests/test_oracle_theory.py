"""Pins from Sec. 3 (Theorem 3.1, Lemma 3.2, Lemma B.1) and the Sec. 4.1 observations,
on the paper's illustrative workload: A 1000 x 100 standard normal, x_true = 1,
1% noise, M = 100 contiguous blocks of ell = 10 rows, r = 0 (Sec. 4.1)."""
import numpy as np
import pytest

import workloads
from oracle import slim, targets, theory

ELL = 10


@pytest.fixture(scope="module")
def problem():
    A, x_true, b = workloads.gaussian_problem(5)
    return A, x_true, b


def _uniform_blocks(rs, steps, M=100):
    return [slim.contiguous_block_ids(int(i), ELL) for i in rs.integers(0, M, size=steps)]


def test_lemma_b1_bounds(problem):
    A, _, b = problem
    for alpha in (1e-3, 1e-1, 1.0, 10.0):
        T = theory.R0Theory(A, b, ELL, alpha)
        ev = np.linalg.eigvalsh(T.Bmat)
        assert T.rho < 1.0                                                        # (i)
        assert ev.min() > 0                                                       # (ii)
        assert T.step_matrix_norms() <= alpha * T.A_max / (1 + alpha * T.A_max) * (1 + 1e-12)  # (iii)
        assert ev.max() <= alpha * T.A_max / (1 + alpha * T.A_max) * (1 + 1e-12)  # (iv) upper
        assert ev.min() >= alpha * T.A_min / (T.M * (1 + alpha * T.A_min))       # (iv) lower


def test_theorem_31_i_mean_iterate(problem):
    # E x_k - x_hat = Q^k (x_0 - x_hat): Monte Carlo mean vs the recursion
    A, _, b = problem
    alpha, k, R = 1.0, 4, 600
    T = theory.R0Theory(A, b, ELL, alpha)
    src = slim.dense_source(A, b)
    rs = np.random.default_rng(0)
    x0 = np.zeros(100)
    finals = []
    for _ in range(R):
        for kk, x, _ in slim.run(src, _uniform_blocks(rs, k), r=0, lam=1.0 / alpha, x0=x0):
            pass
        finals.append(x)
    finals = np.array(finals)
    mean, sd = finals.mean(axis=0), finals.std(axis=0, ddof=1)
    want = T.mean_iterate(x0, k)
    z = np.abs(mean - want) / (sd / np.sqrt(R))
    assert np.max(z) < 4.5
    # and it is the recursion, not x_hat itself, that the mean follows at small k
    assert np.linalg.norm(want - T.x_hat) > 5 * np.linalg.norm(mean - want)
    assert np.linalg.norm(want - T.x_hat) <= T.rho ** k * np.linalg.norm(x0 - T.x_hat) * (1 + 1e-12)


def test_theorem_31_ii_horizon(problem):
    A, _, b = problem
    alpha, R, K = 0.01, 200, 30
    T = theory.R0Theory(A, b, ELL, alpha)
    src = slim.dense_source(A, b)
    rs = np.random.default_rng(1)
    err2 = np.zeros(K)
    for _ in range(R):
        for k, x, _ in slim.run(src, _uniform_blocks(rs, K), r=0, lam=1.0 / alpha):
            err2[k - 1] += np.linalg.norm(x - T.x_hat) ** 2 / R
    bound = np.array([T.horizon_bound(np.zeros(100), k) for k in range(1, K + 1)])
    assert np.all(err2 <= bound)


def test_lemma_32_bias_bound_and_order(problem):
    A, _, b = problem
    xls = targets.x_ls_qr(A, b)
    bias = {}
    for alpha in (1e-6, 1e-5, 1e-3, 1e-1, 1.0):
        T = theory.R0Theory(A, b, ELL, alpha)
        bias[alpha] = np.linalg.norm(T.x_hat - xls)
        assert bias[alpha] <= T.bias_bound()
    # x_hat -> x_LS linearly in alpha (the bias of Fig. 3 grows with alpha)
    assert abs(bias[1e-5] / 1e-5 - bias[1e-6] / 1e-6) <= 0.01 * bias[1e-6] / 1e-6
    vals = [bias[a] for a in sorted(bias)]
    assert all(v1 < v2 for v1, v2 in zip(vals, vals[1:]))


def test_consistent_data_fixed_point():
    # b in range(A): Q_A b = 0, so x_hat = x_LS = x_true (Eq. xh-xls)
    A, x_true, _ = workloads.gaussian_problem(6)
    T = theory.R0Theory(A, A @ x_true, ELL, 1.0)
    assert np.allclose(T.x_hat, x_true, rtol=1e-10, atol=1e-10)


def test_memory_speeds_initial_convergence(problem):
    # Sec. 4.1, Fig. 4: alpha = 1, r in {0,2,4,6,8}, 20 iterations, median error vs x_LS
    A, _, b = problem
    xls = targets.x_ls_qr(A, b)
    src = slim.dense_source(A, b)
    med = []
    for r in (0, 2, 4, 6, 8):
        rs = np.random.default_rng(100 + r)
        errs = []
        for _ in range(60):
            for k, x, _ in slim.run(src, _uniform_blocks(rs, 20), r=r, lam=1.0):
                pass
            errs.append(np.linalg.norm(x - xls) / np.linalg.norm(xls))
        med.append(np.median(errs))
    assert all(a > b for a, b in zip(med, med[1:]))
