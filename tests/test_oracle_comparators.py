"""Pins for the comparators (sg, olbfgs) and the damping schedules.

* The two-loop recursion equals the explicit BFGS inverse updates
  H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T from gamma I, applied to
  the pairs in order; that H is symmetric positive definite and satisfies the
  secant condition H y = s for the newest pair.
* olbfgs with memory 0 is sg.
* sg averaged over all M blocks is one full-gradient step:
  (1/M) sum_i sg_i(x) = x - (alpha/M) A^T (A x - b).
* sg on a single row with alpha = 1/||a||^2 is the Kaczmarz projection,
  Eq. (Kacz): a x_k = b exactly.
* slimLS with r = 0, damping lambda and eta = lambda alpha tends to sg with
  step alpha as lambda grows, with an O(1/lambda) gap (Eq. dbK).
* Each olbfgs step is x - alpha H g with H the explicit BFGS inverse of the
  pairs stored before it, and it stores (x_k - x_{k-1}, A_k^T A_k s).
* The decaying schedule: its values, and on the Gaussian workload of Sec. 4.1
  it gets below the constant-damping horizon of Theorem 3.1(ii).
Mutations planted in the oracle (here, on the CPU) break these pins.
"""
import numpy as np
import pytest

import workloads
from oracle import comparators as cmp, slim, targets


def _pairs(n=12, count=5, seed=0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    H = B @ B.T + n * np.eye(n)           # SPD: every pair has s^T y > 0
    out = []
    for _ in range(count):
        s = rng.standard_normal(n)
        y = H @ s
        out.append((s, y, 1.0 / (s @ y)))
    return out


def _explicit_inverse(pairs, gamma, n):
    H = gamma * np.eye(n)
    for s, y, rho in pairs:
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def test_two_loop_equals_explicit_bfgs_updates():
    n = 12
    pairs = _pairs(n)
    gamma = cmp.initial_scaling(pairs)
    H = _explicit_inverse(pairs, gamma, n)
    g = np.random.default_rng(5).standard_normal(n)
    assert np.linalg.norm(cmp.two_loop(g, pairs, gamma) - H @ g) <= 1e-12 * np.linalg.norm(H @ g)
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0
    s, y, _ = pairs[-1]
    assert np.linalg.norm(cmp.two_loop(y, pairs, gamma) - s) <= 1e-12 * np.linalg.norm(s)
    # gamma is the mean of s^T y / y^T y
    assert gamma == pytest.approx(np.mean([(s @ y) / (y @ y) for s, y, _ in pairs]), rel=1e-15)


def test_olbfgs_without_memory_is_sg():
    A, _, b = workloads.gaussian_problem(4, m=200, n=30)
    src = slim.dense_source(A, b)
    sched = [slim.contiguous_block_ids(i, 10) for i in (3, 7, 3, 19, 0)]
    a = [x for _, x, _ in cmp.run(src, sched, 50.0, "olbfgs", memory=0)]
    c = [x for _, x, _ in cmp.run(src, sched, 50.0, "sg")]
    for xa, xc in zip(a, c):
        assert np.array_equal(xa, xc)


def test_sg_averaged_over_blocks_is_a_gradient_step():
    A, _, b = workloads.gaussian_problem(6, m=100, n=20)
    M, ell, alpha = 10, 10, 0.01
    x = np.random.default_rng(1).standard_normal(20)
    mean = np.mean([cmp.step_sg(x, A[i * ell:(i + 1) * ell], b[i * ell:(i + 1) * ell], alpha)[0]
                    for i in range(M)], axis=0)
    want = x - alpha / M * (A.T @ (A @ x - b))
    assert np.linalg.norm(mean - want) <= 1e-13 * np.linalg.norm(want)


def test_sg_single_row_is_the_kaczmarz_projection():
    A, _, b = workloads.gaussian_problem(7, m=30, n=8)
    x = np.zeros(8)
    for i in (4, 11, 4, 29):
        a = A[i:i + 1]
        x, _ = cmp.step_sg(x, a, b[i:i + 1], 1.0 / float((a @ a.T)[0, 0]))
        assert abs(float((a @ x)[0]) - b[i]) <= 1e-12 * max(1.0, abs(b[i]))


def test_slimls_with_large_damping_tends_to_sg():
    A, _, b = workloads.gaussian_problem(8, m=100, n=15)
    Ak, bk = A[20:30], b[20:30]
    x = np.random.default_rng(2).standard_normal(15)
    alpha = 1e-3
    want, _ = cmp.step_sg(x, Ak, bk, alpha)
    gaps = []
    for lam in (1e4, 1e5, 1e6):
        got, *_ = slim.step_woodbury(x, [Ak], bk, lam, eta=lam * alpha)
        gaps.append(np.linalg.norm(got - want) / np.linalg.norm(want - x))
    assert gaps[0] < 1e-2 and gaps[1] < gaps[0] / 8 and gaps[2] < gaps[1] / 8


def test_olbfgs_steps_against_dense_matrices():
    # each step is x - alpha H g with H the explicit BFGS inverse of the pairs
    # stored before it, and the stored pair is (x_k - x_{k-1}, A_k^T A_k s)
    A, _, b = workloads.gaussian_problem(9, m=120, n=16)
    rng = np.random.default_rng(4)
    opt = cmp.Olbfgs(memory=3)
    x = np.zeros(16)
    for k in range(1, 9):
        i = int(rng.integers(0, 12))
        Ak, bk = A[10 * i:10 * i + 10], b[10 * i:10 * i + 10]
        alpha = 0.02
        pairs = list(opt.pairs)
        gamma = float(np.mean([(p @ q) / (q @ q) for p, q, _ in pairs])) if pairs else 1.0
        H = _explicit_inverse(pairs, gamma, 16)
        want = x - alpha * H @ (Ak.T @ (Ak @ x - bk))
        x_new, _ = opt.step(x, Ak, bk, alpha)
        assert np.linalg.norm(x_new - want) <= 1e-12 * np.linalg.norm(want), k
        s_, y_, rho_ = opt.pairs[-1]
        assert np.array_equal(s_, x_new - x) or np.allclose(s_, x_new - x, rtol=0, atol=1e-15)
        assert np.linalg.norm(y_ - Ak.T @ (Ak @ s_)) <= 1e-13 * np.linalg.norm(y_)
        assert len(opt.pairs) == min(k, 3)
        x = x_new


def test_decaying_schedule_values():
    assert cmp.damping(0.5, 3, decay_after=10) == 0.5
    assert cmp.damping(0.5, 10, decay_after=10) == 0.5
    assert cmp.damping(0.5, 25, decay_after=10) == 0.5 * 25 / 10
    assert cmp.damping(0.5, 2, r=3, ramp=True, decay_after=10) == 0.5 * 4 / 2
    assert cmp.damping(0.5, 40, r=3, ramp=True, decay_after=0) == 0.5


def test_decaying_damping_passes_the_constant_horizon():
    # Sec. 4.1's Gaussian workload (A 1000 x 100, 1% noise, 100 blocks of 10
    # rows), r = 0, alpha = 0.01: after 30 epochs constant damping sits at its
    # horizon (5.5e-3 from x_LS), the 1/k decay after one epoch keeps going
    # toward x_LS (1.5e-3)
    A, _, b = workloads.gaussian_problem(11)
    src = slim.dense_source(A, b)
    x_ls = targets.x_ls_qr(A, b)
    rng = np.random.default_rng(3)
    sched = [slim.contiguous_block_ids(int(i), 10) for i in rng.integers(0, 100, 3000)]

    def err(decay_after):
        x = np.zeros(100)
        for k, ids in enumerate(sched, start=1):
            lam_k = cmp.damping(100.0, k, decay_after=decay_after)
            x, *_ = slim.step_woodbury(x, [src.rows(ids)], src.rhs(ids), lam_k)
        return np.linalg.norm(x - x_ls) / np.linalg.norm(x_ls)

    const, decay = err(0), err(100)
    assert decay < 0.4 * const, (const, decay)


def test_planted_mutations_break_the_pins(monkeypatch):
    n = 12
    pairs = _pairs(n)
    gamma = cmp.initial_scaling(pairs)
    H = _explicit_inverse(pairs, gamma, n)
    g = np.random.default_rng(5).standard_normal(n)

    def gap():
        return np.linalg.norm(cmp.two_loop(g, pairs, gamma) - H @ g) / np.linalg.norm(H @ g)

    assert gap() < 1e-12
    real = cmp.two_loop

    def second_loop_reversed(g_, pairs_, gamma_):
        q = np.array(g_, dtype=np.float64)
        a = []
        for s, y, rho in reversed(pairs_):
            ai = rho * (s @ q)
            q = q - ai * y
            a.append(ai)
        q = gamma_ * q
        for (s, y, rho), ai in zip(reversed(pairs_), a):     # wrong order
            q = q + (ai - rho * (y @ q)) * s
        return q

    monkeypatch.setattr(cmp, "two_loop", second_loop_reversed)
    assert gap() > 1e-3
    monkeypatch.setattr(cmp, "two_loop", real)
    # the averaged scaling replaced by 1
    monkeypatch.setattr(cmp, "initial_scaling", lambda p: 1.0)
    gamma = cmp.initial_scaling(pairs)
    assert gap() > 1e-3
