"""Pins for the oracle's slimLS step, Eq. (ram) with Eq. (B_k), C_k = I.

* Woodbury form == direct n x n form (the identity Sec. 2 cites).
* r = 0 is damped block Kaczmarz, Eq. (dbK) with x_{k-1} in the residual.
* ell = 1, r = 0 has the closed form s = a (a x - b)/(lambda + ||a||^2), and its
  lambda -> 0 limit is randomized Kaczmarz, Eq. (Kacz) with alpha = 1.
* Memory holding every block so far: (lambda I + sum_i A_i^T A_i) x_k =
  lambda x_0 + sum_i A_i^T b_i (induction in the style of Appendix A); with the
  damping ramp of Sec. 4.2 the right side gains sum (lambda_j - lambda_{j-1}) x_{j-1}.
Mutations planted in the oracle (here, on the CPU) must break these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import joseph, slim


def _tiny_tomo(N=16, V=12, D=23, seed=7):
    g = joseph.Geometry(N, V, D)
    x_true = workloads.phantom_2d(N, seed, 4)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, workloads.noise_direction(g.m, seed), 0.01)
    return g, A, b


def test_woodbury_equals_direct_tiny_tomo():
    g, A, b = _tiny_tomo()
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, 3, 12))
    xs_w = [x for _, x, _ in slim.run(src, sched, r=2, lam=1e-2)]
    xs_d = [x for _, x, _ in slim.run(src, sched, r=2, lam=1e-2, form="direct")]
    for xw, xd in zip(xs_w, xs_d):
        assert np.linalg.norm(xw - xd) <= 1e-10 * np.linalg.norm(xd)


def test_woodbury_equals_direct_plain_workload_first_steps():
    cfg = workloads.C1
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, e, cfg.noise)
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, cfg.seed, 5))
    xw = list(slim.run(src, sched, cfg.r, cfg.lam))
    xd = list(slim.run(src, sched, cfg.r, cfg.lam, form="direct"))
    for (_, a, _), (_, c, _) in zip(xw, xd):
        assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(c)


def test_r0_is_damped_block_kaczmarz():
    A, _, b = workloads.gaussian_problem(2, m=200, n=30)
    src = slim.dense_source(A, b)
    lam = 0.3
    sched = [slim.contiguous_block_ids(i, 10) for i in (4, 0, 4, 17, 9)]
    x = np.zeros(30)
    for (k, xk, _), ids in zip(slim.run(src, sched, r=0, lam=lam), sched):
        Ak, bk = A[ids], b[ids]
        x = x - np.linalg.solve(lam * np.eye(30) + Ak.T @ Ak, Ak.T @ (Ak @ x - bk))
        assert np.allclose(xk, x, rtol=1e-12, atol=1e-12)


def test_single_row_closed_form_and_kaczmarz_limit():
    rs = np.random.default_rng(4)
    A = rs.standard_normal((40, 12))
    b = rs.standard_normal(40)
    x = rs.standard_normal(12)
    for i in (0, 17, 39):
        a, bi = A[i], b[i]
        for lam in (1.0, 1e-3):
            xk, _, s, _ = slim.step_woodbury(x, [A[i:i + 1]], b[i:i + 1], lam)
            assert np.allclose(s, a * (a @ x - bi) / (lam + a @ a), rtol=1e-13, atol=1e-15)
        xk, _, _, _ = slim.step_woodbury(x, [A[i:i + 1]], b[i:i + 1], 1e-14)
        kacz = x - (a @ x - bi) / (a @ a) * a
        assert np.allclose(xk, kacz, rtol=1e-10, atol=1e-12)
        assert abs(a @ xk - bi) < 1e-10   # the projection lands on the hyperplane


def _full_memory_check(src, A_rows, b_of, sched, lam, ramp, r):
    n = src.n
    H = np.zeros((n, n))
    rhs = np.zeros(n)
    lam_prev = 0.0
    x_prev = np.zeros(n)
    for (k, xk, _), ids in zip(slim.run(src, sched, r=r, lam=lam, ramp=ramp), sched):
        Ak = A_rows(ids)
        lam_k = slim.damping(lam, k, r, ramp)
        H += Ak.T @ Ak
        rhs += Ak.T @ b_of(ids) + (lam_k - lam_prev) * x_prev
        lhs = lam_k * xk + H @ xk
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs)
        lam_prev, x_prev = lam_k, xk


def test_full_memory_closed_form_gaussian():
    A, _, b = workloads.gaussian_problem(3, m=120, n=25)
    src = slim.dense_source(A, b)
    sched = [slim.contiguous_block_ids(i, 6) for i in (3, 3, 11, 0, 19, 7)]   # repeats allowed
    _full_memory_check(src, lambda ids: A[ids], lambda ids: b[ids], sched, 0.05, False, r=10)


def test_full_memory_closed_form_tomo_with_ramp():
    g, A, b = _tiny_tomo()
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, 11, 5))
    Ad = A.toarray()
    _full_memory_check(src, lambda ids: Ad[ids], lambda ids: b[ids], sched, 1e-2, True, r=6)


def test_ramp_values():
    assert [slim.damping(0.1, k, 3, True) for k in (1, 2, 3, 4, 5)] == \
        pytest.approx([0.4, 0.2, 0.4 / 3, 0.1, 0.1])
    assert slim.damping(0.1, 1, 3, False) == 0.1


def test_eta_scales_the_step():
    g, A, b = _tiny_tomo()
    src = slim.tomo_source(g, b)
    ids = g.view_rays(2)
    x = np.random.default_rng(0).standard_normal(g.n)
    x1, _, s1, _ = slim.step_woodbury(x, [src.rows(ids)], src.rhs(ids), 0.1, eta=1.0)
    x2, _, s2, _ = slim.step_woodbury(x, [src.rows(ids)], src.rhs(ids), 0.1, eta=0.5)
    assert np.allclose(s1, s2) and np.allclose(x - x2, 0.5 * (x - x1))


# --- planted mistakes: the pins above must catch each -----------------------------

def _mutant_rhs_first_block(x_prev, blocks, b_new, lam_k, eta=1.0):
    M = sp.vstack([sp.csr_matrix(B) for B in blocks], format="csr")
    A_k = sp.csr_matrix(blocks[-1])
    ell, p = A_k.shape[0], M.shape[0]
    r_k = A_k @ x_prev - b_new
    K = lam_k * np.eye(p) + (M @ M.T).toarray()
    rhs = np.zeros(p)
    rhs[:ell] = r_k            # wrong block position
    s = M.T @ np.linalg.solve(K, rhs)
    return x_prev - eta * s, r_k, s, None


def _mutant_sign(x_prev, blocks, b_new, lam_k, eta=1.0):
    M = sp.vstack([sp.csr_matrix(B) for B in blocks], format="csr")
    A_k = sp.csr_matrix(blocks[-1])
    ell, p = A_k.shape[0], M.shape[0]
    r_k = b_new - A_k @ x_prev  # wrong sign of the residual
    K = lam_k * np.eye(p) + (M @ M.T).toarray()
    rhs = np.zeros(p)
    rhs[p - ell:] = r_k
    s = M.T @ np.linalg.solve(K, rhs)
    return x_prev - eta * s, r_k, s, None


@pytest.mark.parametrize("mutant", [_mutant_rhs_first_block, _mutant_sign])
def test_planted_mistakes_break_the_pins(monkeypatch, mutant):
    monkeypatch.setattr(slim, "step_woodbury", mutant)
    A, _, b = workloads.gaussian_problem(3, m=120, n=25)
    src = slim.dense_source(A, b)
    sched = [slim.contiguous_block_ids(i, 6) for i in (3, 11, 0, 19)]
    with pytest.raises(AssertionError):
        _full_memory_check(src, lambda ids: A[ids], lambda ids: b[ids], sched, 0.05, False, r=10)
