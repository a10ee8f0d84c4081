"""Pins for the LSQR oracle (the damped least-squares problem of Eq. slimLSstep).

* Converged LSQR equals the closed form (M^T M + d^2 I)^{-1} M^T c.
* Each iterate s_i minimises the damped residual over the Krylov space
  K_i(M^T M, M^T c): checked against an explicit Krylov basis and a small
  dense least-squares solve, for i = 1..6.
* The damped residual never increases from one iterate to the next.
* The normal-equation residual estimate equals ||M^T(c - M s) - d^2 s||.
* damp = 0 on a full-rank tall matrix gives the ordinary least-squares solution.
* On a tomography window the converged step equals the Woodbury step of the
  slimLS oracle.
* SciPy's independent LSQR gives the same iterates at fixed iteration counts.
Mutations planted in the oracle (a flipped sign of theta, a dropped damping
rotation) break these pins (checked at the end).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import joseph, lsqr, slim


def _problem(m=30, n=20, seed=0, dense=True):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((m, n))
    if not dense:
        M[rng.random((m, n)) < 0.6] = 0.0
    c = rng.standard_normal(m)
    return M, c


def _solve(M, c, damp, iters, tol=0.0, trace=None, mod=lsqr):
    return mod.lsqr_damped(lambda v: M @ v, lambda u: M.T @ u, c, M.shape[1], damp, iters, tol,
                           trace)


@pytest.mark.parametrize("m,n,damp", [(30, 20, 0.3), (12, 25, 0.05), (40, 40, 1.0)])
def test_converges_to_closed_form(m, n, damp):
    M, c = _problem(m, n, seed=m + n)
    res = _solve(M, c, damp, 400, tol=1e-14)
    want = np.linalg.solve(M.T @ M + damp * damp * np.eye(n), M.T @ c)
    assert np.linalg.norm(res.s - want) <= 1e-9 * np.linalg.norm(want)


def test_iterates_are_krylov_minimisers():
    M, c = _problem(25, 15, seed=3)
    damp = 0.4
    trace = []
    _solve(M, c, damp, 6, trace=trace)
    K = M.T @ M
    basis = [M.T @ c]
    for i in range(1, 7):
        Q, _ = np.linalg.qr(np.column_stack(basis))           # basis of K_i(M^T M, M^T c)
        stacked = np.vstack([M @ Q, damp * Q])
        y, *_ = np.linalg.lstsq(stacked, np.concatenate([c, np.zeros(15)]), rcond=None)
        want = Q @ y
        assert np.linalg.norm(trace[i - 1] - want) <= 1e-10 * np.linalg.norm(want), i
        basis.append(K @ basis[-1])


def test_damped_residual_decreases_and_estimate_is_exact():
    M, c = _problem(40, 30, seed=5, dense=False)
    damp = 0.2
    trace = []
    _solve(M, c, damp, 25, trace=trace)
    def damped_res(s):
        return math.sqrt(np.linalg.norm(c - M @ s) ** 2 + (damp * np.linalg.norm(s)) ** 2)
    vals = [damped_res(s) for s in trace]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(vals, vals[1:]))
    for i in (1, 5, 12):
        r = _solve(M, c, damp, i)
        exact = np.linalg.norm(M.T @ (c - M @ r.s) - damp ** 2 * r.s)
        assert abs(r.normal_res - exact) <= 1e-8 * exact, i
    assert abs(r.normal_res0 - np.linalg.norm(M.T @ c)) <= 1e-12 * r.normal_res0


def test_undamped_is_ordinary_least_squares():
    M, c = _problem(50, 12, seed=9)
    res = _solve(M, c, 0.0, 200, tol=1e-14)
    want, *_ = np.linalg.lstsq(M, c, rcond=None)
    assert np.linalg.norm(res.s - want) <= 1e-10 * np.linalg.norm(want)


def test_converged_step_equals_woodbury_step():
    N, V, D = 16, 12, 23
    g = joseph.Geometry(N, V, D)
    x_true = workloads.phantom_2d(N, 3, 4)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, workloads.noise_direction(g.m, 3), 0.01)
    src = slim.tomo_source(g, b)
    seed, r, lam = 3, 2, 1e-2
    x = np.random.default_rng(1).standard_normal(g.n) * 0.1
    blocks = [src.rows(slim.view_block_ids(g, seed, k)) for k in (1, 2, 3)]
    b_new = src.rhs(slim.view_block_ids(g, seed, 3))
    xw, rw, sw, _ = slim.step_woodbury(x, blocks, b_new, lam)
    xl, rl, res = lsqr.step_lsqr(x, blocks, b_new, lam, 2000, tol=1e-13)
    assert np.array_equal(rw, rl)
    assert np.linalg.norm(res.s - sw) <= 1e-9 * np.linalg.norm(sw)
    assert np.linalg.norm(xl - xw) <= 1e-9 * np.linalg.norm(xw)


def test_same_iterates_as_scipy_lsqr():
    spla = pytest.importorskip("scipy.sparse.linalg")
    M, c = _problem(35, 22, seed=11, dense=False)
    Ms = sp.csr_matrix(M)
    damp = 0.25
    for iters in (1, 3, 8, 15):
        ours = _solve(M, c, damp, iters).s
        theirs = spla.lsqr(Ms, c, damp=damp, atol=0.0, btol=0.0, conlim=0.0, iter_lim=iters)[0]
        assert np.linalg.norm(ours - theirs) <= 1e-12 * np.linalg.norm(theirs), iters


def test_planted_mutations_break_the_pins():
    # the oracle with a flipped sign of theta, or without the damping
    # rotation, must fail the closed-form pin
    M, c = _problem(30, 20, seed=4)
    damp = 0.3
    want = np.linalg.solve(M.T @ M + damp * damp * np.eye(20), M.T @ c)

    def run(mutation):
        s = np.zeros(20)
        beta = np.linalg.norm(c)
        u = c / beta
        v = M.T @ u
        alpha = np.linalg.norm(v)
        v /= alpha
        w = v.copy()
        rho_bar, phi_bar = alpha, beta
        for _ in range(400):
            u = M @ v - alpha * u
            beta = np.linalg.norm(u)
            u /= beta
            v = M.T @ u - beta * v
            alpha = np.linalg.norm(v)
            v /= alpha
            if mutation == "no_damping":
                c1, rho_hat = 1.0, rho_bar
            else:
                c1, _, rho_hat = lsqr.rotation(rho_bar, damp)
            phi_hat = c1 * phi_bar
            cr, sr, rho = lsqr.rotation(rho_hat, beta)
            theta = sr * alpha * (-1.0 if mutation == "theta_sign" else 1.0)
            rho_bar = -cr * alpha
            phi, phi_bar = cr * phi_hat, sr * phi_hat
            s = s + (phi / rho) * w
            w = v - (theta / rho) * w
        return np.linalg.norm(s - want) / np.linalg.norm(want)

    assert run("none") < 1e-9
    assert run("theta_sign") > 1e-3
    assert run("no_damping") > 1e-3


def test_tik_lsqr_converges_to_the_slimtik_step():
    # the column-scaled damped problem of step_tik_lsqr, solved to 1e-13, is
    # the slimTik step (Woodbury form of the slimTik oracle, itself pinned to
    # the direct form of Eq. slimTik)
    from oracle import tik
    N, V, D = 14, 10, 21
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(N, 5, 4), workloads.noise_direction(g.m, 5),
                            0.01)
    src = slim.tomo_source(g, b)
    cdiag = 0.5 + 1.5 * np.random.default_rng(3).random(g.n)
    x = np.random.default_rng(4).standard_normal(g.n) * 0.1
    blocks = [src.rows(slim.view_block_ids(g, 5, k)) for k in (1, 2, 3)]
    b_new = src.rhs(slim.view_block_ids(g, 5, 3))
    for lam_tik, cd in ((0.8, cdiag), (0.0, cdiag), (0.6, None)):
        xw, *_ = tik.step_woodbury(x, blocks, b_new, 5e-2, lam_tik, V, 3,
                                   None if cd is None else np.sqrt(cd))
        xl, _, res = lsqr.step_tik_lsqr(x, blocks, b_new, 5e-2, lam_tik, V, 3, cd, 5000, 1e-13)
        assert np.linalg.norm(xl - xw) <= 1e-9 * np.linalg.norm(xw), lam_tik
    # C = I and no Tikhonov rows: the plain LSQR step
    xl, _, _ = lsqr.step_tik_lsqr(x, blocks, b_new, 5e-2, 0.0, V, 3, None, 7)
    xp, _, _ = lsqr.step_lsqr(x, blocks, b_new, 5e-2, 7)
    assert np.linalg.norm(xl - xp) <= 1e-12 * np.linalg.norm(xp)   # scaling by diag(1) reorders sums
