"""Pins for the reference solutions and the full-memory limit of the iteration."""
import numpy as np

import workloads
from oracle import joseph, slim, targets


def test_xls_qr_matches_normal_equations():
    A, _, b = workloads.gaussian_problem(8)
    a, c = targets.x_ls_qr(A, b), targets.x_ls_normal(A, b)
    assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)
    # the LS residual is orthogonal to range(A)
    assert np.linalg.norm(A.T @ (A @ a - b)) <= 1e-10 * np.linalg.norm(A.T @ b)


def test_xtik_dense_matches_cgls():
    g = joseph.Geometry(24, 18, 35)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(24, 2, 5), workloads.noise_direction(g.m, 2), 0.01)
    for lam in (1e-1, 1e-3):
        xd = targets.x_tik_dense(A, b, lam)
        xc, it, res = targets.cgls(A, b, lam, tol=1e-13)
        assert res <= 1e-13
        assert np.linalg.norm(xd - xc) <= 1e-9 * np.linalg.norm(xd)
        # optimality of x_tik: A^T(Ax - b) + lam x = 0
        assert np.linalg.norm(A.T @ (A @ xd - b) + lam * xd) <= 1e-10 * np.linalg.norm(A.T @ b)


def test_one_epoch_with_full_memory_is_tikhonov():
    # memory r = M-1, every block exactly once, x_0 = 0  =>  x_M = x_tik(lambda)
    g = joseph.Geometry(16, 10, 23)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(16, 4, 4), workloads.noise_direction(g.m, 4), 0.01)
    lam = 1e-2
    order = np.random.default_rng(3).permutation(g.n_views)
    sched = [g.view_rays(int(a)) for a in order]
    for k, x, _ in slim.run(slim.tomo_source(g, b), sched, r=g.n_views - 1, lam=lam):
        pass
    xt = targets.x_tik_dense(A, b, lam)
    assert np.linalg.norm(x - xt) <= 1e-10 * np.linalg.norm(xt)


def test_full_memory_small_lambda_is_least_squares():
    # Appendix A: with all blocks in memory the iterate after one pass is x_LS (lambda -> 0)
    A, _, b = workloads.gaussian_problem(9, m=300, n=40)
    M = 30
    sched = [slim.contiguous_block_ids(i, 10) for i in np.random.default_rng(2).permutation(M)]
    # (lambda = 1e-6: the gap to x_LS is O(lambda); much smaller lambda makes the
    # p x p Woodbury system of 300 rows in 40 unknowns singular to working precision)
    for k, x, _ in slim.run(slim.dense_source(A, b), sched, r=M - 1, lam=1e-6):
        pass
    xls = targets.x_ls_qr(A, b)
    assert np.linalg.norm(x - xls) <= 1e-7 * np.linalg.norm(xls)
