"""slimTik with a lower-bidiagonal L on the GPU (Eq. slimTik, C_k = L^T L with
(L x)_i = d0_i x_i + d1_i x_{i-1}: the first difference along the image rows
plus a multiple of the identity) against the oracle's direct form of
Eq. (slimTik), the dense n x n system as written.

Trajectories (float64, 1e-10; the mixed solver, 1e-9), slimLS with that C_k
(lam_tik = 0), graph replay, a float32 iterate (1e-5 per step), L set after
some steps (the memory is rebuilt with the new W), the diagonal case against
the diagonal-C path, C_k = I restored, and the argument checks.
"""
import numpy as np
import pytest

import workloads
from oracle import joseph, slim as oslim, tik as otik

from _common import oracle_memory, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _problem(N=24, V=18, D=35, seed=7):
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    return g, b


def _bidiag(n, N, seed):
    rs = np.random.default_rng(seed)
    d0 = 1.0 + 0.5 * rs.random(n)
    d1 = -0.8 * (0.5 + 0.5 * rs.random(n))
    d1[::N] = 0.0                      # no coupling across image rows
    return d0, d1


@pytest.mark.parametrize("lam_tik,solver,tol,graph", [(0.7, 0, 1e-10, False), (0.0, 0, 1e-10, False),
                                                      (0.7, 1, 1e-9, True)])
def test_trajectory_matches_the_direct_form(sl, lam_tik, solver, tol, graph):
    g, b = _problem()
    src = oslim.tomo_source(g, b)
    r, lam, seed, steps = 3, 1e-2, 7, 10
    d0, d1 = _bidiag(g.n, g.N, 1)
    L = otik.bidiagonal(d0, d1)
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in otik.run(src, sched, r, lam, lam_tik, g.n_views, form="direct", L=L)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik,
                solver=solver, refine_iters=2, use_graph=graph)
    s.set_data(b)
    s.set_tik_bidiag(d0, d1)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < tol, k
    s.close()


def _direct_step(g, src, seed, k, r, lam, lam_tik, x_prev, L):
    mem = oracle_memory(g, seed, k, r)
    blocks = [src.rows(ids) for _, _, ids in mem]
    x, *_ = otik.step_direct(x_prev, blocks, src.rhs(mem[-1][2]), lam, lam_tik, g.n_views,
                             otik.window_count(k, r), L)
    return x


def test_float32_single_steps(sl):
    g, b = _problem(seed=8)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 2, 1e-2, 0.5, 8
    d0, d1 = _bidiag(g.n, g.N, 2)
    L = otik.bidiagonal(d0, d1)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik,
                precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED)
    s.set_data(b.astype(np.float32))
    s.set_tik_bidiag(d0, d1)
    x_prev = (np.random.default_rng(3).standard_normal(g.n) * 0.05).astype(np.float32)
    for k in range(1, 7):
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        xo = _direct_step(g, src, seed, k, r, lam, lam_tik, x_prev.astype(np.float64), L)
        assert rel(s.get_x(), xo) < 1e-5, k
        x_prev = xo.astype(np.float32)
    s.close()


def test_L_set_after_steps_and_restored(sl):
    g, b = _problem(seed=9)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 3, 1e-2, 0.6, 9
    d0, d1 = _bidiag(g.n, g.N, 4)
    L = otik.bidiagonal(d0, d1)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
    s.set_data(b)
    s.step(3)                              # C_k = I so far
    x3 = s.get_x()
    s.set_tik_bidiag(d0, d1)               # the window's Gram rows are rebuilt with W
    x_prev = x3
    for k in range(4, 8):
        s.step(1)
        xo = _direct_step(g, src, seed, k, r, lam, lam_tik, x_prev, L)
        assert rel(s.get_x(), xo) < 1e-10, k
        x_prev = s.get_x()
    s.set_tik_bidiag(None)                 # back to C_k = I
    s.step(1)
    I = np.eye(g.n)
    xo = _direct_step(g, src, seed, 8, r, lam, lam_tik, x_prev, I)
    assert rel(s.get_x(), xo) < 1e-10
    s.close()


def test_diagonal_L_matches_the_diagonal_C_path(sl):
    g, b = _problem(seed=10)
    r, lam, lam_tik, seed = 2, 1e-2, 0.8, 10
    d0 = 1.0 + np.random.default_rng(5).random(g.n)
    xs = []
    for use_bidiag in (True, False):
        s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
        s.set_data(b)
        if use_bidiag:
            s.set_tik_bidiag(d0)           # d1 = 0: L = diag(d0), C = diag(d0^2)
        else:
            s.set_c_diag(d0 * d0)
        s.step(8)
        xs.append(s.get_x())
        s.close()
    assert rel(xs[0], xs[1]) < 1e-12


def test_bidiagonal_argument_checks(sl):
    g, b = _problem()
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=0.5)
    d0, d1 = _bidiag(g.n, g.N, 1)
    d0z = d0.copy()
    d0z[5] = 0.0
    with pytest.raises(sl.SlimError) as ei:      # L singular
        s.set_tik_bidiag(d0z, d1)
    assert ei.value.code == sl.SLIM_EINVAL
    with pytest.raises(sl.SlimError) as ei:      # wrong length
        s.set_tik_bidiag(d0[:-1], d1[:-1])
    assert ei.value.code == sl.SLIM_EINVAL
    s.close()
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=0.5, lookahead=2)
    with pytest.raises(sl.SlimError) as ei:      # the pipelined form keeps diagonal C only
        s.set_tik_bidiag(d0, d1)
    assert ei.value.code == sl.SLIM_ENOTSUP
    s.close()
