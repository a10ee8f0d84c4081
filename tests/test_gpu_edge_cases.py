"""Degenerate and boundary configurations of the method against the float64
oracle (Eq. ram / Eq. B_k): one ray per block (the Sherman-Morrison case),
no memory (r = 0, damped block Kaczmarz), one view (every block the same),
the smallest images, a damping so large that the step is lambda^-1 A^T r, a
zero right-hand side, and the damped solve at orders around a tile (1, 63,
64, 65, 129) where the tiled Cholesky pads to a whole tile."""
import numpy as np
import pytest

import workloads
from oracle import joseph, slim as oslim

from _common import rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _data(N, V, D, seed):
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(N, seed, 3), workloads.noise_direction(g.m, seed),
                            0.01)
    return g, b


def _check_trajectory(s, traj, tol=1e-12):
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < tol, k


@pytest.mark.parametrize("r", [0, 4])
def test_one_ray_per_block(sl, r):
    # ell = 1: K is (r+1) x (r+1), padded to one tile; with r = 0 the step is
    # Sherman-Morrison's (lambda + |a|^2)^-1 a r
    N, V, D, lam, seed = 16, 12, 23, 5e-2, 3
    g, b = _data(N, V, D, seed)
    steps = 12
    sched = list(oslim.random_ray_schedule(seed, 1, g.m, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, 1, r, lam, seed, kind=sl.SLIM_BLOCKS_RAYS)
    s.set_data(b)
    _check_trajectory(s, traj)
    s.close()


@pytest.mark.parametrize("tile", [32, 64])
def test_no_memory_view_blocks(sl, tile):
    # r = 0: the damped block Kaczmarz step of Eq. (dbK)
    N, V, D, lam, seed = 20, 15, 29, 1e-2, 4
    g, b = _data(N, V, D, seed)
    steps = 10
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, 0, lam)]
    s = sl.Slim(N, V, D, D, 0, lam, seed, tile=tile)
    s.set_data(b)
    _check_trajectory(s, traj)
    s.close()


@pytest.mark.parametrize("cyclic", [False, True])
def test_a_single_view(sl, cyclic):
    # one view: every block is the same one, so the memory holds r+1 copies of
    # it (duplicates stay, lambda I keeps K definite); the cyclic order's epoch
    # is that one view
    N, V, D, r, lam, seed = 12, 1, 17, 3, 1e-2, 5
    g, b = _data(N, V, D, seed)
    steps = 8
    sched = list(oslim.view_schedule(g, seed, steps, cyclic=cyclic))
    assert all(np.array_equal(blk, sched[0]) for blk in sched)
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, D, r, lam, seed, cyclic=cyclic)
    s.set_data(b)
    _check_trajectory(s, traj)
    s.close()


@pytest.mark.parametrize("N,V,D", [(2, 3, 3), (3, 4, 5), (5, 7, 8)])
def test_smallest_images(sl, N, V, D):
    r, lam, seed = 2, 1e-2, 6
    g, b = _data(N, V, D, seed)
    steps = 9
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, D, r, lam, seed)
    s.set_data(b)
    _check_trajectory(s, traj)
    s.close()


def test_large_damping_is_a_scaled_gradient_step(sl):
    # lambda >> ||M M^T||: z = lambda^-1 [0; r_k] + O(lambda^-2), so the step is
    # x -= lambda^-1 A_k^T r_k to first order; the oracle's step is exact
    N, V, D, r, seed = 16, 12, 23, 2, 7
    lam = 1e6
    g, b = _data(N, V, D, seed)
    steps = 6
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, D, r, lam, seed)
    s.set_data(b)
    _check_trajectory(s, traj)
    A = joseph.full_matrix(g)
    rows = sched[0]
    x1 = -(A[rows].T @ (A[rows] @ np.zeros(g.n) - b[rows])) / lam
    assert rel(traj[0], x1) < 1e-3
    s.close()


def test_zero_data_keeps_zero_iterate(sl):
    N, V, D, r, lam, seed = 16, 12, 23, 3, 1e-2, 8
    s = sl.Slim(N, V, D, D, r, lam, seed, precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED)
    s.set_data(np.zeros(V * D, dtype=np.float32))
    s.step(7)
    assert np.all(s.get_x() == 0.0)
    s.close()


@pytest.mark.parametrize("p", [1, 63, 64, 65, 129])
def test_damped_solve_around_a_tile(sl, p):
    rs = np.random.default_rng(p)
    B = rs.standard_normal((p, p + 3))
    G = B @ B.T / p
    lam = 1e-2
    rhs = rs.standard_normal(p)
    want = np.linalg.solve(lam * np.eye(p) + G, rhs)
    z = torch.zeros(p, dtype=torch.float64, device="cuda")
    sl.damped_solve(torch.tensor(G, device="cuda"), lam, torch.tensor(rhs, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), want) < 1e-11, p
