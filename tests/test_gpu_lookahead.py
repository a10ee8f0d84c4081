"""Pipelined form (geometry chain up to D steps ahead of the iterate chain)
against the float64 oracle: the iterates, the memory and the Gram rows are
those of Eq. (ram)/(B_k) whatever D is."""
import numpy as np
import pytest

import workloads
from oracle import joseph, slim as oslim

from _common import oracle_memory, oracle_step_from, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _problem(N=32, V=20, D=47, seed=7):
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    return g, b


@pytest.mark.parametrize("D,ramp", [(1, False), (2, True), (3, False), (6, False)])
def test_trajectory_fp64(sl, D, ramp):
    g, b = _problem()
    r, lam, seed, steps = 3, 1e-2, 7, 11
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam, ramp=ramp)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, ramp=ramp, lookahead=D)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-12, (D, k)
        if k == 6:
            ids, G, _ = s.get_memory()
            want = np.full(s.p, -1)
            for _, slot, rows in oracle_memory(g, seed, k, r):
                want[slot * g.det_u:(slot + 1) * g.det_u] = rows
            assert np.array_equal(ids, want)
            M = joseph.rows(g, ids)
            Go = (M @ M.T).toarray()
            assert np.max(np.abs(G - Go)) <= 1e-13 * np.max(np.abs(Go))
    assert s.get_iter() == steps
    s.close()


def test_multi_step_call_matches_single_steps(sl):
    g, b = _problem(seed=8)
    r, lam, seed = 2, 1e-2, 8
    sched = list(oslim.view_schedule(g, seed, 9))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, lookahead=2)
    s.set_data(b)
    s.step(4)
    s.step(5)
    assert rel(s.get_x(), traj[-1]) < 1e-12
    s.close()


@pytest.mark.parametrize("D", [1, 3])
def test_mixed_precision_single_step(sl, D):
    g, b = _problem(N=40, V=30, D=57, seed=9)
    r, lam, seed = 5, 1e-2, 9
    sched = list(oslim.view_schedule(g, seed, 8))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, precision=sl.SLIM_PREC_FP32,
                solver=sl.SLIM_SOLVE_MIXED, refine_iters=2, lookahead=D)
    s.set_data(b)
    s.step(7)
    s.set_x(traj[6])      # replaced on the caller's stream, before the next iterate chain
    s.step(1)
    assert rel(s.get_x(), traj[7]) < 1e-5
    s.close()


def test_checkpoint_restore(sl):
    g, b = _problem(seed=10)
    r, lam, seed = 3, 1e-2, 10
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, lookahead=2)
    s.set_data(b)
    s.step(5)
    blob = s.checkpoint()
    s.step(4)
    xa = s.get_x()
    s.restore(blob)
    assert s.get_iter() == 5
    s.step(4)
    assert rel(s.get_x(), xa) < 1e-13
    sched = list(oslim.view_schedule(g, seed, 9))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    assert rel(xa, traj[-1]) < 1e-12
    s.close()


def test_timing_phases(sl):
    g, b = _problem(seed=11)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 11, lookahead=1)
    s.set_data(b)
    s.set_timing(True)
    s.step(3)
    ph, kernels = s.get_timing()
    assert len(ph) == 7 and all(v >= 0.0 for v in ph.values())
    assert kernels == s.kernels_per_step()
    s.close()


def test_unsupported_combinations(sl):
    with pytest.raises(sl.SlimError):
        sl.Slim(32, 20, 47, 20, 2, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, lookahead=1)
    with pytest.raises(sl.SlimError):
        sl.Slim(32, 20, 47, 47, 2, 1e-2, 1, lookahead=11)
    with pytest.raises(sl.SlimError):
        sl.SlimBatch([dict(N=24, n_views=18, det=35, ell=35, r=2, lam=1e-2, seed=1, kind=0,
                           lookahead=1)])


@pytest.mark.parametrize("solver", ["SLIM_SOLVE_MIXED_TC", "SLIM_SOLVE_MIXED_INV"])
@pytest.mark.parametrize("D,r,N,V,det", [(1, 5, 40, 30, 57), (3, 2, 24, 18, 35), (6, 3, 64, 30, 91)])
def test_tensor_core_inverse_solves(sl, D, r, N, V, det, solver):
    # the solves through X = L^{-1} (tensor-core inverse in the geometry
    # chain): the same iterates as the float64 oracle at the float32 bar,
    # on ragged orders (p = 342, 105, 364) and wrapping buffers
    g, b = _problem(N=N, V=V, D=det, seed=9)
    lam, seed = 1e-2, 9
    steps = r + 1 + D + 3
    sched = list(oslim.view_schedule(g, seed, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, precision=sl.SLIM_PREC_FP32,
                solver=getattr(sl, solver), refine_iters=2, lookahead=D)
    s.set_data(b)
    src = oslim.tomo_source(g, b)
    for k in range(1, steps + 1):
        x_prev = traj[k - 2] if k > 1 else np.zeros(g.n)
        s.set_x(x_prev)                  # the oracle's x_{k-1}, rounded to float32
        s.step(1)
        xp = x_prev.astype(np.float32).astype(np.float64)
        xo32, _ = oracle_step_from(g, src, seed, k, r, lam, xp)
        assert rel(s.get_x(), xo32) < 1e-5, (D, k)
    s.close()


def _inverse_depths(T):
    # recursion depths of the triangular inverse over T tiles (a range of n
    # tiles splits into floor(n/2) and ceil(n/2) until single tiles remain)
    return 0 if T <= 1 else 1 + _inverse_depths((T + 1) // 2)


@pytest.mark.parametrize("N,V,det,r", [(32, 20, 47, 2), (64, 30, 91, 3), (256, 180, 363, 5)])
def test_inverse_form_kernels_per_step(sl, N, V, det, r):
    # the launches one step of the pipelined inverse form makes: the geometry
    # chain's six kernels, one persistent factorisation, the inverse (diagonal
    # tiles, a split pass and a product per side at every recursion depth,
    # the mirror) and the cooperative iterate chain
    s = sl.Slim(N, V, det, det, r, 1e-2, 1, precision=sl.SLIM_PREC_FP32,
                solver=sl.SLIM_SOLVE_MIXED_INV, lookahead=2)
    T = (s.p + 63) // 64
    assert s.kernels_per_step() == 6 + 1 + (2 + 4 * _inverse_depths(T)) + 1
    s.close()


@pytest.mark.parametrize("solver", ["SLIM_SOLVE_MIXED_TC", "SLIM_SOLVE_MIXED_INV"])
def test_tensor_core_inverse_argument_checks(sl, solver):
    with pytest.raises(sl.SlimError) as ei:      # needs the pipelined form
        sl.Slim(32, 20, 47, 47, 2, 1e-2, 1, precision=sl.SLIM_PREC_FP32,
                solver=getattr(sl, solver))
    assert ei.value.code == sl.SLIM_ENOTSUP
    with pytest.raises(sl.SlimError) as ei:      # 64-wide tiles only
        sl.Slim(32, 20, 47, 47, 2, 1e-2, 1, precision=sl.SLIM_PREC_FP32,
                solver=getattr(sl, solver), lookahead=2, tile=32)
    assert ei.value.code == sl.SLIM_ENOTSUP
