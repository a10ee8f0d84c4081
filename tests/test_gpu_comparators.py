"""The comparators (sg, olbfgs) and the decaying damping schedule on the GPU
against the float64 oracle: trajectories on the device, single sg steps from
the oracle's iterate, the float32 iterate, slimLS with the decay in the plain
and pipelined forms, and the argument and state checks."""
import numpy as np
import pytest

import workloads
from oracle import comparators as cmp, joseph, slim as oslim

from _common import oracle_memory, rel

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


def _oracle(g, b, seed, steps, lam, method, memory=10, eta=1.0, decay_after=0, x0=None):
    src = oslim.tomo_source(g, b)
    sched = list(oslim.view_schedule(g, seed, steps))
    return [x for _, x, _ in cmp.run(src, sched, lam, method, memory, x0, eta, decay_after)]


@pytest.mark.parametrize("decay_after", [0, 4])
def test_sg_trajectory(sl, decay_after):
    g, b = _problem()
    lam, seed, eta = 40.0, 7, 0.9          # alpha = 1/40
    xs = _oracle(g, b, seed, 15, lam, "sg", eta=eta, decay_after=decay_after)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, solver=sl.SLIM_SOLVE_SG, eta=eta,
                decay_after=decay_after, use_graph=True)
    s.set_data(b)
    for k in (1, 5, 15):
        s.step(k - s.get_iter())
        assert rel(s.get_x(), xs[k - 1]) < 1e-12, k
    s.close()


def test_sg_single_steps_float32(sl):
    g, b = _problem(N=40, V=30, D=57, seed=8)
    src = oslim.tomo_source(g, b)
    lam, seed = 60.0, 8
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, precision=1,
                solver=sl.SLIM_SOLVE_SG)
    s.set_data(b.astype(np.float32))
    x = np.zeros(g.n)
    worst = 0.0
    for k in range(1, 9):
        ids = oslim.view_block_ids(g, seed, k)
        x32 = x.astype(np.float32).astype(np.float64)
        xo, _ = cmp.step_sg(x32, src.rows(ids), src.rhs(ids), 1.0 / lam)
        s.set_x(x.astype(np.float32))
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo))
        x = xo
    assert worst < 1e-6
    s.close()


@pytest.mark.parametrize("memory,decay_after", [(3, 0), (10, 0), (20, 6)])
def test_olbfgs_trajectory(sl, memory, decay_after):
    g, b = _problem(seed=9)
    lam, seed, eta = 30.0, 9, 1.0
    steps = 24
    xs = _oracle(g, b, seed, steps, lam, "olbfgs", memory=memory, eta=eta,
                 decay_after=decay_after)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, solver=sl.SLIM_SOLVE_OLBFGS,
                olbfgs_memory=memory, eta=eta, decay_after=decay_after)
    s.set_data(b)
    for k in (1, 2, 4, 12, steps):
        s.step(k - s.get_iter())
        assert rel(s.get_x(), xs[k - 1]) < 1e-10, (memory, k)
    s.close()


def test_olbfgs_float32_iterate(sl):
    g, b = _problem(N=40, V=30, D=57, seed=10)
    lam, seed = 50.0, 10
    xs = _oracle(g, b, seed, 6, lam, "olbfgs", memory=10)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, precision=1,
                solver=sl.SLIM_SOLVE_OLBFGS, olbfgs_memory=10)
    s.set_data(b.astype(np.float32))
    s.step(6)
    # float32 x (6e-8 relative per rounding) through six steps and five pairs
    assert rel(s.get_x(), xs[-1]) < 1e-5
    s.close()


def test_olbfgs_restart(sl):
    g, b = _problem(seed=11)
    lam, seed = 30.0, 11
    xs = _oracle(g, b, seed, 8, lam, "olbfgs", memory=5)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, solver=sl.SLIM_SOLVE_OLBFGS,
                olbfgs_memory=5)
    s.set_data(b)
    s.step(5)
    s.set_iter(0)                 # drops the pairs; the draws restart at step 1
    s.set_x(np.zeros(g.n))
    s.step(8)
    assert rel(s.get_x(), xs[-1]) < 1e-10
    with pytest.raises(sl.SlimError):
        s.set_iter(3)
    with pytest.raises(sl.SlimError):
        s.checkpoint()
    s.close()


@pytest.mark.parametrize("lookahead", [0, 2])
def test_slimls_with_decaying_damping(sl, lookahead):
    g, b = _problem(seed=12)
    src = oslim.tomo_source(g, b)
    r, lam, seed, K = 2, 1e-2, 12, 4
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, decay_after=K, ramp=True,
                lookahead=lookahead)
    s.set_data(b)
    s.step(12)
    x = np.zeros(g.n)
    for k in range(1, 13):
        mem = oracle_memory(g, seed, k, r)
        blocks = [src.rows(ids) for _, _, ids in mem]
        x, *_ = oslim.step_woodbury(x, blocks, src.rhs(mem[-1][2]),
                                    cmp.damping(lam, k, r, True, K))
    assert rel(s.get_x(), x) < 1e-11
    s.close()


def test_kernels_and_arguments(sl):
    g, b = _problem()
    for solver in (sl.SLIM_SOLVE_SG, sl.SLIM_SOLVE_OLBFGS):
        s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, 10.0, 1, solver=solver)
        s.set_data(b)
        s.set_timing(True)
        s.step(1)
        assert s.get_timing()[1] == 3
        with pytest.raises(sl.SlimError):   # no Gram matrix
            s.get_memory()
        with pytest.raises(sl.SlimError):   # C_k = diag(c) is a Woodbury-form option
            s.set_c_diag(np.ones(g.n))
        s.close()
        with pytest.raises(sl.SlimError):   # the comparators keep no slimLS memory
            sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 10.0, 1, solver=solver)
        with pytest.raises(sl.SlimError):   # pipelined form
            sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, 10.0, 1, solver=solver, lookahead=2)
        with pytest.raises(sl.SlimError):   # slimTik rows
            sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, 10.0, 1, solver=solver, tik_lambda=1.0)
    with pytest.raises(sl.SlimError):       # memory above the largest
        sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, 10.0, 1, solver=sl.SLIM_SOLVE_OLBFGS,
                olbfgs_memory=21)
    with pytest.raises(sl.SlimError):       # negative decay start
        sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, decay_after=-1)


def test_olbfgs_memory_one_and_step_factor(sl):
    g, b = _problem(seed=14)
    lam, seed, eta = 25.0, 14, 0.5
    xs = _oracle(g, b, seed, 10, lam, "olbfgs", memory=1, eta=eta)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, lam, seed, solver=sl.SLIM_SOLVE_OLBFGS,
                olbfgs_memory=1, eta=eta)
    s.set_data(b)
    s.step(10)
    assert rel(s.get_x(), xs[-1]) < 1e-10
    s.close()


@pytest.mark.parametrize("method", ["sg", "olbfgs"])
def test_at_256(sl, method):
    # the 256x256 workload of the bench's step costs, six steps
    cfg = workloads.C2
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = workloads.add_noise(joseph.full_matrix(g) @ x_true, e, cfg.noise)
    lam = 1e3
    xs = _oracle(g, b, cfg.seed, 6, lam, method, memory=10)
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.det, 0, lam, cfg.seed,
                solver=sl.SLIM_SOLVE_SG if method == "sg" else sl.SLIM_SOLVE_OLBFGS)
    s.set_data(b)
    s.step(6)
    assert rel(s.get_x(), xs[-1]) < 1e-11
    s.close()
