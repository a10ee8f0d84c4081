"""Batched form (many independent problems in one graph) and the autotuner,
against the float64 oracle run problem by problem."""
import numpy as np
import pytest

import workloads
from oracle import joseph, rng, slim as oslim

from _common import rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


# uneven problems: sizes, memories, block kinds, tile sizes and CTAs per SM differ
SPECS = [
    dict(N=24, n_views=18, det=35, ell=20, r=3, lam=3e-2, seed=11, kind=1, tile=32, ctas_per_sm=1),
    dict(N=32, n_views=20, det=47, ell=47, r=2, lam=1e-2, seed=12, kind=0, tile=64, ctas_per_sm=3),
    dict(N=20, n_views=30, det=29, ell=37, r=5, lam=5e-3, seed=13, kind=1, tile=0, ctas_per_sm=0),
    dict(N=28, n_views=16, det=41, ell=41, r=1, lam=2e-2, seed=14, kind=0, tile=32, ctas_per_sm=2),
]


def _problem(sp):
    g = joseph.Geometry(sp["N"], sp["n_views"], sp["det"])
    A = joseph.full_matrix(g)
    x_true = workloads.phantom_2d(sp["N"], sp["seed"], 5)
    b = workloads.add_noise(A @ x_true, workloads.noise_direction(g.m, sp["seed"]), 0.01)
    return g, b


def _trajectory(sp, g, b, steps):
    if sp["kind"] == 1:
        sched = oslim.random_ray_schedule(sp["seed"], sp["ell"], g.m, steps)
    else:
        sched = oslim.view_schedule(g, sp["seed"], steps)
    return [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), list(sched), sp["r"], sp["lam"])]


def test_batch_matches_oracle_per_problem(sl):
    steps = 7
    probs = [_problem(sp) for sp in SPECS]
    trajs = [_trajectory(sp, g, b, steps) for sp, (g, b) in zip(SPECS, probs)]
    bt = sl.SlimBatch(SPECS)
    for pb, (_, b) in zip(bt.problems, probs):
        pb.set_data(b)
    bt.step(3)
    bt.sync()
    for i, pb in enumerate(bt.problems):
        assert pb.get_iter() == 3
        assert rel(pb.get_x(), trajs[i][2]) < 1e-12, i
    bt.step(4)
    bt.sync()
    for i, pb in enumerate(bt.problems):
        assert pb.get_iter() == steps
        assert rel(pb.get_x(), trajs[i][-1]) < 1e-12, i
    bt.close()


def test_batch_set_x_between_steps(sl):
    """Work queued on a problem's own stream (set_x) is ordered before the next batch step."""
    sp = SPECS[0]
    g, b = _problem(sp)
    x0 = np.linspace(-1.0, 1.0, g.n)
    sched = list(oslim.random_ray_schedule(sp["seed"], sp["ell"], g.m, 4))
    want = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, sp["r"], sp["lam"])]
    bt = sl.SlimBatch([sp, SPECS[2]])
    g2, b2 = _problem(SPECS[2])
    bt.problems[0].set_data(b)
    bt.problems[1].set_data(b2)
    bt.step(2)
    # x replaced after step 2: steps 3, 4 continue from x0 with the same memory
    bt.problems[0].set_x(x0)
    bt.step(2)
    bt.sync()
    mem = [oslim.tomo_source(g, b).rows(ids) for ids in sched[:4]]
    x = x0
    for k in (3, 4):
        blocks = mem[max(0, k - 1 - sp["r"]):k]
        x = oslim.step_woodbury(x, blocks, b[sched[k - 1]], sp["lam"])[0]
    assert rel(bt.problems[0].get_x(), x) < 1e-12
    assert rel(bt.problems[1].get_x(), _trajectory(SPECS[2], g2, b2, 4)[-1]) < 1e-12
    assert rel(want[-1], x) > 1e-6     # the set_x really changed the path
    bt.close()


def test_batch_mixed_precision_single_step(sl):
    sp = dict(SPECS[1], precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED)
    g, b = _problem(sp)
    want = _trajectory(sp, g, b, 1)[0]
    bt = sl.SlimBatch([sp, SPECS[0]])
    bt.problems[0].set_data(b)
    bt.problems[1].set_data(_problem(SPECS[0])[1])
    bt.step(1)
    bt.sync()
    assert rel(bt.problems[0].get_x(), want) < 1e-5
    bt.close()


def test_autotune_returns_valid_cached_choice(sl):
    sp = dict(N=64, n_views=30, det=91, ell=91, r=3, lam=1e-2, seed=5, kind=0)
    t1 = sl.autotune(sp, steps=3)
    assert t1[0] in (32, 64) and t1[1] in (1, 2, 3) and t1[2] > 0.0
    t2 = sl.autotune(sp, steps=3)
    assert t2 == t1          # cached per size class
    # the tuned options give the same iterates as the defaults
    g = joseph.Geometry(sp["N"], sp["n_views"], sp["det"])
    b = np.random.default_rng(5).standard_normal(g.m)
    xs = []
    for tile, cps in ((0, 0), (t1[0], t1[1])):
        s = sl.Slim(sp["N"], sp["n_views"], sp["det"], sp["ell"], sp["r"], sp["lam"], sp["seed"],
                    tile=tile, ctas_per_sm=cps)
        s.set_data(b)
        s.step(5)
        xs.append(s.get_x())
        s.close()
    assert rel(xs[1], xs[0]) < 1e-12


def test_bad_tile_rejected(sl):
    with pytest.raises(sl.SlimError):
        sl.Slim(32, 20, 47, 47, 2, 1e-2, 1, tile=48)
    with pytest.raises(sl.SlimError):
        sl.Slim(32, 20, 47, 47, 2, 1e-2, 1, ctas_per_sm=5)


@pytest.mark.parametrize("solver,tile,cps", [(0, 32, 1), (0, 64, 3), (1, 32, 2), (1, 64, 1)])
def test_tile_variants_single_step(sl, solver, tile, cps):
    """Each factor precision x tile size, several tiles and a ragged tail."""
    N, V, D, ell, r, lam, seed = 40, 30, 57, 57, 5, 1e-2, 21   # p = 342
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    sched = list(oslim.view_schedule(g, seed, 8))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, ell, r, lam, seed, precision=sl.SLIM_PREC_FP64, solver=solver, tile=tile,
                ctas_per_sm=cps)
    s.set_data(b)
    s.step(7)
    s.set_x(traj[6])
    s.step(1)
    tol = 1e-12 if solver == 0 else 1e-9
    assert rel(s.get_x(), traj[7]) < tol
    s.close()


def test_batch_at_the_mix_extremes(sl):
    # the batched mix's largest order and smallest damping: a 128 x 128 problem
    # with ell = 512 random rays and r = 7 (p = 4096), float64, next to a
    # lambda = 1e-4 problem in the float32 form (float32 iterate, mixed solve
    # with three refinement rounds: at this damping its floor is 1.4e-5 per
    # step, test_gpu_bench_config), and a small one
    big = dict(N=128, n_views=90, det=182, ell=512, r=7, lam=1e-3, seed=31, kind=1, tile=32,
               ctas_per_sm=2)
    small_lam = dict(N=96, n_views=60, det=137, ell=200, r=4, lam=1e-4, seed=32, kind=1,
                     precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED, refine_iters=3)
    specs = [big, small_lam, SPECS[0]]
    probs = [_problem(sp) for sp in specs]
    steps = 3
    bt = sl.SlimBatch(specs)
    assert bt.problems[0].p == 4096
    for pb, (_, b) in zip(bt.problems, probs):
        pb.set_data(b)
    xs = []
    for k in range(1, steps + 1):
        xs.append([pb.get_x() for pb in bt.problems])     # x_{k-1}
        bt.step(1)
        bt.sync()
        for i, (sp, (g, b)) in enumerate(zip(specs, probs)):
            src = oslim.tomo_source(g, b)
            ids = [np.array(rng.random_rays(sp["seed"], kk, sp["ell"], g.m))
                   for kk in range(max(1, k - sp["r"]), k + 1)]
            x_prev = xs[-1][i]
            xo, _, _, _ = oslim.step_woodbury(x_prev, [src.rows(j) for j in ids], src.rhs(ids[-1]),
                                             sp["lam"])
            tol = 2e-5 if sp.get("precision") == sl.SLIM_PREC_FP32 else 1e-12
            assert rel(bt.problems[i].get_x(), xo) < tol, (i, k)
    bt.close()
