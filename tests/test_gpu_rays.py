"""Random-ray blocks (2D) and the 3D streaming form against the FP64 oracle."""
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


def _ring_ids(sched, k, r, ell):
    want = np.full((r + 1) * ell, -1)
    for kk in range(max(1, k - r), k + 1):
        slot = (kk - 1) % (r + 1)
        want[slot * ell:(slot + 1) * ell] = sched[kk - 1]
    return want


def test_random_rays_2d_trajectory_and_gram(sl):
    N, V, D, ell, r, lam, seed = 24, 18, 35, 20, 3, 3e-2, 9
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(N, seed, 5), workloads.noise_direction(g.m, seed), 0.01)
    steps = 10
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, ell, r, lam, seed, kind=sl.SLIM_BLOCKS_RAYS)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-12, k
        if k == 6:
            ids, G, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, ell))
            M = joseph.rows(g, ids)
            Go = (M @ M.T).toarray()
            assert np.max(np.abs(G - Go)) <= 1e-13 * np.max(np.abs(Go))


def _small3d():
    N, V, Du, ell, r, lam, seed, spv = 16, 12, 23, 24, 2, 1e-2, 4, 3
    g = joseph.Geometry(N, V, Du, det_v=N, dim=3)
    b = np.random.default_rng(seed).standard_normal(g.m)
    return g, b, dict(N=N, V=V, Du=Du, ell=ell, r=r, lam=lam, seed=seed, spv=spv)


def test_streaming_3d_trajectory_fp64(sl):
    g, b, c = _small3d()
    steps = 9
    sched = list(oslim.streaming_ray_schedule(c["seed"], c["ell"], c["V"], c["Du"] * c["N"],
                                              c["spv"], steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, c["r"], c["lam"])]
    s = sl.Slim(c["N"], c["V"], c["Du"], c["ell"], c["r"], c["lam"], c["seed"], dim=3, det_v=c["N"],
                kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=c["spv"])
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        if k in (1, 4, 9):
            ids, _, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, c["r"], c["ell"]))
        assert rel(s.get_x(), xo) < 1e-12, k


def test_streaming_3d_single_step_fp32(sl):
    g, b, c = _small3d()
    steps = 8
    sched = list(oslim.streaming_ray_schedule(c["seed"], c["ell"], c["V"], c["Du"] * c["N"],
                                              c["spv"], steps))
    src = oslim.tomo_source(g, b)
    traj = [np.zeros(g.n)] + [x for _, x, _ in oslim.run(src, sched, c["r"], c["lam"])]
    s = sl.Slim(c["N"], c["V"], c["Du"], c["ell"], c["r"], c["lam"], c["seed"], dim=3, det_v=c["N"],
                kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=c["spv"], precision=1, use_graph=True)
    s.set_data(b)
    worst = 0.0
    for k in range(1, steps + 1):
        x32 = traj[k - 1].astype(np.float32)
        mem = sched[max(0, k - 1 - c["r"]):k]
        xo, _, _, _ = oslim.step_woodbury(x32.astype(np.float64), [src.rows(i) for i in mem],
                                          src.rhs(mem[-1]), c["lam"])
        s.set_x(x32)
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo))
    assert worst < 1e-5


def test_streaming_3d_full_size_first_steps(sl):
    # the 256^3 workload (360 views on a 256 x 368 detector, ell = 2048, r = 4):
    # the first two steps (p = 2048, 4096) are still within reach of the dense oracle
    cfg = workloads.C4
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det_u, det_v=cfg.det_v, dim=3)
    b = np.random.default_rng(cfg.seed).standard_normal(g.m)
    spv = 46
    sched = list(oslim.streaming_ray_schedule(cfg.seed, cfg.ell, cfg.n_views,
                                              cfg.det_u * cfg.det_v, spv, 2))
    src = oslim.RowSource(lambda ids: joseph.rows(g, ids), b, g.n)
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det_u, cfg.ell, cfg.r, cfg.lam, cfg.seed, dim=3,
                det_v=cfg.det_v, kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=spv)
    s.set_data(b)
    x = np.zeros(g.n)
    for k in (1, 2):
        mem = sched[:k]
        x, _, _, _ = oslim.step_woodbury(x, [src.rows(i) for i in mem], src.rhs(mem[-1]), cfg.lam)
        s.step(1)
        assert rel(s.get_x(), x) < 1e-11, k


def test_random_rays_2d_decaying_damping(sl):
    # the 1/k decay of the damping after step K, drawn by the random-ray sampler
    from oracle import comparators as cmp
    N, V, D, ell, r, lam, seed, K = 24, 18, 35, 20, 2, 3e-2, 10, 3
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(N, seed, 5), workloads.noise_direction(g.m, seed), 0.01)
    src = oslim.tomo_source(g, b)
    steps = 8
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps))
    x = np.zeros(g.n)
    for k in range(1, steps + 1):
        blocks = [src.rows(sched[j - 1]) for j in range(max(1, k - r), k + 1)]
        x, *_ = oslim.step_woodbury(x, blocks, src.rhs(sched[k - 1]), cmp.damping(lam, k, r, False, K))
    s = sl.Slim(N, V, D, ell, r, lam, seed, kind=sl.SLIM_BLOCKS_RAYS, decay_after=K)
    s.set_data(b)
    s.step(steps)
    assert rel(s.get_x(), x) < 1e-12
    s.close()


# The mapping the autotuner chooses for random-ray blocks: threads per ray of
# the march and scatter, and the pair Gram's cut-off between a thread per pair
# and the whole warp.  Only the order of floating-point sums changes.
@pytest.mark.parametrize("lanes,window", [(8, 16), (16, 64), (32, 8), (8, 256)])
def test_random_rays_2d_thread_mappings(sl, lanes, window):
    N, V, D, ell, r, lam, seed = 40, 24, 57, 37, 3, 2e-2, 12
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ workloads.phantom_2d(N, seed, 5), workloads.noise_direction(g.m, seed), 0.01)
    steps = 8
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, ell, r, lam, seed, kind=sl.SLIM_BLOCKS_RAYS, ray_lanes=lanes,
                pair_window=window)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-12, (lanes, window, k)
        if k == steps:
            ids, G, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, ell))
            M = joseph.rows(g, ids)
            Go = (M @ M.T).toarray()
            assert np.max(np.abs(G - Go)) <= 1e-13 * np.max(np.abs(Go))
    s.close()


@pytest.mark.parametrize("lanes", [8, 16])
def test_streaming_3d_thread_mappings(sl, lanes):
    g, b, c = _small3d()
    steps = 7
    sched = list(oslim.streaming_ray_schedule(c["seed"], c["ell"], c["V"], c["Du"] * c["N"],
                                              c["spv"], steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, c["r"], c["lam"])]
    s = sl.Slim(c["N"], c["V"], c["Du"], c["ell"], c["r"], c["lam"], c["seed"], dim=3, det_v=c["N"],
                kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=c["spv"], ray_lanes=lanes)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-12, (lanes, k)
    s.close()


def test_thread_mapping_argument_checks(sl):
    for kw in (dict(ray_lanes=12), dict(ray_lanes=64), dict(pair_window=4), dict(pair_window=300)):
        with pytest.raises(sl.SlimError) as ei:
            sl.Slim(24, 18, 35, 20, 2, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, **kw)
        assert ei.value.code == sl.SLIM_EINVAL, kw


def test_autotuner_picks_a_ray_mapping(sl):
    spec = dict(N=48, n_views=30, det=69, ell=64, r=2, lam=1e-2, seed=31, kind=sl.SLIM_BLOCKS_RAYS,
                precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED)
    best = sl.autotune_opts(spec, steps=2)
    assert best["tile"] in (32, 64) and best["ctas_per_sm"] in (1, 2, 3)
    assert best["ray_lanes"] in (8, 16, 32) and best["pair_window"] in (16, 32, 64)
    assert 0.0 < best["ms"] < 1e3
    again = sl.autotune_opts(spec, steps=2)          # the size class is cached
    assert again == best
    # the chosen options run
    s = sl.Slim(spec["N"], spec["n_views"], spec["det"], spec["ell"], spec["r"], spec["lam"],
                spec["seed"], precision=spec["precision"], solver=spec["solver"], kind=spec["kind"],
                tile=best["tile"], ctas_per_sm=best["ctas_per_sm"], ray_lanes=best["ray_lanes"],
                pair_window=best["pair_window"])
    s.set_data(np.zeros(spec["n_views"] * spec["det"], dtype=np.float32))
    s.step(4)
    s.sync()
    s.close()
