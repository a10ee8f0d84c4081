"""Block sampling without replacement against the float64 oracle.

  cyclic view blocks (the random cyclic order of Sec. 4.3's walnut
  experiment: a fresh permutation of the views per epoch), in the one-chain
  and the pipelined form, and with_replacement = 0 on view blocks (the same
  order);
  random-ray blocks of distinct rays (Floyd's algorithm), 2D and the 3D
  streaming form.

The ring ids are compared exactly (the samplers are integer work on both
sides) and the iterates at the float64 tolerance, 1e-12.
"""
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


def _problem(N=32, V=20, D=47, seed=7):
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    return g, b


def _ring_ids(sched, k, r, ell):
    want = np.full((r + 1) * ell, -1)
    for kk in range(max(1, k - r), k + 1):
        slot = (kk - 1) % (r + 1)
        want[slot * ell:(slot + 1) * ell] = sched[kk - 1]
    return want


@pytest.mark.parametrize("lookahead,opts", [(0, dict(cyclic=True)),
                                            (0, dict(with_replacement=False)),
                                            (3, dict(cyclic=True))])
def test_cyclic_view_blocks_trajectory(sl, lookahead, opts):
    g, b = _problem()
    r, lam, seed = 3, 1e-2, 7
    steps = 2 * g.n_views + 5           # three epochs: the permutation changes twice
    sched = list(oslim.view_schedule(g, seed, steps, cyclic=True))
    views = [int(ids[0]) // g.det_u for ids in sched]
    for e in range(2):                  # every view once per epoch
        assert sorted(views[e * g.n_views:(e + 1) * g.n_views]) == list(range(g.n_views))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, use_graph=True,
                lookahead=lookahead, **opts)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        if k in (3, g.n_views + 1, 2 * g.n_views + 4):
            ids, _, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, g.det_u)), k
        if k % 7 == 0 or k == steps:
            assert rel(s.get_x(), xo) < 1e-12, k
    s.close()


def test_cyclic_restore_mid_epoch(sl):
    # the permutation is recomputed from the step counter after a jump
    g, b = _problem(seed=8)
    r, lam, seed = 2, 1e-2, 8
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, cyclic=True)
    s.set_data(b)
    s.step(g.n_views + 6)
    blob = s.checkpoint()
    s.step(g.n_views)
    xa = s.get_x()
    s2 = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, cyclic=True)
    s2.set_data(b)
    s2.restore(blob)
    s2.step(g.n_views)
    assert rel(s2.get_x(), xa) < 1e-12
    sched = list(oslim.view_schedule(g, seed, 2 * g.n_views + 6, cyclic=True))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    assert rel(xa, traj[-1]) < 1e-12
    s.close()
    s2.close()


def test_distinct_random_rays_2d(sl):
    N, V, D, ell, r, lam, seed = 24, 18, 35, 40, 3, 3e-2, 9
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    steps = 10
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps, distinct=True))
    assert all(len(set(ids.tolist())) == ell for ids in sched)
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, D, ell, r, lam, seed, kind=sl.SLIM_BLOCKS_RAYS, with_replacement=False)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        if k in (1, 5, 10):
            ids, _, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, ell)), k
        assert rel(s.get_x(), xo) < 1e-12, k
    s.close()


def test_distinct_rays_at_the_largest_block(sl):
    # ell = 2048 distinct rays, the sampler's largest block (its hash set at
    # half load), out of the 8,190 rays of a 64 x 64, 90 x 91 geometry; ids only
    N, V, D, ell, seed = 64, 90, 91, 2048, 11
    s = sl.Slim(N, V, D, ell, 0, 1e-2, seed, kind=sl.SLIM_BLOCKS_RAYS, with_replacement=False)
    s.set_data(np.zeros(V * D))
    for k in range(1, 4):
        s.step(1)
        ids, _, _ = s.get_memory()
        assert np.array_equal(ids, np.array(rng.distinct_rays(seed, k, ell, V * D))), k
    s.close()


def test_distinct_streaming_3d_trajectory(sl):
    N, V, Du, ell, r, lam, seed, spv = 16, 12, 23, 24, 2, 1e-2, 4, 3
    g = joseph.Geometry(N, V, Du, det_v=N, dim=3)
    b = np.random.default_rng(seed).standard_normal(g.m)
    steps = 9
    sched = list(oslim.streaming_ray_schedule(seed, ell, V, Du * N, spv, steps, distinct=True))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = sl.Slim(N, V, Du, ell, r, lam, seed, dim=3, det_v=N, kind=sl.SLIM_BLOCKS_STREAM,
                steps_per_view=spv, with_replacement=False)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        if k in (1, 9):
            ids, _, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, ell)), k
        assert rel(s.get_x(), xo) < 1e-12, k
    s.close()


def test_sampling_argument_checks(sl):
    with pytest.raises(sl.SlimError) as ei:      # random rays have no epoch order
        sl.Slim(24, 18, 35, 20, 2, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, cyclic=True)
    assert ei.value.code == sl.SLIM_ENOTSUP
    with pytest.raises(sl.SlimError) as ei:      # more distinct rays than the problem has
        sl.Slim(8, 2, 5, 11, 0, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, with_replacement=False)
    assert ei.value.code == sl.SLIM_EINVAL
    with pytest.raises(sl.SlimError) as ei:      # above the sampler's block size
        sl.Slim(64, 90, 91, 2049, 0, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, with_replacement=False)
    assert ei.value.code == sl.SLIM_ENOTSUP
