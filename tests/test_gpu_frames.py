"""3D with views from random directions (Sec. 4.3's geometry) on the GPU
against the float64 oracle: A x and A^T y over every ray, the Gram matrix of
the window from the voxel lists, trajectories of random-ray and streaming
blocks, single steps from the oracle's iterate (float64 and the float32 form),
and the argument checks."""
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


def _geom(N=14, V=9, Du=21, Dv=19, seed=3):
    fr = workloads.random_frames(V, seed)
    return joseph.Geometry(N, V, Du, Dv, dim=3, frames=fr), fr


def _data(g, seed):
    x = workloads.phantom_3d(g.N, seed, 6)
    A = joseph.full_matrix(g)
    return A, workloads.add_noise(A @ x, workloads.noise_direction(g.m, seed), 0.01)


def _ctx(sl, g, fr, ell, r, lam, seed, **kw):
    return sl.Slim(g.N, g.n_views, g.det_u, ell, r, lam, seed, dim=3, det_v=g.det_v,
                   kind=kw.pop("kind", sl.SLIM_BLOCKS_RAYS), frames=fr, **kw)


def _ring_ids(sched, k, r, ell):
    want = np.full((r + 1) * ell, -1)
    for kk in range(max(1, k - r), k + 1):
        slot = (kk - 1) % (r + 1)
        want[slot * ell:(slot + 1) * ell] = sched[kk - 1]
    return want


def test_projections_match_the_oracle_rows(sl):
    g, fr = _geom()
    A = joseph.full_matrix(g)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(g.n)
    y = rng.standard_normal(g.m)
    s = _ctx(sl, g, fr, 16, 1, 1e-2, 1)
    xt = torch.tensor(x, device="cuda")
    yt = torch.zeros(g.m, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()   # inputs filled on torch's stream; the projections
    s.project(xt, yt)          # run on the context's own stream
    s.sync()
    want = A @ x
    assert np.abs(yt.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()
    bt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    yd = torch.tensor(y, device="cuda")
    torch.cuda.synchronize()
    s.backproject(yd, bt)
    s.sync()
    want = A.T @ y
    assert np.abs(bt.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()
    # a subset of rays by id
    ids = torch.tensor([0, 5, g.m - 1, 77, 5], dtype=torch.int32, device="cuda")
    ys = torch.zeros(5, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s.project(xt, ys, ids)
    s.sync()
    assert np.abs(ys.cpu().numpy() - (A @ x)[[0, 5, g.m - 1, 77, 5]]).max() <= 1e-13 * np.abs(
        A @ x).max()
    s.close()


@pytest.mark.parametrize("solver", ["fp64", "mixed"])
def test_random_rays_trajectory_and_gram(sl, solver):
    g, fr = _geom(seed=4)
    A, b = _data(g, 4)
    ell, r, lam, seed, steps = 30, 2, 3e-2, 4, 9
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = _ctx(sl, g, fr, ell, r, lam, seed, refine_iters=3,
             solver=sl.SLIM_SOLVE_MIXED if solver == "mixed" else sl.SLIM_SOLVE_FP64)
    s.set_data(b)
    for k, xo in enumerate(traj, start=1):
        s.step(1)
        assert rel(s.get_x(), xo) < (1e-12 if solver == "fp64" else 1e-9), k
        if k == 5:
            ids, G, _ = s.get_memory()
            assert np.array_equal(ids, _ring_ids(sched, k, r, ell))
            M = joseph.rows(g, ids)
            Go = (M @ M.T).toarray()
            assert np.max(np.abs(G - Go)) <= 1e-13 * np.max(np.abs(Go))
            assert np.count_nonzero(Go) < Go.size    # rays that share no voxel
    s.close()


def test_streaming_trajectory(sl):
    g, fr = _geom(N=12, V=8, Du=18, Dv=17, seed=5)
    A, b = _data(g, 5)
    ell, r, lam, seed, spv, steps = 25, 3, 1e-2, 5, 2, 12
    sched = list(oslim.streaming_ray_schedule(seed, ell, g.n_views, g.rays_per_view, spv, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam, ramp=True)]
    s = _ctx(sl, g, fr, ell, r, lam, seed, kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=spv,
             ramp=True, use_graph=True)
    s.set_data(b)
    s.step(steps)
    assert rel(s.get_x(), traj[-1]) < 1e-11
    s.close()


def test_single_steps_float32(sl):
    g, fr = _geom(N=16, V=10, Du=24, Dv=24, seed=6)
    A, b = _data(g, 6)
    src = oslim.tomo_source(g, b)
    ell, r, lam, seed = 40, 3, 1e-2, 6
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, 8))
    s = _ctx(sl, g, fr, ell, r, lam, seed, precision=1, solver=sl.SLIM_SOLVE_MIXED)
    s.set_data(b.astype(np.float32))
    x = np.zeros(g.n)
    worst = 0.0
    for k in range(1, 9):
        blocks = [src.rows(sched[j - 1]) for j in range(max(1, k - r), k + 1)]
        x32 = x.astype(np.float32).astype(np.float64)
        xo, *_ = oslim.step_woodbury(x32, blocks, src.rhs(sched[k - 1]), lam)
        s.set_x(x.astype(np.float32))
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo))
        x = xo
    assert worst < 1e-5
    s.close()


def test_arguments(sl):
    g, fr = _geom()
    bad = fr.copy()
    bad[2, 3:6] *= 1.01                  # u not unit length
    with pytest.raises(sl.SlimError):
        _ctx(sl, g, bad, 16, 1, 1e-2, 1)
    with pytest.raises(sl.SlimError):    # view blocks
        sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 1, 1e-2, 1, dim=3, det_v=g.det_v, frames=fr)
    with pytest.raises(sl.SlimError):    # frames in 2D
        sl.Slim(g.N, g.n_views, g.det_u, 16, 1, 1e-2, 1, kind=sl.SLIM_BLOCKS_RAYS, frames=fr)
    with pytest.raises(sl.SlimError):    # the LSQR form
        _ctx(sl, g, fr, 16, 1, 1e-2, 1, solver=sl.SLIM_SOLVE_LSQR, lsqr_max_iter=5)
    s = _ctx(sl, g, fr, 16, 1, 1e-2, 1)
    s.set_timing(True)
    s.set_data(np.zeros(g.m))
    s.step(1)
    assert s.get_timing()[1] >= 6         # sample, march, Gram, K, factor, solves, scatter
    s.close()


def test_rays_missing_the_volume(sl):
    # a detector much wider than the volume's shadow: many rays cross no voxel
    # (zero rows of A, zero Gram rows and columns)
    N = 8
    fr = workloads.random_frames(6, 7)
    g = joseph.Geometry(N, 6, 30, 28, dim=3, frames=fr)
    A, b = _data(g, 7)
    empty = np.diff(A.indptr) == 0
    assert empty.mean() > 0.3
    ell, r, lam, seed, steps = 40, 2, 1e-2, 7, 8
    sched = list(oslim.random_ray_schedule(seed, ell, g.m, steps))
    traj = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)]
    s = _ctx(sl, g, fr, ell, r, lam, seed)
    s.set_data(b)
    s.step(steps)
    assert rel(s.get_x(), traj[-1]) < 1e-12
    s.close()


def test_projection_at_full_size_on_sampled_rays(sl):
    # the bench's geometry (256^3, 360 directions, 368 x 368 detector): A x on
    # 300 sampled rays against the oracle's rows, one by one
    cfg = workloads.C4R
    fr = workloads.random_frames(cfg.n_views, cfg.seed)
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det_u, cfg.det_v, dim=3, frames=fr)
    rng = np.random.default_rng(17)
    ids = np.sort(rng.choice(g.m, 300, replace=False)).astype(np.int32)
    x = rng.standard_normal(g.n)
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det_u, cfg.ell, cfg.r, cfg.lam, cfg.seed, dim=3,
                det_v=cfg.det_v, kind=sl.SLIM_BLOCKS_STREAM, steps_per_view=46, frames=fr)
    xt = torch.tensor(x, device="cuda")
    yt = torch.zeros(len(ids), dtype=torch.float64, device="cuda")
    idt = torch.tensor(ids, device="cuda")
    torch.cuda.synchronize()   # inputs filled on torch's stream; the projection
    s.project(xt, yt, idt)     # runs on the context's own stream
    s.sync()
    got = yt.cpu().numpy()
    for i, ray in enumerate(ids):
        idx, w = joseph.ray_taps(g, int(ray))
        want = float(w @ x[idx])
        assert abs(got[i] - want) <= 1e-12 * max(1.0, float(np.abs(w).sum())), int(ray)
    s.close()
