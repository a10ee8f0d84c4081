"""slimTik on the GPU (Eq. slimTik, C_k = diag(c), Woodbury form) against the
float64 slimTik oracle: single steps from the oracle's iterate, trajectories on
the device with both readings of the Tikhonov count and the damping ramp, the
256x256 workload, the float32 iterate, graph replay, a change of C_k after
steps, the full-memory identity on the GPU's own iterates, and the argument
checks."""
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


def _problem(N=32, V=20, D=47, seed=7):
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    return g, b


def _cdiag(n, seed):
    return 0.5 + 1.5 * np.random.default_rng(seed).random(n)


def _oracle_step(g, src, seed, k, r, lam, lam_tik, x_prev, c=None, ramp=False, reading="window",
                 eta=1.0):
    mem = oracle_memory(g, seed, k, r)
    blocks = [src.rows(ids) for _, _, ids in mem]
    lam_k = oslim.damping(lam, k, r, ramp)
    cnt = otik.window_count(k, r, reading)
    l = None if c is None else np.sqrt(c)
    x, *_ = otik.step_woodbury(x_prev, blocks, src.rhs(mem[-1][2]), lam_k, lam_tik, g.n_views,
                               cnt, l, eta)
    return x


@pytest.mark.parametrize("reading", [0, 1])
def test_single_steps_match_the_oracle(sl, reading):
    g, b = _problem()
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 3, 1e-2, 0.7, 7
    c = _cdiag(g.n, 1)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik,
                tik_reading=reading)
    s.set_data(b)
    s.set_c_diag(c)
    x_prev = np.random.default_rng(2).standard_normal(g.n) * 0.05
    rd = ("window", "printed")[reading]
    for k in range(1, 9):
        xo = _oracle_step(g, src, seed, k, r, lam, lam_tik, x_prev, c, reading=rd)
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-11, k
        x_prev = xo
    s.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_trajectory_with_the_ramp(sl, use_graph):
    g, b = _problem(seed=8)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed, eta = 2, 1e-2, 1.3, 8, 0.8
    c = _cdiag(g.n, 3)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik, ramp=True,
                eta=eta, use_graph=use_graph)
    s.set_data(b)
    s.set_c_diag(c)
    x = np.zeros(g.n)
    for k in range(1, 13):
        x = _oracle_step(g, src, seed, k, r, lam, lam_tik, x, c, ramp=True, eta=eta)
    s.step(12)
    assert rel(s.get_x(), x) < 1e-10
    s.close()


def test_identity_c_and_no_tikhonov_rows(sl):
    # tik_lambda > 0 with C = I; and C = diag(c) with tik_lambda = 0 (slimLS
    # with a diagonal C_k, Eq. B_k)
    g, b = _problem(seed=9)
    src = oslim.tomo_source(g, b)
    r, lam, seed = 2, 1e-2, 9
    c = _cdiag(g.n, 4)
    for lam_tik, cd in ((0.9, None), (0.0, c)):
        s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
        s.set_data(b)
        if cd is not None:
            s.set_c_diag(cd)
        x = np.zeros(g.n)
        for k in range(1, 8):
            x = _oracle_step(g, src, seed, k, r, lam, lam_tik, x, cd)
        s.step(7)
        assert rel(s.get_x(), x) < 1e-10, lam_tik
        s.close()


def test_changing_c_rebuilds_the_memory(sl):
    g, b = _problem(seed=10)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 3, 1e-2, 0.6, 10
    c = _cdiag(g.n, 5)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
    s.set_data(b)
    s.step(3)                     # C = I
    s.set_c_diag(c)               # the three retained blocks' Gram entries change
    s.step(3)
    x = np.zeros(g.n)
    for k in range(1, 7):
        x = _oracle_step(g, src, seed, k, r, lam, lam_tik, x, None if k <= 3 else c)
    assert rel(s.get_x(), x) < 1e-10
    s.set_c_diag(None)            # back to C = I
    s.step(1)
    x = _oracle_step(g, src, seed, 7, r, lam, lam_tik, x, None)
    assert rel(s.get_x(), x) < 1e-10
    s.close()


def test_full_memory_identity_on_the_gpu_iterates(sl):
    # r >= k-1: (lambda C + k beta C + sum A_i^T A_i) x_k = lambda C x_0 +
    # sum A_i^T b_i for the blocks the GPU drew (any sample sequence)
    g, b = _problem(N=16, V=12, D=23, seed=11)
    A = joseph.full_matrix(g)
    r, lam, lam_tik, seed = 9, 3e-2, 0.8, 11
    c = _cdiag(g.n, 6)
    x0 = np.random.default_rng(7).standard_normal(g.n) * 0.1
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
    s.set_data(b)
    s.set_c_diag(c)
    s.set_x(x0)
    beta = lam_tik ** 2 / g.n_views
    H = np.zeros((g.n, g.n))
    rhs = lam * c * x0
    for k in range(1, r + 2):
        s.step(1)
        ids = oslim.view_block_ids(g, seed, k)
        Ak = A[ids].toarray()
        H += Ak.T @ Ak
        rhs = rhs + Ak.T @ b[ids]
        xk = s.get_x()
        lhs = (lam + k * beta) * c * xk + H @ xk
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs), k
    s.close()


@pytest.mark.parametrize("lookahead,solver", [(2, "fp64"), (6, "mixed")])
def test_pipelined_form(sl, lookahead, solver):
    # the factored matrix mu_k I + M_k C^{-1} M_k^T is prepared up to D steps
    # ahead; the right-hand side and the update take x when the step runs
    g, b = _problem(seed=15)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 3, 1e-2, 0.8, 15
    c = _cdiag(g.n, 16)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik, ramp=True,
                lookahead=lookahead, refine_iters=3,
                solver=sl.SLIM_SOLVE_MIXED if solver == "mixed" else sl.SLIM_SOLVE_FP64)
    s.set_data(b)
    s.step(2)                     # C = I, two steps (and D more prepared)
    s.set_c_diag(c)               # prepared again with the new C
    s.step(8)
    x = np.zeros(g.n)
    for k in range(1, 11):
        x = _oracle_step(g, src, seed, k, r, lam, lam_tik, x, None if k <= 2 else c, ramp=True)
    # float32 factor: each of the 1 + 3 solves leaves about kappa(K) u_32 ~ 1e-3
    # of the error of the one before (kappa ~ 1e4 here)
    tol = 1e-10 if solver == "fp64" else 1e-8
    assert rel(s.get_x(), x) < tol
    s.close()


def test_single_steps_at_256(sl):
    cfg = workloads.C2
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = workloads.add_noise(joseph.full_matrix(g) @ x_true, e, cfg.noise)
    src = oslim.tomo_source(g, b)
    lam_tik = 2.0
    c = _cdiag(g.n, 12)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, cfg.r, cfg.lam, cfg.seed, tik_lambda=lam_tik)
    s.set_data(b)
    s.set_c_diag(c)
    x_prev = np.zeros(g.n)
    for k in range(1, 8):
        xo = _oracle_step(g, src, cfg.seed, k, cfg.r, cfg.lam, lam_tik, x_prev, c)
        if k in (1, 2, 6, 7):
            s.set_x(x_prev)
            s.set_iter(k - 1)
            s.step(1)
            assert rel(s.get_x(), xo) < 1e-10, k
        x_prev = xo
    s.close()


@pytest.mark.parametrize("solver", ["fp64", "mixed"])
def test_float32_iterate(sl, solver):
    g, b = _problem(N=40, V=30, D=57, seed=13)
    src = oslim.tomo_source(g, b)
    r, lam, lam_tik, seed = 4, 1e-2, 0.9, 13
    c = _cdiag(g.n, 14)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, precision=1, tik_lambda=lam_tik,
                solver=sl.SLIM_SOLVE_MIXED if solver == "mixed" else sl.SLIM_SOLVE_FP64)
    s.set_data(b.astype(np.float32))
    s.set_c_diag(c.astype(np.float32))
    c32 = c.astype(np.float32).astype(np.float64)
    x_prev = np.zeros(g.n)
    worst = 0.0
    for k in range(1, 9):
        x32 = x_prev.astype(np.float32).astype(np.float64)
        xo = _oracle_step(g, src, seed, k, r, lam, lam_tik, x32, c32)
        s.set_x(x_prev.astype(np.float32))
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo))
        x_prev = xo
    assert worst < 1e-5
    s.close()


def test_kernels_per_step(sl):
    g, b = _problem()
    s0 = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1)
    s1 = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=0.5)
    counts = []
    for s in (s0, s1):
        s.set_data(b)
        s.set_timing(True)
        s.step(1)
        counts.append(s.get_timing()[1])
        s.close()
    assert counts[1] == counts[0] + 2


def test_unsupported_and_invalid(sl):
    g, b = _problem()
    with pytest.raises(sl.SlimError):   # negative lam_tik
        sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=-1.0)
    with pytest.raises(sl.SlimError):   # unknown reading
        sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=1.0, tik_reading=2)
    with pytest.raises(sl.SlimError):   # random-ray blocks
        sl.Slim(g.N, g.n_views, g.det_u, 20, 2, 1e-2, 1, tik_lambda=1.0, kind=sl.SLIM_BLOCKS_RAYS)
    s = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1, tik_lambda=1.0)
    s.set_data(b)
    bad = np.ones(g.n)
    bad[17] = 0.0
    with pytest.raises(sl.SlimError):   # C not positive definite
        s.set_c_diag(bad)
    with pytest.raises(sl.SlimError):   # wrong length
        s.set_c_diag(np.ones(g.n - 1))
    s.close()
    sg = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 0, 10.0, 1, solver=sl.SLIM_SOLVE_SG)
    with pytest.raises(sl.SlimError):   # the comparators take C = I only
        sg.set_c_diag(np.ones(g.n))
    sg.close()


def test_checkpoint_and_restore(sl):
    # a context restored from a checkpoint (x, k) with the same options and C
    # continues the trajectory (the memory is rebuilt with C)
    g, b = _problem(seed=16)
    r, lam, lam_tik, seed = 2, 1e-2, 0.7, 16
    c = _cdiag(g.n, 17)
    a = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
    a.set_data(b)
    a.set_c_diag(c)
    a.step(5)
    blob = a.checkpoint()
    a.step(4)
    want = a.get_x()
    a.close()
    d = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, tik_lambda=lam_tik)
    d.set_data(b)
    d.set_c_diag(c)
    d.restore(blob)
    d.step(4)
    assert rel(d.get_x(), want) < 1e-12
    d.close()
