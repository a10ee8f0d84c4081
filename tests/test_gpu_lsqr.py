"""The LSQR inner solver (Eq. slimLSstep by LSQR, Sec. 4.2) on the GPU
against the float64 LSQR oracle: single steps from the oracle's iterate at
fixed iteration counts (the same iterates up to rounding), to a tolerance
(against the oracle at that tolerance and the Woodbury step), at 256x256,
with a float32 iterate, and the edge cases.

Element-wise parity at a fixed iteration count holds before LSQR loses the
orthogonality of its Lanczos vectors: on these windows a 1e-15 change of the
right-hand side moves the 8th iterate by about 1e-15 but the 30th of a
94-row window by 7e-7 and the 60th by 4e-3 (the float64 oracle against
itself), and the damped objective by up to 2e-4 there.  Counts beyond the
onset are therefore checked where the result is unique: converged to a
tolerance, against the oracle at that tolerance and the exact Woodbury step."""
import numpy as np
import pytest

import workloads
from oracle import joseph, lsqr as olsqr, slim as oslim, tik as otik

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


def _oracle_lsqr_step(g, src, seed, k, r, lam, x_prev, iters, tol=0.0, ramp=False):
    mem = oracle_memory(g, seed, k, r)
    blocks = [src.rows(ids) for _, _, ids in mem]
    lam_k = oslim.damping(lam, k, r, ramp)
    return olsqr.step_lsqr(x_prev, blocks, src.rhs(mem[-1][2]), lam_k, iters, tol)


def _ctx(sl, g, r, lam, seed, iters, tol, precision=0, **kw):
    return sl.Slim(g.N, g.n_views, g.det_u, g.det_u, r, lam, seed, precision=precision,
                   solver=sl.SLIM_SOLVE_LSQR, lsqr_max_iter=iters, lsqr_tol=tol, **kw)


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_fixed_iterations_match_the_oracle(sl, iters):
    g, b = _problem()
    src = oslim.tomo_source(g, b)
    r, lam, seed = 3, 1e-2, 7
    s = _ctx(sl, g, r, lam, seed, iters, 0.0)
    s.set_data(b)
    x_prev = np.zeros(g.n)
    for k in range(1, 8):
        xo, _, res = _oracle_lsqr_step(g, src, seed, k, r, lam, x_prev, iters)
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-11, (iters, k)
        it, nres, nres0 = s.lsqr_info()
        assert it == res.iters == iters
        assert abs(nres0 - res.normal_res0) <= 1e-12 * res.normal_res0
        assert abs(nres - res.normal_res) <= 1e-8 * res.normal_res0
        x_prev = xo
    s.close()


def test_tolerance_matches_the_oracle_and_the_woodbury_step(sl):
    g, b = _problem(seed=8)
    src = oslim.tomo_source(g, b)
    r, lam, seed, tol = 2, 1e-2, 8, 1e-10
    s = _ctx(sl, g, r, lam, seed, 20000, tol)
    s.set_data(b)
    x_prev = np.zeros(g.n)
    from _common import oracle_step_from
    for k in range(1, 7):
        xo, _, res = _oracle_lsqr_step(g, src, seed, k, r, lam, x_prev, 20000, tol)
        xw, _ = oracle_step_from(g, src, seed, k, r, lam, x_prev)
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        xg = s.get_x()
        it, nres, nres0 = s.lsqr_info()
        assert nres <= tol * nres0 and abs(it - res.iters) <= 2, (k, it, res.iters)
        assert rel(xg - x_prev, xo - x_prev) < 1e-8, k      # the steps s_k agree
        assert rel(xg - x_prev, xw - x_prev) < 1e-6, k      # and are the exact step
        x_prev = xw
    s.close()


def test_trajectory_with_the_damping_ramp(sl):
    # consecutive steps on the device (x never leaves it), ramped damping
    g, b = _problem(seed=9)
    src = oslim.tomo_source(g, b)
    r, lam, seed, iters = 2, 1e-2, 9, 8
    s = _ctx(sl, g, r, lam, seed, iters, 0.0, ramp=True)
    s.set_data(b)
    x = np.zeros(g.n)
    for k in range(1, 10):
        x, _, _ = _oracle_lsqr_step(g, src, seed, k, r, lam, x, iters, ramp=True)
    s.step(9)
    assert rel(s.get_x(), x) < 1e-10
    s.close()


def test_single_steps_at_256(sl):
    cfg = workloads.C2
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = workloads.add_noise(joseph.full_matrix(g) @ x_true, e, cfg.noise)
    src = oslim.tomo_source(g, b)
    iters = 10
    s = _ctx(sl, g, cfg.r, cfg.lam, cfg.seed, iters, 0.0)
    s.set_data(b)
    x_prev = np.zeros(g.n)
    for k in range(1, 8):
        xo, _, _ = _oracle_lsqr_step(g, src, cfg.seed, k, cfg.r, cfg.lam, x_prev, iters)
        if k in (1, 2, 6, 7):
            s.set_x(x_prev)
            s.set_iter(k - 1)
            s.step(1)
            # 10 iterations: a 1e-15 change of c moves the oracle's x_k by
            # ~1e-15 here (by 1e-8 to 4e-8 at 20 iterations on the 2,178-row
            # windows of steps 6 and 7)
            assert rel(s.get_x(), xo) < 1e-11, k
        x_prev = xo
    s.close()


def test_float32_iterate(sl):
    g, b = _problem(N=40, V=30, D=57, seed=10)
    src = oslim.tomo_source(g, b)
    r, lam, seed, iters = 4, 1e-2, 10, 8
    s = _ctx(sl, g, r, lam, seed, iters, 0.0, precision=1)
    s.set_data(b.astype(np.float32))
    x_prev = np.zeros(g.n)
    worst = 0.0
    for k in range(1, 9):
        xo, _, _ = _oracle_lsqr_step(g, src, seed, k, r, lam, x_prev, iters)
        x32 = x_prev.astype(np.float32).astype(np.float64)
        xo32, _, _ = _oracle_lsqr_step(g, src, seed, k, r, lam, x32, iters)
        s.set_x(x_prev.astype(np.float32))
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo32))
        x_prev = xo
    assert worst < 1e-5
    s.close()


def test_zero_residual_leaves_x(sl):
    # b = 0 and x = 0: r_k = A_k 0 - 0 is exactly zero, so c = 0, s = 0 and
    # no iteration runs
    g, _ = _problem(seed=11)
    s = _ctx(sl, g, 2, 1e-2, 11, 10, 0.0)
    s.set_data(np.zeros(g.m))
    s.set_x(np.zeros(g.n))
    s.step(3)
    assert s.lsqr_info()[0] == 0
    assert not s.get_x().any()
    s.close()


def test_unsupported_and_invalid(sl):
    g, _ = _problem()
    with pytest.raises(sl.SlimError):   # no iterations
        _ctx(sl, g, 2, 1e-2, 1, 0, 0.0)
    with pytest.raises(sl.SlimError):   # negative tolerance
        _ctx(sl, g, 2, 1e-2, 1, 10, -1.0)
    with pytest.raises(sl.SlimError):   # pipelined form
        _ctx(sl, g, 2, 1e-2, 1, 10, 0.0, lookahead=2)
    with pytest.raises(sl.SlimError):   # random-ray blocks
        sl.Slim(g.N, g.n_views, g.det_u, 20, 2, 1e-2, 1, solver=sl.SLIM_SOLVE_LSQR,
                lsqr_max_iter=10, kind=sl.SLIM_BLOCKS_RAYS)
    with pytest.raises(sl.SlimError):   # stored matrix
        _ctx(sl, g, 2, 1e-2, 1, 10, 0.0, a_mode=sl.A_CSR_F32)
    s = _ctx(sl, g, 2, 1e-2, 1, 10, 0.0)
    s.set_data(np.zeros(g.m))
    s.step(1)
    ids, G, z = None, None, None
    with pytest.raises(sl.SlimError):   # LSQR keeps no Gram matrix
        s.get_memory()
    s.close()
    wb = sl.Slim(g.N, g.n_views, g.det_u, g.det_u, 2, 1e-2, 1)
    with pytest.raises(sl.SlimError):   # not an LSQR context
        wb.lsqr_info()
    wb.close()


def _tik_problem(sl, iters, tol, seed=12, lam_tik=0.8, reading=0):
    g, b = _problem(seed=seed)
    src = oslim.tomo_source(g, b)
    r, lam = 3, 1e-2
    cdiag = 0.5 + 1.5 * np.random.default_rng(seed).random(g.n)
    s = _ctx(sl, g, r, lam, seed, iters, tol, tik_lambda=lam_tik, tik_reading=reading)
    s.set_data(b)
    s.set_c_diag(cdiag)
    return g, b, src, r, lam, cdiag, s


@pytest.mark.parametrize("iters", [3, 8])
def test_slimtik_fixed_iterations_match_the_oracle(sl, iters):
    # slimTik with C_k = diag(c) by LSQR on the column-scaled window
    g, b, src, r, lam, cdiag, s = _tik_problem(sl, iters, 0.0)
    lam_tik = 0.8
    x_prev = np.random.default_rng(2).standard_normal(g.n) * 0.05
    for k in range(1, 7):
        mem = oracle_memory(g, 12, k, r)
        blocks = [src.rows(ids) for _, _, ids in mem]
        xo, _, res = olsqr.step_tik_lsqr(x_prev, blocks, src.rhs(mem[-1][2]),
                                         oslim.damping(lam, k, r, False), lam_tik, g.n_views,
                                         otik.window_count(k, r), cdiag, iters)
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        assert rel(s.get_x(), xo) < 1e-11, (iters, k)
        assert s.lsqr_info()[0] == res.iters
        x_prev = xo
    s.close()


def test_slimtik_converged_is_the_woodbury_step(sl):
    g, b, src, r, lam, cdiag, s = _tik_problem(sl, 20000, 1e-10, seed=13, lam_tik=1.1)
    x_prev = np.zeros(g.n)
    for k in range(1, 6):
        mem = oracle_memory(g, 13, k, r)
        blocks = [src.rows(ids) for _, _, ids in mem]
        xw, *_ = otik.step_woodbury(x_prev, blocks, src.rhs(mem[-1][2]),
                                    oslim.damping(lam, k, r, False), 1.1, g.n_views,
                                    otik.window_count(k, r), np.sqrt(cdiag))
        s.set_x(x_prev)
        s.set_iter(k - 1)
        s.step(1)
        assert rel(s.get_x() - x_prev, xw - x_prev) < 1e-6, k
        x_prev = xw
    s.set_timing(True)
    s.step(1)
    assert s.get_timing()[1] == 4     # sample, march, slimTik right-hand side, LSQR
    s.close()
