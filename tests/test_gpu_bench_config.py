"""The launch configuration the bench times, at the bench's own size, against
the float64 oracle (Eq. ram / Eq. B_k).

The headline runs the 256 x 256 workload (p = 2178) pipelined: the geometry
chain six steps ahead of the iterate chain, the extended ring of r+1+D slots,
D+1 factor buffers, the window factored in chronological order with the
short first forward sweep, one persistent-factorisation CTA per SM shared by
the factorisations in flight, CUDA graphs.  These tests run exactly that
context for more than r+1+D steps, so that the extended ring and the factor
buffers wrap, and compare sampled steps element-wise with the oracle's step
taken from the GPU's own previous iterate:

  float32 form (float32 factor + 2 float64-residual refinements): 1e-5
  float64 form (float64 factor, same pipeline):                     1e-12

They also compare the memory (ring ids, exact) and the Gram matrix of the
window (1e-13 of its largest entry) with the oracle's, and run the mixed
solver at lambda = 1e-4, where kappa(lambda I + G) is about 1e7.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import joseph, slim as oslim

from _common import oracle_memory, oracle_step_from, rel, tomo_problem

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
              pytest.mark.usefixtures("torch_side_stream")]

LOOKAHEAD = 6


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


@pytest.fixture(scope="module")
def c2():
    return tomo_problem(workloads.C2)


def _context(sl, cfg, form, refine_iters=2, **kw):
    """The bench's chosen form (`mixed`) or the same pipeline with the float64
    factor (`fp64`), on torch's current stream."""
    common = dict(lookahead=LOOKAHEAD, ctas_per_sm=1, use_graph=True)
    common.update(kw)
    if form == "mixed":
        s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.det, cfg.r, cfg.lam, cfg.seed,
                    precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED,
                    refine_iters=refine_iters, **common)
    else:
        s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.det, cfg.r, cfg.lam, cfg.seed,
                    precision=sl.SLIM_PREC_FP64, solver=sl.SLIM_SOLVE_FP64, **common)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    return s


def _check_memory(s, g, seed, k, r):
    ids, G, _ = s.get_memory()
    want = np.full(s.p, -1)
    for _, slot, rows in oracle_memory(g, seed, k, r):
        want[slot * g.det_u:(slot + 1) * g.det_u] = rows
    assert np.array_equal(ids, want), k
    M = joseph.rows(g, want)
    Go = (M @ M.T).toarray()
    assert np.max(np.abs(G - Go)) <= 1e-13 * np.max(np.abs(Go)), k


def _run_sampled(s, g, b, cfg, steps, check, tol, mem_at=()):
    src = oslim.tomo_source(g, b)
    worst = 0.0
    for k in range(1, steps + 1):
        x_prev = s.get_x() if k in check else None     # synchronises every stream
        s.step(1)
        if k in check:
            xo, _ = oracle_step_from(g, src, cfg.seed, k, cfg.r, cfg.lam, x_prev)
            e = rel(s.get_x(), xo)
            worst = max(worst, e)
            assert e < tol, (k, e)
        if k in mem_at:
            _check_memory(s, g, cfg.seed, k, cfg.r)
    return worst


@pytest.mark.parametrize("form,tol", [("mixed", 1e-5), ("fp64", 1e-12)])
def test_bench_configuration_at_full_size(sl, c2, form, tol):
    cfg = workloads.C2
    g, _, _, b = c2
    s = _context(sl, cfg, form)
    s.set_data(b.astype(np.float32) if form == "mixed" else b)
    steps = cfg.r + 1 + LOOKAHEAD + 4            # the extended ring (12 slots) wraps
    check = {1, 2, 6, 7, 12, 13, 14, 15, 16}
    _run_sampled(s, g, b, cfg, steps, check, tol, mem_at=(7, 13, 16))
    assert s.get_iter() == steps
    s.close()


def test_mixed_solver_at_lambda_1e4(sl):
    # a problem of the batched mix's range: 128 x 128, 90 views x 182 bins,
    # r = 8 (p = 1638), lambda = 1e-4, pipelined as the bench runs it.  Each
    # refinement round shrinks the error by about kappa * u32 (0.66 here
    # against 0.09 at the 256 x 256 workload): two rounds leave 1.3e-5 at
    # k = 9, three reach the float32 floor
    cfg = workloads.Tomo2D("mixed-1e-4", N=128, n_views=90, det=182, ell=182, r=8, lam=1e-4,
                           seed=5)
    g, _, _, b = tomo_problem(cfg)
    k = cfg.r + 3
    ids = np.concatenate([rows for _, _, rows in oracle_memory(g, cfg.seed, k, cfg.r)])
    M = joseph.rows(g, ids)
    ev = sla.eigvalsh((M @ M.T).toarray() + cfg.lam * np.eye(M.shape[0]))
    kappa = ev[-1] / ev[0]
    assert kappa > 5e6, kappa        # kappa * u32 about 0.66: refinement still contracts
    s = _context(sl, cfg, "mixed", refine_iters=3)
    s.set_data(b.astype(np.float32))
    worst = _run_sampled(s, g, b, cfg, 14, {1, 5, 9, 11, 14}, 1e-5)
    assert worst < 1e-5, (worst, kappa)
    s.close()
