"""Stored-matrix variant (float32 / bfloat16 CSR of A) against the oracle on the same A."""
import numpy as np
import pytest

import workloads
from oracle import csr, joseph, slim as oslim

from _common import rel, tomo_problem

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
              pytest.mark.usefixtures("torch_side_stream")]

KIND_MODE = {"f32": 1, "bf16": 2}


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


@pytest.fixture(scope="module")
def c1():
    return tomo_problem(workloads.C1)


def _make(sl, cfg, kind, **kw):
    """Context on torch's current stream (a side stream, see conftest), so
    that its passes are ordered with the tensors the tests fill and read."""
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.det, cfg.r, cfg.lam, cfg.seed,
                precision=kw.pop("precision", 1), solver=kw.pop("solver", 1),
                a_mode=KIND_MODE[kind], **kw)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    return s


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_stored_matrix_is_the_oracle_matrix(sl, c1, kind):
    cfg = workloads.C1
    g = c1[0]
    S = csr.stored_matrix(g, kind)
    s = _make(sl, cfg, kind)
    rp, col, val = s.get_csr()
    assert np.array_equal(rp, S.indptr) and np.array_equal(col, S.indices)
    assert np.array_equal(val.astype(np.float64), S.data)


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_full_passes(sl, c1, kind):
    cfg = workloads.C1
    g = c1[0]
    S = csr.stored_matrix(g, kind)
    s = _make(sl, cfg, kind)
    rs = np.random.default_rng(3)
    xv, yv = rs.standard_normal(g.n), rs.standard_normal(g.m)
    x = torch.tensor(xv, dtype=torch.float32, device="cuda")
    y = torch.zeros(g.m, dtype=torch.float32, device="cuda")
    s.project(x, y)
    x32 = xv.astype(np.float32).astype(np.float64)
    scale = np.abs(S) @ np.abs(x32) + 1e-30
    assert np.max(np.abs(y.double().cpu().numpy() - S @ x32) / scale) < 2e-6
    yt = torch.tensor(yv, dtype=torch.float32, device="cuda")
    xb = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    s.backproject(yt, xb)
    y32 = yv.astype(np.float32).astype(np.float64)
    scale = np.abs(S.T) @ np.abs(y32) + 1e-30
    assert np.max(np.abs(xb.double().cpu().numpy() - S.T @ y32) / scale) < 2e-6
    ids = torch.tensor(rs.integers(0, g.m, 41), dtype=torch.int32, device="cuda")
    ys = torch.zeros(41, dtype=torch.float32, device="cuda")
    s.project(x, ys, ids)
    # the subset goes through the same rows; only the summation order may differ
    assert np.allclose(ys.cpu().numpy(), y.cpu().numpy()[ids.cpu().numpy()], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_full_forward_pass_float64(sl, c1, kind):
    # float64 iterate over the stored float32 / bfloat16 values (the staged
    # full pass instantiated for double): exact products, float64 sums
    cfg = workloads.C1
    g = c1[0]
    S = csr.stored_matrix(g, kind)
    s = _make(sl, cfg, kind, precision=0, solver=0)
    xv = np.random.default_rng(4).standard_normal(g.n)
    y = torch.zeros(g.m, dtype=torch.float64, device="cuda")
    s.project(torch.tensor(xv, device="cuda"), y)
    scale = np.abs(S) @ np.abs(xv) + 1e-300
    assert np.max(np.abs(y.cpu().numpy() - S @ xv) / scale) < 1e-13
    s.close()


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_single_steps_on_the_stored_matrix(sl, c1, kind):
    cfg = workloads.C1
    g, A, _, b = c1
    S = csr.stored_matrix(g, kind)
    src = oslim.RowSource(csr.stored_rows_fn(S), b, g.n)
    s = _make(sl, cfg, kind)
    s.set_data(b)
    x_prev = np.zeros(g.n)
    worst = 0.0
    for k in range(1, 25):
        mem = [oslim.view_block_ids(g, cfg.seed, kk) for kk in range(max(1, k - cfg.r), k + 1)]
        x32 = x_prev.astype(np.float32).astype(np.float64)
        xo, _, _, _ = oslim.step_woodbury(x32, [src.rows(ids) for ids in mem], src.rhs(mem[-1]),
                                          cfg.lam)
        s.set_x(x_prev.astype(np.float32))
        s.set_iter(k - 1)
        s.step(1)
        worst = max(worst, rel(s.get_x(), xo))
        x_prev = xo
    assert worst < 1e-5


def test_stored_matrix_at_the_256_workload(sl):
    # the 256 x 256, 180 x 363 workload: build both stores and spot-check rows
    cfg = workloads.C2
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    rows = np.random.default_rng(5).integers(0, g.m, 300)
    for kind in ("f32", "bf16"):
        s = _make(sl, cfg, kind)
        rp, col, val = s.get_csr()
        for r in rows:
            idx, w = joseph.ray_taps(g, int(r))
            seg = slice(rp[r], rp[r + 1])
            assert np.array_equal(col[seg], idx)
            assert np.array_equal(val[seg].astype(np.float64), csr.round_values(w, kind))
        # the full forward pass over all 65,340 rays (staged tiles of
        # consecutive rays), checked on the sampled rows against the stored
        # entries just verified
        xv = np.random.default_rng(6).standard_normal(g.n).astype(np.float32)
        y = torch.full((g.m,), np.nan, dtype=torch.float32, device="cuda")
        s.project(torch.tensor(xv, device="cuda"), y)
        yh = y.cpu().numpy().astype(np.float64)
        assert np.isfinite(yh).all()
        x64 = xv.astype(np.float64)
        for r in rows:
            seg = slice(rp[r], rp[r + 1])
            want = np.dot(val[seg].astype(np.float64), x64[col[seg]])
            mag = np.dot(np.abs(val[seg].astype(np.float64)), np.abs(x64[col[seg]]))
            assert abs(yh[r] - want) <= 2e-6 * mag + 1e-30, (kind, int(r))
        s.close()
