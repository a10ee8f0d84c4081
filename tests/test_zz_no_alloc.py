"""The allocation-free damped Gram solve against the allocating one.

slim_damped_solve_noalloc serves callers that cannot allocate device memory
when they solve (an application whose device memory is reserved by its own
pool allocator, or a latency-critical loop that must not call cudaMalloc or
cudaFree, which synchronise the device).  It keeps its scratch in one static
device array shared by every call, so this test makes two calls in a row of
different sizes -- the second must not see the first call's leftovers -- and
compares each with slim_damped_solve at the tolerance of the other solve tests.
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _system(p, seed):
    rs = np.random.default_rng(seed)
    B = rs.standard_normal((p, p + 20)) / np.sqrt(p)
    return B @ B.T, rs.standard_normal(p)


def test_noalloc_matches_allocating_solve_on_two_calls(sl):
    for call, (p, lam) in enumerate([(1000, 1e-2), (300, 1e-3)]):
        G, rhs = _system(p, 40 + call)
        Gt = torch.tensor(G, device="cuda")
        rt = torch.tensor(rhs, device="cuda")
        z_ref = torch.zeros(p, dtype=torch.float64, device="cuda")
        z_new = torch.full((p,), float("nan"), dtype=torch.float64, device="cuda")
        sl.damped_solve(Gt, lam, rt, z_ref)
        sl.damped_solve_noalloc(Gt, lam, rt, z_new)
        torch.cuda.synchronize()
        a, b = z_new.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b), call


def test_noalloc_rejects_orders_above_its_limit(sl):
    p = sl.NOALLOC_MAX_P + 1
    Gt = torch.eye(p, dtype=torch.float64, device="cuda")
    rt = torch.ones(p, dtype=torch.float64, device="cuda")
    zt = torch.zeros(p, dtype=torch.float64, device="cuda")
    with pytest.raises(sl.SlimError) as ei:
        sl.damped_solve_noalloc(Gt, 1.0, rt, zt)
    assert ei.value.code == sl.SLIM_EINVAL
