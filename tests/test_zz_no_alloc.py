"""The allocation-free damped Gram solve.

slim_damped_solve_noalloc serves callers that cannot allocate device memory
when they solve (an application whose device memory is reserved by its own
pool allocator, or a latency-critical loop that must not call cudaMalloc or
cudaFree, which synchronise the device).  It keeps its scratch in one static
device array shared by every call, so these tests make two calls in a row of
different sizes -- the second must not see the first call's leftovers -- and
compare each with numpy's dense solve and with slim_damped_solve, at the
tolerance of the other damped-solve tests.  One test runs in a fresh process
whose first solve is the allocation-free one (its one-time set-up included).
This file is collected last on purpose.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-11


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _system(p, seed):
    rs = np.random.default_rng(seed)
    B = rs.standard_normal((p, p + 20)) / np.sqrt(p)
    return B @ B.T, rs.standard_normal(p)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_dense_and_allocating_solve_on_two_calls(sl):
    for call, (p, lam) in enumerate([(1000, 1e-2), (300, 1e-3)]):
        G, rhs = _system(p, 40 + call)
        want = np.linalg.solve(lam * np.eye(p) + G, rhs)
        Gt = torch.tensor(G, device="cuda")
        rt = torch.tensor(rhs, device="cuda")
        z_new = torch.full((p,), float("nan"), dtype=torch.float64, device="cuda")
        z_ref = torch.zeros(p, dtype=torch.float64, device="cuda")
        sl.damped_solve_noalloc(Gt, lam, rt, z_new)
        sl.damped_solve(Gt, lam, rt, z_ref)
        torch.cuda.synchronize()
        a, b = z_new.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert _rel(a, want) < TOL, call
        assert _rel(a, b) < TOL, call


def test_noalloc_first_in_a_fresh_process():
    code = f"""
import sys
sys.path.insert(0, {ROOT!r})
import numpy as np, torch
from paper_1912_07962_gb300 import build, slim
build.build()
for call, (p, lam, seed) in enumerate([(777, 1e-2, 5), (64, 1e-1, 6)]):
    rs = np.random.default_rng(seed)
    B = rs.standard_normal((p, p + 20)) / np.sqrt(p)
    G, rhs = B @ B.T, rs.standard_normal(p)
    want = np.linalg.solve(lam * np.eye(p) + G, rhs)
    z = torch.full((p,), float("nan"), dtype=torch.float64, device="cuda")
    slim.damped_solve_noalloc(torch.tensor(G, device="cuda"), lam,
                              torch.tensor(rhs, device="cuda"), z)
    torch.cuda.synchronize()
    got = z.cpu().numpy()
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert np.all(np.isfinite(got)) and err < {TOL!r}, (call, err)
print("ok")
"""
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         cwd=ROOT, timeout=600)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stderr[-3000:]


def test_noalloc_rejects_orders_above_its_limit(sl):
    p = sl.NOALLOC_MAX_P + 1
    Gt = torch.eye(p, dtype=torch.float64, device="cuda")
    rt = torch.ones(p, dtype=torch.float64, device="cuda")
    zt = torch.zeros(p, dtype=torch.float64, device="cuda")
    with pytest.raises(sl.SlimError) as ei:
        sl.damped_solve_noalloc(Gt, 1.0, rt, zt)
    assert ei.value.code == sl.SLIM_EINVAL
