"""Failure detection on the GPU without a fault: a bounded device wait (the
grid barrier of the cooperative solvers) is made to run out by an arrival
that never comes; the kernel records SLIM_ETIMEOUT and ends, and the device
then runs the method correctly."""
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


def test_bounded_wait_reports_a_timeout_and_the_device_stays_usable(sl):
    assert sl.selftest_wait(0) == sl.SLIM_ETIMEOUT
    N, V, D, r, lam, seed = 24, 16, 35, 2, 1e-2, 3
    g = joseph.Geometry(N, V, D)
    b = workloads.add_noise(joseph.full_matrix(g) @ workloads.phantom_2d(N, seed, 5),
                            workloads.noise_direction(g.m, seed), 0.01)
    sched = list(oslim.view_schedule(g, seed, 6))
    want = [x for _, x, _ in oslim.run(oslim.tomo_source(g, b), sched, r, lam)][-1]
    s = sl.Slim(N, V, D, D, r, lam, seed)
    s.set_data(b)
    s.step(6)
    assert rel(s.get_x(), want) < 1e-12
    s.close()
