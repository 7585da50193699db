"""Failure detection of the tensor-core kernels, made without a fault: a
bounded mbarrier wait on a barrier that nothing completes runs out, raises
the error flag and returns, and the context stays usable afterwards."""
import time

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def test_wait_with_arrival_succeeds(G):
    assert G.wait_selftest(True) == (0, 1)


def test_wait_without_arrival_runs_out_and_context_survives(G):
    t0 = time.time()
    err, ok = G.wait_selftest(False)
    dt = time.time() - t0
    assert (err, ok) == (1, 0)
    assert dt < 60, dt
    # the same context still runs the tensor-core GEMM correctly
    e, ref = G.tc_selftest(2, 200, 48, 40, 3, seed=5)
    assert e <= 2e-5 * max(ref, 11.0)
    assert G.wait_selftest(True) == (0, 1)
