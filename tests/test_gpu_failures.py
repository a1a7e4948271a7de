"""Failure detection without a GPU fault: a bounded device wait that runs out
reports AMG_ERR_TIMEOUT and leaves the context usable; Krylov breakdown on an
indefinite system is reported, by the oracle and by the library alike."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import setup_both  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    for blocks in (1, 8, 32):
        assert amg.amg_selftest_wait_timeout(blocks) == amg.AMG_ERR_TIMEOUT
    # the device still works: a normal solve right after
    s = W.poisson2d(16)
    h, oh, b = setup_both(s, coarse_max=16)
    x = torch.zeros_like(b)
    assert amg.pcg_solve(h, b, x, rtol=1e-8).status == amg.AMG_OK


def test_pcg_breakdown_on_indefinite_system():
    # diag(1, -1): with the exact (one-level) preconditioner (r, z) = 0 and
    # (p, A p) = 0 in the first iteration
    s = W.from_dense(np.diag([1.0, -1.0]), np.array([1.0, 1.0]))
    h, oh, b = setup_both(s)
    x_o, info_o = oh.pcg(s.b, rtol=1e-10)
    assert info_o.status == O.ERR_BREAKDOWN
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-10)
    assert info.status == amg.AMG_ERR_BREAKDOWN
