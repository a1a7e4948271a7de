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


def test_bicgstab_breakdown_on_indefinite_system():
    # two copies of [[1, 3], [3, 1]], omega = 1, coarsest level of 2 rows: the
    # V-cycle is exact in binary and (A M^-1 b, b) = 0 for b = (3, 1, 2, 2), so
    # the first BiCGStab step divides by zero (the oracle's pins work it by hand)
    a = np.kron(np.eye(2), np.array([[1.0, 3.0], [3.0, 1.0]]))
    s = W.from_dense(a, np.array([3.0, 1.0, 2.0, 2.0]))
    h, oh, b = setup_both(s, coarse_max=2, omega=1.0)
    assert h.sizes() == oh.sizes() == [4, 2]
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    np.testing.assert_array_equal(z.cpu().numpy(), oh.vcycle(s.b))
    _, info_o = oh.bicgstab(s.b, rtol=1e-10)
    assert info_o.status == O.ERR_BREAKDOWN
    x = torch.zeros_like(b)
    info = amg.bicgstab_solve(h, b, x, rtol=1e-10)
    assert info.status == amg.AMG_ERR_BREAKDOWN
    # the same hierarchy with a right-hand side off the breakdown converges
    b2 = b.clone()
    b2[3] = 1.0
    x2 = torch.zeros_like(b2)
    assert amg.bicgstab_solve(h, b2, x2, rtol=1e-12).status == amg.AMG_OK
