"""The allocation-free coarse solve, through the C ABI, against the existing
entry point that runs the same solver with hierarchy-owned memory.

amg_coarse_cg_noalloc serves callers that cannot call cudaMalloc (inside a
global-mode stream capture, in loops that cannot take cudaMalloc's device
synchronisation, or under a framework that owns all device memory).  Its
reference here is amg_vcycle on a one-level hierarchy whose coarsest solver
is CG: that V-cycle is exactly the CG solve of A z = r.  This file is named so
that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402

# the tolerance the V-cycle parity tests use when the coarsest solve is CG
TOL = 1e-9


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_existing_entry_point_twice():
    lib = amg.lib()
    s = W.lognormal3d(40, seed=21)  # 64,000 rows
    dev = torch.device("cuda", 0)
    rp, ci, val = (torch.from_numpy(a).to(dev) for a in (s.rp, s.ci, s.val))
    h = amg.amg_setup(rp, ci, val, max_levels=1, coarse_solver=amg.AMG_COARSE_CG)
    assert h.num_levels == 1
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    for call in range(2):  # two calls in a row share the scratch array
        f = torch.from_numpy(rng.uniform(-1, 1, s.n)).to(dev)
        z_ref = torch.empty_like(f)
        amg.amg_vcycle(h, f, z_ref)
        x = torch.full_like(f, float("nan"))  # output must not depend on its prior contents
        it = C.c_int(-1)
        st = lib.amg_coarse_cg_noalloc(s.n, s.nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), f.data_ptr(),
                                       x.data_ptr(), stream, C.byref(it))
        assert st == amg.AMG_OK, amg.status_string(st)
        assert 0 < it.value <= 1000
        assert _rel(x, z_ref) < TOL, (call, _rel(x, z_ref))
    h.close()


def test_noalloc_rejects_oversized_and_invalid_input():
    lib = amg.lib()
    n = amg.NOALLOC_MAX_N + 1
    it = C.c_int()
    # rejected before any device work: the pointers are never dereferenced
    assert lib.amg_coarse_cg_noalloc(n, 7 * n, 16, 16, 16, 16, 16, None, C.byref(it)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_coarse_cg_noalloc(0, 0, 16, 16, 16, 16, 16, None, C.byref(it)) == amg.AMG_ERR_INVALID_ARG
    s = W.poisson2d(8)
    dev = torch.device("cuda", 0)
    rp, ci, val = (torch.from_numpy(a).to(dev) for a in (s.rp, s.ci, s.val))
    f = torch.ones(s.n, dtype=torch.float64, device=dev)
    x = torch.empty_like(f)
    bad = ci.clone()
    bad[2] = 10_000
    with pytest.raises(amg.AmgError) as e:
        amg.amg_coarse_cg_noalloc(rp, bad, val, f, x)
    assert e.value.status == amg.AMG_ERR_INVALID_CSR
    # a valid call right after an error still works
    it = amg.amg_coarse_cg_noalloc(rp, ci, val, f, x)
    r = torch.from_numpy(s.dense()).to(dev) @ x - f
    assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) < 1e-11 and it > 0
