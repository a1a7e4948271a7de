"""The allocation-free coarse solve, through the C ABI, against the existing
entry point that runs the same solver with hierarchy-owned memory.

amg_coarse_cg_noalloc serves callers that cannot call cudaMalloc (code under
a framework that owns all device memory, or loops that cannot take
cudaMalloc's device synchronisation).  Its reference here is amg_vcycle on a
one-level hierarchy whose coarsest solver is CG: that V-cycle is exactly the
CG solve of A z = r.  This file is named so that pytest collects it last."""
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
    # x must not be f
    assert lib.amg_coarse_cg_noalloc(s.n, s.nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), f.data_ptr(),
                                     f.data_ptr(), None, C.byref(it)) == amg.AMG_ERR_INVALID_ARG
    # a valid call right after an error still works
    it = amg.amg_coarse_cg_noalloc(rp, ci, val, f, x)
    r = torch.from_numpy(s.dense()).to(dev) @ x - f
    assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) < 1e-11 and it > 0


def _shifted_poisson(m, shift):
    s = W.poisson2d(m)
    rows = np.repeat(np.arange(s.n), np.diff(s.rp))
    val = s.val.copy()
    val[s.ci == rows] += shift
    return s.rp, s.ci, val


def test_noalloc_at_the_size_limit():
    """Exactly NOALLOC_MAX_N rows (a 512 x 512 grid, shifted to keep CG short):
    the scratch carve at its largest, against amg_vcycle on a one-level CG
    hierarchy and against the residual recomputed here."""
    lib = amg.lib()
    rp_h, ci_h, val_h = _shifted_poisson(512, 1.0)
    n = len(rp_h) - 1
    assert n == amg.NOALLOC_MAX_N
    dev = torch.device("cuda", 0)
    rp, ci, val = (torch.from_numpy(a).to(dev) for a in (rp_h, ci_h, val_h))
    f = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, n)).to(dev)
    h = amg.amg_setup(rp, ci, val, max_levels=1, coarse_solver=amg.AMG_COARSE_CG)
    z_ref = torch.empty_like(f)
    amg.amg_vcycle(h, f, z_ref)
    x = torch.full_like(f, float("nan"))
    it = C.c_int(-1)
    st = lib.amg_coarse_cg_noalloc(n, len(ci_h), rp.data_ptr(), ci.data_ptr(), val.data_ptr(), f.data_ptr(),
                                   x.data_ptr(), torch.cuda.current_stream().cuda_stream, C.byref(it))
    assert st == amg.AMG_OK, amg.status_string(st)
    assert _rel(x, z_ref) < TOL
    a = torch.sparse_csr_tensor(rp.long(), ci.long(), val, size=(n, n))
    r = torch.mv(a, x) - f
    assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) < 1e-10
    h.close()


def test_noalloc_reports_non_convergence():
    """A 1D Laplacian of 20,000 rows needs far more than the solver's 1000 CG
    iterations to reach 1e-12: the call returns AMG_ERR_NOT_CONVERGED with the
    iteration count at the limit."""
    lib = amg.lib()
    n = 20000
    rp = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                cols.append(j)
                vals.append(v)
        rp[i + 1] = len(cols)
    dev = torch.device("cuda", 0)
    rp_d = torch.from_numpy(rp).to(dev)
    ci_d = torch.tensor(cols, dtype=torch.int32, device=dev)
    val_d = torch.tensor(vals, dtype=torch.float64, device=dev)
    f = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, n)).to(dev)
    x = torch.empty_like(f)
    it = C.c_int(-1)
    st = lib.amg_coarse_cg_noalloc(n, len(cols), rp_d.data_ptr(), ci_d.data_ptr(), val_d.data_ptr(), f.data_ptr(),
                                   x.data_ptr(), torch.cuda.current_stream().cuda_stream, C.byref(it))
    assert st == amg.AMG_ERR_NOT_CONVERGED, amg.status_string(st)
    assert it.value == 1000
    assert torch.isfinite(x).all()
