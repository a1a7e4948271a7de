"""The full-size workloads of the benchmark, in the configurations bench.py
times, checked where the oracle cannot run whole (minutes of serial CPU):
by properties that hold at any size and by sampled outputs recomputed from
their definitions.

- lognormal3d_128 with the autotuned kernels the benchmark uses: same
  iterations and solution as the default kernels (which
  test_gpu_solve.py::test_full_size_lognormal_128_pcg matches to the oracle);
- anisotropic3d_256 (16.8M unknowns) in FP64, FP32 and FP16 storage: true
  residual, mixed-precision error against the FP64 solution, the level-0
  aggregates as a partition into pairs-of-pairs (Sec. 2.1, two passes), and
  sampled Galerkin entries (A_c)_IJ = sum_{i in I, j in J} a_ij (Sec. 2.1);
- convdiff2d_2048 with BiCGStab (Algorithm 5) and the FP32 V-cycle.
"""
import numpy as np
import pytest
import torch

from gpu_util import rel_err, to_cuda
from paper_2007_00056_gb300 import amg
from paper_2007_00056_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_lognormal_128_autotuned_matches_default_kernels():
    s = W.lognormal3d(128, seed=1)
    rp, ci, val, b = to_cuda(s)
    xs, its = [], []
    for tune in (False, True):
        h = amg.amg_setup(rp, ci, val)
        if tune:
            amg.amg_autotune(h)
        x = torch.zeros_like(b)
        info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
        assert info.status == amg.AMG_OK and info.rel_res_true <= 1.01e-8
        xs.append(x.cpu().numpy())
        its.append(info.iterations)
        h.close()
    assert its[0] == its[1]
    assert rel_err(xs[1], xs[0]) < 1e-11


@pytest.fixture(scope="module")
def aniso256():
    s = W.config_anisotropic3d_256()
    return s, to_cuda(s)


def test_anisotropic_256_precisions(aniso256):
    s, (rp, ci, val, b) = aniso256
    xs = {}
    for prec in (amg.AMG_FP64, amg.AMG_FP32, amg.AMG_FP16_STORAGE):
        h = amg.amg_setup(rp, ci, val, amg.amg_default_params(precision=prec))
        x = torch.zeros_like(b)
        info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
        assert info.status == amg.AMG_OK, info
        assert info.rel_res_true <= 1.01e-8, info
        xs[prec] = x
        h.close()
    ref = xs[amg.AMG_FP64]
    for prec in (amg.AMG_FP32, amg.AMG_FP16_STORAGE):
        d = torch.linalg.vector_norm(xs[prec] - ref) / torch.linalg.vector_norm(ref)
        assert d.item() < 1e-6


def test_anisotropic_256_aggregates_and_sampled_galerkin(aniso256):
    s, (rp, ci, val, b) = aniso256
    h = amg.amg_setup(rp, ci, val)
    n0, _ = amg.amg_level_info(h, 0)
    n1, _ = amg.amg_level_info(h, 1)
    agg = torch.empty(n0, dtype=torch.int32, device=b.device)
    amg.amg_level_info(h, 0, agg)
    a = agg.cpu().numpy().astype(np.int64)
    # a partition of the fine nodes into n1 aggregates of 1..4 nodes (two pairwise passes)
    assert a.min() == 0 and a.max() == n1 - 1
    sizes = np.bincount(a, minlength=n1)
    assert sizes.min() >= 1 and sizes.max() <= 4
    # aggregate ids ranked by smallest member: first members appear in increasing order
    first = np.full(n1, n0, dtype=np.int64)
    np.minimum.at(first, a, np.arange(n0))
    assert np.all(np.diff(first) > 0)
    # sampled coarse rows: (A_c)_IJ = sum over i in I, j in J of a_ij
    crp, cci, cval = (t.cpu().numpy() for t in amg.amg_export_level(h, 1))
    rp0, ci0, v0 = s.rp, s.ci, s.val
    members = [[] for _ in range(n1)]
    rows = np.random.default_rng(3).integers(0, n1, 200)
    want = set(rows.tolist())
    for i in np.flatnonzero(np.isin(a, rows)):
        members[a[i]].append(i)
    for I in want:
        acc = {}
        for i in members[I]:
            for e in range(rp0[i], rp0[i + 1]):
                J = int(a[ci0[e]])
                acc[J] = acc.get(J, 0.0) + v0[e]
        got = {int(cci[e]): cval[e] for e in range(crp[I], crp[I + 1])}
        assert sorted(got) == sorted(acc)
        for J, v in acc.items():
            assert abs(got[J] - v) <= 1e-12 * max(1.0, abs(v))
    h.close()


@pytest.mark.parametrize("peclet", [10.0, 100.0, 1000.0])
def test_convdiff_2048_bicgstab_fp32_vcycle(peclet):
    s = W.config_convdiff2d_2048(peclet=peclet)
    rp, ci, val, b = to_cuda(s)
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(precision=amg.AMG_FP32))
    x = torch.zeros_like(b)
    info = amg.bicgstab_solve(h, b, x, rtol=1e-8)
    assert info.status == amg.AMG_OK, info
    assert info.rel_res_true <= 1.01e-8, info
    h.close()
