"""Dense coarsest solve on the GPU against the oracle's dense LU (Algorithm 1,
coarsest level solved exactly).

The library inverts the coarsest matrix by blocked Gauss-Jordan elimination:
in FP64 up to 2048 rows, above that in FP32 with FP64 refinement in every
coarse solve.  Either way the coarse solve must reach FP64 accuracy, so a
one-level hierarchy's V-cycle equals the dense solve to 1e-12.
"""
import numpy as np
import pytest
import torch

from gpu_util import rel_err, setup_both, to_cuda
from paper_2007_00056_gb300 import amg
from paper_2007_00056_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    # (name, system, parameters): sizes chosen to hit both inversion paths
    ("poisson2d_32_fp64_m1024", lambda: W.poisson2d(32), dict(coarse_max=1024)),
    ("random_spd_m1031_fp64_ragged_panels", lambda: W.random_spd(1031, 0.01, 5), dict(coarse_max=1031)),
    ("convdiff2d_45_nonsymmetric_fp64_m2025", lambda: W.convdiff2d(45, peclet=300.0), dict(coarse_max=4096)),
    ("poisson2d_64_fp32_m4096", lambda: W.poisson2d(64), dict(coarse_max=4096)),
    ("random_spd_m2083_fp32_ragged_panels", lambda: W.random_spd(2083, 0.004, 6), dict(coarse_max=2083)),
    ("convdiff2d_48_nonsymmetric_fp32_m2304", lambda: W.convdiff2d(48, peclet=300.0), dict(coarse_max=4096)),
    ("lognormal3d_14_fp32_m2744", lambda: W.lognormal3d(14, seed=3), dict(coarse_max=4096)),
    ("fem_p1_50_fp32_m2500", lambda: W.fem_p1_jittered(50, seed=3), dict(coarse_max=2500)),
    ("fem_p1_60_fp32_m3600", lambda: W.fem_p1_jittered(60, seed=4), dict(coarse_max=4096)),
    ("aniso3d_20_two_levels", lambda: W.anisotropic3d(20), dict(coarse_max=2100)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_dense_coarse_vcycle_matches_oracle(name, make, kw):
    s = make()
    h, oh, b = setup_both(s, **kw)
    assert h.sizes() == oh.sizes()
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    z_o = oh.vcycle(s.b)
    assert rel_err(z.cpu().numpy(), z_o) < 1e-12
    if h.num_levels == 1:
        # one level: the V-cycle is the exact solve
        x = np.linalg.solve(s.dense(), s.b)
        assert rel_err(z.cpu().numpy(), x) < 1e-11


def test_dense_coarse_exact_preconditioner_converges_in_one_iteration():
    s = W.poisson2d(64)
    h, _, b = setup_both(s, coarse_max=4096)
    assert h.num_levels == 1
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8)
    assert info.status == amg.AMG_OK and info.iterations == 1
    assert info.rel_res_true < 1e-12


def test_dense_coarse_fp32_vcycle():
    s = W.poisson2d(64)
    h, oh, b = setup_both(s, coarse_max=4096, precision=amg.AMG_FP32)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    # FP32 storage of the right-hand side and the result bounds the accuracy
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-6


@pytest.mark.parametrize("make", [lambda: W.fem_p1_jittered(50, seed=3), lambda: W.lognormal3d(14, seed=3)],
                         ids=["fem_p1_50", "lognormal3d_14"])
def test_real_valued_coarsest_keeps_fp32_inverse(make):
    """Matrices with non-integer entries round A v in FP64, so no solve can
    return v to the last bit; the refinement is accepted on its backward error
    and the FP32 inverse is kept (the batched solver, which needs an FP64
    inverse, then refuses the hierarchy)."""
    s = make()
    rp, ci, val, b = to_cuda(s)
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=4096))
    assert h.num_levels == 1 and s.n > 2048
    with pytest.raises(amg.AmgError) as e:
        amg.amg_batch_pcg([h], [b], [torch.zeros_like(b)], rtol=1e-8)
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    x = np.linalg.solve(s.dense(), s.b)
    assert rel_err(z.cpu().numpy(), x) < 1e-11


def test_batched_solver_requires_fp64_inverse():
    s = W.poisson2d(48)  # 2304 rows, one level: FP32 inverse
    rp, ci, val, b = to_cuda(s)
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=2400))
    x = torch.zeros_like(b)
    with pytest.raises(amg.AmgError):
        amg.amg_batch_pcg([h], [b], [x], rtol=1e-8)


def test_dense_max_gives_a_stalled_coarsest_level_the_direct_solve():
    """A lognormal hierarchy stalls well above a stop size of 100 rows; with
    dense_max above its coarsest size the coarsest level is inverted instead
    of solved by CG, and the V-cycle is the oracle's dense-coarse cycle."""
    s = W.lognormal3d(24, seed=2)
    p = amg.amg_default_params(coarse_max=100)
    rp, ci, val, b = to_cuda(s)
    h_cg = amg.amg_setup(rp, ci, val, p)
    n_l = h_cg.sizes()[-1]
    assert n_l > 100 and amg.amg_coarse_cg_cluster_size(h_cg) >= 0
    h_cg.close()
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, dense_max=n_l))
    assert h.sizes()[-1] == n_l and amg.amg_coarse_cg_cluster_size(h) == -1
    import oracle as O
    oh = O.Hierarchy(s.rp, s.ci, s.val, params=O.Params(coarse_max=100, coarse_solver=1))
    assert oh.sizes() == h.sizes()
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-12
    h.close()
    # below the coarsest size the CG stays
    h2 = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, dense_max=n_l - 1))
    assert amg.amg_coarse_cg_cluster_size(h2) >= 0
    h2.close()
