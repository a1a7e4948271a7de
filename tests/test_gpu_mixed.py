"""Mixed precision (FP32 hierarchy values and V-cycle, FP64 outer Krylov and
coarsest solve) against the FP64 oracle.

Tolerances: an FP32 V-cycle differs from the FP64 one by FP32 rounding
(unit roundoff 6e-8) accumulated over a few passes per level and amplified by
the coarse correction, so 1e-5 relative is a safe bound.  Flexible PCG with
the FP32 preconditioner keeps an FP64 residual recurrence and stops at the
same 1e-8; its solution then differs from the FP64 oracle's by at most about
cond(A) times the residual difference, checked here at 1e-6."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, setup_both, to_cuda  # noqa: E402

VCYCLE_TOL_FP32 = 1e-5
# FP16 storage rounds every stored value of D^-1/2 A D^-1/2 to 11 significant
# bits (relative 4.9e-4); the V-cycle then approximates the FP64 one to
# roughly that size times the coarse-correction gain, bounded here by 2e-2.
VCYCLE_TOL_FP16 = 2e-2

CASES = [
    ("poisson2d_64", lambda: W.poisson2d(64), dict(coarse_max=64)),
    ("aniso3d_24", lambda: W.anisotropic3d(24), dict(coarse_max=100)),
    ("lognormal3d_24", lambda: W.lognormal3d(24, seed=1), dict()),
    ("lognormal3d_32_cg", lambda: W.lognormal3d(32, seed=1), dict(coarse_max=2000, coarse_solver=2)),
    ("fem_p1_60", lambda: W.fem_p1_jittered(60, seed=4), dict(coarse_max=60)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_fp32_vcycle_close_to_fp64_oracle(case):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, precision=amg.AMG_FP32, **kw)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < VCYCLE_TOL_FP32


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_fp32_flexible_pcg_reaches_fp64_accuracy(case):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, precision=amg.AMG_FP32, **kw)
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
    x_o, info_o = oh.pcg(s.b, rtol=1e-8, flexible=True)
    assert info.status == amg.AMG_OK
    assert info.rel_res_true <= 1e-8
    assert info.iterations <= info_o.iterations + 2
    assert rel_err(x.cpu().numpy(), x_o) < 1e-6


def test_fp32_hierarchy_is_the_fp64_hierarchy():
    """Values are rounded after the FP64 setup: aggregates and patterns match."""
    s = W.lognormal3d(20, seed=8)
    rp, ci, val, b = to_cuda(s)
    h64 = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=300))
    h32 = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=300, precision=amg.AMG_FP32))
    assert h64.sizes() == h32.sizes()
    for k in range(h64.num_levels):
        for a, c in zip(amg.amg_export_level(h64, k), amg.amg_export_level(h32, k)):
            assert torch.equal(a, c)


def test_fp32_bicgstab_convdiff():
    s = W.convdiff2d(96, peclet=100.0)
    h, oh, b = setup_both(s, precision=amg.AMG_FP32, coarse_max=64)
    x = torch.zeros_like(b)
    info = amg.bicgstab_solve(h, b, x, rtol=1e-8, max_iter=300)
    x_o, info_o = oh.bicgstab(s.b, rtol=1e-8, max_iter=300)
    assert info.status == amg.AMG_OK and info.rel_res_true <= 1e-8
    # BiCGStab is not flexible: the FP32 V-cycle is a perturbed (slightly
    # nonlinear) preconditioner, which may cost a few more iterations than
    # the FP64 oracle's; bounded by 10% plus two
    assert info.iterations <= int(1.1 * info_o.iterations) + 2
    assert rel_err(x.cpu().numpy(), x_o) < 1e-6


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_fp16_storage_vcycle_and_flexible_pcg(case):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, precision=amg.AMG_FP16_STORAGE, **kw)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < VCYCLE_TOL_FP16
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
    x_o, info_o = oh.pcg(s.b, rtol=1e-8, flexible=True)
    assert info.status == amg.AMG_OK and info.rel_res_true <= 1e-8
    assert info.iterations <= int(1.5 * info_o.iterations) + 2
    assert rel_err(x.cpu().numpy(), x_o) < 1e-6


def test_fp16_storage_kernel_variants():
    s = W.lognormal3d(18, seed=2)
    h, oh, b = setup_both(s, precision=amg.AMG_FP16_STORAGE, coarse_max=200)
    z_o = oh.vcycle(s.b)
    for tpr in (0, 1, 4):
        for fp in (0, 1):
            for fq in (0, 1):
                for k in range(h.num_levels):
                    try:
                        amg.amg_level_set_config(h, k, tpr, fp, fq)
                    except amg.AmgError:
                        amg.amg_level_set_config(h, k, 1, fp, fq)
                z = torch.empty_like(b)
                amg.amg_vcycle(h, b, z)
                assert rel_err(z.cpu().numpy(), z_o) < VCYCLE_TOL_FP16
    amg.amg_autotune(h)
