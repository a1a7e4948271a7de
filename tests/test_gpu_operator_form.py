"""Residual-operator form of a zero-guess cycle visit against the explicit
sweeps and the oracle.

With x = omega D^-1 f the first presmoothing sweep from zero, the visit's
residual is t = f - A x = C f with C = I - omega A D^-1, and prolongation plus
the postsmoothing sweep give y = Q x_c + omega D^-1 (f + t) with
Q = P - omega D^-1 A P (Algorithm 1 rearranged; the paper's V-cycle in exact
arithmetic).  Only the rounding differs from the explicit kernels, so FP64
V-cycles agree with the oracle to the same 1e-12 as the explicit form, and the
two forms agree with each other to a few ulps.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, setup_both, to_cuda  # noqa: E402

CASES = [
    ("poisson2d_97_ragged", lambda: W.poisson2d(97), dict(coarse_max=50)),
    ("lognormal3d_24", lambda: W.lognormal3d(24, seed=1), dict()),
    ("aniso3d_24", lambda: W.anisotropic3d(24), dict(coarse_max=100)),
    ("fem_p1_60", lambda: W.fem_p1_jittered(60, seed=4), dict(coarse_max=60)),
    ("convdiff2d_64_nonsymmetric", lambda: W.convdiff2d(64, peclet=200.0), dict(coarse_max=64)),
    ("lognormal3d_32_cg_coarse", lambda: W.lognormal3d(32, seed=1), dict(coarse_max=2000, coarse_solver=2)),
]


def _set_form(h, on):
    for k in range(h.num_levels - 1):
        amg.amg_level_set_operator_form(h, k, on)


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_operator_form_equals_explicit_sweeps_and_oracle(case):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, **kw)
    assert all(amg.amg_level_operator_form(h, k) for k in range(h.num_levels - 1))
    assert not amg.amg_level_operator_form(h, h.num_levels - 1)  # the coarsest level is solved
    z_o = oh.vcycle(s.b)
    tol = 1e-12 if oh.dense_coarse else 1e-9
    z_op = torch.empty_like(b)
    amg.amg_vcycle(h, b, z_op)
    _set_form(h, False)
    z_ex = torch.empty_like(b)
    amg.amg_vcycle(h, b, z_ex)
    assert rel_err(z_op.cpu().numpy(), z_o) < tol
    assert rel_err(z_ex.cpu().numpy(), z_o) < tol
    if oh.dense_coarse:
        assert rel_err(z_op.cpu().numpy(), z_ex.cpu().numpy()) < 1e-13
    np.testing.assert_allclose(z_op.cpu().numpy(), z_o, rtol=tol * 100, atol=tol * np.abs(z_o).max())


@pytest.mark.parametrize("cycle", [amg.AMG_CYCLE_W, amg.AMG_CYCLE_F])
def test_operator_form_in_w_and_f_cycles(cycle):
    """Zero-guess visits use C and Q; the second visits of the W- and F-cycles
    (from a guess) use the explicit sweeps; together they are the oracle's cycle."""
    s = W.lognormal3d(20, seed=5)
    h, oh, b = setup_both(s, coarse_max=100, cycle=cycle)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-12


def test_operator_form_fp32_close_to_fp64_oracle():
    s = W.anisotropic3d(24)
    h, oh, b = setup_both(s, coarse_max=100, precision=amg.AMG_FP32)
    z_o = oh.vcycle(s.b)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), z_o) < 1e-5
    _set_form(h, False)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), z_o) < 1e-5


def test_operator_form_off_and_unavailable():
    s = W.lognormal3d(16, seed=2)
    rp, ci, val, b = to_cuda(s)
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, operator_form=0))
    assert not any(amg.amg_level_operator_form(h, k) for k in range(h.num_levels))
    with pytest.raises(amg.AmgError) as e:
        amg.amg_level_set_operator_form(h, 0, True)
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED
    # FP16 storage and more than one sweep have no operator form
    for kw in (dict(precision=amg.AMG_FP16_STORAGE), dict(nu_pre=2)):
        h2 = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, **kw))
        assert not any(amg.amg_level_operator_form(h2, k) for k in range(h2.num_levels))
    with pytest.raises(amg.AmgError):
        amg.amg_setup(rp, ci, val, amg.amg_default_params(operator_form=2))
    with pytest.raises(IndexError):
        amg.amg_level_operator_form(h, 99)


def test_pcg_with_operator_form_matches_oracle_at_fixed_iterations():
    s = W.lognormal3d(28, seed=7)
    h, oh, b = setup_both(s, coarse_max=300)
    x_o, info_o = oh.pcg(s.b, rtol=1e-8)
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8)
    assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
    assert info.rel_res_true <= 1e-8
    x = torch.zeros_like(b)
    amg.pcg_solve(h, b, x, rtol=0.0, max_iter=info_o.iterations)
    assert rel_err(x.cpu().numpy(), x_o) < 1e-10


def test_dense_inverse_falls_back_to_pivoting():
    """A well-conditioned coarsest matrix on which elimination without row
    interchanges is unstable (2 x 2 blocks [[1e-9, 1], [1, 1]]: a tiny leading
    pivot, then cancellation of terms of size 1e9 in FP32): the library must
    still return the exact solve, through the partially pivoted inverse."""
    m = 2200  # above the FP64 inverse limit: the FP32 inverse with refinement
    blk = np.array([[1e-9, 1.0], [1.0, 1.0]])
    a = np.kron(np.eye(m // 2), blk)
    rng = np.random.default_rng(9)
    s = W.from_dense(a, rng.uniform(-1, 1, m))
    h, oh, b = setup_both(s, max_levels=1, coarse_solver=amg.AMG_COARSE_DENSE)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), np.linalg.solve(a, s.b)) < 1e-11
