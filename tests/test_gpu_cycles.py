"""W- and F-cycles (Sec. 2 names V, W and F) and AMG as a stand-alone solver
(Sec. 3.1, compared with AMG-PCG in Sec. 4.4) on the GPU against the oracle.

Tolerances follow test_gpu_solve.py: a cycle differs from the oracle's only by
summation order and fused multiply-adds, so 1e-12 relative with a dense
coarsest solve; a CG coarsest solve stops at 1e-12 and is called many times
per W-cycle, so 1e-9.  Iteration counts of a solve agree within one; at the
oracle's count the iterates agree to 1e-10."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, setup_both, to_cuda  # noqa: E402

TOL_DENSE = 1e-12
TOL_CG = 1e-9
SOLUTION_TOL = 1e-10
KINDS = {"V": amg.AMG_CYCLE_V, "W": amg.AMG_CYCLE_W, "F": amg.AMG_CYCLE_F}

CASES = [
    ("poisson2d_64", lambda: W.poisson2d(64), dict(coarse_max=64)),
    ("poisson2d_97_ragged", lambda: W.poisson2d(97), dict(coarse_max=50)),
    ("lognormal3d_24", lambda: W.lognormal3d(24, seed=1), dict(coarse_max=200)),
    ("lognormal3d_32_cg_coarse", lambda: W.lognormal3d(32, seed=1), dict(coarse_max=2000, coarse_solver=2)),
    ("aniso3d_24", lambda: W.anisotropic3d(24), dict(coarse_max=100)),
    ("fem_p1_60", lambda: W.fem_p1_jittered(60, seed=4), dict(coarse_max=60)),
    ("convdiff2d_64_nonsymmetric", lambda: W.convdiff2d(64, peclet=100.0), dict(coarse_max=64)),
    ("lognormal3d_16_nu2_3", lambda: W.lognormal3d(16, seed=3), dict(coarse_max=30, nu_pre=2, nu_post=3)),
    ("lognormal3d_16_nopost", lambda: W.lognormal3d(16, seed=3), dict(coarse_max=30, nu_post=0)),
]


def _tol(oh):
    return TOL_DENSE if oh.dense_coarse else TOL_CG


@pytest.mark.parametrize("kind", ["W", "F"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_cycle_matches_oracle(case, kind):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, cycle=KINDS[kind], **kw)
    assert h.num_levels >= 3
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    z_o = oh.vcycle(s.b)
    tol = _tol(oh)
    assert rel_err(z.cpu().numpy(), z_o) < tol
    np.testing.assert_allclose(z.cpu().numpy(), z_o, rtol=tol * 100, atol=tol * np.abs(z_o).max())


def test_cycle_kinds_differ_and_launch_more_on_coarse_levels():
    """Four levels: the W-cycle visits level k 2^k times, the F-cycle k+1
    times (levels below the coarsest), so their results and launch counts
    differ from the V-cycle's."""
    s = W.poisson2d(64)
    zs, launches = {}, {}
    for name, kind in KINDS.items():
        h, _, b = setup_both(s, coarse_max=64, cycle=kind)
        assert h.sizes() == [4096, 1024, 256, 64]
        z = torch.empty_like(b)
        amg.amg_vcycle(h, b, z)  # warm-up
        torch.cuda.synchronize()
        n0 = amg.amg_kernel_launches()
        amg.amg_vcycle(h, b, z)
        torch.cuda.synchronize()
        launches[name] = amg.amg_kernel_launches() - n0
        zs[name] = z.cpu().numpy()
    assert launches["V"] < launches["F"] < launches["W"]
    assert rel_err(zs["W"], zs["V"]) > 1e-6 and rel_err(zs["F"], zs["W"]) > 1e-6


SOLVER_CASES = [CASES[0], CASES[2], CASES[3], CASES[5], CASES[6]]


@pytest.mark.parametrize("kind", ["V", "W", "F"])
@pytest.mark.parametrize("case", SOLVER_CASES, ids=lambda c: c[0])
def test_amg_solver_matches_oracle(case, kind):
    _, make, kw = case
    s = make()
    h, oh, b = setup_both(s, cycle=KINDS[kind], **kw)
    x = torch.zeros_like(b)
    info = amg.amg_solve(h, b, x, rtol=1e-8, max_iter=2000)
    x_o, info_o = oh.amg_solve(s.b, rtol=1e-8, max_iter=2000)
    assert info.status == amg.AMG_OK and info_o.status == O.OK, (info, info_o)
    assert abs(info.iterations - info_o.iterations) <= 1
    assert info.rel_res_true <= 1e-8
    # same number of cycles: the iterates agree to 1e-10
    x = torch.zeros_like(b)
    info = amg.amg_solve(h, b, x, rtol=0.0, max_iter=info_o.iterations)
    assert info.iterations == info_o.iterations and info.status == amg.AMG_ERR_NOT_CONVERGED
    assert rel_err(x.cpu().numpy(), x_o) < SOLUTION_TOL


@pytest.mark.parametrize("kind", ["W", "F"])
def test_pcg_with_w_and_f_cycles_matches_oracle(kind):
    s = W.lognormal3d(24, seed=1)
    h, oh, b = setup_both(s, coarse_max=200, cycle=KINDS[kind])
    flexible = kind == "F"  # the F-cycle's M^{-1} is not symmetric
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=flexible)
    x_o, info_o = oh.pcg(s.b, rtol=1e-8, flexible=flexible)
    assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
    x = torch.zeros_like(b)
    amg.pcg_solve(h, b, x, rtol=0.0, max_iter=info_o.iterations, flexible=flexible)
    assert rel_err(x.cpu().numpy(), x_o) < SOLUTION_TOL


def test_bicgstab_with_w_cycle_matches_oracle():
    s = W.convdiff2d(64, peclet=300.0)
    h, oh, b = setup_both(s, coarse_max=64, cycle=amg.AMG_CYCLE_W)
    x = torch.zeros_like(b)
    info = amg.bicgstab_solve(h, b, x, rtol=1e-8)
    x_o, info_o = oh.bicgstab(s.b, rtol=1e-8)
    assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
    assert info.rel_res_true <= 1.01e-8


@pytest.mark.parametrize("precision", [amg.AMG_FP32, amg.AMG_FP16_STORAGE])
@pytest.mark.parametrize("kind", ["W", "F"])
def test_mixed_precision_cycles_and_solver(precision, kind):
    """FP32 / FP16-storage cycles stay within the mixed-precision bounds of
    test_gpu_mixed.py of the FP64 oracle's cycle; the stationary solver, whose
    residual is FP64, still reaches 1e-8."""
    s = W.lognormal3d(24, seed=1)
    h, oh, b = setup_both(s, coarse_max=200, cycle=KINDS[kind], precision=precision)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    bound = 1e-5 if precision == amg.AMG_FP32 else 2e-2
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < bound
    x = torch.zeros_like(b)
    info = amg.amg_solve(h, b, x, rtol=1e-8, max_iter=2000)
    assert info.status == amg.AMG_OK and info.rel_res_true <= 1e-8
    _, info_o = oh.amg_solve(s.b, rtol=1e-8, max_iter=2000)
    assert info.iterations <= info_o.iterations + 3


def test_amg_solver_edge_cases():
    s = W.poisson2d(40)
    h, oh, b = setup_both(s, coarse_max=100)
    # b = 0: x = 0 after 0 cycles, whatever x0 was
    x = torch.ones_like(b)
    info = amg.amg_solve(h, torch.zeros_like(b), x, rtol=1e-8)
    assert info.status == amg.AMG_OK and info.iterations == 0 and not torch.any(x)
    # max_iter = 0: not converged, x0 returned unchanged
    x0 = torch.full_like(b, 0.5)
    x = x0.clone()
    info = amg.amg_solve(h, b, x, rtol=1e-8, max_iter=0)
    assert info.status == amg.AMG_ERR_NOT_CONVERGED and info.iterations == 0 and torch.equal(x, x0)
    # an initial guess that already meets the tolerance: 0 cycles
    xs = torch.from_numpy(np.linalg.solve(s.dense(), s.b)).to(b.device)
    x = xs.clone()
    info = amg.amg_solve(h, b, x, rtol=1e-8)
    assert info.status == amg.AMG_OK and info.iterations == 0 and torch.equal(x, xs)
    # a nonzero initial guess: same iterates as the oracle from that guess
    g = np.random.default_rng(5).uniform(-1, 1, s.n)
    x = torch.from_numpy(g.copy()).to(b.device)
    info = amg.amg_solve(h, b, x, rtol=0.0, max_iter=7)
    x_o, _ = oh.amg_solve(s.b, x0=g, rtol=0.0, max_iter=7)
    assert info.iterations == 7 and rel_err(x.cpu().numpy(), x_o) < SOLUTION_TOL
    # bad arguments
    with pytest.raises(amg.AmgError):
        amg.amg_solve(h, b, torch.zeros_like(b), rtol=-1.0)
    with pytest.raises(amg.AmgError):
        amg.amg_solve(h, b, torch.zeros_like(b), max_iter=-1)


def test_amg_solver_graph_replay_is_deterministic():
    """The second solve on a hierarchy replays a captured CUDA graph of one
    cycle; it gives the first solve's result bit for bit."""
    s = W.lognormal3d(24, seed=2)
    h, _, b = setup_both(s, coarse_max=200, cycle=amg.AMG_CYCLE_W)
    xs = []
    for _ in range(3):
        x = torch.zeros_like(b)
        info = amg.amg_solve(h, b, x, rtol=1e-9)
        assert info.status == amg.AMG_OK
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0].view(np.int64), xs[1].view(np.int64))
    assert np.array_equal(xs[0].view(np.int64), xs[2].view(np.int64))


def test_cycle_parameter_checks():
    s = W.poisson2d(40)
    rp, ci, val, b = to_cuda(s)
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, ci, val, amg.amg_default_params(cycle=3))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    # the batched solver runs V-cycles only
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, cycle=amg.AMG_CYCLE_W))
    with pytest.raises(amg.AmgError) as e:
        amg.amg_batch_pcg([h], [b], [torch.zeros_like(b)], rtol=1e-8)
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED


def test_full_size_lognormal_128_amg_solver_and_w_cycle_pcg():
    """The benchmark system solved by AMG as a solver (V-cycles) and by PCG
    with W-cycles; the true residual is recomputed on the host from the
    returned x (scipy CSR product in FP64)."""
    sp = pytest.importorskip("scipy.sparse")
    s = W.lognormal3d(128, seed=1)
    rp, ci, val, b = to_cuda(s)
    A = sp.csr_matrix((s.val, s.ci, s.rp), shape=(s.n, s.n))
    bn = np.linalg.norm(s.b)
    h = amg.amg_setup(rp, ci, val)
    x = torch.zeros_like(b)
    info = amg.amg_solve(h, b, x, rtol=1e-8, max_iter=5000)
    assert info.status == amg.AMG_OK, info
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) / bn <= 1.01e-8
    its_solver = info.iterations
    x = torch.zeros_like(b)
    info_v = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
    assert info_v.iterations < its_solver  # Krylov acceleration needs fewer cycles (Sec. 4.4)
    h.close()
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(cycle=amg.AMG_CYCLE_W))
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
    assert info.status == amg.AMG_OK
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) / bn <= 1.01e-8
    assert info.iterations <= info_v.iterations
    h.close()
