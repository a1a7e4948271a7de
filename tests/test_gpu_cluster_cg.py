"""The coarsest-level CG on one thread block cluster (coarsest levels of at
most 2048 rows) against the dense solve, the oracle's CG and the grid-wide CG
kernel (which the allocation-free entry point always uses).

Both CG forms stop at a relative residual of 1e-12 (Sec. 4.2's CG coarse
solver), so each agrees with the exact solve to about cond(A) * 1e-12 and
with the other to the same order; their iteration counts differ only by
rounding (the same recurrences summed in a different order)."""
import numpy as np
import pytest

sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, setup_both, to_cuda  # noqa: E402

ONE_LEVEL = [
    ("lognormal3d_12", lambda: W.lognormal3d(12, seed=4)),          # 1728 rows
    ("poisson2d_45_ragged", lambda: W.poisson2d(45)),              # 2025 rows, not a multiple of 16
    ("fem_p1_40", lambda: W.fem_p1_jittered(40, seed=2)),          # 1600 rows
    ("random_spd_2048", lambda: W.random_spd(2048, 0.003, 9)),     # the largest cluster size
    ("random_spd_5", lambda: W.random_spd(5, 0.6, 7)),              # fewer rows than CTAs
    ("random_spd_1", lambda: W.random_spd(1, 1.0, 3)),
]


@pytest.mark.parametrize("name,make", ONE_LEVEL, ids=[c[0] for c in ONE_LEVEL])
def test_cluster_cg_one_level_solve(name, make):
    """A one-level hierarchy with the CG coarse solver: its cycle is the CG
    solve itself; against the dense solve, the oracle's CG (same iteration
    count within a few) and the grid-wide kernel."""
    s = make()
    h, oh, b = setup_both(s, max_levels=1, coarse_solver=amg.AMG_COARSE_CG)
    assert h.num_levels == 1
    assert amg.amg_coarse_cg_cluster_size(h) in (8, 16)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    zc = z.cpu().numpy()
    A = sp.csr_matrix((s.val, s.ci, s.rp), shape=(s.n, s.n))
    bn = np.linalg.norm(s.b)
    # the stopping rule is ||r|| <= 1e-12 ||b|| on the recurrence residual; the
    # true residual of the pipelined recurrences drifts from it by rounding
    assert np.linalg.norm(s.b - A @ zc) <= 1e-10 * bn
    x = spla.spsolve(A.tocsc(), s.b)
    assert rel_err(zc, x) < 1e-8
    assert rel_err(zc, oh.vcycle(s.b)) < 1e-8
    rp, ci, val, _ = to_cuda(s)
    xg = torch.zeros_like(b)
    its_grid = amg.amg_coarse_cg_noalloc(rp, ci, val, b, xg)
    assert rel_err(zc, xg.cpu().numpy()) < 1e-8
    assert abs(its_grid - oh.last_coarse_cg_iters) <= max(3, oh.last_coarse_cg_iters // 7)


def test_cluster_cg_inside_multilevel_cycles_and_mixed_precision():
    """A stalled lognormal hierarchy whose coarsest level (a few thousand rows)
    goes to the cluster: V-cycle and W-cycle equal the oracle's to the CG
    tolerance, FP64 PCG matches the oracle's iterations, the FP32 cycle stays
    within its bound."""
    s = W.lognormal3d(32, seed=1)
    h, oh, b = setup_both(s, coarse_max=100)
    assert not oh.dense_coarse and h.sizes()[-1] <= 2048
    assert amg.amg_coarse_cg_cluster_size(h) in (8, 16)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-9
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=True)
    x_o, info_o = oh.pcg(s.b, rtol=1e-8, flexible=True)
    assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
    x = torch.zeros_like(b)
    amg.pcg_solve(h, b, x, rtol=0.0, max_iter=info_o.iterations, flexible=True)
    assert rel_err(x.cpu().numpy(), x_o) < 1e-10
    hw, ohw, _ = setup_both(s, coarse_max=100, cycle=amg.AMG_CYCLE_W)
    amg.amg_vcycle(hw, b, z)
    assert rel_err(z.cpu().numpy(), ohw.vcycle(s.b)) < 1e-9
    h32, _, _ = setup_both(s, coarse_max=100, precision=amg.AMG_FP32)
    assert amg.amg_coarse_cg_cluster_size(h32) in (8, 16)
    amg.amg_vcycle(h32, b, z)
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-5


def test_cluster_cg_is_deterministic_and_size_limit():
    s = W.lognormal3d(32, seed=1)
    h, _, b = setup_both(s, coarse_max=100)
    zs = []
    for _ in range(3):
        z = torch.empty_like(b)
        amg.amg_vcycle(h, b, z)
        zs.append(z.cpu().numpy())
    assert np.array_equal(zs[0].view(np.int64), zs[1].view(np.int64))
    assert np.array_equal(zs[0].view(np.int64), zs[2].view(np.int64))
    # above 2048 rows the whole GPU solves the coarsest level
    big = W.lognormal3d(14, seed=1)  # 2744 rows, one level
    rp, ci, val, bb = to_cuda(big)
    hb = amg.amg_setup(rp, ci, val, amg.amg_default_params(max_levels=1, coarse_solver=amg.AMG_COARSE_CG))
    assert amg.amg_coarse_cg_cluster_size(hb) == 0
    zb = torch.empty_like(bb)
    amg.amg_vcycle(hb, bb, zb)
    A = sp.csr_matrix((big.val, big.ci, big.rp), shape=(big.n, big.n))
    assert np.linalg.norm(big.b - A @ zb.cpu().numpy()) <= 1e-10 * np.linalg.norm(big.b)
    # a dense coarsest level reports -1
    hd = amg.amg_setup(*to_cuda(W.poisson2d(20))[:3])
    assert amg.amg_coarse_cg_cluster_size(hd) == -1
