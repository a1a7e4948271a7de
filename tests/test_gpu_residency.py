"""Level matrices in host memory during the solve phase (Sec. 3.1.1, the
hybrid CPU/GPU-CI algorithm): the same kernels read the same numbers from
pinned host memory (mapped) or from device buffers that a copy stream fills
one visit ahead (staged), so every result must equal the resident
hierarchy's bit for bit, and the oracle's to its usual tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, setup_both, to_cuda  # noqa: E402

MODES = [(amg.AMG_HOST_MAPPED, 0), (amg.AMG_HOST_STAGED, 0), (amg.AMG_HOST_STAGED, 1), (amg.AMG_HOST_MAPPED, 2)]


def _bits(t):
    return t.cpu().numpy().view(np.int64)


def _pcg(h, b, flexible=True):
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=1e-10, max_iter=500, flexible=flexible, check=True)
    return x, info.iterations


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32, amg.AMG_FP16_STORAGE])
@pytest.mark.parametrize("mode", MODES, ids=lambda m: f"{['resident', 'mapped', 'staged'][m[0]]}_from{m[1]}")
def test_host_levels_give_the_resident_result(mode, precision):
    s = W.lognormal3d(28, seed=3)
    h, oh, b = setup_both(s, coarse_max=200, precision=precision)
    assert h.num_levels >= 4
    z_res = torch.empty_like(b)
    amg.amg_vcycle(h, b, z_res)
    x_res, it_res = _pcg(h, b)
    before = amg.amg_memory_info(h)
    assert before["host_bytes"] == 0 and before["staging_bytes"] == 0
    amg.amg_set_residency(h, mode[0], mode[1])
    moved = amg.amg_memory_info(h)
    assert moved["host_bytes"] > 0
    assert moved["device_bytes"] - moved["staging_bytes"] + moved["host_bytes"] == before["device_bytes"]
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    np.testing.assert_array_equal(_bits(z), _bits(z_res))
    for _ in range(2):  # the second solve would replay a graph on a resident hierarchy
        x, it = _pcg(h, b)
        assert it == it_res
        np.testing.assert_array_equal(_bits(x), _bits(x_res))
    if precision == amg.AMG_FP64:
        assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-12
    # and back
    amg.amg_set_residency(h, amg.AMG_RESIDENT)
    assert amg.amg_memory_info(h)["device_bytes"] == before["device_bytes"]
    x, it = _pcg(h, b)
    np.testing.assert_array_equal(_bits(x), _bits(x_res))


@pytest.mark.parametrize("cycle", [amg.AMG_CYCLE_W, amg.AMG_CYCLE_F])
def test_staged_w_and_f_cycles(cycle):
    """Visits the V-cycle prediction does not foresee are copied on demand."""
    s = W.lognormal3d(20, seed=5)
    h, oh, b = setup_both(s, coarse_max=100, cycle=cycle)
    z_res = torch.empty_like(b)
    amg.amg_vcycle(h, b, z_res)
    x_res = torch.zeros_like(b)
    i_res = amg.amg_solve(h, b, x_res, rtol=1e-9, check=True)
    amg.amg_set_residency(h, amg.AMG_HOST_STAGED, 0)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    np.testing.assert_array_equal(_bits(z), _bits(z_res))
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-12
    x = torch.zeros_like(b)
    i = amg.amg_solve(h, b, x, rtol=1e-9, check=True)
    assert i.iterations == i_res.iterations
    np.testing.assert_array_equal(_bits(x), _bits(x_res))


@pytest.mark.parametrize("nu", [(1, 1), (2, 3), (1, 0)])
def test_staged_explicit_sweeps(nu):
    s = W.poisson2d(97)
    h, oh, b = setup_both(s, coarse_max=50, nu_pre=nu[0], nu_post=nu[1], operator_form=0)
    z_res = torch.empty_like(b)
    amg.amg_vcycle(h, b, z_res)
    amg.amg_set_residency(h, amg.AMG_HOST_STAGED, 0)
    z = torch.empty_like(b)
    amg.amg_vcycle(h, b, z)
    np.testing.assert_array_equal(_bits(z), _bits(z_res))
    assert rel_err(z.cpu().numpy(), oh.vcycle(s.b)) < 1e-12


def test_staging_copies_each_matrix_once_per_v_cycle():
    """With the V-cycle prediction every visit finds its matrix already copied
    (or on its way), so a cycle copies each staged array exactly once."""
    s = W.anisotropic3d(32)
    h, _, b = setup_both(s, coarse_max=100)
    amg.amg_set_residency(h, amg.AMG_HOST_STAGED, 0)
    z = torch.empty_like(b)
    copied = [amg.amg_memory_info(h)["copied_bytes"]]
    for _ in range(4):
        amg.amg_vcycle(h, b, z)
        copied.append(amg.amg_memory_info(h)["copied_bytes"])
    per_cycle = np.diff(copied)
    info = amg.amg_memory_info(h)
    # level 0's A stays resident; C and Q of every level, and the column
    # indices of A (which C shares) below level 0, are copied
    assert per_cycle[1] == per_cycle[2] == per_cycle[3] > 0
    assert per_cycle[1] < info["host_bytes"]
    assert per_cycle[0] >= per_cycle[1]


def test_batched_solve_on_a_host_level_hierarchy():
    """The batched kernel reads a host-resident hierarchy through the link."""
    systems = [W.poisson2d(40, seed=7 + i) for i in range(3)]
    hs, bs, xr, xs = [], [], [], []
    for s in systems:
        rp, ci, val, b = to_cuda(s)
        hs.append(amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=64)))
        bs.append(b)
    xr = [torch.zeros_like(b) for b in bs]
    amg.amg_batch_pcg(hs, bs, xr, rtol=1e-10, flexible=True)
    for h in hs:
        amg.amg_set_residency(h, amg.AMG_HOST_MAPPED, 0)
    xs = [torch.zeros_like(b) for b in bs]
    infos = amg.amg_batch_pcg(hs, bs, xs, rtol=1e-10, flexible=True)
    assert all(i.status == amg.AMG_OK for i in infos)
    for a, r in zip(xs, xr):
        np.testing.assert_array_equal(_bits(a), _bits(r))


def test_residency_errors():
    s = W.poisson2d(64)
    rp, ci, val, b = to_cuda(s)
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=64))
    L = h.num_levels - 1
    for mode, first in [(3, 0), (-1, 0), (amg.AMG_HOST_MAPPED, -1), (amg.AMG_HOST_STAGED, L)]:
        with pytest.raises(amg.AmgError) as e:
            amg.amg_set_residency(h, mode, first)
        assert e.value.status == amg.AMG_ERR_INVALID_ARG
    amg.amg_set_residency(h, amg.AMG_HOST_STAGED, 0)
    with pytest.raises(amg.AmgError) as e:
        amg.amg_autotune(h)
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED
    amg.amg_set_residency(h, amg.AMG_RESIDENT)
    amg.amg_autotune(h)
    h.close()
