"""GPU setup phase vs the oracle: aggregates, P/A_c patterns and values bit-exact.

Covers the paper's worked example, tie-heavy uniform grids (many handshake
rounds), lognormal coefficients (hub-star coarsening), anisotropy,
nonsymmetric values, P1 finite elements, random graphs, and the full-size
128^3 lognormal system of the benchmark."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.conftest import read_golden  # noqa: E402
from tests.gpu_util import assert_hierarchy_bitexact, setup_both, to_cuda  # noqa: E402


def test_worked_example_on_gpu():
    g = read_golden("worked_example.txt")
    s = W.from_dense(g["A"])
    # one pass, one coarsening step: P and A_c of the worked example
    h, oh, _ = setup_both(s, passes=1, coarse_max=3)
    assert h.sizes() == [6, 3]
    agg = torch.empty(6, dtype=torch.int32, device="cuda")
    amg.amg_level_info(h, 0, agg)
    P = np.zeros((6, 3))
    P[np.arange(6), agg.cpu().numpy()] = 1
    np.testing.assert_array_equal(P, g["P"])
    rp, ci, val = amg.amg_export_level(h, 1)
    ac = np.zeros((3, 3))
    rows = np.repeat(np.arange(3), np.diff(rp.cpu().numpy()))
    ac[rows, ci.cpu().numpy()] = val.cpu().numpy()
    np.testing.assert_array_equal(ac, g["Ac"])
    assert amg.amg_setup_rounds(h, 0, 0) == 2  # one productive round + the empty one
    assert_hierarchy_bitexact(h, oh)


@pytest.mark.parametrize("case", [
    ("poisson2d_64", lambda: W.poisson2d(64), dict(coarse_max=64)),
    ("poisson2d_97_ragged", lambda: W.poisson2d(97), dict(coarse_max=50)),
    ("aniso3d_16", lambda: W.anisotropic3d(16), dict(coarse_max=64)),
    ("aniso3d_33", lambda: W.anisotropic3d(33, eps_z=1e-2, seed=5), dict(coarse_max=100)),
    ("lognormal3d_24", lambda: W.lognormal3d(24, seed=1), dict()),
    ("lognormal3d_40", lambda: W.lognormal3d(40, seed=7), dict(coarse_max=500)),
    ("convdiff2d_48", lambda: W.convdiff2d(48, peclet=300.0), dict(coarse_max=40)),
    ("fem_p1_50", lambda: W.fem_p1_jittered(50, seed=3), dict(coarse_max=30)),
    ("random_ties", lambda: W.random_spd(700, 0.01, 3, int_weights=True), dict(coarse_max=20)),
    ("one_pass_six_levels", lambda: W.lognormal3d(20, seed=2), dict(passes=1, max_levels=6, coarse_max=10)),
    ("three_passes", lambda: W.poisson2d(70), dict(passes=3, coarse_max=30)),
], ids=lambda c: c[0])
def test_hierarchy_bitexact(case):
    _, make, kw = case
    s = make()
    h, oh, _ = setup_both(s, **kw)
    assert_hierarchy_bitexact(h, oh)


def test_handshake_round_counts_match_literal_rounds():
    s = W.poisson2d(64)
    h, oh, _ = setup_both(s, coarse_max=64, matcher=1)
    assert_hierarchy_bitexact(h, oh)
    for k in range(oh.num_levels - 1):
        rounds = oh.level_info(k)[2]
        for p in range(2):
            assert amg.amg_setup_rounds(h, k, p) == rounds[p]
    assert amg.amg_setup_rounds(h, 0, 0) == 96


def test_full_size_lognormal_128_setup_bitexact():
    """The 128^3 lognormal system (2.1M unknowns): whole hierarchy bit-exact."""
    s = W.lognormal3d(128, seed=1)
    h, oh, _ = setup_both(s)
    assert_hierarchy_bitexact(h, oh)
    assert oh.num_levels >= 4 and not oh.dense_coarse


def test_setup_errors():
    s = W.poisson2d(8)
    rp, ci, val, _ = to_cuda(s)
    bad_ci = ci.clone()
    bad_ci[3] = 1000
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, bad_ci, val)
    assert e.value.status == amg.AMG_ERR_INVALID_CSR
    unsorted = ci.clone()
    unsorted[0], unsorted[1] = ci[1].item(), ci[0].item()
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, unsorted, val)
    assert e.value.status == amg.AMG_ERR_INVALID_CSR
    zero_diag = val.clone()
    zero_diag[0] = 0.0  # row 0 starts with its diagonal
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, ci, zero_diag, coarse_max=4)
    assert e.value.status == amg.AMG_ERR_ZERO_DIAG
    nan = val.clone()
    nan[5] = float("nan")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, ci, nan)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    # structurally nonsymmetric pattern is reported, not mis-coarsened
    a = s.dense()
    a[0, 20] = -0.5
    ns = W.from_dense(a)
    rp2, ci2, val2, _ = to_cuda(ns)
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp2, ci2, val2, coarse_max=4)
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED


def test_degenerate_inputs():
    # 1 x 1 system, diagonal matrix (no edges), matrix at or below coarse_max
    for a in (np.array([[3.0]]), np.diag(np.arange(1.0, 40.0))):
        s = W.from_dense(a)
        h, oh, _ = setup_both(s, coarse_max=1 if a.shape[0] > 1 else 4)
        assert h.num_levels == 1
        assert_hierarchy_bitexact(h, oh)
    s = W.poisson2d(10)
    h, oh, _ = setup_both(s)  # 100 <= 4096: coarsest level only
    assert h.num_levels == 1


def test_setup_is_deterministic():
    s = W.lognormal3d(30, seed=11)
    rp, ci, val, _ = to_cuda(s)
    p = amg.amg_default_params(coarse_max=200)
    h1 = amg.amg_setup(rp, ci, val, p)
    h2 = amg.amg_setup(rp, ci, val, p)
    for k in range(h1.num_levels):
        for a, b in zip(amg.amg_export_level(h1, k), amg.amg_export_level(h2, k)):
            assert torch.equal(a, b)
