"""Matching options on the GPU against the oracle, bit for bit: Algorithm 3's
own tie order (its edge list sorted lexicographically descending, so equal
weights go to the larger index) and the diagonally scaled edge weight
max(|a_ij|,|a_ji|) / sqrt(|a_ii a_jj|) (an option outside the paper).

Tie-heavy uniform grids exercise the tie order (many handshake rounds); the
lognormal systems exercise the scaled weight, which keeps coarsening where the
plain weight stalls."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import assert_hierarchy_bitexact, rel_err, setup_both, to_cuda  # noqa: E402

CASES = [
    ("poisson2d_63_odd", lambda: W.poisson2d(63), dict(coarse_max=40)),
    ("poisson2d_97_ragged", lambda: W.poisson2d(97), dict(coarse_max=50)),
    ("aniso3d_17", lambda: W.anisotropic3d(17), dict(coarse_max=64)),
    ("lognormal3d_24", lambda: W.lognormal3d(24, seed=1), dict(coarse_max=100)),
    ("lognormal3d_40", lambda: W.lognormal3d(40, seed=7), dict(coarse_max=500)),
    ("convdiff2d_48_nonsymmetric", lambda: W.convdiff2d(48, peclet=300.0), dict(coarse_max=40)),
    ("fem_p1_50", lambda: W.fem_p1_jittered(50, seed=3), dict(coarse_max=30)),
    ("random_ties", lambda: W.random_spd(700, 0.01, 3, int_weights=True), dict(coarse_max=20)),
]
OPTIONS = [
    ("tie_larger", dict(tie_break=amg.AMG_TIE_LARGER)),
    ("scaled_weight", dict(edge_weight=amg.AMG_WEIGHT_SCALED)),
    ("both", dict(tie_break=amg.AMG_TIE_LARGER, edge_weight=amg.AMG_WEIGHT_SCALED)),
]


@pytest.mark.parametrize("opt", OPTIONS, ids=lambda o: o[0])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hierarchy_bitexact_with_option(case, opt):
    _, make, kw = case
    s = make()
    h, oh, _ = setup_both(s, **kw, **opt[1])
    assert_hierarchy_bitexact(h, oh)


def test_literal_rounds_with_larger_ties():
    """Round counts of the device handshakes equal the oracle's literal rounds
    under the descending tie order too."""
    s = W.poisson2d(63)
    h, oh, _ = setup_both(s, coarse_max=40, matcher=1, tie_break=amg.AMG_TIE_LARGER)
    assert_hierarchy_bitexact(h, oh)
    for k in range(oh.num_levels - 1):
        rounds = oh.level_info(k)[2]
        for p in range(2):
            assert amg.amg_setup_rounds(h, k, p) == rounds[p]


def test_scaled_weight_breaks_the_lognormal_stall_and_solves():
    """With the plain weight the 48^3 lognormal hierarchy stops on a stalled
    level of thousands of rows; the scaled weight keeps coarsening.  Both
    hierarchies precondition PCG to 1e-8, with the same iterates as the
    oracle's at the oracle's iteration count."""
    s = W.lognormal3d(48, seed=1)
    sizes = {}
    for name, kw in (("abs", {}), ("scaled", dict(edge_weight=amg.AMG_WEIGHT_SCALED))):
        h, oh, b = setup_both(s, **kw)
        assert h.sizes() == oh.sizes()
        sizes[name] = h.sizes()
        flexible = not oh.dense_coarse
        x = torch.zeros_like(b)
        info = amg.pcg_solve(h, b, x, rtol=1e-8, flexible=flexible)
        x_o, info_o = oh.pcg(s.b, rtol=1e-8, flexible=flexible)
        assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
        x = torch.zeros_like(b)
        amg.pcg_solve(h, b, x, rtol=0.0, max_iter=info_o.iterations, flexible=flexible)
        assert rel_err(x.cpu().numpy(), x_o) < 1e-10
    assert sizes["scaled"][-1] < sizes["abs"][-1]


def test_option_parameter_checks_and_zero_diagonal():
    s = W.poisson2d(20)
    rp, ci, val, b = to_cuda(s)
    for kw in (dict(tie_break=2), dict(tie_break=-1), dict(edge_weight=2)):
        with pytest.raises(amg.AmgError) as e:
            amg.amg_setup(rp, ci, val, amg.amg_default_params(**kw))
        assert e.value.status == amg.AMG_ERR_INVALID_ARG
    # a zero diagonal entry is reported by the scaled weight before any matching
    v = s.val.copy()
    d0 = int(np.flatnonzero(s.ci[s.rp[5]:s.rp[6]] == 5)[0]) + s.rp[5]
    v[d0] = 0.0
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup(rp, ci, torch.from_numpy(v).to(b.device),
                      amg.amg_default_params(edge_weight=amg.AMG_WEIGHT_SCALED))
    assert e.value.status == amg.AMG_ERR_ZERO_DIAG


def test_full_size_lognormal_128_scaled_weight_bitexact():
    """The benchmark system with the scaled weight: whole hierarchy bit-exact
    against the oracle, and far smaller coarsest level than the plain one."""
    s = W.lognormal3d(128, seed=1)
    h, oh, _ = setup_both(s, edge_weight=amg.AMG_WEIGHT_SCALED)
    assert_hierarchy_bitexact(h, oh)
    assert h.sizes()[-1] < 20000
