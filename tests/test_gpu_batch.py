"""Batched PCG (one thread block per system, or a cluster of 2, 4 or 8 blocks
for systems above 8192, 24576 and 65536 rows): each system's result is
bitwise the same alone and in any batch, and agrees with the oracle like
pcg_solve."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import rel_err, to_cuda  # noqa: E402


def _systems():
    return [W.poisson2d(31, seed=5), W.lognormal3d(12, seed=7), W.fem_p1_jittered(40, seed=3),
            W.anisotropic3d(14, seed=4), W.poisson2d(70, seed=9), W.lognormal3d(9, seed=2),
            W.fem_p1_jittered(23, seed=8)]


def _setup(systems, precision, coarse_max=200, **kw):
    hs, bs = [], []
    for s in systems:
        rp, ci, val, b = to_cuda(s)
        hs.append(amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=coarse_max, precision=precision,
                                                                    **kw)))
        bs.append(b)
    return hs, bs


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32])
def test_batch_alone_equals_in_mix_bitwise(precision):
    systems = _systems()
    hs, bs = _setup(systems, precision)
    xs = [torch.zeros_like(b) for b in bs]
    infos = amg.amg_batch_pcg(hs, bs, xs, rtol=1e-8, flexible=True)
    assert all(i.status == amg.AMG_OK for i in infos)
    for k in range(len(systems)):
        x1 = torch.zeros_like(bs[k])
        i1 = amg.amg_batch_pcg([hs[k]], [bs[k]], [x1], rtol=1e-8, flexible=True)[0]
        assert i1.iterations == infos[k].iterations
        assert torch.equal(x1, xs[k]), f"system {k} differs alone vs in the batch"
    # a different batch composition and order: still identical
    order = [5, 2, 0]
    xs2 = [torch.zeros_like(bs[k]) for k in order]
    amg.amg_batch_pcg([hs[k] for k in order], [bs[k] for k in order], xs2, rtol=1e-8, flexible=True)
    for j, k in enumerate(order):
        assert torch.equal(xs2[j], xs[k])


def test_batch_matches_oracle_fp64():
    systems = _systems()
    hs, bs = _setup(systems, amg.AMG_FP64)
    xs = [torch.zeros_like(b) for b in bs]
    infos = amg.amg_batch_pcg(hs, bs, xs, rtol=1e-8)
    for s, h, info, x in zip(systems, hs, infos, xs):
        oh = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=200)
        assert oh.sizes() == h.sizes()
        x_o, info_o = oh.pcg(s.b, rtol=1e-8)
        assert info.status == amg.AMG_OK and abs(info.iterations - info_o.iterations) <= 1
        assert info.rel_res_true <= 1.01e-8
    # fixed iteration count: solutions within 1e-10 of the oracle's
    ks = [0, 1, 2]
    outs = [torch.zeros_like(bs[k]) for k in ks]
    its = []
    for k in ks:
        oh = O.Hierarchy(systems[k].rp, systems[k].ci, systems[k].val, coarse_max=200)
        _, io = oh.pcg(systems[k].b, rtol=1e-8)
        its.append(io.iterations)
    for k, out, it in zip(ks, outs, its):
        amg.amg_batch_pcg([hs[k]], [bs[k]], [out], rtol=0.0, max_iter=it)
        oh = O.Hierarchy(systems[k].rp, systems[k].ci, systems[k].val, coarse_max=200)
        x_o, _ = oh.pcg(systems[k].b, rtol=0.0, max_iter=it)
        assert rel_err(out.cpu().numpy(), x_o) < 1e-10


def test_batch_agrees_with_single_solve():
    systems = _systems()[:3]
    hs, bs = _setup(systems, amg.AMG_FP32)
    xs = [torch.zeros_like(b) for b in bs]
    infos = amg.amg_batch_pcg(hs, bs, xs, rtol=1e-8, flexible=True)
    for h, b, x, info in zip(hs, bs, xs, infos):
        y = torch.zeros_like(b)
        i2 = amg.pcg_solve(h, b, y, rtol=1e-8, flexible=True)
        assert abs(i2.iterations - info.iterations) <= 1
        assert rel_err(x.cpu().numpy(), y.cpu().numpy()) < 1e-7


def test_batch_rejections():
    s = W.poisson2d(20)
    hs, bs = _setup([s, s], amg.AMG_FP64)
    xs = [torch.zeros_like(b) for b in bs]
    with pytest.raises(amg.AmgError) as e:  # the same hierarchy twice
        amg.amg_batch_pcg([hs[0], hs[0]], bs, xs)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    h32, b32 = _setup([s], amg.AMG_FP32)
    with pytest.raises(amg.AmgError) as e:  # mixed precisions
        amg.amg_batch_pcg([hs[0], h32[0]], [bs[0], b32[0]], [xs[0], torch.zeros_like(b32[0])])
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    rp, ci, val, b = to_cuda(W.lognormal3d(30, seed=1))
    hcg = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=100, coarse_solver=amg.AMG_COARSE_CG))
    with pytest.raises(amg.AmgError) as e:  # coarsest level not dense
        amg.amg_batch_pcg([hcg], [b], [torch.zeros_like(b)])
    assert e.value.status == amg.AMG_ERR_UNSUPPORTED
    # b = 0 inside a batch
    xz = [torch.ones_like(bs[0]), torch.zeros_like(bs[1])]
    infos = amg.amg_batch_pcg(hs, [torch.zeros_like(bs[0]), bs[1]], xz, rtol=1e-8)
    assert infos[0].iterations == 0 and torch.all(xz[0] == 0) and infos[1].status == amg.AMG_OK


def _large_systems():
    # one, two, four and eight blocks per system
    return [W.poisson2d(60, seed=3), W.poisson2d(100, seed=4), W.fem_p1_jittered(170, seed=5),
            W.anisotropic3d(42, seed=6)]


@pytest.mark.parametrize("precision", [amg.AMG_FP64, amg.AMG_FP32])
def test_cluster_teams_alone_equal_in_mix_and_match_oracle(precision):
    systems = _large_systems()
    assert [s.n for s in systems] == [3600, 10000, 28900, 74088]
    # a stalled coarsest level keeps the dense solve the batched kernel needs
    hs, bs = _setup(systems, precision, coarse_max=256, dense_max=2048)
    xs = [torch.zeros_like(b) for b in bs]
    infos = amg.amg_batch_pcg(hs, bs, xs, rtol=1e-8, flexible=True)
    assert all(i.status == amg.AMG_OK and i.rel_res_true <= 1e-8 for i in infos), infos
    for k in range(len(systems)):
        x1 = torch.zeros_like(bs[k])
        i1 = amg.amg_batch_pcg([hs[k]], [bs[k]], [x1], rtol=1e-8, flexible=True)[0]
        assert i1.iterations == infos[k].iterations
        assert torch.equal(x1, xs[k]), f"system {k} differs alone vs in the batch"
    # the same system twice in one launch of its team size (two hierarchies)
    h2, b2 = _setup([systems[2]], precision, coarse_max=256, dense_max=2048)
    xa, xb = torch.zeros_like(bs[2]), torch.zeros_like(b2[0])
    amg.amg_batch_pcg([hs[2], h2[0]], [bs[2], b2[0]], [xa, xb], rtol=1e-8, flexible=True)
    assert torch.equal(xa, xb) and torch.equal(xa, xs[2])
    for s, h, info, x in zip(systems, hs, infos, xs):
        oh = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=256)
        assert oh.sizes() == h.sizes()
        x_o, info_o = oh.pcg(s.b, rtol=1e-12, flexible=True)
        # both stop at a relative residual of 1e-8 or below: the error is at
        # most cond(A) 1e-8, a few 1e-5 for these systems
        assert rel_err(x.cpu().numpy(), x_o) < 1e-5
        if precision == amg.AMG_FP64:
            _, io = oh.pcg(s.b, rtol=1e-8, flexible=True)
            assert abs(info.iterations - io.iterations) <= 1
