"""Hierarchies set up and solved at the same time on several host threads and
streams (the server's pattern): every result must equal the one computed
alone, bit for bit.  Coarsest levels of different sizes exercise the
process-wide kernel attributes (shared-memory limits) that one thread's setup
must not lower under another thread's launch."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2007_00056_gb300 import amg  # noqa: E402
from paper_2007_00056_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import to_cuda  # noqa: E402


def _solve(s, params, stream):
    with torch.cuda.stream(stream):
        rp, ci, val, b = to_cuda(s)
        h = amg.amg_setup(rp, ci, val, params, stream=stream)
        x = torch.zeros_like(b)
        info = amg.pcg_solve(h, b, x, rtol=1e-9, flexible=True, stream=stream)
        stream.synchronize()
        sizes = h.sizes()
        h.close()
    return info, x.cpu().numpy(), sizes


def test_concurrent_setups_and_solves_equal_sequential():
    # lognormal hierarchies stall at a few percent of N: coarsest levels of a
    # few hundred to about 2000 rows, each solved by the cluster CG with its
    # own shared-memory size
    systems = [W.lognormal3d(n, seed=40 + n) for n in (18, 21, 24, 27, 30, 33, 36, 39)]
    params = amg.amg_default_params(precision=amg.AMG_FP32, coarse_max=128)
    alone = [_solve(s, params, torch.cuda.Stream()) for s in systems]
    assert len({a[2][-1] for a in alone}) >= 4  # coarsest sizes differ
    results = {}
    errors = []

    def worker(t):
        stream = torch.cuda.Stream()
        try:
            for rep in range(3):
                for i in range(t, len(systems), 4):
                    results[(rep, i)] = _solve(systems[i], params, stream)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for (rep, i), (info, x, sizes) in results.items():
        assert info.status == amg.AMG_OK, (i, amg.status_string(info.status))
        assert info.iterations == alone[i][0].iterations
        np.testing.assert_array_equal(x.view(np.int64), alone[i][1].view(np.int64))
