"""Host-side logic of the solve server, on the CPU: request fingerprints,
device-memory estimates, per-request parameters and the least-recently-used
eviction under the memory budget (no GPU: the server object is assembled
without its worker threads and its hierarchies are stand-ins)."""
import collections
import threading

import numpy as np

from paper_2007_00056_gb300 import amg
from paper_2007_00056_gb300 import serving as S
from paper_2007_00056_gb300 import workloads as W


def test_fingerprint_identifies_the_matrix():
    s = W.poisson2d(10)
    k = S.fingerprint(s.rp, s.ci, s.val)
    assert k == S.fingerprint(s.rp.copy(), s.ci.copy(), s.val.copy())
    v = s.val.copy()
    v[3] = np.nextafter(v[3], 0.0)
    assert S.fingerprint(s.rp, s.ci, v) != k
    t = W.poisson2d(11)
    assert S.fingerprint(t.rp, t.ci, t.val) != k
    assert k.startswith(f"{s.n}:{s.nnz}:")


def test_memory_estimate_grows_with_the_system_and_the_fp32_copies():
    a = S.estimate_bytes(1000, 5000, amg.AMG_FP64)
    b = S.estimate_bytes(2000, 10000, amg.AMG_FP64)
    assert 0 < a < b
    assert S.estimate_bytes(1000, 5000, amg.AMG_FP32) > a
    # at least the input CSR and the hierarchy's share of it
    assert a >= 5000 * 12 + 4 * 1001


class _FakeH:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def _bare_server(budget):
    srv = S.SolveServer.__new__(S.SolveServer)
    srv.budget = budget
    srv.precision = amg.AMG_FP32
    srv.small_max_n = 5000
    srv.batch_coarse_max = 256
    srv.big_coarse_max = 1024
    srv.big_dense_max = 8192
    srv.params = {"edge_weight": amg.AMG_WEIGHT_SCALED}
    srv._lock = threading.Condition()
    srv._in_use = 0
    srv._cache = collections.OrderedDict()
    srv._cache_bytes = 0
    srv.stats = collections.Counter()
    return srv


def test_eviction_is_lru_over_idle_hierarchies_only():
    srv = _bare_server(budget=100)
    hs = {}
    for key, nbytes, users in (("a", 30, 0), ("b", 30, 1), ("c", 30, 0)):
        hs[key] = _FakeH()
        e = S._Entry(hs[key], nbytes, key)
        e.users = users
        srv._cache[key] = e
        srv._cache_bytes += nbytes
    # room for 10 more: nothing evicted
    assert srv._evict_for(10) and not any(h.closed for h in hs.values())
    # 40 more: the least recent idle entry ("a") goes; "b" is in use and stays
    assert srv._evict_for(40)
    assert hs["a"].closed and not hs["b"].closed and not hs["c"].closed
    assert list(srv._cache) == ["b", "c"] and srv._cache_bytes == 60
    # 70 more needs "c" too; 80 more cannot be found while "b" is in use
    assert srv._evict_for(70) and hs["c"].closed
    assert not srv._evict_for(80)
    assert srv.stats["evicted"] == 2


def test_cache_hit_moves_the_entry_to_most_recent():
    srv = _bare_server(budget=1000)
    for key in ("x", "y", "z"):
        srv._cache[key] = S._Entry(_FakeH(), 10, key)
    e = srv._cache_get("x")
    assert e is not None and e.users == 1
    assert list(srv._cache) == ["y", "z", "x"]
    assert srv._cache_get("missing") is None


def test_small_and_large_requests_get_their_coarse_limits():
    srv = _bare_server(budget=1000)
    small = srv._params_for(4000)
    large = srv._params_for(6000)
    assert small.coarse_max == 256 and large.coarse_max == 1024
    # a large hierarchy that stalls above its stop size keeps the dense coarsest solve
    assert small.dense_max == 0 and large.dense_max == 8192
    assert small.precision == large.precision == amg.AMG_FP32
    assert small.cycle == amg.AMG_CYCLE_V  # the batched kernel runs V-cycles
    assert small.edge_weight == large.edge_weight == amg.AMG_WEIGHT_SCALED
    srv.params = {"edge_weight": amg.AMG_WEIGHT_ABS, "operator_form": 0}
    p = srv._params_for(6000)
    assert p.edge_weight == amg.AMG_WEIGHT_ABS and p.operator_form == 0 and p.dense_max == 8192


def test_batcher_hands_a_failed_batch_back_to_the_workers(monkeypatch):
    """A batch that fails as a whole returns every system to its worker (info
    None: the worker then solves it alone) instead of leaving it waiting."""
    import queue

    srv = _bare_server(budget=100)
    srv.dev = None
    srv.max_batch = 8
    srv.batch_window_s = 0.001
    srv._stop = False
    monkeypatch.setattr(S.torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(S.torch.cuda, "Stream", lambda device=None: None)

    def failing_batch(*args, **kwargs):
        raise RuntimeError("batch failed")

    monkeypatch.setattr(S.amg, "amg_batch_pcg", failing_batch)
    bq = queue.Queue()
    items = [(object(), None, None, threading.Event(), {}) for _ in range(3)]
    for it in items:
        bq.put(it)
    t = threading.Thread(target=srv._batch_loop, args=(bq, 1), daemon=True)
    t.start()
    try:
        for it in items:
            assert it[3].wait(5.0)
    finally:
        srv._stop = True
        t.join(5.0)
    assert not t.is_alive()
    assert all(it[4]["info"] is None for it in items)
    assert srv.stats["batch_errors"] >= 1 and srv.stats["batches"] == 0
