"""Continuous-batching solve server over the C ABI.

Requests (a CSR system and a right-hand side, arriving over time) go through:

1. admission: FIFO, admitted only while the estimated device memory of the
   requests in flight plus the hierarchy cache stays inside a budget (default
   half of the free device memory at start); a finished request releases its
   memory, and the least recently used cached hierarchies are evicted when
   an admission needs room;
2. setup on a worker thread with its own CUDA stream: host-to-device copy and
   ``amg_setup`` (or a hit in the device hierarchy cache, keyed by a
   fingerprint of the matrix);
3. solve: a request whose hierarchy fits the batched kernel (dense coarsest
   level, at most ``small_max_n`` rows) joins the batch queue of its size
   class (``batch_classes``: rows up to 5000, 20000, 60000); a batcher thread
   per class (each with its own stream) launches ``amg_batch_pcg`` on
   whatever became ready within a short window, again and again, so requests
   that become ready while a batch runs join the next one, and batches of
   different classes overlap with each other and with the large solves on
   the worker streams.  Classes keep a batch's systems of similar size: a
   batch returns when its slowest system converges.  A team of one to eight
   thread blocks per system outruns the whole-GPU solve in throughput once a
   few systems of a class are ready together (measured: 32 systems of 60,000
   rows 2,142 solves/s batched against 259/s one at a time, 4 of them 490/s
   against 278/s; 64 of 8,100 rows 12,057/s against 440/s), but a lone
   mid-size system is 2-3x slower on its team than on the whole GPU; so a
   class launches the batched kernel only with at least ``batch_min``
   systems and otherwise hands them back to their workers.  Under a backlog
   the batches fill; at a light load the requests take the whole-GPU path.
   Requests whose matrix is already cached share its hierarchy and take
   turns on it (its work vectors serve one solve at a time).  Larger
   requests run ``pcg_solve`` on their worker's stream (16 workers by
   default), with the whole GPU.  Their hierarchies stop at 1024 rows
   (``big_coarse_max``) rather than the
   library's 4096: the dense inverse of the coarsest level costs 2 N_L^3
   operations, while one more level costs far less.  A hierarchy whose
   coarsening stalls above that (the P1 systems near 10^6 rows stop at a few
   thousand rows) still gets the dense inverse up to ``big_dense_max`` rows:
   a coarse CG would run hundreds of grid-wide iterations in every cycle.
   Every setup uses the scaled edge weight by default (``params``), which
   keeps the lognormal systems coarsening past the paper's weight's stall;
4. completion: the solution is copied to host memory; the latency is
   completion time minus arrival time.

Every solve is deterministic and independent of the others (block-local
reductions in the batched kernel, fixed-grid reductions elsewhere), so a
request's solution is the same alone and in any mix.
"""
from __future__ import annotations

import collections
import dataclasses
import hashlib
import queue
import threading
import time

import numpy as np
import torch

from . import amg


@dataclasses.dataclass
class ServeResult:
    rid: int
    x: np.ndarray
    iterations: int
    rel_res_true: float
    status: int
    arrival: float
    admitted: float
    finished: float
    path: str  # "batch" or "single"
    started: float = 0.0      # a worker picked the request up
    setup_done: float = 0.0   # input on the device and hierarchy ready

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def fingerprint(rp: np.ndarray, ci: np.ndarray, val: np.ndarray) -> str:
    """Cache key of a matrix: its sizes and the SHA-256 of its CSR bytes.  SHA-256
    runs on the CPUs' hash instructions, about twice as fast as BLAKE2 here, and
    a request hashes its whole matrix (up to about 80 MB) on its worker."""
    h = hashlib.sha256()
    for a in (rp, ci, val):
        h.update(np.ascontiguousarray(a).view(np.uint8))
    return f"{len(rp) - 1}:{len(ci)}:{h.hexdigest()}"


def estimate_bytes(n: int, nnz: int, precision: int) -> int:
    """Device bytes of a request in flight: its input, a hierarchy of about
    2.5x the fine CSR (geometric level sizes), FP32 copies in mixed modes,
    and the V-cycle and Krylov work vectors."""
    csr = nnz * 12 + 4 * (n + 1)
    hier = int(2.5 * csr) + (int(1.5 * nnz * 4) if precision != amg.AMG_FP64 else 0)
    vectors = n * 8 * 24
    return csr + hier + vectors + (1 << 20)


class _Entry:
    __slots__ = ("h", "bytes", "users", "key", "lock")

    def __init__(self, h, nbytes, key):
        self.h = h
        self.bytes = nbytes
        self.users = 0
        self.key = key
        # a hierarchy's work vectors serve one solve at a time: requests with
        # the same matrix (a cache hit) take turns
        self.lock = threading.Lock()


class SolveServer:
    def __init__(self, device: int = 0, memory_budget: int | None = None, precision: int = amg.AMG_FP32,
                 rtol: float = 1e-8, max_iter: int = 1000, workers: int = 16, small_max_n: int = 60000,
                 batch_coarse_max: int = 256, big_coarse_max: int = 1024, big_dense_max: int = 8192,
                 max_batch: int = 256,
                 cache_entries: int = 64, batch_classes=(5000, 20000, 60000), batch_window_s: float = 0.001,
                 batch_min=(1, 2, 3), params=None):
        self.dev = torch.device("cuda", device)
        # amg_params fields for every request's setup.  Default: the scaled
        # edge weight max(|a_ij|,|a_ji|)/sqrt(|a_ii a_jj|), an option the paper
        # does not have; with the paper's weight the variable-coefficient
        # systems stall at a few percent of N and their coarse CG dominates the
        # stream's GPU time (measured: 141 against 206 solves/s of capacity)
        self.params = {"edge_weight": amg.AMG_WEIGHT_SCALED} if params is None else dict(params)
        torch.cuda.set_device(self.dev)
        amg.lib()
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            memory_budget = free // 2
        self.budget = int(memory_budget)
        self.precision = precision
        self.rtol = rtol
        self.max_iter = max_iter
        self.small_max_n = small_max_n
        self.batch_coarse_max = batch_coarse_max
        self.big_coarse_max = big_coarse_max
        self.big_dense_max = big_dense_max
        self.max_batch = max_batch
        self.cache_entries = cache_entries
        self.batch_window_s = batch_window_s
        self._lock = threading.Condition()
        self._in_use = 0                      # bytes of admitted requests (inputs + work)
        self._cache: "collections.OrderedDict[str, _Entry]" = collections.OrderedDict()
        self._cache_bytes = 0
        self._pending: "collections.deque" = collections.deque()  # admitted, waiting for a worker
        self.batch_classes = tuple(sorted(c for c in batch_classes if c < small_max_n)) + (small_max_n,)
        # fewest systems a batch of each class needs to beat solving them one
        # by one on the worker streams (the batched kernel gives a system a
        # team of one to four thread blocks here, so a lone mid-size system
        # is faster on the whole GPU)
        bm = tuple(batch_min) + (batch_min[-1],) * len(self.batch_classes)
        self.batch_min = bm[:len(self.batch_classes)]
        self._batchqs = [queue.Queue() for _ in self.batch_classes]
        self._results: dict[int, ServeResult] = {}
        self._stop = False
        self.stats = collections.Counter()
        self._workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        self._batchers = [threading.Thread(target=self._batch_loop, args=(q, m), daemon=True)
                          for q, m in zip(self._batchqs, self.batch_min)]
        for t in self._workers + self._batchers:
            t.start()

    # ------------------------------------------------------------------ admission
    def _params_for(self, n: int):
        extra = getattr(self, "params", {})
        if n <= self.small_max_n:
            return amg.amg_default_params(**{"precision": self.precision, "coarse_max": self.batch_coarse_max,
                                             **extra})
        return amg.amg_default_params(**{"precision": self.precision, "coarse_max": self.big_coarse_max,
                                         "dense_max": self.big_dense_max, **extra})

    def _evict_for(self, need: int) -> bool:
        """Evicts idle cached hierarchies (least recent first) until `need` fits."""
        while self._in_use + self._cache_bytes + need > self.budget:
            victim = next((k for k, e in self._cache.items() if e.users == 0), None)
            if victim is None:
                return False
            e = self._cache.pop(victim)
            self._cache_bytes -= e.bytes
            e.h.close()
            self.stats["evicted"] += 1
        return True

    def submit(self, rid: int, rp, ci, val, b, arrival: float) -> None:
        n, nnz = len(rp) - 1, len(ci)
        need = estimate_bytes(n, nnz, self.precision)
        if need > self.budget:
            raise MemoryError(f"request {rid} needs about {need} bytes, above the whole budget {self.budget}")
        with self._lock:
            while not self._evict_for(need):
                self._lock.wait(timeout=0.05)
            self._in_use += need
            self._pending.append((rid, rp, ci, val, b, arrival, time.perf_counter(), need))
            self._lock.notify_all()

    # ------------------------------------------------------------------ workers
    def _cache_get(self, key):
        e = self._cache.get(key)
        if e is not None:
            self._cache.move_to_end(key)
            e.users += 1
        return e

    def _worker(self):
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(device=self.dev)
        while True:
            with self._lock:
                while not self._pending and not self._stop:
                    self._lock.wait(timeout=0.05)
                if self._stop and not self._pending:
                    return
                job = self._pending.popleft()
            try:
                self._run(job, stream)
            except Exception as exc:  # report, do not kill the server
                rid = job[0]
                with self._lock:
                    self._results[rid] = ServeResult(rid, np.zeros(0), 0, float("nan"), -1, job[5], job[6],
                                                     time.perf_counter(), f"error: {exc}")
                    self._in_use -= job[7]
                    self._lock.notify_all()

    def _run(self, job, stream):
        rid, rp, ci, val, b, arrival, admitted, need = job
        started = time.perf_counter()
        n = len(rp) - 1
        key = fingerprint(rp, ci, val)
        with torch.cuda.stream(stream):
            d_rp = torch.from_numpy(rp).to(self.dev, non_blocking=True)
            d_ci = torch.from_numpy(ci).to(self.dev, non_blocking=True)
            d_val = torch.from_numpy(val).to(self.dev, non_blocking=True)
            d_b = torch.from_numpy(b).to(self.dev, non_blocking=True)
            with self._lock:
                entry = self._cache_get(key)
            if entry is None:
                h = amg.amg_setup(d_rp, d_ci, d_val, self._params_for(n), stream=stream)
                nbytes = estimate_bytes(n, len(ci), self.precision) // 2
                with self._lock:
                    entry = self._cache.get(key)
                    if entry is None:
                        entry = _Entry(h, nbytes, key)
                        entry.users = 1
                        self._cache[key] = entry
                        self._cache_bytes += nbytes
                        while len(self._cache) > self.cache_entries and self._evict_one_idle():
                            pass
                    else:  # another worker built it meanwhile
                        h.close()
                        entry.users += 1
                self.stats["setup"] += 1
            else:
                self.stats["cache_hit"] += 1
            try:
                x = torch.zeros_like(d_b)
                h = entry.h
                stream.synchronize()
                setup_done = time.perf_counter()
                batchable = (n <= self.small_max_n and h.sizes()[-1] <= self.batch_coarse_max
                             and self._dense_coarse(h))
                with entry.lock:
                    info = None
                    path = "single"
                    if batchable:
                        done = threading.Event()
                        slot = {}
                        cls = next(k for k, c in enumerate(self.batch_classes) if n <= c)
                        self._batchqs[cls].put((h, d_b, x, done, slot))
                        done.wait()
                        info = slot["info"]  # None: the batcher handed the system back
                        if info is not None:
                            path = "batch"
                    if info is None:
                        info = amg.pcg_solve(h, d_b, x, rtol=self.rtol, max_iter=self.max_iter, flexible=True,
                                             stream=stream)
                    hx = x.to("cpu", non_blocking=True)
                    stream.synchronize()
            except BaseException:
                # the worker reports the error; the cached hierarchy becomes evictable again
                with self._lock:
                    entry.users -= 1
                raise
        fin = time.perf_counter()
        with self._lock:
            entry.users -= 1
            self._in_use -= need
            self._results[rid] = ServeResult(rid, hx.numpy(), info.iterations, info.rel_res_true, info.status,
                                             arrival, admitted, fin, path, started, setup_done)
            self._lock.notify_all()

    def _evict_one_idle(self) -> bool:
        victim = next((k for k, e in self._cache.items() if e.users == 0), None)
        if victim is None:
            return False
        e = self._cache.pop(victim)
        self._cache_bytes -= e.bytes
        e.h.close()
        self.stats["evicted"] += 1
        return True

    @staticmethod
    def _dense_coarse(h) -> bool:
        # the coarsest level is solved with the dense inverse
        return amg.amg_coarse_cg_cluster_size(h) < 0

    # ------------------------------------------------------------------ batcher
    def _batch_loop(self, bq, min_batch):
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(device=self.dev)
        while True:
            try:
                first = bq.get(timeout=0.05)
            except queue.Empty:
                if self._stop:
                    return
                continue
            # gather what becomes ready within a short window after the first request
            group = [first]
            deadline = time.perf_counter() + self.batch_window_s
            while len(group) < self.max_batch:
                left = deadline - time.perf_counter()
                try:
                    group.append(bq.get(timeout=left) if left > 0 else bq.get_nowait())
                except queue.Empty:
                    break
            if len(group) < min_batch:
                # hand the systems back: each runs the whole-GPU solve on its worker's stream
                for g in group:
                    g[4]["info"] = None
                    g[3].set()
                self.stats["unbatched"] += len(group)
                continue
            try:
                infos = amg.amg_batch_pcg([g[0] for g in group], [g[1] for g in group], [g[2] for g in group],
                                          rtol=self.rtol, max_iter=self.max_iter, flexible=True, stream=stream)
            except Exception:
                # the batch failed as a whole: hand its systems back, each worker
                # then solves (or reports) its own system alone
                for g in group:
                    g[4]["info"] = None
                    g[3].set()
                self.stats["batch_errors"] += 1
                continue
            self.stats["batches"] += 1
            self.stats["batched"] += len(group)
            for g, info in zip(group, infos):
                g[4]["info"] = info
                g[3].set()

    # ------------------------------------------------------------------ driving
    def wait(self, rids, timeout: float = 600.0):
        t0 = time.perf_counter()
        with self._lock:
            while not all(r in self._results for r in rids):
                if time.perf_counter() - t0 > timeout:
                    raise TimeoutError("requests did not finish")
                self._lock.wait(timeout=0.05)
            return [self._results[r] for r in rids]

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        for t in self._workers + self._batchers:
            t.join(timeout=10)
        with self._lock:
            for e in self._cache.values():
                e.h.close()
            self._cache.clear()
            self._cache_bytes = 0


def serve_stream(server: SolveServer, requests, systems, time_scale: float = 1.0):
    """Feeds requests at their arrival times (seconds, scaled by time_scale) and
    returns (results, wall seconds).  systems[i] is the System of requests[i]."""
    t0 = time.perf_counter()
    base = requests[0].arrival_s if requests else 0.0
    for req, s in zip(requests, systems):
        due = t0 + (req.arrival_s - base) * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        server.submit(req.rid, s.rp, s.ci, s.val, s.b, arrival=max(due, t0))
    results = server.wait([r.rid for r in requests])
    return results, time.perf_counter() - t0


def latency_summary(results):
    lat = np.array([r.latency for r in results])
    out = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
    done = [r for r in results if r.started > 0]
    if done:
        # where the time goes: waiting for a worker, setup (copy + hierarchy), solve
        out["mean_queue_ms"] = float(np.mean([r.started - r.arrival for r in done]) * 1e3)
        out["mean_setup_ms"] = float(np.mean([r.setup_done - r.started for r in done]) * 1e3)
        out["mean_solve_ms"] = float(np.mean([r.finished - r.setup_done for r in done]) * 1e3)
    return out
