#!/usr/bin/env python
"""Benchmark of the GB300 aggregation-AMG PCG solver.

Workload (one step): the 3D 7-point anisotropic diffusion system on a 256^3
grid (16,777,216 unknowns, 117,047,296 nonzeros, off-diagonals -1, -1 and
-1e-3 in z, FP64 CSR, b ~ U[-1,1] seed 2): device AMG setup (pairwise
heavy-edge matching, two passes per level, Galerkin products, coarsest
inverse) followed by FP64 flexible AMG-preconditioned CG from x = 0 to a
relative residual of 1e-8.  Inputs are resident in HBM when the timed region
starts; the level-0 matrix (1.47 GB) is far larger than the 129 MB L2, so no
flush is needed between steps.

Printed: one JSON line (rank 0).  value = solves per second over all ranks
(replicas: every rank solves its own copy; no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AMG-PCG time to 1e-8 rel. residual; V-cycle HBM GB/s; batched solves/s + p99"
UNIT = "solves/s"
WORKLOAD = ("anisotropic3d_256: 3D 7-pt anisotropic diffusion, 256^3 grid (16,777,216 unknowns, 117,047,296 "
            "nonzeros), eps_z = 1e-3, b ~ U[-1,1] seed 2, FP64 CSR; AMG setup + FP64 flexible PCG to 1e-8")
RTOL = 1e-8
# FP64 peak of GB300: 152 SMs x 2 FMA per clock x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
HBM_SPEC_GBS = 7900.0  # GB300 HBM3e nominal; the measured copy bandwidth is the primary denominator
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernel, keyed by profiler kind at level 0 of the 256^3 system (scaled from
# the capture named in profiles/ by rows); absent once the kernel changes
DRAM_BYTES_PER_LAUNCH = {
    # k_op_residual<1, double, double> at level 0 of anisotropic3d_128: 213,434,624 bytes
    # (profiles/level_kernels_anisotropic3d_128.md), times 8.0217, the ratio of the
    # launch's algorithmic bytes at 256^3 and at 128^3
    ("op_residual", 0): 213434624 * 8.0217,
    # k_pcg_spmv<1> (the outer q = A p) at level 0 of anisotropic3d_128: 212,622,208 bytes, the
    # mean of two launches (profiles/krylov_spmv_anisotropic3d_128.md), times 8.0202, the ratio
    # of the launch's algorithmic bytes at 256^3 and at 128^3
    ("krylov_spmv", 0): 212622208 * 8.0202,
}
# DRAM bytes per launch of the coarse CG on the 128^3 lognormal coarsest
# level (profiles/coarse_cg_lognormal3d_128.md): its matrix and vectors live
# in shared memory, so these bytes stand for the solve's HBM traffic
COARSE_CG_DRAM_BYTES = 10576128 + 169216


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--grid", type=int, default=128, help="cells per side of the lognormal system")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2048,
                    help="requests of the serving stream added to the line (2048: the whole stream; 0: none)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (256^3 mixed precision, 2048^2 BiCGStab, 64^2 Poisson)")
    ap.add_argument("--workload", choices=["solve", "serving", "batched"], default="solve",
                    help="serving: run the full 2048-request stream and print only its line; batched: the "
                         "batched kernel against single solves, alone")
    ap.add_argument("--profile-case", default=None,
                    help="one setup + FP64 flexible PCG solve of a named system for profiler captures, e.g. "
                         "anisotropic3d_128, anisotropic3d_256, lognormal3d_128 (prints one line, no timing)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu_index)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = max(smax, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(v: float, world: int) -> float:
    """Max of a per-rank value over all ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return world * units_per_rank / (max_ms * 1e-3)


def shard(items, rank: int, world: int):
    """Round-robin share of independent work items for one rank (replicas)."""
    return items[rank::world]


# ---------------------------------------------------------------------------
# oracle timings (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_full_solve(conn):
    """Child process: one complete oracle solve of the headline system on one
    host core (setup + flexible PCG to 1e-8), every part timed, nothing
    extrapolated.  Sends a dict through conn."""
    try:
        import oracle as O
        from paper_2007_00056_gb300 import workloads as W

        s = W.config_anisotropic3d_256()
        t0 = time.perf_counter()
        oh = O.Hierarchy(s.rp, s.ci, s.val)
        t1 = time.perf_counter()
        _, info = oh.pcg(s.b, rtol=RTOL, flexible=True)
        t2 = time.perf_counter()
        conn.send({"setup_s": t1 - t0, "solve_s": t2 - t1, "iterations": info.iterations,
                   "rel_res_true": info.rel_res_true, "levels": oh.sizes()})
    except Exception as e:  # reported in the line, never fatal to the GPU measurement
        conn.send({"error": repr(e)})
    conn.close()


def start_cpu_baseline():
    """Starts the oracle's full solve in a spawned child on its own host core;
    it runs while the later GPU lines are measured.  Returns (process,
    connection)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    rd, wr = ctx.Pipe(duplex=False)
    p = ctx.Process(target=oracle_full_solve, args=(wr,), daemon=True)
    p.start()
    wr.close()
    return p, rd


def finish_cpu_baseline(proc, conn, timeout_s=900.0):
    if proc is None:
        return None
    r = conn.recv() if conn.poll(timeout_s) else {"error": f"no result within {timeout_s:.0f} s"}
    proc.join(5)
    if "error" in r:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r["error"]}
    t = r["setup_s"] + r["solve_s"]
    return {"value": 1.0 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one complete solve of the full 256^3 system by the serial FP64 oracle on one host core: "
                       f"setup {r['setup_s']:.1f} s + flexible PCG {r['solve_s']:.1f} s ({r['iterations']} "
                       f"iterations to 1e-8), timed whole, nothing extrapolated; it ran in a child process while "
                       f"the GPU lines between the end-to-end timing and the serving stream were measured"),
            "time_to_solution_s": t, "iterations": r["iterations"], "rel_res_true": r["rel_res_true"],
            "levels": r["levels"]}


def run_reference(args):
    """Oracle arm: the serial FP64 oracle on one host core, headline workload.
    The first warm-up step is one complete solve (setup + flexible PCG to
    1e-8), timed whole: its time gives `value`.  The other W - 1 warm-up steps
    and the K timed steps are bounded samples of the same workload, one
    oracle PCG iteration each (a call with max_iter = 1 on the already built
    hierarchy: initial residual, one V-cycle, one SpMV, the updates and the
    final true residual), whose mean is ms_per_step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2007_00056_gb300 import workloads as W

    s = W.config_anisotropic3d_256()
    t0 = time.perf_counter()
    oh = O.Hierarchy(s.rp, s.ci, s.val)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, info = oh.pcg(s.b, rtol=RTOL, flexible=True)
    t_pcg = time.perf_counter() - t0
    full = t_setup + t_pcg
    for _ in range(max(0, args.warmup - 1)):
        oh.pcg(s.b, rtol=0.0, max_iter=1, flexible=True)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oh.pcg(s.b, rtol=0.0, max_iter=1, flexible=True)
        ts.append(time.perf_counter() - t0)
    value = 1.0 / full
    sample = (f"warm-up step 1: one complete oracle solve of the full system timed whole (setup {t_setup:.1f} s + "
              f"flexible PCG {t_pcg:.1f} s, {info.iterations} iterations), which gives the value; "
              f"the {args.steps} timed steps are one-iteration PCG samples on the same hierarchy "
              f"({statistics.mean(ts):.3f} s each)")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ts) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": s.n, "nnz": s.nnz, "rtol": RTOL},
        "time_to_solution_s": full, "iterations": info.iterations, "rel_res_true": info.rel_res_true,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# serving stream (continuous batching)
# ---------------------------------------------------------------------------
def _gen_request(req):
    s = req.system()
    return req.rid, s.rp, s.ci, s.val, s.b


def generate_requests(count: int):
    """The first `count` requests of the 2048-request stream (Poisson arrivals at
    200/s, N log-uniform in [1e3, 1e6]) and their systems, generated on the host
    by a spawn-context process pool (safe after CUDA initialisation)."""
    import multiprocessing as mp

    from paper_2007_00056_gb300 import workloads as W

    reqs = W.request_stream(count=2048)[:count]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        out = pool.map(_gen_request, reqs, chunksize=1)
    systems = {rid: W.System(f"req{rid}", rp, ci, val, b) for rid, rp, ci, val, b in out}
    return reqs, [systems[r.rid] for r in reqs]


def oracle_serving_sample(reqs, systems, count=16):
    """The oracle (serial FP64, one host core) serving the first `count` requests
    one at a time at their arrival times: its own solves/s and p50/p99, for
    context beside the GPU server.  Each request is its setup (the server's
    stop sizes and edge weight) plus flexible PCG to 1e-8."""
    import numpy as np

    import oracle as O

    times = []
    for req, s in list(zip(reqs, systems))[:count]:
        t0 = time.perf_counter()
        cm = 256 if s.n <= 60000 else 1024
        oh = O.Hierarchy(s.rp, s.ci, s.val, params=O.Params(coarse_max=cm, edge_weight=1))
        oh.pcg(s.b, rtol=RTOL, flexible=True)
        times.append(time.perf_counter() - t0)
    done, lat = 0.0, []
    for (rq, _), t in zip(list(zip(reqs, systems))[:count], times):
        done = max(done, rq.arrival_s) + t
        lat.append((done - rq.arrival_s) * 1e3)
    return {"requests": len(times), "cores": 1, "kind": "oracle",
            "solves_per_s": len(times) / sum(times),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "sample": f"the first {len(times)} requests of the stream, one at a time at their arrival times, "
                      f"by the serial FP64 oracle on one host core (setup with the server's stop sizes and "
                      f"scaled edge weight, flexible PCG to 1e-8)"}


def run_serving(reqs, systems, plain_sample=256):
    """Serves the stream at its arrival times (latency), then all at once
    (capacity), then the plain FP64 method one request at a time on the first
    `plain_sample` requests (context)."""
    import numpy as np
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import serving as S

    import inspect

    total_n = sum(s.n for s in systems)
    srv_defaults = {k: v.default for k, v in inspect.signature(S.SolveServer).parameters.items()}
    # untimed warm-up on a throwaway server (first launches of every kernel,
    # growth of the memory pools): a cold server fell 1.5 s behind in the
    # stream's first requests, and at an arrival rate this close to its
    # capacity that backlog never drained
    warm = min(64, len(reqs))
    srv = S.SolveServer()
    S.serve_stream(srv, reqs[:warm], systems[:warm], time_scale=0.0)
    srv.close()
    srv = S.SolveServer()
    res, wall = S.serve_stream(srv, reqs, systems)
    stats = dict(srv.stats)
    srv.close()
    srv = S.SolveServer()
    res_cap, wall_cap = S.serve_stream(srv, reqs, systems, time_scale=0.0)
    srv.close()
    ok = sum(r.status == amg.AMG_OK and r.rel_res_true <= 1e-8 for r in res)
    # the same stream with the paper's edge weight max(|a_ij|, |a_ji|)
    paper = {}
    for tag, scale in (("", 1.0), ("capacity_", 0.0)):
        srv = S.SolveServer(params={"edge_weight": amg.AMG_WEIGHT_ABS})
        rp_, wp_ = S.serve_stream(srv, reqs, systems, time_scale=scale)
        srv.close()
        lp = S.latency_summary(rp_)
        paper.update({f"{tag}solves_per_s": len(rp_) / wp_, f"{tag}p50_ms": lp["p50_ms"], f"{tag}p99_ms": lp["p99_ms"],
                      f"{tag}converged_1e-8": int(sum(r.status == amg.AMG_OK and r.rel_res_true <= 1e-8 for r in rp_))})
    # the queue stays bounded when late requests wait no longer than early ones
    q = len(res) // 4
    lat_first = S.latency_summary(res[:q]) if q else None
    lat_last = S.latency_summary(res[-q:]) if q else None
    # plain FP64 method: setup + pcg_solve per request, sequential, same device
    dev = torch.device("cuda", torch.cuda.current_device())
    sample = list(zip(reqs, systems))[:plain_sample]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_request = []
    for _, s in sample:
        tr = time.perf_counter()
        rp, ci, val, b = (torch.from_numpy(a).to(dev) for a in (s.rp, s.ci, s.val, s.b))
        # the server's hierarchy shape (coarsest size) in plain FP64
        cm = srv_defaults["batch_coarse_max"] if s.n <= srv_defaults["small_max_n"] else srv_defaults["big_coarse_max"]
        h = amg.amg_setup(rp, ci, val, amg.amg_default_params(coarse_max=cm))
        x = torch.zeros_like(b)
        amg.pcg_solve(h, b, x, rtol=RTOL, flexible=not h.sizes()[-1] <= 4096)
        x.cpu()
        h.close()
        per_request.append(time.perf_counter() - tr)
    plain = time.perf_counter() - t0
    # the plain method serving the same arrivals one request at a time
    done, plain_lat = 0.0, []
    for (rq, _), t in zip(sample, per_request):
        done = max(done, rq.arrival_s) + t
        plain_lat.append((done - rq.arrival_s) * 1e3)
    lat = S.latency_summary(res)
    return {
        "requests": len(reqs), "unknowns_total": int(total_n), "converged_1e-8": int(ok),
        "arrival_rate_hz": 200.0, "solves_per_s": len(reqs) / wall, "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"],
        "max_ms": lat["max_ms"],
        "p50_ms_first_quarter": lat_first["p50_ms"] if lat_first else None,
        "p50_ms_last_quarter": lat_last["p50_ms"] if lat_last else None,
        "mean_queue_ms": lat.get("mean_queue_ms"), "mean_setup_ms": lat.get("mean_setup_ms"),
        "mean_solve_ms": lat.get("mean_solve_ms"),
        "capacity_solves_per_s": len(reqs) / wall_cap,
        "capacity_p50_ms": S.latency_summary(res_cap)["p50_ms"],
        "plain_fp64_sequential_sample": len(sample),
        "plain_fp64_sequential_solves_per_s": len(sample) / plain,
        "plain_fp64_sequential_p50_ms": float(np.percentile(plain_lat, 50)),
        "plain_fp64_sequential_p99_ms": float(np.percentile(plain_lat, 99)),
        "batched_requests": int(stats.get("batched", 0)), "batches": int(stats.get("batches", 0)),
        "precision": "fp32 V-cycle, fp64 flexible PCG",
        "edge_weight": "max(|a_ij|,|a_ji|)/sqrt(|a_ii a_jj|) (option; the server's default)",
        "workers": srv_defaults["workers"],
        "paper_edge_weight": paper,
        "oracle_one_at_a_time": oracle_serving_sample(reqs, systems),
    }


def run_batched(dev, groups=((2000, 48), (16000, 48), (30000, 24), (60000, 24))):
    """The batched kernel against the same systems solved one at a time.

    Each group holds `k` systems of about `n` rows, the three families of the
    serving stream in turn (seed 5000 + j), set up as the server sets up a
    batchable request (FP32 V-cycle, coarsest at most 256 rows, dense, scaled
    edge weight). Timed with CUDA events, solve phase only (hierarchies
    already built): one `amg_batch_pcg` call over the group; `pcg_solve` on each
    system in turn with the same hierarchies; and the plain FP64 method (FP64
    hierarchies, PCG with the fixed preconditioner) in turn."""
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def dense_coarse(h):
        return amg.amg_coarse_cg_cluster_size(h) < 0

    lines = []
    for n_target, k in groups:
        systems = [W.Request(j, 0.0, W.FAMILIES[j % 3], n_target, 5000 + j).system() for j in range(k)]
        p32 = amg.amg_default_params(precision=amg.AMG_FP32, coarse_max=256, edge_weight=amg.AMG_WEIGHT_SCALED)
        p64 = amg.amg_default_params(coarse_max=256, edge_weight=amg.AMG_WEIGHT_SCALED)
        h32, h64, bs = [], [], []
        for s in systems:
            rp, ci, val, b = (torch.from_numpy(a).to(dev) for a in (s.rp, s.ci, s.val, s.b))
            h = amg.amg_setup(rp, ci, val, p32)
            if h.sizes()[-1] > 256 or not dense_coarse(h):
                h.close()
                continue
            h32.append(h)
            h64.append(amg.amg_setup(rp, ci, val, p64))
            bs.append(b)
        m = len(h32)
        if m == 0:
            lines.append({"n_target": n_target, "systems": 0, "status": "no batchable hierarchy"})
            continue

        def batch():
            xs = [torch.zeros_like(b) for b in bs]
            return xs, amg.amg_batch_pcg(h32, bs, xs, rtol=RTOL, flexible=True)

        def single(hs, flexible):
            xs, infos = [], []
            for h, b in zip(hs, bs):
                x = torch.zeros_like(b)
                infos.append(amg.pcg_solve(h, b, x, rtol=RTOL, flexible=flexible))
                xs.append(x)
            return xs, infos

        batch()  # warm-up: first launches of each team size
        single(h32[:1], True)
        single(h64[:1], False)
        ms_b, (xb, ib) = timed(batch)
        ms_s, (_, is_) = timed(lambda: single(h32, True))
        ms_p, (xp, ip) = timed(lambda: single(h64, False))
        err = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(xb, xp))
        lines.append({
            "n_target": n_target, "systems": m, "rows_total": int(sum(b.numel() for b in bs)),
            "team_blocks": sorted({1 if b.numel() <= 8192 else 2 if b.numel() <= 24576 else 4 if b.numel() <= 65536
                                   else 8 for b in bs}),
            "batched_solves_per_s": m / (ms_b * 1e-3),
            "single_fp32_solves_per_s": m / (ms_s * 1e-3),
            "plain_fp64_single_solves_per_s": m / (ms_p * 1e-3),
            "batched_over_single": ms_s / ms_b, "batched_over_plain_fp64": ms_p / ms_b,
            "iterations_batched": [min(i.iterations for i in ib), max(i.iterations for i in ib)],
            "iterations_plain_fp64": [min(i.iterations for i in ip), max(i.iterations for i in ip)],
            "converged_1e-8": int(sum(i.status == amg.AMG_OK and i.rel_res_true <= RTOL for i in ib)),
            "rel_res_true_max": max(i.rel_res_true for i in ib),
            "max_rel_err_vs_plain_fp64": err,
        })
        for h in h32 + h64:
            h.close()
    return {"note": "solve phase only, hierarchies built beforehand; FP32 V-cycle in FP64 flexible PCG for the "
                    "batched and single lines, the FP64 V-cycle in PCG for the plain method; CUDA events",
            "lines": lines}


VCYCLE_KINDS = {"jacobi0", "jacobi", "residual", "restrict", "prolong_jacobi", "prolong", "coarse_dense",
                "coarse_cg", "cast", "op_residual", "op_post"}
# kinds that are one kernel each and stream the level's matrix or vectors from HBM
HBM_KERNEL_KINDS = ("op_residual", "op_post", "krylov_spmv", "residual", "jacobi", "jacobi0", "restrict", "prolong",
                    "prolong_jacobi")


def b_v_bytes(h, s_v, s_x, coarse_bytes=None):
    """Algorithmic bytes of one V-cycle (one pre- and one post-sweep, zero
    guess) by the measurement plan's count: per level k below the coarsest,
    two matrix passes B_A(k) = nnz_k (s_v + 4) + 4 (N_k + 1), nine vector
    passes of N_k s_x and the aggregate map (4 N_k); plus the coarsest solve,
    8 N_L^2 for the dense inverse, or `coarse_bytes` (the DRAM bytes ncu
    measured) for a coarse CG that works from shared memory."""
    from paper_2007_00056_gb300 import amg

    sizes = [amg.amg_level_info(h, k) for k in range(h.num_levels)]
    total = 0.0
    for n, nnz in sizes[:-1]:
        total += 2.0 * (nnz * (s_v + 4) + 4.0 * (n + 1)) + 9.0 * n * s_x + 4.0 * n
    n_l = sizes[-1][0]
    total += 8.0 * n_l * n_l if coarse_bytes is None else float(coarse_bytes)
    return total


def vcycle_rate(h, b, bv, reps=20):
    """Rate of the whole V-cycle: its algorithmic bytes bv (b_v_bytes) over
    the time of `reps` V-cycles run back to back with the profiler off (CUDA
    events on the current stream).  Returns (GB/s, ms per V-cycle)."""
    import torch

    from paper_2007_00056_gb300 import amg

    stream = torch.cuda.current_stream()
    z = torch.empty_like(b)
    amg.amg_profile_enable(h, False)
    for _ in range(3):
        amg.amg_vcycle(h, b, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        amg.amg_vcycle(h, b, z)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return bv / (ms * 1e-3) / 1e9, ms


def _solve_timed(sys_, params, krylov, dev, profile=False, tune=False, coarse_bytes=None):
    """Setup + solve of one system from device-resident inputs ("pcg": flexible
    PCG, "bicgstab", or "amg": AMG as a stationary solver); CUDA events on the
    current stream.  Returns times, the solve info, x and (with profile) the
    V-cycle's rate by the measurement plan's algorithmic bytes (coarse_bytes:
    DRAM bytes of a shared-memory coarse CG)."""
    import torch

    from paper_2007_00056_gb300 import amg

    stream = torch.cuda.current_stream()
    rp, ci, val, b = (torch.from_numpy(a).to(dev) for a in (sys_.rp, sys_.ci, sys_.val, sys_.b))
    x = torch.zeros_like(b)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record(stream)
    h = amg.amg_setup(rp, ci, val, params)
    e1.record(stream)
    if tune:  # later setups of the same level shapes reuse the tuned kernels
        amg.amg_autotune(h)
    if profile:
        amg.amg_profile_enable(h, True)
    solve = {"pcg": amg.pcg_solve, "bicgstab": amg.bicgstab_solve, "amg": amg.amg_solve}[krylov]
    kw = {"flexible": True} if krylov == "pcg" else {}
    info = solve(h, b, x, rtol=RTOL, max_iter=5000 if krylov == "amg" else 1000, **kw)
    e2.record(stream)
    torch.cuda.synchronize()
    vc_bytes = vc_ms = 0.0
    top = []
    if profile:
        table = amg.amg_profile_table(h)
        for r in table:
            if r["kind"] in VCYCLE_KINDS:
                vc_bytes += r["bytes"]
                vc_ms += r["ms"]
        for r in sorted(table, key=lambda r: -r["ms"])[:5]:
            top.append({"kernel": f"{r['kind']}@{r['level']}", "ms": r["ms"],
                        "gbs": r["bytes"] / (r["ms"] * 1e-3) / 1e9 if r["ms"] > 0 else None})
        sv, sx = {amg.AMG_FP64: (8, 8), amg.AMG_FP32: (4, 4), amg.AMG_FP16_STORAGE: (2, 4)}[params.precision]
        dense = amg.amg_coarse_cg_cluster_size(h) < 0
        bv = b_v_bytes(h, sv, sx, None if dense else coarse_bytes)
        level_nnz = [amg.amg_level_info(h, k) for k in range(h.num_levels)]
        vc_gbs_unprofiled, vc_ms_unprofiled = vcycle_rate(h, b, bv)
        cms = sum(r["ms"] for r in table if r["kind"] in ("coarse_dense", "coarse_cg"))
        coarse_share = cms / vc_ms if vc_ms > 0 else None
    levels = h.sizes()
    h.close()
    out = dict(setup_ms=e0.elapsed_time(e1), solve_ms=e1.elapsed_time(e2), info=info, x=x, levels=levels,
               vc_bytes=vc_bytes, vc_ms=vc_ms, top=top)
    if profile:
        out.update(vc_gbs=vc_gbs_unprofiled, vc_cycle_ms=vc_ms_unprofiled, vc_coarse_share=coarse_share,
                   vc_bv_bytes=bv, table=table, level_nnz=level_nnz)
    return out


def coarse_cg_roofline(table, level_nnz):
    """FP64 rate of the coarse CG (the coarsest solve of the 128^3 lognormal
    hierarchy, whose rows and matrix slice live in shared memory, so its bound
    is the FP64 pipe and its grid barrier, not HBM).  Flops per iteration are
    the method's Jacobi-PCG work, 2 nnz_L (the product) + 13 N_L (three
    vector updates, the Jacobi scaling, three inner products); the iteration
    count per launch is the profiler's byte total over its per-iteration
    charge (one matrix pass plus ten FP64 vectors)."""
    rows = [r for r in table if r["kind"] == "coarse_cg"]
    if not rows:
        return None
    r = rows[0]
    n_l, nnz_l = level_nnz[r["level"]]
    charge = nnz_l * 12 + 4 * (n_l + 1) + 80 * n_l
    iters = r["bytes"] / r["launches"] / charge
    ms = r["ms"] / r["launches"]
    flops = (2.0 * nnz_l + 13.0 * n_l) * iters
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "pipe": "fp64", "kernel": f"coarse_cg@level{r['level']}", "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": COARSE_CG_DRAM_BYTES,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)",
            "flops_per_iteration": "2 nnz_L + 13 N_L", "iterations_per_launch": iters, "ms_per_launch": ms,
            "us_per_iteration": ms * 1e3 / iters}


def run_residency(dev, x64_main=None):
    """The hybrid CPU/GPU-CI placement of Sec. 3.1.1 on the 256^3 system (FP64
    flexible PCG): the level matrices in pinned host memory, read over the
    host-device link (mapped) or copied one cycle visit ahead into two device
    buffers (staged), against the resident hierarchy.  Per mode: device and
    host bytes of the hierarchy, the solve time (setup excluded: the
    placement changes after setup), iterations, whether x equals the resident
    solution bit for bit, and the bytes the staging copied per solve."""
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    s3 = W.config_anisotropic3d_256()
    rp, ci, val, b = (torch.from_numpy(a).to(dev) for a in (s3.rp, s3.ci, s3.val, s3.b))
    h = amg.amg_setup(rp, ci, val, amg.amg_default_params())
    del rp, ci, val
    stream = torch.cuda.current_stream()
    lines = []
    x_res = None
    for mode, first in ((amg.AMG_RESIDENT, 0), (amg.AMG_HOST_STAGED, 1), (amg.AMG_HOST_STAGED, 0),
                        (amg.AMG_HOST_MAPPED, 1), (amg.AMG_HOST_MAPPED, 0)):
        amg.amg_set_residency(h, mode, first)
        x = torch.zeros_like(b)
        amg.pcg_solve(h, b, x, rtol=RTOL, flexible=True)  # warm-up (prefetch state, page mappings)
        mem0 = amg.amg_memory_info(h)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        info = amg.pcg_solve(h, b, x, rtol=RTOL, flexible=True)
        e1.record(stream)
        torch.cuda.synchronize()
        mem = amg.amg_memory_info(h)
        if x_res is None:
            x_res = x.clone()
        ms = e0.elapsed_time(e1)
        copied = mem["copied_bytes"] - mem0["copied_bytes"]
        lines.append({"mode": ["resident", "host_mapped", "host_staged"][mode], "first_level": first,
                      "device_bytes": mem["device_bytes"], "host_bytes": mem["host_bytes"],
                      "staging_bytes": mem["staging_bytes"], "solve_ms": ms, "iterations": info.iterations,
                      "status": amg.status_string(info.status), "rel_res_true": info.rel_res_true,
                      "x_bitwise_equal_resident": bool(torch.equal(x.view(torch.int64), x_res.view(torch.int64))),
                      "staged_bytes_per_solve": copied,
                      "staged_gbs": copied / (ms * 1e-3) / 1e9 if copied else None})
    amg.amg_set_residency(h, amg.AMG_RESIDENT)
    h.close()
    del b
    torch.cuda.empty_cache()
    return {"system": "anisotropic3d_256 FP64 flexible PCG", "lines": lines}


def run_configs(dev, peak, x64_main=None):
    """The other workloads of the method, measured on this GPU: the 256^3
    anisotropic system in both mixed-precision forms (flexible PCG; error
    against the FP64 solution of the headline), the 128^3 lognormal system in
    FP64 (its coarsest level is solved by the coarse CG), the 2048^2 upwind
    convection-diffusion system with BiCGStab (FP32 V-cycle, FP64 outer) at
    three Peclet numbers, and the 64^2 Poisson system (coarsest level 64
    rows).  Each line: setup and solve time (a second solve after one untimed
    warm-up whose hierarchy is autotuned, as in the headline), iterations,
    true relative residual, and the V-cycle's rate by the measurement plan's
    algorithmic bytes over the time of unprofiled V-cycles."""
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    out = []

    def line(name, sys_, prec, krylov, x_ref=None, coarse_bytes=None, **kw):
        params = amg.amg_default_params(precision=prec, **kw)
        _solve_timed(sys_, params, krylov, dev, tune=True)  # warm-up; its hierarchy is autotuned
        r = _solve_timed(sys_, params, krylov, dev)
        p = _solve_timed(sys_, params, krylov, dev, profile=True, coarse_bytes=coarse_bytes)
        info = r["info"]
        gbs = p["vc_gbs"]
        d = {"config": name, "n": sys_.n, "nnz": sys_.nnz, "krylov": krylov,
             "precision": {amg.AMG_FP64: "fp64", amg.AMG_FP32: "fp32 V-cycle / fp64 outer",
                           amg.AMG_FP16_STORAGE: "fp16-storage V-cycle / fp64 outer"}[prec],
             "status": amg.status_string(info.status),
             "iterations": info.iterations, "rel_res_true": info.rel_res_true,
             "setup_ms": r["setup_ms"], "solve_ms": r["solve_ms"], "time_to_solution_ms": r["setup_ms"] + r["solve_ms"],
             "levels": r["levels"], "vcycle_gbs": gbs, "vcycle_bytes": p["vc_bv_bytes"],
             "vcycle_frac_of_measured_peak": (gbs / peak) if gbs else None,
             "vcycle_frac_of_spec": (gbs / HBM_SPEC_GBS) if gbs else None,
             "vcycle_ms": p["vc_cycle_ms"], "vcycle_coarsest_share": p["vc_coarse_share"],
             "top_kernels_profiled_solve": p["top"]}
        if x_ref is not None:
            d["rel_diff_vs_fp64_solution"] = float(torch.linalg.vector_norm(r["x"] - x_ref) /
                                                   torch.linalg.vector_norm(x_ref))
        out.append(d)
        return d, p

    s3 = W.config_anisotropic3d_256()
    for prec in (amg.AMG_FP32, amg.AMG_FP16_STORAGE):
        line("anisotropic3d_256 eps_z=1e-3", s3, prec, "pcg", x64_main)
    del s3
    torch.cuda.empty_cache()
    s2 = W.config_lognormal3d_128()
    d, p = line("lognormal3d_128 sigma=1", s2, amg.AMG_FP64, "pcg", coarse_bytes=COARSE_CG_DRAM_BYTES)
    if p.get("table"):
        d["coarse_cg_roofline"] = coarse_cg_roofline(p["table"], p["level_nnz"])
    del s2
    for pe in (10.0, 100.0, 1000.0):
        s4 = W.config_convdiff2d_2048(peclet=pe)
        line(f"convdiff2d_2048 upwind Pe={pe:g}", s4, amg.AMG_FP32, "bicgstab")
        del s4
    # the 64^2 Poisson configuration coarsens to 64 rows (4096 -> 1024 -> 256 -> 64); with the
    # library's default stop size (4096) it would be a single dense level, a direct solve
    line("poisson2d_64 coarse_max=64", W.config_poisson2d_64(), amg.AMG_FP64, "pcg", coarse_max=64)
    torch.cuda.empty_cache()
    return out


def run_cycles(dev, sys_main):
    """AMG as a stand-alone solver against AMG-PCG (Sec. 4.4 compares the
    two), each with the V-, W- and F-cycle, on the benchmark system and on a
    1024^2 P1 finite-element system (Table 1's P1 shape, 1,048,576 unknowns).
    Each line: setup and solve time of a second run after a warm-up whose
    hierarchy is autotuned, cycles or iterations, true relative residual.
    `amg_solver_over_pcg` is the time to solution of AMG as a solver over that
    of AMG-PCG, both with V-cycles."""
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    lines, ratios = [], {}
    for name, s in (("lognormal3d_128", sys_main), ("fem_p1_1024 jitter 0.25", W.fem_p1_jittered(1024, seed=0))):
        t = {}
        for method in ("pcg", "amg"):
            for cname, kind in (("V", amg.AMG_CYCLE_V), ("W", amg.AMG_CYCLE_W), ("F", amg.AMG_CYCLE_F)):
                params = amg.amg_default_params(cycle=kind)
                _solve_timed(s, params, method, dev, tune=True)  # warm-up; its hierarchy is autotuned
                r = _solve_timed(s, params, method, dev)
                info = r["info"]
                tts = r["setup_ms"] + r["solve_ms"]
                t[(method, cname)] = tts
                lines.append({"system": name, "n": s.n,
                              "method": "AMG-PCG (flexible)" if method == "pcg" else "AMG as a solver",
                              "cycle": cname, "status": amg.status_string(info.status),
                              "iterations": info.iterations, "rel_res_true": info.rel_res_true,
                              "setup_ms": r["setup_ms"], "solve_ms": r["solve_ms"], "time_to_solution_ms": tts,
                              "ms_per_iteration": r["solve_ms"] / max(1, info.iterations), "levels": r["levels"]})
        ratios[name] = t[("amg", "V")] / t[("pcg", "V")]
        torch.cuda.empty_cache()
    return {"lines": lines, "amg_solver_over_pcg": ratios, "rtol": RTOL}


def run_scaled_weight(dev, sys_main):
    """The benchmark system with the diagonally scaled edge weight, an option
    outside the paper (max(|a_ij|,|a_ji|)/sqrt(|a_ii a_jj|)): hierarchy sizes,
    setup and FP64 flexible PCG time, second run after an autotuned warm-up.
    Not the headline: the headline uses the paper's weight |a_ij|."""
    from paper_2007_00056_gb300 import amg

    params = amg.amg_default_params(edge_weight=amg.AMG_WEIGHT_SCALED)
    _solve_timed(sys_main, params, "pcg", dev, tune=True)
    r = _solve_timed(sys_main, params, "pcg", dev)
    info = r["info"]
    return {"system": "lognormal3d_128", "edge_weight": "max(|a_ij|,|a_ji|)/sqrt(|a_ii a_jj|)",
            "status": amg.status_string(info.status), "iterations": info.iterations,
            "rel_res_true": info.rel_res_true, "levels": r["levels"], "setup_ms": r["setup_ms"],
            "solve_ms": r["solve_ms"], "time_to_solution_ms": r["setup_ms"] + r["solve_ms"]}


def run_complexity(dev):
    """Complexity of AMG as a solver (Sec. 4.3 measures it on P1 finite
    elements at four uniform refinements, Table 1): the P1 family at
    312^2, 626^2, 1253^2 and 2507^2 unknowns (Table 1's P1L1-P1L4 sizes within
    0.3%), V-cycles, FP64, time to 1e-8 (setup + solve: the median of three
    runs after an autotuned warm-up, all three reported), and the exponent p
    of a least-squares fit t ~ N^p.
    Also the coarsest-solver comparison of Sec. 4.2 on the 1253^2 system,
    whose hierarchy stops at 7,089 rows: the same hierarchy with its coarsest
    level solved by the dense inverse (forced above the default size limit)
    or by CG."""
    import math

    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    lines = []
    coarse = []
    for m in (312, 626, 1253, 2507):
        s = W.fem_p1_jittered(m, seed=0)
        params = amg.amg_default_params()
        _solve_timed(s, params, "amg", dev, tune=True)
        runs = [_solve_timed(s, params, "amg", dev) for _ in range(3)]
        runs_ms = [x["setup_ms"] + x["solve_ms"] for x in runs]
        r = runs[sorted(range(3), key=lambda k: runs_ms[k])[1]]
        info = r["info"]
        lines.append({"system": f"fem_p1_{m}", "n": s.n, "nnz": s.nnz, "status": amg.status_string(info.status),
                      "cycles": info.iterations, "rel_res_true": info.rel_res_true, "setup_ms": r["setup_ms"],
                      "solve_ms": r["solve_ms"], "time_to_solution_ms": r["setup_ms"] + r["solve_ms"],
                      "runs_ms": runs_ms, "levels": r["levels"]})
        if m == 1253:
            for name, cs in (("dense inverse", amg.AMG_COARSE_DENSE), ("CG", amg.AMG_COARSE_CG)):
                pc = amg.amg_default_params(coarse_solver=cs)
                _solve_timed(s, pc, "amg", dev, tune=True)
                rc = _solve_timed(s, pc, "amg", dev)
                coarse.append({"system": f"fem_p1_{m}", "coarsest_solver": name, "coarsest_rows": rc["levels"][-1],
                               "cycles": rc["info"].iterations, "setup_ms": rc["setup_ms"],
                               "solve_ms": rc["solve_ms"], "time_to_solution_ms": rc["setup_ms"] + rc["solve_ms"]})
        del s
        torch.cuda.empty_cache()
    xs = [math.log(l["n"]) for l in lines]
    ys = [math.log(l["time_to_solution_ms"]) for l in lines]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    p = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sum((x - mx) ** 2 for x in xs)
    return {"lines": lines, "exponent": p, "coarsest_solver": coarse,
            "note": "AMG as a solver, V-cycle, FP64, rtol 1e-8; the paper reports about N^1.1 on its CPU/GPU "
                    "implementations"}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def run_profile_case(name):
    """One setup and one FP64 flexible PCG solve of a named system (family and
    grid size, the benchmark's generators and seeds), for profiler captures:
    no warm-up, no timing."""
    import torch

    from paper_2007_00056_gb300 import amg
    from paper_2007_00056_gb300 import workloads as W

    fam, _, size = name.rpartition("_")
    gen = {"anisotropic3d": lambda n: W.anisotropic3d(n, eps_z=1e-3, seed=2),
           "lognormal3d": lambda n: W.lognormal3d(n, seed=1), "poisson2d": lambda n: W.poisson2d(n)}[fam]
    s = gen(int(size))
    dev = torch.device("cuda", 0)
    amg.lib(build_if_missing=True)
    rp, ci, val, b = (torch.from_numpy(a).to(dev) for a in (s.rp, s.ci, s.val, s.b))
    h = amg.amg_setup(rp, ci, val)
    x = torch.zeros_like(b)
    info = amg.pcg_solve(h, b, x, rtol=RTOL, flexible=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "n": s.n, "levels": h.sizes(), "iterations": info.iterations,
                      "status": amg.status_string(info.status)}), flush=True)
    h.close()



def main():
    args = parse_args()
    from paper_2007_00056_gb300 import workloads as W

    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.workload == "serving":
        reqs, systems = generate_requests(2048)
        from paper_2007_00056_gb300 import amg

        amg.lib(build_if_missing=True)
        out = run_serving(reqs, systems)
        out.update({"metric": METRIC, "unit": "solves/s", "value": out["solves_per_s"], "n_gpus": 1,
                    "higher_is_better": True, "data": "synthetic", "dtype": "f32/f64",
                    "config": {"workload": "serving stream, 2048 requests, Poisson arrivals 200/s"}})
        print(json.dumps(out), flush=True)
        return
    if args.workload == "batched":
        import torch

        from paper_2007_00056_gb300 import amg

        amg.lib(build_if_missing=True)
        out = run_batched(torch.device("cuda", 0))
        print(json.dumps({"metric": "batched AMG-PCG solves/s against single solves", "unit": "solves/s",
                          "n_gpus": 1, "data": "synthetic", "batched": out}), flush=True)
        return

    rank, world, local = dist_setup(args)
    import torch

    from paper_2007_00056_gb300 import amg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    amg.lib(build_if_missing=True)
    sys_ = W.config_anisotropic3d_256()
    rp = torch.from_numpy(sys_.rp).to(dev)
    ci = torch.from_numpy(sys_.ci).to(dev)
    val = torch.from_numpy(sys_.val).to(dev)
    b = torch.from_numpy(sys_.b).to(dev)
    x = torch.zeros_like(b)
    params = amg.amg_default_params()
    stream = torch.cuda.current_stream()

    def step(profile=False):
        h = amg.amg_setup(rp, ci, val, params)
        if profile:
            amg.amg_profile_enable(h, True)
        x.zero_()
        ev_mid = torch.cuda.Event(enable_timing=True)
        ev_mid.record(stream)
        info = amg.pcg_solve(h, b, x, rtol=RTOL, max_iter=1000, flexible=True)
        return h, info, ev_mid

    # warm-up; the first warm-up hierarchy is autotuned and every later setup of
    # the same level shapes reuses the tuned kernel configuration
    levels = []
    for w in range(max(args.warmup, 1)):
        h, info, _ = step()
        if w == 0 and not args.no_autotune:
            amg.amg_autotune(h)
        levels = h.sizes()
        level_cfg = [amg.amg_level_config(h, k) + (amg.amg_level_operator_form(h, k),) for k in range(h.num_levels)]
        h.close()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = amg.amg_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    setup_ms, iters, rel_true = [], [], []
    # NVTX range "timed": lets a profiler capture exactly the timed launches
    # (ncu --nvtx --nvtx-include "timed/")
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    last = ev0
    for _ in range(args.steps):
        h, info, ev_mid = step()
        ev_end = torch.cuda.Event(enable_timing=True)
        ev_end.record(stream)
        setup_ms.append((last, ev_mid))
        iters.append(info.iterations)
        rel_true.append(info.rel_res_true)
        if info.status != amg.AMG_OK:
            raise RuntimeError(f"PCG did not converge: {info}")
        h.close()
        last = ev_end
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    launches = amg.amg_kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    total_ms = ev0.elapsed_time(ev1)
    setup_t = [a.elapsed_time(bv) for a, bv in setup_ms]
    max_ms = allreduce_max(total_ms, world)
    ms_per_step = max_ms / args.steps
    value = job_throughput(args.steps, world, max_ms)
    setup_mean = statistics.mean(setup_t)
    solve_mean = ms_per_step - setup_mean
    x_main = x.clone()

    # live per-kernel timing of the same step (CUDA events on the launching stream)
    peak, peak_kind = measured_peaks()
    table_acc = {}
    level_nnz = []
    vc = (None, None)
    bv = None
    for ps in range(args.profile_steps):
        h, info, _ = step(profile=True)
        level_nnz = [amg.amg_level_info(h, k) for k in range(h.num_levels)]
        for r in amg.amg_profile_table(h):
            key = (r["kind"], r["level"])
            acc = table_acc.setdefault(key, dict(kind=r["kind"], level=r["level"], ms=0.0, bytes=0.0, launches=0,
                                                 step_ms=[]))
            acc["ms"] += r["ms"]
            acc["bytes"] += r["bytes"]
            acc["launches"] += r["launches"]
            acc["step_ms"].append(r["ms"])
        if ps == args.profile_steps - 1:
            bv = b_v_bytes(h, 8, 8)
            vc = vcycle_rate(h, b, bv)
        h.close()
    # each kernel's time is its median over the profiled steps, times their
    # number (one step's timings can be disturbed by the node's other work)
    for acc in table_acc.values():
        acc["ms"] = statistics.median(acc["step_ms"]) * len(acc["step_ms"])
    table = sorted(table_acc.values(), key=lambda r: -r["ms"])
    # dominant single kernel of the step among the solve-phase kernels
    top = next((r for r in table if r["kind"] in HBM_KERNEL_KINDS), None)
    roofline = None
    if top:
        per_launch_bytes = top["bytes"] / top["launches"]
        per_launch_ms = top["ms"] / top["launches"]
        achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"{top['kind']}@level{top['level']}", "achieved": achieved,
                    "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": DRAM_BYTES_PER_LAUNCH.get((top["kind"], top["level"])),
                    "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
                    "launches_per_step": top["launches"] / args.profile_steps,
                    "share_of_profiled_solve": top["ms"] / sum(r["ms"] for r in table)}
    hbm_level0 = []
    for r in table:
        if r["level"] == 0 and r["kind"] in HBM_KERNEL_KINDS and r["ms"] > 0:
            g = r["bytes"] / (r["ms"] * 1e-3) / 1e9
            hbm_level0.append({"kernel": f"{r['kind']}@0", "gbs": g, "frac": g / peak, "frac_of_spec": g / HBM_SPEC_GBS,
                               "bytes_per_launch": r["bytes"] / r["launches"],
                               "traffic": DRAM_BYTES_PER_LAUNCH.get((r["kind"], 0))})
    kernels = [dict(kernel=f"{r['kind']}@{r['level']}", ms_per_step=r["ms"] / args.profile_steps,
                    launches_per_step=r["launches"] / args.profile_steps,
                    gbs=(r["bytes"] / (r["ms"] * 1e-3) / 1e9) if r["ms"] > 0 else 0.0) for r in table[:14]]

    # end to end through the public API from pinned host buffers
    h_rp = torch.from_numpy(sys_.rp).pin_memory()
    h_ci = torch.from_numpy(sys_.ci).pin_memory()
    h_val = torch.from_numpy(sys_.val).pin_memory()
    h_b = torch.from_numpy(sys_.b).pin_memory()
    h_x = torch.empty_like(h_b).pin_memory()
    d_rp, d_ci, d_val, d_b = (torch.empty_like(t, device=dev) for t in (h_rp, h_ci, h_val, h_b))
    h2d = sum(t.numel() * t.element_size() for t in (h_rp, h_ci, h_val, h_b))
    d2h = h_x.numel() * h_x.element_size()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps = max(1, args.e2e_steps)
    phases = []  # per step: events after the input copies, after the solve, after the result copy
    for _ in range(e2e_steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        for d, hsrc in ((d_rp, h_rp), (d_ci, h_ci), (d_val, h_val), (d_b, h_b)):
            d.copy_(hsrc, non_blocking=True)
        ev[1].record(stream)
        he = amg.amg_setup(d_rp, d_ci, d_val, params)
        xe = torch.zeros_like(d_b)
        amg.pcg_solve(he, d_b, xe, rtol=RTOL, max_iter=1000, flexible=True)
        ev[2].record(stream)
        h_x.copy_(xe, non_blocking=True)
        ev[3].record(stream)
        torch.cuda.current_stream().synchronize()
        he.close()
        phases.append(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allreduce_max(e0.elapsed_time(e1), world)
    e2e_value = job_throughput(e2e_steps, world, e2e_ms)
    e2e_phase_ms = {k: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in phases)
                    for i, k in enumerate(("h2d_ms", "setup_solve_ms", "d2h_ms"))}
    e2e_step_ms = [ev[0].elapsed_time(ev[3]) for ev in phases]
    del d_rp, d_ci, d_val, d_b, h_rp, h_ci, h_val

    # the oracle's full solve runs in a spawned child process on one host core
    # while the remaining GPU lines are measured; it starts only now, so that
    # it shares no host memory bandwidth with the headline and end-to-end
    # timings above (a spawned child is safe to start after CUDA work)
    cpu_proc = cpu_conn = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc, cpu_conn = start_cpu_baseline()

    configs = cycles = complexity = scaled = residency = batched = None
    if rank == 0 and world == 1 and not args.no_configs:
        configs = run_configs(dev, peak, x_main)
        try:
            batched = run_batched(dev)
        except Exception as e:  # recorded in the line; the other workloads still run
            batched = {"error": f"{type(e).__name__}: {e}"}
        residency = run_residency(dev)
        s2 = W.config_lognormal3d_128()
        cycles = run_cycles(dev, s2)
        complexity = run_complexity(dev)
        scaled = run_scaled_weight(dev, s2)
        del s2

    # the oracle's child is joined before the serving stream: the server's host
    # threads and copies must not share the host with it either
    cpu = finish_cpu_baseline(cpu_proc, cpu_conn) if rank == 0 else None

    serving = None
    if rank == 0 and world == 1 and args.serving_requests > 0:
        reqs, systems = generate_requests(args.serving_requests)
        serving = run_serving(reqs, systems)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": sys_.n, "nnz": sys_.nnz, "rtol": RTOL, "precision": "fp64",
                       "krylov": "flexible PCG", "levels": levels, "parallelism": f"replicas{world}",
                       "level_kernels": [dict(zip(("tpr", "fuse_pre", "fuse_post", "operator_form"), c))
                                         for c in level_cfg],
                       "l2": "inputs larger than L2 (level-0 CSR 1.47 GB > 129 MB); no flush"},
            "time_to_solution_ms": ms_per_step, "setup_ms": setup_mean, "solve_ms": solve_mean,
            "iterations": iters[0], "rel_res_true_max": max(rel_true),
            "vcycle": {"gbs": vc[0], "ms_per_cycle": vc[1], "bytes_per_cycle": bv, "peak": peak,
                       "frac": vc[0] / peak if vc[0] else None,
                       "frac_of_spec": vc[0] / HBM_SPEC_GBS if vc[0] else None,
                       "note": "algorithmic bytes of one V-cycle by the measurement plan's count (two matrix "
                               "passes, nine vector passes and the aggregate map per level, 8 N_L^2 for the dense "
                               "coarsest inverse) over the time of twenty V-cycles run with the profiler off"},
            "roofline": roofline, "hbm_level0": hbm_level0, "kernels": kernels,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "mean_phase_ms": e2e_phase_ms, "step_ms": e2e_step_ms,
                    "h2d_gbs": h2d / (e2e_phase_ms["h2d_ms"] * 1e-3) / 1e9 if e2e_phase_ms["h2d_ms"] > 0 else None},
            "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu,
            "configs_measured": configs, "cycles": cycles, "complexity": complexity,
            "option_scaled_weight": scaled, "host_resident_levels": residency, "batched": batched,
            "serving": serving,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
