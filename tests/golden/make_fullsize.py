"""Writes the stored oracle results of the full-size workloads.

Runs the serial FP64 oracle (and nothing else) on the two largest benchmark
systems and stores what the GPU parity tests compare against:

- anisotropic3d_256 (16,777,216 unknowns, eps_z = 1e-3, seed 2): the whole
  hierarchy (SHA-256 of every level's row pointers, columns, FP64 values and
  aggregate map), flexible AMG-PCG (Algorithm 4) to a relative residual of
  1e-8, and its solution: 2-norm, 4096 sampled entries and a 32-row
  Rademacher sketch S x (S from ``numpy.random.default_rng(11)``);
- convdiff2d_2048 at Peclet 100 (4,194,304 unknowns, seed 3): the hierarchy
  hashes, AMG-BiCGStab (Algorithm 5, FP64 V-cycle) to 1e-8 and to 1e-12, and
  the 1e-12 solution in the same compressed form.

Every record is keyed by the SHA-256 of the input (row pointers, columns,
values, right-hand side): a test whose regenerated input hashes differently
recomputes the record with ``record(name)`` instead of using the stored one.

    python tests/golden/make_fullsize.py [anisotropic3d_256] [convdiff2d_2048_pe100]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SAMPLE_SEED, SAMPLES = 7, 4096
SKETCH_SEED, SKETCH_ROWS = 11, 32


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def system(name: str):
    from paper_2007_00056_gb300 import workloads as W

    if name == "anisotropic3d_256":
        return W.config_anisotropic3d_256()
    if name == "convdiff2d_2048_pe100":
        return W.config_convdiff2d_2048(peclet=100.0)
    raise KeyError(name)


def input_hash(s) -> str:
    return sha(s.rp, s.ci, s.val, s.b)


def sample_indices(n: int) -> np.ndarray:
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, size=min(SAMPLES, n), replace=False))


def sketch(x: np.ndarray) -> list[float]:
    """S x for the SKETCH_ROWS x n matrix S of independent +-1 entries drawn
    row by row from default_rng(SKETCH_SEED); E ||S e||^2 = SKETCH_ROWS ||e||^2."""
    rng = np.random.default_rng(SKETCH_SEED)
    out = []
    for _ in range(SKETCH_ROWS):
        sgn = rng.integers(0, 2, size=len(x), dtype=np.int8).astype(np.float64) * 2.0 - 1.0
        out.append(float(sgn @ x))
    return out


def solution_record(x: np.ndarray) -> dict:
    idx = sample_indices(len(x))
    return {"norm2": float(np.linalg.norm(x)), "sample_idx": idx.tolist(), "sample_x": x[idx].tolist(),
            "sketch": sketch(x)}


def hierarchy_record(oh) -> list[dict]:
    out = []
    for k in range(oh.num_levels):
        rp, ci, val, agg = oh.level(k)
        out.append({"n": int(len(rp) - 1), "nnz": int(len(ci)), "rp": sha(rp), "ci": sha(ci), "val": sha(val),
                    "agg": sha(agg) if agg is not None else None})
    return out


def record(name: str) -> dict:
    """The oracle's record for one workload (minutes of serial CPU)."""
    import oracle as O

    s = system(name)
    t0 = time.perf_counter()
    oh = O.Hierarchy(s.rp, s.ci, s.val)
    rec = {"workload": name, "n": s.n, "nnz": s.nnz, "input_sha256": input_hash(s),
           "oracle_setup_s": time.perf_counter() - t0, "levels": hierarchy_record(oh)}
    if name == "anisotropic3d_256":
        t0 = time.perf_counter()
        x, info = oh.pcg(s.b, rtol=1e-8, flexible=True)
        rec["pcg_flexible"] = {"rtol": 1e-8, "iterations": info.iterations, "status": info.status,
                               "rel_res_recurrence": info.rel_res_recurrence, "rel_res_true": info.rel_res_true,
                               "oracle_solve_s": time.perf_counter() - t0, "solution": solution_record(x)}
    else:
        for rtol, key in ((1e-8, "bicgstab_1e-8"), (1e-12, "bicgstab_1e-12")):
            t0 = time.perf_counter()
            x, info = oh.bicgstab(s.b, rtol=rtol, max_iter=5000)
            rec[key] = {"rtol": rtol, "iterations": info.iterations, "status": info.status,
                        "rel_res_recurrence": info.rel_res_recurrence, "rel_res_true": info.rel_res_true,
                        "oracle_solve_s": time.perf_counter() - t0}
            if rtol == 1e-12:
                rec[key]["solution"] = solution_record(x)
    return rec


def path(name: str) -> str:
    return os.path.join(HERE, f"fullsize_{name}.json")


def load(name: str) -> dict:
    with open(path(name)) as f:
        return json.load(f)


if __name__ == "__main__":
    names = sys.argv[1:] or ["anisotropic3d_256", "convdiff2d_2048_pe100"]
    for nm in names:
        r = record(nm)
        with open(path(nm), "w") as f:
            json.dump(r, f)
        print(nm, r["input_sha256"], flush=True)
