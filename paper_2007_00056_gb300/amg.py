"""Python binding of the C ABI in ``include/amg.h`` (argument marshalling only).

Every function has the name of the C entry point it wraps and takes torch
CUDA tensors; all computation runs in the CUDA library.  There is no CPU
fallback: if ``libamg_gb300.so`` has not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

AMG_OK = 0
STATUS = {
    0: "AMG_OK", 1: "AMG_ERR_INVALID_ARG", 2: "AMG_ERR_INVALID_CSR", 3: "AMG_ERR_ZERO_DIAG",
    4: "AMG_ERR_OOM", 5: "AMG_ERR_BREAKDOWN", 6: "AMG_ERR_NOT_CONVERGED", 7: "AMG_ERR_TIMEOUT",
    8: "AMG_ERR_CUDA", 9: "AMG_ERR_UNSUPPORTED",
}
AMG_ERR_INVALID_ARG, AMG_ERR_INVALID_CSR, AMG_ERR_ZERO_DIAG, AMG_ERR_OOM = 1, 2, 3, 4
AMG_ERR_BREAKDOWN, AMG_ERR_NOT_CONVERGED, AMG_ERR_TIMEOUT, AMG_ERR_CUDA, AMG_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
AMG_FP64, AMG_FP32, AMG_FP16_STORAGE = 0, 1, 2
AMG_COARSE_AUTO, AMG_COARSE_DENSE, AMG_COARSE_CG = 0, 1, 2
AMG_CYCLE_V, AMG_CYCLE_W, AMG_CYCLE_F = 0, 1, 2
AMG_TIE_SMALLER, AMG_TIE_LARGER = 0, 1
AMG_WEIGHT_ABS, AMG_WEIGHT_SCALED = 0, 1
AMG_RESIDENT, AMG_HOST_MAPPED, AMG_HOST_STAGED = 0, 1, 2

# every symbol include/amg.h declares
EXPORTS = (
    "amg_default_params", "amg_setup", "amg_vcycle", "amg_solve", "pcg_solve", "bicgstab_solve", "amg_num_levels",
    "amg_level_info", "amg_export_level", "amg_setup_rounds", "amg_destroy", "amg_status_string",
    "amg_kernel_launches", "amg_profile_enable", "amg_profile_reset", "amg_profile_read",
    "amg_coarse_cg_noalloc", "amg_autotune", "amg_level_config", "amg_level_set_config", "amg_batch_pcg",
    "amg_selftest_wait_timeout", "amg_selftest_convert", "amg_last_cuda_error", "amg_coarse_cg_cluster_size",
    "amg_level_operator_form", "amg_level_set_operator_form", "amg_set_residency", "amg_memory_info",
)
KERNEL_KINDS = ("jacobi0", "jacobi", "residual", "restrict", "prolong_jacobi", "prolong", "coarse_dense",
                "coarse_cg", "cast", "krylov_spmv", "krylov_vec", "op_residual", "op_post")


class AmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = status_string(status)
        if status in (8, 4):  # AMG_ERR_CUDA, AMG_ERR_OOM: name the CUDA error behind it
            try:
                detail += f"; {lib().amg_last_cuda_error().decode()}"
            except Exception:
                pass
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


class amg_params(C.Structure):
    _fields_ = [
        ("passes", C.c_int),
        ("max_levels", C.c_int),
        ("coarse_max", C.c_int),
        ("stall_ratio", C.c_double),
        ("omega", C.c_double),
        ("nu_pre", C.c_int),
        ("nu_post", C.c_int),
        ("coarse_solver", C.c_int),
        ("precision", C.c_int),
        ("cycle", C.c_int),
        ("tie_break", C.c_int),
        ("edge_weight", C.c_int),
        ("operator_form", C.c_int),
        ("dense_max", C.c_int),
        ("graphs", C.c_int),
    ]


class amg_solve_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("rel_res_recurrence", C.c_double),
        ("rel_res_true", C.c_double),
        ("status", C.c_int),
    ]

    def __repr__(self):
        return (f"amg_solve_info(iterations={self.iterations}, rel_res={self.rel_res_recurrence:.3e}, "
                f"true={self.rel_res_true:.3e}, status={STATUS.get(self.status, self.status)})")


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Loads libamg_gb300.so; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                if build_if_missing:
                    _build.build()
                else:
                    raise RuntimeError(f"CUDA library not built: {path} is missing "
                                       "(run __graft_entry__.build() first)")
            l = C.CDLL(path)
            vp, i32, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
            l.amg_default_params.argtypes = [C.POINTER(amg_params)]
            l.amg_setup.argtypes = [i32, i64, vp, vp, vp, C.POINTER(amg_params), vp, C.POINTER(vp)]
            l.amg_vcycle.argtypes = [vp, vp, vp, vp]
            l.amg_solve.argtypes = [vp, vp, vp, d, i32, vp, C.POINTER(amg_solve_info)]
            l.pcg_solve.argtypes = [vp, vp, vp, d, i32, i32, vp, C.POINTER(amg_solve_info)]
            l.bicgstab_solve.argtypes = [vp, vp, vp, d, i32, vp, C.POINTER(amg_solve_info)]
            l.amg_num_levels.argtypes = [vp]
            l.amg_level_info.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i64), vp, vp]
            l.amg_export_level.argtypes = [vp, i32, vp, vp, vp, vp]
            l.amg_setup_rounds.argtypes = [vp, i32, i32]
            l.amg_destroy.argtypes = [vp]
            l.amg_destroy.restype = None
            l.amg_status_string.argtypes = [i32]
            l.amg_status_string.restype = C.c_char_p
            l.amg_kernel_launches.argtypes = []
            l.amg_kernel_launches.restype = C.c_ulonglong
            l.amg_profile_enable.argtypes = [vp, i32]
            l.amg_profile_reset.argtypes = [vp]
            l.amg_profile_read.argtypes = [vp, i32, i32, C.POINTER(d), C.POINTER(d), C.POINTER(C.c_longlong)]
            l.amg_autotune.argtypes = [vp, vp]
            l.amg_selftest_wait_timeout.argtypes = [i32, vp]
            l.amg_selftest_convert.argtypes = [i64, vp, vp, vp, vp]
            l.amg_last_cuda_error.argtypes = []
            l.amg_last_cuda_error.restype = C.c_char_p
            l.amg_batch_pcg.argtypes = [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), d, i32, i32, vp,
                                        C.POINTER(amg_solve_info)]
            l.amg_level_set_config.argtypes = [vp, i32, i32, i32, i32]
            l.amg_level_config.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
            l.amg_coarse_cg_noalloc.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, C.POINTER(i32)]
            l.amg_coarse_cg_cluster_size.argtypes = [vp]
            l.amg_level_operator_form.argtypes = [vp, i32]
            l.amg_level_set_operator_form.argtypes = [vp, i32, i32]
            l.amg_set_residency.argtypes = [vp, i32, i32, vp]
            u64p = C.POINTER(C.c_uint64)
            l.amg_memory_info.argtypes = [vp, u64p, u64p, u64p, u64p]
            _lib = l
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().amg_status_string(int(status)).decode()
    except Exception:  # library not loadable: still give the symbolic name
        return STATUS.get(status, str(status))


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def amg_default_params(**overrides) -> amg_params:
    p = amg_params()
    st = lib().amg_default_params(C.byref(p))
    if st != AMG_OK:
        raise AmgError(st, "amg_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Hierarchy:
    """Owning handle of a device hierarchy (amg_destroy on close / garbage collection)."""

    def __init__(self, handle: C.c_void_p, n: int, params: amg_params):
        self._h = handle
        self.n = n
        self.params = params

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("hierarchy already destroyed")
        return self._h

    def close(self):
        if self._h is not None:
            lib().amg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self) -> int:
        return lib().amg_num_levels(self.handle)

    def sizes(self):
        return [amg_level_info(self, k)[0] for k in range(self.num_levels)]


def amg_setup(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, params: amg_params | None = None,
              stream=None, **overrides) -> Hierarchy:
    """Setup phase on the device; returns the hierarchy (raises AmgError on failure)."""
    n = row_ptr.numel() - 1
    nnz = col.numel()
    if params is None:
        params = amg_default_params(**overrides)
    out = C.c_void_p()
    st = lib().amg_setup(n, nnz, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                         _dev(val, torch.float64, "val"), C.byref(params), _stream(stream), C.byref(out))
    if st != AMG_OK:
        raise AmgError(st, "amg_setup")
    return Hierarchy(out, n, params)


def amg_vcycle(h: Hierarchy, r: torch.Tensor, z: torch.Tensor, stream=None) -> None:
    st = lib().amg_vcycle(h.handle, _dev(r, torch.float64, "r"), _dev(z, torch.float64, "z"), _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_vcycle")


def amg_solve(h: Hierarchy, b: torch.Tensor, x: torch.Tensor, rtol: float = 1e-8, max_iter: int = 1000,
              stream=None, check: bool = False) -> amg_solve_info:
    """AMG as a solver (stationary cycles).  x holds x0 on entry.  Returns the
    solve info; with check=True a status other than AMG_OK raises."""
    info = amg_solve_info()
    st = lib().amg_solve(h.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"), float(rtol),
                         int(max_iter), _stream(stream), C.byref(info))
    if st not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN) or (check and st != AMG_OK):
        raise AmgError(st, "amg_solve")
    info.status = st
    return info


def pcg_solve(h: Hierarchy, b: torch.Tensor, x: torch.Tensor, rtol: float = 1e-8, max_iter: int = 1000,
              flexible: bool = False, stream=None, check: bool = False) -> amg_solve_info:
    """x holds x0 on entry.  Returns the solve info; with check=True a status other
    than AMG_OK raises."""
    info = amg_solve_info()
    st = lib().pcg_solve(h.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"), float(rtol),
                         int(max_iter), int(bool(flexible)), _stream(stream), C.byref(info))
    if st not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN) or (check and st != AMG_OK):
        raise AmgError(st, "pcg_solve")
    info.status = st
    return info


def bicgstab_solve(h: Hierarchy, b: torch.Tensor, x: torch.Tensor, rtol: float = 1e-8, max_iter: int = 1000,
                   stream=None, check: bool = False) -> amg_solve_info:
    info = amg_solve_info()
    st = lib().bicgstab_solve(h.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"), float(rtol),
                              int(max_iter), _stream(stream), C.byref(info))
    if st not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN) or (check and st != AMG_OK):
        raise AmgError(st, "bicgstab_solve")
    info.status = st
    return info


def amg_num_levels(h: Hierarchy) -> int:
    return lib().amg_num_levels(h.handle)


def amg_level_info(h: Hierarchy, level: int, agg_out: torch.Tensor | None = None, stream=None):
    """(n, nnz) of a level; fills agg_out (int32, length n) with its aggregate map if given."""
    n = C.c_int()
    nnz = C.c_int64()
    ptr = _dev(agg_out, torch.int32, "agg_out") if agg_out is not None else None
    st = lib().amg_level_info(h.handle, int(level), C.byref(n), C.byref(nnz), ptr, _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_level_info")
    return n.value, nnz.value


def amg_export_level(h: Hierarchy, level: int, stream=None):
    """Level CSR as device tensors (row_ptr, col, val)."""
    n, nnz = amg_level_info(h, level)
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
    st = lib().amg_export_level(h.handle, int(level), rp.data_ptr(), ci.data_ptr(), val.data_ptr(), _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_export_level")
    return rp, ci[:nnz], val[:nnz]


def amg_setup_rounds(h: Hierarchy, level: int, p: int) -> int:
    return lib().amg_setup_rounds(h.handle, int(level), int(p))


def amg_destroy(h: Hierarchy) -> None:
    h.close()


def amg_kernel_launches() -> int:
    return int(lib().amg_kernel_launches())


def amg_profile_enable(h: Hierarchy, on: bool = True) -> None:
    st = lib().amg_profile_enable(h.handle, int(bool(on)))
    if st != AMG_OK:
        raise AmgError(st, "amg_profile_enable")


def amg_profile_reset(h: Hierarchy) -> None:
    st = lib().amg_profile_reset(h.handle)
    if st != AMG_OK:
        raise AmgError(st, "amg_profile_reset")


def amg_profile_read(h: Hierarchy, kind, level: int = 0):
    """(ms, bytes, launches) accumulated for a kernel kind (name or index) at a level."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ms, by, n = C.c_double(), C.c_double(), C.c_longlong()
    st = lib().amg_profile_read(h.handle, k, int(level), C.byref(ms), C.byref(by), C.byref(n))
    if st != AMG_OK:
        raise AmgError(st, "amg_profile_read")
    return ms.value, by.value, n.value


def amg_profile_table(h: Hierarchy):
    """Every (kind, level) with launches: list of dicts sorted by time, descending."""
    rows = []
    for ki, kind in enumerate(KERNEL_KINDS):
        for lev in range(max(1, h.num_levels)):
            ms, by, n = amg_profile_read(h, ki, lev)
            if n:
                rows.append(dict(kind=kind, level=lev, ms=ms, bytes=by, launches=n,
                                 gbs=(by / (ms * 1e-3) / 1e9) if ms > 0 else 0.0))
    rows.sort(key=lambda r: -r["ms"])
    return rows


def amg_coarse_cg_cluster_size(h: Hierarchy) -> int:
    """CTAs of the cluster that solves the coarsest level by CG (0: the whole
    GPU; -1: dense inverse)."""
    return lib().amg_coarse_cg_cluster_size(h.handle)


NOALLOC_MAX_N = 262144


def amg_coarse_cg_noalloc(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, f: torch.Tensor,
                          x: torch.Tensor, stream=None) -> int:
    """Jacobi-PCG solve of A x = f (to 1e-12) using only the library's fixed
    scratch array (no device allocation); returns the iteration count."""
    it = C.c_int(0)
    st = lib().amg_coarse_cg_noalloc(row_ptr.numel() - 1, col.numel(), _dev(row_ptr, torch.int32, "row_ptr"),
                                     _dev(col, torch.int32, "col"), _dev(val, torch.float64, "val"),
                                     _dev(f, torch.float64, "f"), _dev(x, torch.float64, "x"), _stream(stream),
                                     C.byref(it))
    if st != AMG_OK:
        raise AmgError(st, "amg_coarse_cg_noalloc")
    return it.value


def amg_autotune(h: Hierarchy, stream=None) -> None:
    """Times kernel variants on h's levels, keeps the fastest and caches them by level shape."""
    st = lib().amg_autotune(h.handle, _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_autotune")


def amg_level_config(h: Hierarchy, level: int):
    """(lanes per row, fused presmoothing, fused prolongation) of a level."""
    t, a, b = C.c_int(), C.c_int(), C.c_int()
    if lib().amg_level_config(h.handle, int(level), C.byref(t), C.byref(a), C.byref(b)) != 0:
        raise IndexError(level)
    return t.value, a.value, b.value


def amg_level_set_config(h: Hierarchy, level: int, tpr: int, fuse_pre: bool, fuse_post: bool) -> None:
    st = lib().amg_level_set_config(h.handle, int(level), int(tpr), int(bool(fuse_pre)), int(bool(fuse_post)))
    if st != AMG_OK:
        raise AmgError(st, "amg_level_set_config")


def amg_level_operator_form(h: Hierarchy, level: int) -> bool:
    """Whether zero-guess visits of a level use the residual-operator form."""
    r = lib().amg_level_operator_form(h.handle, int(level))
    if r < 0:
        raise IndexError(level)
    return bool(r)


def amg_level_set_operator_form(h: Hierarchy, level: int, on: bool) -> None:
    st = lib().amg_level_set_operator_form(h.handle, int(level), int(bool(on)))
    if st != AMG_OK:
        raise AmgError(st, "amg_level_set_operator_form")


def amg_set_residency(h: Hierarchy, residency: int, first_level: int = 0, stream=None) -> None:
    """Moves the matrix arrays of levels first_level..L-1 to pinned host memory
    (AMG_HOST_MAPPED, AMG_HOST_STAGED) or everything back (AMG_RESIDENT)."""
    st = lib().amg_set_residency(h.handle, int(residency), int(first_level), _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_set_residency")


def amg_memory_info(h: Hierarchy) -> dict:
    """Device bytes, pinned host bytes, staging bytes and bytes copied by the staging."""
    v = [C.c_uint64() for _ in range(4)]
    st = lib().amg_memory_info(h.handle, *[C.byref(x) for x in v])
    if st != AMG_OK:
        raise AmgError(st, "amg_memory_info")
    return dict(zip(("device_bytes", "host_bytes", "staging_bytes", "copied_bytes"), (x.value for x in v)))


def amg_batch_pcg(hs, bs, xs, rtol: float = 1e-8, max_iter: int = 1000, flexible: bool = False, stream=None):
    """Solves len(hs) systems in one persistent launch per team size (a thread
    block, or a cluster of 2, 4 or 8 blocks, per system by its row count).
    Returns the list of per-system solve infos; raises AmgError only for
    errors other than non-convergence or breakdown."""
    k = len(hs)
    if not (len(bs) == len(xs) == k) or k == 0:
        raise ValueError("hs, bs and xs must have the same non-zero length")
    H = (C.c_void_p * k)(*[h.handle for h in hs])
    B = (C.c_void_p * k)(*[_dev(b, torch.float64, "b") for b in bs])
    X = (C.c_void_p * k)(*[_dev(x, torch.float64, "x") for x in xs])
    infos = (amg_solve_info * k)()
    st = lib().amg_batch_pcg(k, H, B, X, float(rtol), int(max_iter), int(bool(flexible)), _stream(stream), infos)
    if st not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN):
        raise AmgError(st, "amg_batch_pcg")
    return list(infos)


def amg_selftest_convert(x: torch.Tensor, stream=None):
    """The library's FP64 -> FP32 -> FP64 conversions of a CUDA float64 tensor:
    returns (x rounded to FP32, that widened back to FP64)."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("x must be a CUDA float64 tensor")
    x = x.contiguous()
    f32 = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    f64 = torch.empty_like(x)
    st = lib().amg_selftest_convert(x.numel(), x.data_ptr(), f32.data_ptr(), f64.data_ptr(), _stream(stream))
    if st != AMG_OK:
        raise AmgError(st, "amg_selftest_convert")
    return f32, f64


def amg_selftest_wait_timeout(blocks: int = 8, stream=None) -> int:
    """Runs the bounded-wait self-test; returns the status (AMG_ERR_TIMEOUT expected)."""
    return lib().amg_selftest_wait_timeout(int(blocks), _stream(stream))
