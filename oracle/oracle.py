"""ctypes wrapper of the serial FP64 oracle (``amg_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Every function here forwards to the C oracle; the
wrapper converts numpy arrays and owns the hierarchy handle.  Nothing here
touches a GPU.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_trace_lock = threading.Lock()
_lib = None

# status codes of the oracle (mirrors the meaning, not the code, of the library's)
OK, ERR_INVALID_ARG, ERR_INVALID_CSR, ERR_ZERO_DIAG, ERR_OOM, ERR_BREAKDOWN, ERR_NOT_CONVERGED = range(7)


def build(force: bool = False) -> str:
    """Compile amg_oracle.c into oracle/_build/liboracle.so (plain gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    """Oracle parameters; defaults follow the method's configuration (2 pairwise
    passes, damped Jacobi omega = 2/3 with one pre and one post sweep, V-cycle;
    cycle = 1 selects the W-cycle, 2 the F-cycle).  matcher: 0 the greedy
    edge-order matching (Algorithm 3), 1 its literal handshake rounds, 2 the
    node-based matching of Algorithm 2 with the scan direction alternating
    between passes (Sec. 2.1.1)."""

    _fields_ = [
        ("passes", C.c_int),
        ("max_levels", C.c_int),
        ("coarse_max", C.c_int),
        ("stall_ratio", C.c_double),
        ("omega", C.c_double),
        ("nu_pre", C.c_int),
        ("nu_post", C.c_int),
        ("coarse_solver", C.c_int),
        ("matcher", C.c_int),
        ("cycle", C.c_int),
        ("tie_break", C.c_int),
        ("edge_weight", C.c_int),
    ]

    def __init__(self, **kw):
        super().__init__()
        lib().orc_default_params(C.byref(self))
        for k, v in kw.items():
            setattr(self, k, v)


class _Info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("rel_res_recurrence", C.c_double),
        ("rel_res_true", C.c_double),
        ("status", C.c_int),
    ]


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # AMG_ORACLE_SO lets the mutation tests load a deliberately broken copy
            l = C.CDLL(os.environ.get("AMG_ORACLE_SO") or build())
            l.orc_default_params.argtypes = [C.POINTER(Params)]
            l.orc_spmv.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
            l.orc_check_csr.argtypes = [C.c_int, C.c_longlong, _i32p, _i32p]
            l.orc_match_greedy.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p]
            l.orc_match_rounds.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, C.POINTER(C.c_int)]
            l.orc_match_greedy_opt.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, C.c_int, _i32p]
            l.orc_match_rounds_opt.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, C.c_int, _i32p,
                                               C.POINTER(C.c_int)]
            l.orc_nhem.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p]
            l.orc_nhem_dir.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, _i32p]
            l.orc_aggregates.argtypes = [C.c_int, _i32p, _i32p]
            l.orc_galerkin.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, C.c_int, _i32p, _i32p, _f64p]
            l.orc_galerkin.restype = C.c_longlong
            l.orc_dense_solve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
            l.orc_setup.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.POINTER(Params), C.POINTER(C.c_void_p)]
            l.orc_destroy.argtypes = [C.c_void_p]
            l.orc_num_levels.argtypes = [C.c_void_p]
            l.orc_dense_coarse.argtypes = [C.c_void_p]
            l.orc_last_coarse_cg_iters.argtypes = [C.c_void_p]
            l.orc_level_info.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
            l.orc_level_export.argtypes = [C.c_void_p, C.c_int, _i32p, _i32p, _f64p, C.c_void_p]
            l.orc_vcycle.argtypes = [C.c_void_p, _f64p, _f64p]
            l.orc_pcg.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int, C.c_int, C.POINTER(_Info)]
            l.orc_set_pcg_trace.argtypes = [C.c_void_p, C.c_int]
            l.orc_bicgstab.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int, C.POINTER(_Info)]
            l.orc_amg_solve.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int, C.POINTER(_Info)]
            _lib = l
    return _lib


def _csr(rp, ci, val):
    return (np.ascontiguousarray(rp, dtype=np.int32), np.ascontiguousarray(ci, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def spmv(rp, ci, val, x):
    rp, ci, val = _csr(rp, ci, val)
    n = len(rp) - 1
    y = np.empty(n)
    lib().orc_spmv(n, rp, ci, val, np.ascontiguousarray(x, dtype=np.float64), y)
    return y


def check_csr(rp, ci):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    return lib().orc_check_csr(len(rp) - 1, int(rp[-1]) if len(rp) else 0, rp, ci)


def match_greedy(rp, ci, val, tie_break=0, edge_weight=0):
    """Greedy edge-based HEM (Algorithm 3): mate array.  tie_break 0 orders
    equal weights by smaller index, 1 by larger (Algorithm 3's descending
    sort); edge_weight 1 divides by sqrt(|a_ii a_jj|)."""
    rp, ci, val = _csr(rp, ci, val)
    n = len(rp) - 1
    mate = np.empty(n, dtype=np.int32)
    if tie_break == 0 and edge_weight == 0:
        lib().orc_match_greedy(n, rp, ci, val, mate)
    else:
        lib().orc_match_greedy_opt(n, rp, ci, val, int(tie_break), int(edge_weight), mate)
    return mate


def match_rounds(rp, ci, val, tie_break=0, edge_weight=0):
    """Synchronous handshake rounds run to their fixed point: (mate, rounds)."""
    rp, ci, val = _csr(rp, ci, val)
    n = len(rp) - 1
    mate = np.empty(n, dtype=np.int32)
    r = C.c_int(0)
    if tie_break == 0 and edge_weight == 0:
        lib().orc_match_rounds(n, rp, ci, val, mate, C.byref(r))
    else:
        lib().orc_match_rounds_opt(n, rp, ci, val, int(tie_break), int(edge_weight), mate, C.byref(r))
    return mate, r.value


def nhem(rp, ci, val, descending=False):
    """Literal node-based HEM of Algorithm 2: (agg, n_c).  descending scans
    the nodes from the last index down (the alternate direction of Sec. 2.1.1);
    aggregates are numbered in visit order either way."""
    rp, ci, val = _csr(rp, ci, val)
    n = len(rp) - 1
    agg = np.empty(n, dtype=np.int32)
    nc = lib().orc_nhem_dir(n, rp, ci, val, int(bool(descending)), agg)
    return agg, nc


def aggregates(mate):
    mate = np.ascontiguousarray(mate, dtype=np.int32)
    agg = np.empty(len(mate), dtype=np.int32)
    nc = lib().orc_aggregates(len(mate), mate, agg)
    return agg, nc


def galerkin(rp, ci, val, agg, nc):
    """A_c = P^T A P for the piecewise-constant P of agg: (rp_c, ci_c, val_c)."""
    rp, ci, val = _csr(rp, ci, val)
    n = len(rp) - 1
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    nnz = int(rp[-1])
    rpc = np.empty(nc + 1, dtype=np.int32)
    cic = np.empty(max(nnz, 1), dtype=np.int32)
    valc = np.empty(max(nnz, 1))
    m = lib().orc_galerkin(n, rp, ci, val, agg, nc, rpc, cic, valc)
    if m < 0:
        raise MemoryError("oracle galerkin")
    return rpc, cic[:m].copy(), valc[:m].copy()


def dense_solve(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    x = np.empty(a.shape[0])
    st = lib().orc_dense_solve(a.shape[0], a, np.ascontiguousarray(b, dtype=np.float64), x)
    if st != OK:
        raise np.linalg.LinAlgError("singular")
    return x


class SolveInfo:
    def __init__(self, info: _Info):
        self.iterations = info.iterations
        self.rel_res_recurrence = info.rel_res_recurrence
        self.rel_res_true = info.rel_res_true
        self.status = info.status

    def __repr__(self):
        return (f"SolveInfo(iterations={self.iterations}, rel_res={self.rel_res_recurrence:.3e}, "
                f"true={self.rel_res_true:.3e}, status={self.status})")


class Hierarchy:
    """Oracle AMG hierarchy (setup phase) with its cycle (V, W or F), AMG as a
    solver, PCG and BiCGStab."""

    def __init__(self, rp, ci, val, params: Params | None = None, **kw):
        self._rp, self._ci, self._val = _csr(rp, ci, val)
        self.n = len(self._rp) - 1
        self.params = params if params is not None else Params(**kw)
        h = C.c_void_p()
        st = lib().orc_setup(self.n, self._rp, self._ci, self._val, C.byref(self.params), C.byref(h))
        if st != OK:
            raise ValueError(f"oracle setup failed with status {st}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_destroy(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return lib().orc_num_levels(self._h)

    @property
    def dense_coarse(self) -> bool:
        return bool(lib().orc_dense_coarse(self._h))

    @property
    def last_coarse_cg_iters(self) -> int:
        return lib().orc_last_coarse_cg_iters(self._h)

    def level_info(self, k):
        n = C.c_int()
        nnz = C.c_longlong()
        rounds = (C.c_int * 8)()
        st = lib().orc_level_info(self._h, k, C.byref(n), C.byref(nnz), rounds)
        if st != OK:
            raise IndexError(k)
        return n.value, nnz.value, list(rounds)

    def level(self, k):
        """(rp, ci, val, agg) of level k; agg is None at the coarsest level."""
        n, nnz, _ = self.level_info(k)
        rp = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        val = np.empty(max(nnz, 1))
        agg = np.empty(max(n, 1), dtype=np.int32) if k < self.num_levels - 1 else None
        lib().orc_level_export(self._h, k, rp, ci, val,
                               agg.ctypes.data_as(C.c_void_p) if agg is not None else None)
        return rp, ci[:nnz], val[:nnz], (agg[:n] if agg is not None else None)

    def sizes(self):
        return [self.level_info(k)[0] for k in range(self.num_levels)]

    def vcycle(self, r):
        """z = M^{-1} r: one cycle of the configured kind (V, W or F) from zero."""
        z = np.empty(self.n)
        lib().orc_vcycle(self._h, np.ascontiguousarray(r, dtype=np.float64), z)
        return z

    def pcg(self, b, x0=None, rtol=1e-8, max_iter=1000, flexible=False):
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        info = _Info()
        lib().orc_pcg(self._h, np.ascontiguousarray(b, dtype=np.float64), x, rtol, max_iter,
                      int(flexible), C.byref(info))
        return x, SolveInfo(info)

    def pcg_directions(self, b, rtol=1e-8, max_iter=1000, flexible=False):
        """PCG as pcg() does, also returning its search directions: (x, info,
        P) with P[j - 1] the direction p_j of iteration j."""
        P = np.zeros((max(max_iter, 1), self.n))
        with _trace_lock:
            lib().orc_set_pcg_trace(P.ctypes.data_as(C.c_void_p), max_iter)
            try:
                x, info = self.pcg(b, rtol=rtol, max_iter=max_iter, flexible=flexible)
            finally:
                lib().orc_set_pcg_trace(None, 0)
        return x, info, P[:info.iterations]

    def amg_solve(self, b, x0=None, rtol=1e-8, max_iter=1000):
        """AMG as a solver: x_{j+1} = x_j + M^{-1}(b - A x_j) until the tolerance."""
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        info = _Info()
        lib().orc_amg_solve(self._h, np.ascontiguousarray(b, dtype=np.float64), x, rtol, max_iter,
                            C.byref(info))
        return x, SolveInfo(info)

    def bicgstab(self, b, x0=None, rtol=1e-8, max_iter=1000):
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        info = _Info()
        lib().orc_bicgstab(self._h, np.ascontiguousarray(b, dtype=np.float64), x, rtol, max_iter,
                           C.byref(info))
        return x, SolveInfo(info)
