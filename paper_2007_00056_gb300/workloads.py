"""Seeded synthetic linear systems shaped like the method's workloads.

This module only assembles test problems (matrices in CSR and right-hand
sides).  It holds none of the AMG method's arithmetic and imports neither the
CUDA library nor the oracle; both sides are fed from here.

Conventions (all generators): square CSR with int32 row pointers and column
indices, columns strictly ascending in every row, FP64 values; unknowns are
numbered lexicographically with x fastest; Dirichlet boundary nodes are
eliminated; every random draw comes from ``numpy.random.default_rng(seed)``
(PCG64), so a (generator, size, seed) triple fixes the bytes.

The paper evaluates on finite-element matrices of a scalar convection-diffusion
equation (Sec. 4.1, Table 1: P1-P4 elements, 55k-6.3M unknowns, about seven
nonzeros per row for P1) and on SuiteSparse matrices (Table 4); neither set is
available, so these generators stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    """A CSR system A x = b."""

    name: str
    rp: np.ndarray  # int32, n+1
    ci: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    b: np.ndarray  # float64, n
    symmetric: bool = True

    @property
    def n(self) -> int:
        return len(self.rp) - 1

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rp))
        a[rows, self.ci] = self.val
        return a


def _compress(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray):
    """(n, k) candidate columns (ascending per row) + existence mask -> CSR."""
    counts = mask.sum(axis=1)
    rp = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    ci = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    assert rp[-1] < 2**31
    return rp.astype(np.int32), ci, val


def _grid_stencil(shape, offsets, coefs_fn):
    """Generic structured-grid stencil assembly.

    shape: grid extents, x fastest (nx, ny[, nz]).  offsets: list of integer
    offset tuples in ascending column order (the diagonal is the zero tuple).
    coefs_fn(k, idx) returns the (N,) values of offset k given the (d, N)
    coordinate array idx.  Entries whose neighbour falls outside the grid are
    dropped (Dirichlet elimination)."""
    dims = len(shape)
    N = int(np.prod(shape))
    strides = [1]
    for d in range(1, dims):
        strides.append(strides[-1] * shape[d - 1])
    lin = np.arange(N, dtype=np.int64)
    idx = []
    rem = lin.copy()
    for d in range(dims):
        idx.append(rem % shape[d])
        rem //= shape[d]
    idx = np.stack(idx)
    K = len(offsets)
    cols = np.empty((N, K), dtype=np.int64)
    vals = np.empty((N, K), dtype=np.float64)
    mask = np.ones((N, K), dtype=bool)
    for k, off in enumerate(offsets):
        c = lin.copy()
        for d in range(dims):
            if off[d]:
                nd = idx[d] + off[d]
                mask[:, k] &= (nd >= 0) & (nd < shape[d])
                c += off[d] * strides[d]
        cols[:, k] = c
        vals[:, k] = coefs_fn(k, idx)
    cols[~mask] = 0
    return _compress(cols, vals, mask)


_OFF2 = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
_OFF3 = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def poisson2d(n: int, seed: int = 0) -> System:
    """2D 5-point Poisson [-1,-1,4,-1,-1] on an n x n interior grid; b ~ U[-1,1] from seed."""
    def coef(k, idx):
        return np.full(idx.shape[1], 4.0 if k == 2 else -1.0)

    rp, ci, val = _grid_stencil((n, n), _OFF2, coef)
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, n * n)
    return System(f"poisson2d_{n}", rp, ci, val, b)


def anisotropic3d(n: int, eps_z: float = 1e-3, seed: int = 2) -> System:
    """3D 7-point diffusion with coefficients (1, 1, eps_z): off-diagonals -1, -1,
    -eps_z; diagonal 2(2 + eps_z) on every row (Dirichlet eliminated)."""
    d = 2.0 * (2.0 + eps_z)
    per = [-eps_z, -1.0, -1.0, d, -1.0, -1.0, -eps_z]

    def coef(k, idx):
        return np.full(idx.shape[1], per[k])

    rp, ci, val = _grid_stencil((n, n, n), _OFF3, coef)
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, n ** 3)
    return System(f"anisotropic3d_{n}_eps{eps_z:g}", rp, ci, val, b)


def lognormal3d(n: int, seed: int = 1, sigma: float = 1.0) -> System:
    """3D cell-centred finite-volume diffusion on n^3 cells with cell
    coefficients k = exp(sigma * N(0,1)) drawn in grid order.  Interior face
    transmissibility T = 2 k_a k_b / (k_a + k_b), Dirichlet wall face T = 2 k
    (half cell to the wall); diagonal = sum of the six face T's, off-diagonal
    = -T.  b is the same generator's next U[-1,1] draw."""
    rng = np.random.default_rng(seed)
    N = n ** 3
    kc = np.exp(sigma * rng.standard_normal(N))
    b = rng.uniform(-1.0, 1.0, N)
    k3 = kc.reshape(n, n, n)  # [z, y, x]

    def faces(axis):
        a = k3
        lo = np.take(a, range(0, n - 1), axis=axis)
        hi = np.take(a, range(1, n), axis=axis)
        return 2.0 * lo * hi / (lo + hi)

    # transmissibility toward the neighbour in direction (axis, sign); wall faces 2k
    def trans(axis, sign):
        t = np.empty((n, n, n))
        f = faces(axis)
        sl_all = [slice(None)] * 3
        if sign < 0:
            sl_in = list(sl_all); sl_in[axis] = slice(1, n)
            sl_b = list(sl_all); sl_b[axis] = slice(0, 1)
        else:
            sl_in = list(sl_all); sl_in[axis] = slice(0, n - 1)
            sl_b = list(sl_all); sl_b[axis] = slice(n - 1, n)
        t[tuple(sl_in)] = f
        t[tuple(sl_b)] = 2.0 * k3[tuple(sl_b)]
        return t.reshape(N)

    # axes of k3: 0 = z, 1 = y, 2 = x
    tz_m, ty_m, tx_m = trans(0, -1), trans(1, -1), trans(2, -1)
    tx_p, ty_p, tz_p = trans(2, +1), trans(1, +1), trans(0, +1)
    diag = ((((tz_m + ty_m) + tx_m) + tx_p) + ty_p) + tz_p
    per = [-tz_m, -ty_m, -tx_m, diag, -tx_p, -ty_p, -tz_p]

    def coef(k, idx):
        return per[k]

    rp, ci, val = _grid_stencil((n, n, n), _OFF3, coef)
    return System(f"lognormal3d_{n}_s{seed}", rp, ci, val, b)


def convdiff2d(n: int, peclet: float = 100.0, seed: int = 3) -> System:
    """-Lap u + w . grad u on (0,1)^2, first-order upwind finite differences,
    scaled by h^2 (h = 1/(n+1)), w(x, y) = Pe (cos 2 pi y, sin 2 pi x) at the
    node.  west = -1 - h max(w_x,0), east = -1 + h min(w_x,0), likewise
    south/north with w_y, diagonal 4 + h|w_x| + h|w_y|.  Nonsymmetric
    M-matrix with a symmetric pattern."""
    h = 1.0 / (n + 1)
    ii = np.arange(n * n) % n
    jj = np.arange(n * n) // n
    x = (ii + 1) * h
    y = (jj + 1) * h
    wx = peclet * np.cos(2 * np.pi * y)
    wy = peclet * np.sin(2 * np.pi * x)
    south = -1.0 - h * np.maximum(wy, 0.0)
    west = -1.0 - h * np.maximum(wx, 0.0)
    diag = 4.0 + h * np.abs(wx) + h * np.abs(wy)
    east = -1.0 + h * np.minimum(wx, 0.0)
    north = -1.0 + h * np.minimum(wy, 0.0)
    per = [south, west, diag, east, north]

    def coef(k, idx):
        return per[k]

    rp, ci, val = _grid_stencil((n, n), _OFF2, coef)
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, n * n)
    return System(f"convdiff2d_{n}_pe{peclet:g}", rp, ci, val, b, symmetric=False)


def fem_p1_jittered(n: int, seed: int = 0, jitter: float = 0.25) -> System:
    """P1 finite-element Laplacian on the unit square: (n+2)^2 vertices on a
    uniform grid, interior vertices moved by U[-jitter h, jitter h] in x and y,
    every cell split along its (i,j)-(i+1,j+1) diagonal, Dirichlet boundary
    vertices eliminated.  Seven-point pattern, like the P1 matrices of Table 1
    (about seven nonzeros per row).  b ~ U[-1,1] from the same generator."""
    rng = np.random.default_rng(seed)
    m = n + 2
    h = 1.0 / (n + 1)
    gx, gy = np.meshgrid(np.arange(m) * h, np.arange(m) * h, indexing="xy")
    px = gx.copy()
    py = gy.copy()
    jit = rng.uniform(-jitter * h, jitter * h, size=(2, n, n))
    px[1:-1, 1:-1] += jit[0]
    py[1:-1, 1:-1] += jit[1]
    vid = np.arange(m * m).reshape(m, m)  # [y, x]
    v00 = vid[:-1, :-1].ravel(); v10 = vid[:-1, 1:].ravel()
    v01 = vid[1:, :-1].ravel(); v11 = vid[1:, 1:].ravel()
    tris = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    X = px.ravel()[tris]
    Y = py.ravel()[tris]
    # gradients of the barycentric functions: grad phi_i = (y_j - y_k, x_k - x_j) / (2 area)
    det = (X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0]) - (X[:, 2] - X[:, 0]) * (Y[:, 1] - Y[:, 0])
    area = 0.5 * det
    assert np.all(area > 0), "jitter produced an inverted triangle"
    gxs = np.stack([Y[:, 1] - Y[:, 2], Y[:, 2] - Y[:, 0], Y[:, 0] - Y[:, 1]], 1) / det[:, None]
    gys = np.stack([X[:, 2] - X[:, 1], X[:, 0] - X[:, 2], X[:, 1] - X[:, 0]], 1) / det[:, None]
    K = (gxs[:, :, None] * gxs[:, None, :] + gys[:, :, None] * gys[:, None, :]) * area[:, None, None]
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    vals = K.ravel()
    # keep interior vertices only, renumbered lexicographically (x fastest)
    interior = np.full(m * m, -1, dtype=np.int64)
    iy, ix = np.meshgrid(np.arange(1, m - 1), np.arange(1, m - 1), indexing="ij")
    interior[vid[iy, ix].ravel()] = np.arange(n * n)
    r = interior[rows]
    c = interior[cols]
    keep = (r >= 0) & (c >= 0)
    r, c, vals = r[keep], c[keep], vals[keep]
    N = n * n
    key = r * N + c
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uk, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(vals, start)
    ur = uk // N
    uc = uk % N
    rp = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rp, ur + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    b = rng.uniform(-1.0, 1.0, N)
    return System(f"fem_p1_{n}_s{seed}", rp, uc.astype(np.int32), sums.astype(np.float64), b)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_poisson2d_64() -> System:
    """2D 5-point Poisson on a 64 x 64 interior grid (N = 4096), b ~ U[-1,1] seed 0."""
    return poisson2d(64, seed=0)


def config_lognormal3d_128() -> System:
    """3D 7-point lognormal(0,1) finite-volume diffusion on 128^3 cells (2.1M unknowns), seed 1."""
    return lognormal3d(128, seed=1)


def config_anisotropic3d_256() -> System:
    """3D 7-point anisotropic diffusion on 256^3 (16.8M unknowns), eps_z = 1e-3, seed 2."""
    return anisotropic3d(256, eps_z=1e-3, seed=2)


def config_convdiff2d_2048(peclet: float = 100.0) -> System:
    """2D upwind convection-diffusion on 2048^2 (4.2M unknowns), seed 3."""
    return convdiff2d(2048, peclet=peclet, seed=3)


@dataclass
class Request:
    """One solve request of the serving stream."""

    rid: int
    arrival_s: float
    family: str
    n_target: int
    seed: int

    def system(self) -> System:
        if self.family == "poisson2d":
            n = max(2, int(round(math.sqrt(self.n_target))))
            return poisson2d(n, seed=self.seed)
        if self.family == "lognormal3d":
            n = max(2, int(round(self.n_target ** (1.0 / 3.0))))
            return lognormal3d(n, seed=self.seed)
        if self.family == "fem_p1":
            n = max(2, int(round(math.sqrt(self.n_target))))
            return fem_p1_jittered(n, seed=self.seed)
        raise ValueError(self.family)


FAMILIES = ("poisson2d", "lognormal3d", "fem_p1")


def request_stream(count: int = 2048, rate_hz: float = 200.0, n_lo: float = 1e3, n_hi: float = 1e6,
                   seed: int = 4) -> list[Request]:
    """Serving stream: Poisson arrivals (exponential gaps of mean 1/rate), family
    uniform over the three SPD families, N = round(10^U[log10 n_lo, log10 n_hi]),
    per-request seed 1000 + r."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, count)
    arrivals = np.cumsum(gaps)
    fam = rng.integers(0, len(FAMILIES), count)
    ns = np.round(10.0 ** rng.uniform(math.log10(n_lo), math.log10(n_hi), count)).astype(np.int64)
    return [Request(r, float(arrivals[r]), FAMILIES[int(fam[r])], int(ns[r]), 1000 + r) for r in range(count)]


def worked_example() -> System:
    """The 6 x 6 matrix of the worked example in Sec. 2.1.1 (b = ones)."""
    a = np.array([
        [4, -2, 0, 0, 1, 0],
        [-2, 4, 1, 0, 0, 0],
        [0, 1, 4, 1, 2, 0],
        [0, 0, 1, 4, 0, 2],
        [1, 0, 2, 0, 4, 0],
        [0, 0, 0, 2, 0, 4],
    ], dtype=np.float64)
    return from_dense(a, np.ones(6), "worked_example")


def from_dense(a: np.ndarray, b: np.ndarray | None = None, name: str = "dense",
               keep_zeros: np.ndarray | None = None) -> System:
    """CSR of the nonzeros of a dense matrix (plus positions flagged in keep_zeros)."""
    a = np.asarray(a, dtype=np.float64)
    mask = a != 0
    if keep_zeros is not None:
        mask |= keep_zeros
    n = a.shape[0]
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = np.cumsum(mask.sum(1))
    rows, cols = np.nonzero(mask)
    return System(name, rp, cols.astype(np.int32), a[rows, cols].copy(),
                  np.ones(n) if b is None else np.asarray(b, dtype=np.float64),
                  symmetric=bool(np.allclose(a, a.T)))


def random_spd(n: int, density: float, seed: int, int_weights: bool = False) -> System:
    """Random sparse symmetric diagonally dominant matrix (SPD) with symmetric
    pattern.  int_weights draws off-diagonals from {-1,-2,-3} to force ties."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    pick = rng.random(len(iu[0])) < density
    if int_weights:
        w = -rng.integers(1, 4, pick.sum()).astype(np.float64)
    else:
        w = -rng.uniform(0.1, 1.0, pick.sum())
    a[iu[0][pick], iu[1][pick]] = w
    a = a + a.T
    a[np.diag_indices(n)] = np.abs(a).sum(1) + 1.0
    return from_dense(a, rng.uniform(-1, 1, n), f"random_spd_{n}_{seed}")
