"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
value printed in the paper, a closed form, an invariant, a textbook routine
(numpy dense algebra) or brute force on tiny inputs.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2007_00056_gb300 import workloads as W
from tests.conftest import read_golden


def _P(agg, nc):
    P = np.zeros((len(agg), nc))
    P[np.arange(len(agg)), agg] = 1.0
    return P


def _dense(rp, ci, val, n):
    a = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    a[rows, ci] = val
    return a


# --------------------------------------------------------------------------
# Sec. 2.1.1 worked example (printed A, P, A_c)
# --------------------------------------------------------------------------

def test_worked_example_matches_paper():
    g = read_golden("worked_example.txt")
    s = W.from_dense(g["A"])
    mate = O.match_greedy(s.rp, s.ci, s.val)
    agg, nc = O.aggregates(mate)
    assert nc == 3
    np.testing.assert_array_equal(_P(agg, nc), g["P"])
    rpc, cic, vc = O.galerkin(s.rp, s.ci, s.val, agg, nc)
    np.testing.assert_array_equal(_dense(rpc, cic, vc, nc), g["Ac"])
    # the handshake rounds reach the same pairs (one productive round + one empty round)
    mate_r, rounds = O.match_rounds(s.rp, s.ci, s.val)
    np.testing.assert_array_equal(mate_r, mate)
    assert rounds == 2
    # the paper's own Algorithm 2 (node-based) produces the printed P too
    agg_n, nc_n = O.nhem(s.rp, s.ci, s.val)
    np.testing.assert_array_equal(_P(agg_n, nc_n), g["P"])


def test_galerkin_diagonal_formula():
    """(A_c)_kk = a_ij + a_ji + a_ii + a_jj for a pair k = {i, j} (Sec. 2.1.1)."""
    for seed in range(5):
        s = W.random_spd(40, 0.15, seed)
        a = s.dense()
        a = a + np.triu(np.random.default_rng(seed).uniform(-0.1, 0.1, a.shape), 1) * (a != 0)
        s2 = W.from_dense(a)
        mate = O.match_greedy(s2.rp, s2.ci, s2.val)
        agg, nc = O.aggregates(mate)
        rpc, cic, vc = O.galerkin(s2.rp, s2.ci, s2.val, agg, nc)
        ac = _dense(rpc, cic, vc, nc)
        for i in range(s2.n):
            j = mate[i]
            if j > i:
                k = agg[i]
                assert ac[k, k] == pytest.approx(a[i, j] + a[j, i] + a[i, i] + a[j, j], rel=1e-15, abs=1e-15)
            elif j < 0:
                assert ac[agg[i], agg[i]] == a[i, i]


# --------------------------------------------------------------------------
# Galerkin product against dense P^T A P
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_galerkin_equals_dense_triple_product(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    mask = rng.random((n, n)) < 0.2
    np.fill_diagonal(mask, True)
    a = np.where(mask, rng.standard_normal((n, n)), 0.0)
    # plant explicit zeros that must survive as structural entries
    zeros = mask & (rng.random((n, n)) < 0.1)
    a[zeros] = 0.0
    s = W.from_dense(a, keep_zeros=mask)
    nc = int(rng.integers(1, n + 1))
    agg = np.concatenate([np.arange(nc), rng.integers(0, nc, n - nc)]).astype(np.int32)
    rng.shuffle(agg)
    # renumber so that aggregate ids follow the smallest member (any map works for P^T A P)
    rpc, cic, vc = O.galerkin(s.rp, s.ci, s.val, agg, nc)
    P = _P(agg, nc)
    np.testing.assert_allclose(_dense(rpc, cic, vc, nc), P.T @ a @ P, rtol=1e-13, atol=1e-13)
    # structural pattern: (I,J) stored iff some stored (i,j) maps to it
    pat = (P.T @ mask.astype(float) @ P) > 0
    got = np.zeros((nc, nc), dtype=bool)
    rows = np.repeat(np.arange(nc), np.diff(rpc))
    got[rows, cic] = True
    np.testing.assert_array_equal(got, pat)
    # columns strictly ascending per row
    for I in range(nc):
        assert np.all(np.diff(cic[rpc[I]:rpc[I + 1]]) > 0)


def test_galerkin_symmetric_stays_exactly_symmetric():
    for seed in range(4):
        s = W.random_spd(80, 0.08, seed)
        mate = O.match_greedy(s.rp, s.ci, s.val)
        agg, nc = O.aggregates(mate)
        rpc, cic, vc = O.galerkin(s.rp, s.ci, s.val, agg, nc)
        ac = _dense(rpc, cic, vc, nc)
        np.testing.assert_array_equal(ac, ac.T)


# --------------------------------------------------------------------------
# Matching: brute force, invariants, handshake rounds
# --------------------------------------------------------------------------

def _edges(a):
    n = a.shape[0]
    E = {}
    for i in range(n):
        for j in range(n):
            if i != j and a[i, j] != 0:
                u, v = min(i, j), max(i, j)
                E[(u, v)] = max(E.get((u, v), 0.0), abs(a[i, j]))
    return E


def _bruteforce_greedy(a):
    """Lexicographically first maximal matching in the edge order (w desc,
    min asc, max asc), found by enumerating every matching."""
    E = _edges(a)
    order = sorted(E, key=lambda e: (-E[e], e[0], e[1]))
    rank = {e: r for r, e in enumerate(order)}
    n = a.shape[0]
    best = None
    edges = list(E)
    for k in range(0, n // 2 + 1):
        for combo in itertools.combinations(edges, k):
            used = set()
            ok = True
            for u, v in combo:
                if u in used or v in used:
                    ok = False
                    break
                used.add(u); used.add(v)
            if not ok:
                continue
            if any(u not in used and v not in used for u, v in edges):
                continue  # not maximal
            key = sorted(rank[e] for e in combo)
            if best is None or key < best[0]:
                best = (key, combo)
    mate = -np.ones(n, dtype=np.int32)
    for u, v in best[1]:
        mate[u], mate[v] = v, u
    return mate


@pytest.mark.parametrize("seed", range(40))
def test_greedy_matching_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 9))
    mask = np.triu(rng.random((n, n)) < 0.5, 1)
    w = -rng.integers(1, 3, (n, n)).astype(float)  # ties on purpose
    a = np.where(mask, w, 0.0)
    if seed % 2:  # nonsymmetric values on a symmetric pattern
        a = a + np.where(mask, -rng.integers(1, 3, (n, n)), 0.0).T
    else:
        a = a + a.T
    a[np.diag_indices(n)] = 10.0
    s = W.from_dense(a)
    np.testing.assert_array_equal(O.match_greedy(s.rp, s.ci, s.val), _bruteforce_greedy(a))


@pytest.mark.parametrize("seed", range(60))
def test_handshake_rounds_reach_greedy_matching(seed):
    """Synchronous mutual-heaviest handshakes, run to the fixed point, give the
    greedy edge-order matching (locally dominant edges are greedy edges)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 80))
    s = W.random_spd(n, float(rng.uniform(0.05, 0.4)), seed, int_weights=bool(seed % 3))
    mate_g = O.match_greedy(s.rp, s.ci, s.val)
    mate_r, rounds = O.match_rounds(s.rp, s.ci, s.val)
    np.testing.assert_array_equal(mate_r, mate_g)
    assert rounds >= 1


def test_matching_is_maximal_and_consistent():
    for seed in range(10):
        s = W.random_spd(100, 0.05, seed, int_weights=True)
        mate = O.match_greedy(s.rp, s.ci, s.val)
        a = s.dense()
        for i in range(s.n):
            if mate[i] >= 0:
                assert mate[mate[i]] == i and a[i, mate[i]] != 0
        for (u, v) in _edges(a):
            assert mate[u] >= 0 or mate[v] >= 0, "an edge with both ends free remains"


def test_numbering_invariance_distinct_weights():
    """EHEM is invariant to the numbering when the weights are distinct (Sec. 2.1.2)."""
    for seed in range(5):
        s = W.random_spd(60, 0.1, seed)
        a = s.dense()
        perm = np.random.default_rng(seed).permutation(s.n)
        ap = a[np.ix_(perm, perm)]  # new index k is old node perm[k]
        sp = W.from_dense(ap)
        m0 = O.match_greedy(s.rp, s.ci, s.val)
        m1 = O.match_greedy(sp.rp, sp.ci, sp.val)
        inv = np.argsort(perm)
        for k in range(s.n):
            old = perm[k]
            if m0[old] < 0:
                assert m1[k] < 0
            else:
                assert m1[k] == inv[m0[old]]


def test_aggregates_partition_and_numbering():
    s = W.random_spd(200, 0.03, 7, int_weights=True)
    mate = O.match_greedy(s.rp, s.ci, s.val)
    agg, nc = O.aggregates(mate)
    assert agg.min() == 0 and agg.max() == nc - 1
    counts = np.bincount(agg, minlength=nc)
    assert np.all((counts >= 1) & (counts <= 2))  # pairs or singletons
    assert nc >= s.n / 2  # coarsening ratio slightly below two per pass
    # aggregate id = rank of the smallest member
    first = np.array([np.min(np.nonzero(agg == I)[0]) for I in range(nc)])
    assert np.all(np.diff(first) > 0)


# --------------------------------------------------------------------------
# Hierarchy shapes
# --------------------------------------------------------------------------

def test_uniform_grid_hierarchy_quarters_each_level():
    s = W.poisson2d(64)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=64)
    assert h.sizes() == [4096, 1024, 256, 64]
    s = W.anisotropic3d(16)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=64)
    assert h.sizes() == [4096, 1024, 256, 64]


def test_hierarchy_levels_are_galerkin_products():
    s = W.lognormal3d(10, seed=3)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=50)
    assert h.num_levels >= 3
    for k in range(h.num_levels - 1):
        rp, ci, val, agg = h.level(k)
        rpc, cic, vc, _ = h.level(k + 1)
        n, nc = len(rp) - 1, len(rpc) - 1
        counts = np.bincount(agg, minlength=nc)
        assert counts.min() >= 1 and counts.max() <= 4  # two pairwise passes
        P = _P(agg, nc)
        np.testing.assert_allclose(_dense(rpc, cic, vc, nc), P.T @ _dense(rp, ci, val, n) @ P,
                                   rtol=1e-12, atol=1e-12)


def _two_pass_level_sizes(s, levels):
    """Sizes of the candidate levels of s built from the pinned building blocks
    (greedy matching, numbering by smallest member, Galerkin product), two
    pairwise passes per level, without any stop rule."""
    rp, ci, val = s.rp, s.ci, s.val
    sizes = [len(rp) - 1]
    for _ in range(levels):
        for _ in range(2):
            agg, nc = O.aggregates(O.match_greedy(rp, ci, val))
            rp, ci, val = O.galerkin(rp, ci, val, agg, nc)
        sizes.append(len(rp) - 1)
    return sizes


def test_hierarchy_stops_before_a_stalled_level():
    """Reading of Table 2's level rule: a level is not added when its size
    ratio N_{k+1}/N_k to the level above exceeds stall_ratio.  On a lognormal
    8^3 system the hub-star stall sets in after four levels (ratios 0.31, 0.38,
    0.57, 0.77, then 0.89): with coarse_max = 1 and 30 allowed levels, only the
    stall can stop the hierarchy, and it must stop exactly there.  A ratio
    equal to stall_ratio does not stop it (the rule is a strict >)."""
    s = W.lognormal3d(8, seed=1)
    cand = _two_pass_level_sizes(s, 8)
    ratios = [cand[k + 1] / cand[k] for k in range(len(cand) - 1)]
    first_stall = next(k for k, r in enumerate(ratios) if r > 0.85)
    assert first_stall >= 3  # the stall is measured against the level above, not the finest
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=1, max_levels=30, stall_ratio=0.85)
    assert h.sizes() == cand[:first_stall + 1]
    # stall_ratio equal to the ratio of the last kept level: that level stays
    eq = ratios[first_stall - 1]
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=1, max_levels=30, stall_ratio=eq)
    assert h.sizes() == cand[:first_stall + 1]
    # just below it: that level is the first stalled one and is not added
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=1, max_levels=30, stall_ratio=np.nextafter(eq, 0.0))
    assert h.sizes() == cand[:first_stall]


def _path(m):
    a = np.diag([2.0] * m) + np.diag([-1.0] * (m - 1), 1) + np.diag([-1.0] * (m - 1), -1)
    return W.from_dense(a)


def test_node_based_matching_scans_both_ways_by_hand():
    """Algorithm 2 on a 5-node path with equal weights, worked by hand.  From
    the first index: 0 takes 1, 2 takes 3 (1 is taken), 4 stays single; ids in
    visit order.  From the last index (the alternate direction of Sec. 2.1.1):
    4 takes 3, 2 takes 1, 0 stays single, ids again in visit order.  A node
    with two equally heavy free neighbours keeps the last one in stored order
    (Algorithm 2's max(k, |a_ij|) = |a_ij| test)."""
    s = _path(5)
    agg, nc = O.nhem(s.rp, s.ci, s.val)
    assert nc == 3 and agg.tolist() == [0, 0, 1, 1, 2]
    agg, nc = O.nhem(s.rp, s.ci, s.val, descending=True)
    assert nc == 3 and agg.tolist() == [2, 1, 1, 0, 0]
    # a 3-node path: from the first index 0 takes 1; from the last, 2 takes 1
    p3 = _path(3)
    assert O.nhem(p3.rp, p3.ci, p3.val)[0].tolist() == [0, 0, 1]
    assert O.nhem(p3.rp, p3.ci, p3.val, descending=True)[0].tolist() == [1, 0, 0]
    # node 0 with two equally heavy free neighbours 1 and 2 keeps the last (2)
    s3 = W.from_dense(np.array([[3.0, -1.0, -1.0], [-1.0, 2.0, 0.0], [-1.0, 0.0, 2.0]]))
    assert O.nhem(s3.rp, s3.ci, s3.val)[0].tolist() == [0, 1, 0]


@pytest.mark.parametrize("seed", range(10))
def test_node_based_matching_is_maximal_both_ways(seed):
    s = W.random_spd(40, 0.15, seed, int_weights=True)
    a = s.dense()
    for desc in (False, True):
        agg, nc = O.nhem(s.rp, s.ci, s.val, descending=desc)
        sizes = np.bincount(agg, minlength=nc)
        assert sizes.min() >= 1 and sizes.max() <= 2
        single = np.flatnonzero(sizes[agg] == 1)
        for i in single:  # no edge joins two singletons
            for j in single:
                assert i == j or a[i, j] == 0.0


def test_alternating_node_based_hierarchy():
    """matcher = 2: pass p of the hierarchy (counted over all levels) scans from
    the first index when p is even and from the last when p is odd; every
    level is the Galerkin product of its composed aggregates."""
    s = W.lognormal3d(10, seed=5)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=30, matcher=2)
    assert h.num_levels >= 3
    rp, ci, val = s.rp, s.ci, s.val
    p = 0
    for k in range(h.num_levels - 1):
        n = len(rp) - 1
        comp = np.arange(n)
        for _ in range(2):
            agg, nc = O.nhem(rp, ci, val, descending=(p % 2 == 1))
            comp = agg[comp]
            rp, ci, val = O.galerkin(rp, ci, val, agg, nc)
            p += 1
        _, _, _, agg_h = h.level(k)
        np.testing.assert_array_equal(agg_h, comp)
        rpc, cic, vc, _ = h.level(k + 1)
        np.testing.assert_array_equal(rpc, rp)
        np.testing.assert_array_equal(cic, ci)
        np.testing.assert_array_equal(vc, val)


# --------------------------------------------------------------------------
# Coarse solve, V-cycle, Krylov
# --------------------------------------------------------------------------

def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 17, 40):
        a = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal(n)
        np.testing.assert_allclose(O.dense_solve(a, b), np.linalg.solve(a, b), rtol=1e-12, atol=1e-12)
    # pivoting is needed: zero leading entry
    a = np.array([[0.0, 1.0], [2.0, 3.0]])
    np.testing.assert_allclose(O.dense_solve(a, np.array([1.0, 5.0])), [1.0, 1.0])


def _block2x2(nblocks, a_, b_):
    blk = np.array([[a_, -b_], [-b_, a_]])
    return np.kron(np.eye(nblocks), blk)


def test_vcycle_closed_form_on_2x2_blocks():
    """Two-grid cycle on blockdiag([[a,-b],[-b,a]]): each block is one aggregate.
    Smooth rhs (1,1) is solved exactly: the presmoothed guess w f/a plus the
    coarse correction (1 - w(a-b)/a)/(a-b) gives 1/(a-b).  Oscillatory rhs
    (1,-1) restricts to zero, so the result is two Jacobi steps:
    w/a + (w/a)(1 - w(a+b)/a); for a=4, b=1, w=2/3 that is 7/36."""
    a_, b_ = 4.0, 1.0
    s = W.from_dense(_block2x2(8, a_, b_))
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=8)
    assert h.sizes() == [16, 8]
    smooth = np.ones(16)
    np.testing.assert_allclose(h.vcycle(smooth), smooth / (a_ - b_), rtol=1e-15)
    osc = np.tile([1.0, -1.0], 8)
    np.testing.assert_allclose(h.vcycle(osc), osc * 7.0 / 36.0, rtol=1e-15)


def test_single_level_vcycle_is_exact_solve():
    s = W.random_spd(30, 0.2, 1)
    h = O.Hierarchy(s.rp, s.ci, s.val)  # N <= coarse_max: coarsest level only
    assert h.num_levels == 1 and h.dense_coarse
    np.testing.assert_allclose(h.vcycle(s.b), np.linalg.solve(s.dense(), s.b), rtol=1e-12)


def _vcycle_matrix(h, n):
    return np.column_stack([h.vcycle(e) for e in np.eye(n)])


def test_vcycle_operator_symmetric_and_contracting():
    """With identical pre/post Jacobi sweeps and an exact coarse solve, M^{-1}
    is symmetric for symmetric A and the error propagator I - M^{-1} A has
    spectral radius below one (two-grid and multi-level)."""
    s = W.poisson2d(16)
    for coarse_max, levels in ((64, 2), (16, 3)):
        h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=coarse_max)
        assert h.num_levels == levels
        M = _vcycle_matrix(h, s.n)
        np.testing.assert_allclose(M, M.T, atol=1e-13)
        E = np.eye(s.n) - M @ s.dense()
        rho = np.max(np.abs(np.linalg.eigvals(E)))
        assert rho < 1.0
    s = W.lognormal3d(6, seed=5)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=20)
    E = np.eye(s.n) - _vcycle_matrix(h, s.n) @ s.dense()
    assert np.max(np.abs(np.linalg.eigvals(E))) < 1.0


def test_residual_operator_form_equals_algorithm_1():
    """The device evaluates a zero-guess visit of level k (one pre- and one
    post-sweep) as t = C f and y = Q x_c + omega D^-1 (f + t), with
    C = I - omega A D^-1 and Q = P - omega D^-1 A P formed at setup.  Expanding
    Algorithm 1: x1 = omega D^-1 f, t = f - A x1 = C f, f_c = P^T t,
    x2 = x1 + P x_c and y = x2 + omega D^-1 (f - A x2) = Q x_c + omega D^-1 (f + t).
    The rewritten recursion, built from the oracle's own levels, gives the
    oracle's V-cycle on symmetric and nonsymmetric hierarchies of three or
    more levels."""
    omega = 2.0 / 3.0
    for s, cm in ((W.poisson2d(12), 16), (W.lognormal3d(6, seed=3), 16), (W.convdiff2d(12, peclet=50.0), 10)):
        oh = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=cm)
        L = oh.num_levels
        assert L >= 3 and oh.dense_coarse
        lev = [oh.level(k) for k in range(L)]
        A = [_dense(rp, ci, val, len(rp) - 1) for rp, ci, val, _ in lev]
        P = [_P(lev[k][3], A[k + 1].shape[0]) for k in range(L - 1)]

        def op_cycle(k, f, q_sign=-1.0):
            if k == L - 1:
                return np.linalg.solve(A[k], f)
            dinv = 1.0 / np.diag(A[k])
            C = np.eye(len(f)) - omega * A[k] * dinv[None, :]
            Q = P[k] + q_sign * (omega * dinv)[:, None] * (A[k] @ P[k])
            t = C @ f
            x_c = op_cycle(k + 1, P[k].T @ t, q_sign)
            return Q @ x_c + omega * dinv * (f + t)

        f = np.random.default_rng(5).uniform(-1.0, 1.0, s.n)
        z = oh.vcycle(f)
        assert np.linalg.norm(op_cycle(0, f) - z) <= 1e-12 * np.linalg.norm(z)
        # the check sees a planted mistake (Q with its second term's sign flipped)
        assert np.linalg.norm(op_cycle(0, f, q_sign=1.0) - z) > 1e-3 * np.linalg.norm(z)


def test_coarse_cg_solver_agrees_with_dense():
    s = W.lognormal3d(8, seed=2)
    hd = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=60, coarse_solver=1)
    hc = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=60, coarse_solver=2)
    assert hd.dense_coarse and not hc.dense_coarse
    np.testing.assert_allclose(hc.vcycle(s.b), hd.vcycle(s.b), rtol=1e-9, atol=1e-12)
    # conjugate gradients end within n_L steps (finite termination), far below the cap
    n_coarse = hc.sizes()[-1]
    assert 1 <= hc.last_coarse_cg_iters <= n_coarse
    s = W.lognormal3d(12, seed=2)
    hc = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=400, coarse_solver=2)
    hd = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=400, coarse_solver=1)
    np.testing.assert_allclose(hc.vcycle(s.b), hd.vcycle(s.b), rtol=1e-9, atol=1e-12)
    assert 1 <= hc.last_coarse_cg_iters <= hc.sizes()[-1] // 4


@pytest.mark.parametrize("seed", range(6))
def test_pcg_tiny_spd_converges_within_n_steps(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 30))
    s = W.random_spd(n, 0.3, seed)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=3)
    x, info = h.pcg(s.b, rtol=1e-12, max_iter=n)
    assert info.status == O.OK and info.iterations <= n
    np.testing.assert_allclose(x, np.linalg.solve(s.dense(), s.b), rtol=1e-9, atol=1e-11)


def test_pcg_matches_dense_solve_to_1e10():
    s = W.lognormal3d(9, seed=4)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=40)
    x_ref = np.linalg.solve(s.dense(), s.b)
    for flexible in (False, True):
        x, info = h.pcg(s.b, rtol=1e-14, max_iter=200, flexible=flexible)
        assert info.status == O.OK
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10
        assert info.rel_res_true < 1e-13


def test_pcg_rtol_and_recurrence_residual():
    s = W.poisson2d(32)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=16)
    x, info = h.pcg(s.b, rtol=1e-8)
    assert info.status == O.OK and info.rel_res_recurrence <= 1e-8
    r = s.b - s.dense() @ x
    assert np.linalg.norm(r) / np.linalg.norm(s.b) == pytest.approx(info.rel_res_true, rel=1e-6)
    # one iteration fewer does not meet the tolerance
    _, info2 = h.pcg(s.b, rtol=0.0, max_iter=info.iterations - 1)
    assert info2.rel_res_recurrence > 1e-8


def test_pcg_edge_cases():
    s = W.poisson2d(8)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=4)
    x, info = h.pcg(np.zeros(s.n))
    assert info.iterations == 0 and np.all(x == 0)
    x_ref = np.linalg.solve(s.dense(), s.b)
    x, info = h.pcg(s.b, x0=x_ref)  # already converged start
    assert info.iterations == 0
    x, info = h.pcg(s.b, rtol=1e-30, max_iter=3)
    assert info.status == O.ERR_NOT_CONVERGED and info.iterations == 3


def test_bicgstab_nonsymmetric_matches_dense():
    s = W.convdiff2d(14, peclet=200.0)
    assert not np.allclose(s.dense(), s.dense().T)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=20)
    x, info = h.bicgstab(s.b, rtol=1e-13, max_iter=200)
    assert info.status == O.OK
    x_ref = np.linalg.solve(s.dense(), s.b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10
    assert info.rel_res_true < 1e-12


def test_bicgstab_spd_and_exact_preconditioner():
    s = W.random_spd(20, 0.3, 3)
    h = O.Hierarchy(s.rp, s.ci, s.val)  # single level: M^{-1} = A^{-1}
    x, info = h.bicgstab(s.b, rtol=1e-12)
    # with an exact preconditioner the first half step already solves the system
    assert info.iterations == 1 and info.status == O.OK
    np.testing.assert_allclose(x, np.linalg.solve(s.dense(), s.b), rtol=1e-11)


def _bicgstab_breakdown_system():
    """Two copies of [[1, 3], [3, 1]] (eigenvalues 4 and -2), omega = 1 and a
    coarsest level of 2 rows: pairs {0,1} and {2,3}, A_c = diag(8, 8).  Every
    step of the V-cycle is exact in binary.  Worked by hand from Algorithm 1:
    A M^-1 = I on the pair-constant vectors and -8 I on the pair-alternating
    ones.  For b = 2 (1,1,0,0) + (1,-1,0,0) + 2 (0,0,1,1) = (3, 1, 2, 2),
    (A M^-1 b, b) = 2 (4 - 8 + 4) = 0 exactly."""
    a = np.kron(np.eye(2), np.array([[1.0, 3.0], [3.0, 1.0]]))
    return a, np.array([3.0, 1.0, 2.0, 2.0])


def test_bicgstab_breakdown_when_the_first_direction_meets_the_shadow_residual_at_zero():
    """R11's breakdown rule: with r_0 = rbar_0 = b and p~ = M^-1 b, the first
    step divides by (A p~, rbar_0); when that is 0 the solve stops with
    ERR_BREAKDOWN and leaves x at the initial guess.  A b whose product is not
    0 (the last entry changed) converges instead."""
    a, b = _bicgstab_breakdown_system()
    s = W.from_dense(a, b)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=2, omega=1.0)
    assert h.sizes() == [4, 2] and h.dense_coarse
    z = h.vcycle(b)
    np.testing.assert_array_equal(z, [4.5, -3.5, 0.5, 0.5])  # Algorithm 1 by hand
    assert (a @ z) @ b == 0.0
    x, info = h.bicgstab(b, rtol=1e-10)
    assert info.status == O.ERR_BREAKDOWN and not np.any(x)
    b2 = np.array([3.0, 1.0, 2.0, 1.0])
    assert (a @ h.vcycle(b2)) @ b2 != 0.0
    x2, info2 = h.bicgstab(b2, rtol=1e-12)
    assert info2.status == O.OK
    np.testing.assert_allclose(x2, np.linalg.solve(a, b2), rtol=0, atol=1e-12)


def test_check_csr_rejects_bad_input():
    s = W.poisson2d(4)
    assert O.check_csr(s.rp, s.ci) == O.OK
    ci = s.ci.copy(); ci[3] = 99
    assert O.check_csr(s.rp, ci) == O.ERR_INVALID_CSR
    ci = s.ci.copy(); ci[1], ci[2] = ci[2], ci[1]
    assert O.check_csr(s.rp, ci) == O.ERR_INVALID_CSR


def test_krylov_finite_termination_two_eigenvalues():
    """On blockdiag([[4,-1],[-1,4]]) the two-grid preconditioned operator has
    exactly two eigenvalues (1 on the pair-constant vectors, 35/36 on the
    pair-alternating ones, from the closed form above), so PCG and BiCGStab
    reach rounding level within two iterations for any right-hand side."""
    s = W.from_dense(_block2x2(10, 4.0, 1.0))
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=10)
    b = np.random.default_rng(0).uniform(-1, 1, s.n)
    _, info = h.pcg(b, rtol=1e-13, max_iter=50)
    assert info.status == O.OK and info.iterations <= 2
    _, info = h.bicgstab(b, rtol=1e-13, max_iter=50)
    assert info.status == O.OK and info.iterations <= 2


@pytest.mark.parametrize("coarse_solver", [1, 2])
def test_flexible_beta_keeps_consecutive_directions_a_conjugate(coarse_solver):
    """Flexible CG (reading R-C9): beta = (z_{j+1}, r_{j+1} - r_j)/(z_j, r_j).
    With r_{j+1} - r_j = -alpha A p_j and alpha = (r_j, z_j)/(p_j, A p_j) this
    beta equals -(z_{j+1}, A p_j)/(p_j, A p_j), so p_{j+1} = z_{j+1} + beta p_j
    is A-conjugate to p_j for ANY preconditioner.  The F-cycle is a fixed but
    nonsymmetric M^{-1} (pinned below), where the Fletcher-Reeves beta loses
    that property; the check therefore tells the two formulas apart."""
    s = W.lognormal3d(12, seed=3)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=100, cycle=2, coarse_solver=coarse_solver)
    a = s.dense()

    def worst(P):
        out = 0.0
        for j in range(len(P) - 1):
            ap = a @ P[j]
            out = max(out, abs(P[j + 1] @ ap) / np.sqrt((P[j + 1] @ (a @ P[j + 1])) * (P[j] @ ap)))
        return out

    x, info, P = h.pcg_directions(s.b, rtol=1e-10, max_iter=60, flexible=True)
    assert info.status == O.OK and len(P) >= 10
    assert worst(P) < 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(a, s.b), rtol=1e-8, atol=1e-10)
    # the same check on Fletcher-Reeves directions fails by orders of magnitude
    _, _, P_fr = h.pcg_directions(s.b, rtol=1e-10, max_iter=60, flexible=False)
    assert worst(P_fr) > 1e-6


def test_coarse_cg_finite_termination_two_eigenvalues():
    """A one-level hierarchy with the CG coarse solver: the V-cycle is a
    Jacobi-PCG solve of A z = r.  On blockdiag([[a,-b],[-b,a]]) the operator
    D^-1 A has exactly two eigenvalues, (a - b)/a and (a + b)/a, so CG ends
    within two iterations and returns A^{-1} r."""
    a = np.kron(np.eye(30), np.array([[4.0, -1.0], [-1.0, 4.0]]))
    s = W.from_dense(a, np.random.default_rng(2).uniform(-1, 1, 60))
    h = O.Hierarchy(s.rp, s.ci, s.val, max_levels=1, coarse_solver=2)
    z = h.vcycle(s.b)
    assert h.last_coarse_cg_iters <= 2
    np.testing.assert_allclose(z, np.linalg.solve(a, s.b), rtol=1e-12)


# --------------------------------------------------------------------------
# W- and F-cycles (Sec. 2 names V, W and F) and AMG as a solver (Sec. 3.1)
# --------------------------------------------------------------------------

def _levels_dense(h):
    """Dense A_k and P_k of an oracle hierarchy (the setup is pinned above)."""
    As, Ps = [], []
    for k in range(h.num_levels):
        rp, ci, val, agg = h.level(k)
        n = len(rp) - 1
        As.append(_dense(rp, ci, val, n))
        if agg is not None:
            Ps.append(_P(agg, h.level_info(k + 1)[0]))
    return As, Ps


def _error_propagators(As, Ps, omega=2.0 / 3.0, nu_pre=1, nu_post=1):
    """Textbook multigrid recursion of the error propagator of one cycle at
    level k: E_k = S_k^nu_post (I - P_k C_{k+1} P_k^T A_k) S_k^nu_pre with
    S_k = I - omega D_k^{-1} A_k and C_{k+1} the coarse approximate inverse:
    A_L^{-1} at the coarsest level, else (I - E_{k+1}) A_{k+1}^{-1} (V),
    (I - E_{k+1}^2) A_{k+1}^{-1} (W: two cycles, the second from the first's
    result) or (I - E^V_{k+1} E^F_{k+1}) A_{k+1}^{-1} (F: an F-cycle, then a
    V-cycle).  Returns {kind: E_0} for kind 0 (V), 1 (W), 2 (F)."""
    L = len(As) - 1
    E = {0: [None] * (L + 1), 1: [None] * (L + 1), 2: [None] * (L + 1)}
    for k in range(L - 1, -1, -1):
        A = As[k]
        n = A.shape[0]
        S = np.eye(n) - omega * A / np.diag(A)[:, None]
        Ac_inv = np.linalg.inv(As[k + 1])
        for kind in (0, 1, 2):
            if k + 1 == L:
                C = Ac_inv
            elif kind == 0:
                C = (np.eye(len(Ac_inv)) - E[0][k + 1]) @ Ac_inv
            elif kind == 1:
                C = (np.eye(len(Ac_inv)) - E[1][k + 1] @ E[1][k + 1]) @ Ac_inv
            else:
                C = (np.eye(len(Ac_inv)) - E[0][k + 1] @ E[2][k + 1]) @ Ac_inv
            P = Ps[k]
            E[kind][k] = (np.linalg.matrix_power(S, nu_post) @ (np.eye(n) - P @ C @ P.T @ A)
                          @ np.linalg.matrix_power(S, nu_pre))
    return {kind: E[kind][0] for kind in (0, 1, 2)}


_CYCLE_SYSTEMS = [
    ("poisson2d_16_four_levels", lambda: W.poisson2d(16), 4),
    ("lognormal3d_6", lambda: W.lognormal3d(6, seed=5), 8),
    ("convdiff2d_14_nonsymmetric", lambda: W.convdiff2d(14, peclet=200.0), 6),
]


@pytest.mark.parametrize("name,make,coarse_max", _CYCLE_SYSTEMS, ids=[c[0] for c in _CYCLE_SYSTEMS])
def test_cycles_match_error_propagation_recursion(name, make, coarse_max):
    """M^{-1} of each cycle kind equals (I - E_0) A^{-1} of the textbook
    recursion; needs at least four levels so that W and F differ."""
    s = make()
    A = s.dense()
    Ms = {}
    for kind in (0, 1, 2):
        h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=coarse_max, cycle=kind)
        assert h.num_levels >= 4, h.sizes()
        Ms[kind] = np.column_stack([h.vcycle(e) for e in np.eye(s.n)])
    As, Ps = _levels_dense(h)
    Es = _error_propagators(As, Ps)
    Ainv = np.linalg.inv(A)
    for kind in (0, 1, 2):
        want = (np.eye(s.n) - Es[kind]) @ Ainv
        assert np.max(np.abs(Ms[kind] - want)) <= 1e-11 * np.max(np.abs(want)), kind
    # the three kinds are different operators here
    assert np.max(np.abs(Ms[1] - Ms[0])) > 1e-6 and np.max(np.abs(Ms[2] - Ms[1])) > 1e-6


def test_cycle_kinds_coincide_on_two_and_three_levels():
    """With two levels every kind is one exact coarse solve; with three the
    level-1 cycles of W and F both end in the exact solve, so W = F (bitwise),
    while W differs from V by the second level-1 cycle."""
    s = W.poisson2d(16)
    for coarse_max, levels in ((64, 2), (16, 3)):
        z = {}
        for kind in (0, 1, 2):
            h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=coarse_max, cycle=kind)
            assert h.num_levels == levels
            z[kind] = h.vcycle(s.b)
        assert np.array_equal(z[1], z[2])
        if levels == 2:
            assert np.array_equal(z[0], z[1])
        else:
            assert not np.array_equal(z[0], z[1])


def test_w_cycle_symmetric_f_cycle_not():
    """Same pre/post smoothing and an exact coarsest solve keep the W-cycle's
    M^{-1} symmetric for symmetric A; the F-cycle's coarse correction (an F-
    then a V-cycle) is not symmetric, which is why it needs flexible PCG."""
    s = W.poisson2d(16)
    M = {}
    for kind in (1, 2):
        h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=4, cycle=kind)
        M[kind] = np.column_stack([h.vcycle(e) for e in np.eye(s.n)])
    assert np.max(np.abs(M[1] - M[1].T)) < 1e-13
    assert np.max(np.abs(M[2] - M[2].T)) > 1e-8


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_amg_solver_iterates_closed_form(kind):
    """AMG as a solver from x_0 = 0: the error after j cycles is E^j x*, so
    x_j = (I - E^j) A^{-1} b; the iteration count is the first j whose true
    residual meets the tolerance."""
    s = W.lognormal3d(6, seed=5)
    A = s.dense()
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=8, cycle=kind)
    E = _error_propagators(*_levels_dense(h))[kind]
    xs = np.linalg.solve(A, s.b)
    for j in (1, 2, 5):
        x, info = h.amg_solve(s.b, rtol=0.0, max_iter=j)
        assert info.iterations == j and info.status == O.ERR_NOT_CONVERGED
        want = xs - np.linalg.matrix_power(E, j) @ xs
        assert np.linalg.norm(x - want) <= 1e-11 * np.linalg.norm(xs)
    rtol = 1e-8
    bn = np.linalg.norm(s.b)
    Ej = np.eye(s.n)
    for j in range(1, 200):
        Ej = E @ Ej
        rel = np.linalg.norm(s.b - A @ (xs - Ej @ xs)) / bn
        if rel <= rtol:
            break
    assert abs(rel / rtol - 1.0) > 1e-3  # not a borderline count
    x, info = h.amg_solve(s.b, rtol=rtol)
    assert info.status == O.OK and info.iterations == j
    assert info.rel_res_true <= rtol


def test_amg_solver_edge_cases():
    s = W.poisson2d(12)
    h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=16)
    x, info = h.amg_solve(np.zeros(s.n), x0=np.ones(s.n))
    assert info.iterations == 0 and info.status == O.OK and not np.any(x)
    xs = np.linalg.solve(s.dense(), s.b)
    x, info = h.amg_solve(s.b, x0=xs, rtol=1e-8)
    assert info.iterations == 0 and info.status == O.OK and np.array_equal(x, xs)
    x, info = h.amg_solve(s.b, rtol=1e-8, max_iter=0)
    assert info.iterations == 0 and info.status == O.ERR_NOT_CONVERGED and not np.any(x)
    # a stationary iteration converges linearly: residuals fall every cycle
    rels = [h.amg_solve(s.b, rtol=0.0, max_iter=j)[1].rel_res_true for j in range(1, 8)]
    assert all(b < a for a, b in zip(rels, rels[1:]))


# --------------------------------------------------------------------------
# Matching options: Algorithm 3's own tie order, diagonally scaled weights
# --------------------------------------------------------------------------

def _bruteforce_greedy_key(a, key, weight=None):
    """Lexicographically first maximal matching in the edge order `key`
    (enumerating every matching); weight(i, j, a_ij) replaces |a_ij|."""
    n = a.shape[0]
    E = {}
    for i in range(n):
        for j in range(n):
            if i != j and a[i, j] != 0:
                u, v = min(i, j), max(i, j)
                w = abs(a[i, j]) if weight is None else weight(i, j, a[i, j])
                E[(u, v)] = max(E.get((u, v), 0.0), w)
    order = sorted(E, key=lambda e: key(E[e], e[0], e[1]))
    rank = {e: r for r, e in enumerate(order)}
    best = None
    edges = list(E)
    for k in range(0, n // 2 + 1):
        for combo in itertools.combinations(edges, k):
            ends = [x for e in combo for x in e]
            if len(set(ends)) < len(ends):
                continue
            used = set(ends)
            if any(u not in used and v not in used for u, v in edges):
                continue
            r = sorted(rank[e] for e in combo)
            if best is None or r < best[0]:
                best = (r, combo)
    mate = -np.ones(n, dtype=np.int32)
    for u, v in best[1]:
        mate[u], mate[v] = v, u
    return mate


def _tiny_tied(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 9))
    mask = np.triu(rng.random((n, n)) < 0.5, 1)
    a = np.where(mask, -rng.integers(1, 3, (n, n)).astype(float), 0.0)
    a = a + a.T
    a[np.diag_indices(n)] = rng.integers(4, 7, n).astype(float)
    return a


@pytest.mark.parametrize("seed", range(30))
def test_descending_tie_order_bruteforce(seed):
    """Algorithm 3 sorts its edge list lexicographically descending: equal
    weights go to the larger (max, then min) endpoint."""
    a = _tiny_tied(seed)
    s = W.from_dense(a)
    want = _bruteforce_greedy_key(a, lambda w, u, v: (-w, -v, -u))
    np.testing.assert_array_equal(O.match_greedy(s.rp, s.ci, s.val, tie_break=1), want)
    mate_r, _ = O.match_rounds(s.rp, s.ci, s.val, tie_break=1)
    np.testing.assert_array_equal(mate_r, want)


@pytest.mark.parametrize("seed", range(20))
def test_descending_tie_order_is_the_reversed_numbering(seed):
    """Renumbering i -> N-1-i turns the descending tie order into the default
    (smaller index) one, on graphs with many ties."""
    rng = np.random.default_rng(seed)
    s = W.random_spd(int(rng.integers(5, 120)), float(rng.uniform(0.05, 0.3)), seed, int_weights=True)
    a = s.dense()
    r = a[::-1, ::-1].copy()
    sr = W.from_dense(r)
    m_desc = O.match_greedy(s.rp, s.ci, s.val, tie_break=1)
    m_rev = O.match_greedy(sr.rp, sr.ci, sr.val)
    n = s.n
    back = np.where(m_rev[::-1] >= 0, n - 1 - m_rev[::-1], -1)
    np.testing.assert_array_equal(m_desc, back)
    mate_r, _ = O.match_rounds(s.rp, s.ci, s.val, tie_break=1)
    np.testing.assert_array_equal(mate_r, m_desc)


@pytest.mark.parametrize("seed", range(20))
def test_scaled_weight_bruteforce_and_invariance(seed):
    """Weight max(|a_ij|,|a_ji|)/sqrt(|a_ii a_jj|): brute force on tiny graphs;
    invariant under a symmetric positive diagonal scaling D A D; equal to the
    plain matching when the diagonal is constant."""
    a = _tiny_tied(seed)
    d = np.abs(np.diag(a))
    s = W.from_dense(a)
    want = _bruteforce_greedy_key(a, lambda w, u, v: (-w, u, v),
                                  weight=lambda i, j, x: abs(x) / np.sqrt(d[i] * d[j]))
    np.testing.assert_array_equal(O.match_greedy(s.rp, s.ci, s.val, edge_weight=1), want)
    np.testing.assert_array_equal(O.match_rounds(s.rp, s.ci, s.val, edge_weight=1)[0], want)
    rng = np.random.default_rng(seed)
    b = W.random_spd(int(rng.integers(5, 100)), 0.2, seed)  # real weights: no ties
    D = rng.uniform(0.5, 2.0, b.n)
    sc = W.from_dense(D[:, None] * b.dense() * D[None, :])
    np.testing.assert_array_equal(O.match_greedy(sc.rp, sc.ci, sc.val, edge_weight=1),
                                  O.match_greedy(b.rp, b.ci, b.val, edge_weight=1))
    p = W.poisson2d(9)  # constant diagonal 4
    np.testing.assert_array_equal(O.match_greedy(p.rp, p.ci, p.val, edge_weight=1),
                                  O.match_greedy(p.rp, p.ci, p.val))


def test_matching_options_reach_the_hierarchy():
    """The options change the aggregates of a tie-heavy grid (descending order)
    and of a lognormal system (scaled weights), and every level stays the
    Galerkin product of its aggregates."""
    s = W.poisson2d(11)  # odd rows: the two tie orders pair a row from opposite ends
    a0 = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=16).level(0)[3]
    a1 = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=16, tie_break=1).level(0)[3]
    assert not np.array_equal(a0, a1)
    s = W.lognormal3d(8, seed=2)
    for kw in (dict(tie_break=1), dict(edge_weight=1)):
        h = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=20, **kw)
        for k in range(h.num_levels - 1):
            rp, ci, val, agg = h.level(k)
            A = _dense(rp, ci, val, len(rp) - 1)
            P = _P(agg, h.level_info(k + 1)[0])
            rpc, cic, valc, _ = h.level(k + 1)
            np.testing.assert_allclose(_dense(rpc, cic, valc, P.shape[1]), P.T @ A @ P, rtol=1e-13, atol=1e-13)
    sizes_plain = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=20).sizes()
    sizes_scaled = O.Hierarchy(s.rp, s.ci, s.val, coarse_max=20, edge_weight=1).sizes()
    assert sizes_scaled != sizes_plain
