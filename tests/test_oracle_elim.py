"""Pins of the oracle's low-degree elimination (Sec. 3.2; option elim = 1).

Each pin checks the elimination levels against something other than the
oracle itself:
the dense Schur complement (numpy), the greedy independent set taken by its
definition, the series-conductance closed form on a path, exactness on trees,
the dense pseudo-inverse, and the paper's stated reason for elimination (grids
coarsen better after it).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _dense(g):
    return oracle.laplacian_dense(g.n, g.rp, g.col, g.w)


def _level_dense(h, l):
    rp, col, w = h.csr(l)
    return oracle.laplacian_dense(len(rp) - 1, rp, col, w)


def _elim_order(n, l, seed=1):
    # the sweep order of reading R20: decreasing splitmix64(key + u), ties to the
    # lower index; key = the level's colour key with the top bit set
    key = oracle.splitmix64(oracle.splitmix64(seed) ^ ((2 * l + 1) << 32) ^ (1 << 63))
    p = [oracle.splitmix64((key + u) & (2**64 - 1)) for u in range(n)]
    return sorted(range(n), key=lambda u: (-p[u], u))


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    u = list(perm[:-1]) + list(rng.integers(0, n, m))
    v = list(perm[1:]) + list(rng.integers(0, n, m))
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(lo[lo != hi].astype(np.int64) * n + hi[lo != hi])
    return W.from_edges(n, key // n, key % n, rng.uniform(0.5, 2.0, key.size), f"rand{n}")


GRAPHS = {
    "grid": lambda: W.grid2d(16, 14),
    "chung_lu": lambda: W.chung_lu(900, seed=41),
    "random": lambda: _random_graph(400, 300, 42),
}


@pytest.mark.parametrize("gname", list(GRAPHS))
def test_first_level_is_the_dense_schur_complement(gname):
    g = GRAPHS[gname]()
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    assert h.info(0)["elim"]
    cidx = h.elim(0)
    Fs, Cs = np.flatnonzero(cidx < 0), np.flatnonzero(cidx >= 0)
    assert np.array_equal(cidx[Cs], np.arange(Cs.size))          # C keeps the fine order
    A = _dense(g)
    S = A[np.ix_(Cs, Cs)] - A[np.ix_(Cs, Fs)] @ np.diag(1.0 / np.diag(A)[Fs]) @ A[np.ix_(Fs, Cs)]
    Ac = _level_dense(h, 1)
    assert np.max(np.abs(Ac - S)) <= 1e-13 * np.max(np.abs(S))    # Eq. (3.1)
    rp, col, w = h.csr(1)
    W1 = np.zeros_like(Ac)
    W1[np.repeat(np.arange(len(rp) - 1), np.diff(rp)), col] = w
    assert np.array_equal(W1, W1.T)                                # bit-symmetric coarse weights
    assert np.all(np.abs(Ac.sum(axis=1)) <= 1e-12 * np.abs(Ac).max())   # again a Laplacian


@pytest.mark.parametrize("gname", list(GRAPHS))
def test_eliminated_set_is_the_greedy_low_degree_independent_set(gname):
    g = GRAPHS[gname]()
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    for l in range(h.num_levels - 1):
        if not h.info(l)["elim"]:
            continue
        rp, col, _ = h.csr(l)
        deg = np.diff(rp)
        inF = h.elim(l) < 0
        # the sweep of Sec. 3.2 by its definition: in the sweep order, an eligible
        # node of degree 1..4 joins F and its neighbours become ineligible
        want = np.zeros(deg.size, bool)
        inel = np.zeros(deg.size, bool)
        for u in _elim_order(deg.size, l):
            if not inel[u] and 1 <= deg[u] <= 4:
                want[u] = True
                inel[col[rp[u]:rp[u + 1]]] = True
        assert np.array_equal(inF, want), l
        assert h.info(l)["nF"] == want.sum()
        for u in np.flatnonzero(inF):                                 # independent
            assert not inF[col[rp[u]:rp[u + 1]]].any()


def test_path_coarsens_by_series_conductance():
    # On a weighted path the coarse graph is again a path.  An eliminated interior
    # node f joins its two neighbours by the series conductance w1 w2 / (w1 + w2);
    # two neighbouring C nodes keep their edge; an eliminated end adds nothing.
    n = 400
    rng = np.random.default_rng(5)
    wt = rng.uniform(0.5, 2.0, n - 1)
    g = W.from_edges(n, np.arange(n - 1), np.arange(1, n), wt, "wpath")
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    cidx = h.elim(0)
    Cs = np.flatnonzero(cidx >= 0)
    rp, col, w = h.csr(1)
    assert len(rp) - 1 == Cs.size and np.all(np.diff(rp) <= 2)
    for k in range(Cs.size - 1):                   # coarse nodes k, k+1 = fine Cs[k] < Cs[k+1]
        a, b = Cs[k], Cs[k + 1]
        if b == a + 1:
            want = wt[a]
        else:
            assert b == a + 2 and cidx[a + 1] < 0  # exactly one eliminated node between
            want = wt[a] * wt[a + 1] / (wt[a] + wt[a + 1])
        e = rp[k] + np.searchsorted(col[rp[k]:rp[k + 1]], k + 1)
        assert col[e] == k + 1
        assert w[e] == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("tree", ["path", "random_tree", "caterpillar"])
def test_trees_are_solved_exactly_in_one_cycle(tree):
    rng = np.random.default_rng(6)
    if tree == "path":
        g = W.path(3000)
    elif tree == "random_tree":
        n = 3000
        parent = np.array([rng.integers(0, i) for i in range(1, n)])
        g = W.from_edges(n, parent, np.arange(1, n), rng.uniform(0.5, 2.0, n - 1), "tree")
    else:   # a spine with two legs per spine node (every node degree <= 4)
        s = 1000
        u = list(range(s - 1)) + list(range(s)) + list(range(s))
        v = list(range(1, s)) + list(range(s, 2 * s)) + list(range(2 * s, 3 * s))
        g = W.from_edges(3 * s, np.array(u), np.array(v), np.ones(len(u)), "caterpillar")
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    kinds = [h.info(l)["elim"] for l in range(h.num_levels - 1)]
    assert all(kinds)                                   # only elimination levels above the coarsest
    b = W.zero_sum_rhs(g.n, 7)
    x, hist = h.solve(b, tol=1e-11, max_cycles=5)
    assert len(hist) - 1 == 1                           # exact: one cycle
    assert hist[-1] <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("gname", ["grid", "chung_lu", "rgg"])
def test_solution_with_elimination_matches_dense_pseudoinverse(gname):
    g = {"grid": W.grid2d(40, 40), "chung_lu": W.chung_lu(2000, seed=21), "rgg": W.rgg2d(1800, seed=22)}[gname]
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    assert any(h.info(l)["elim"] for l in range(h.num_levels))
    b = W.zero_sum_rhs(g.n, 23)
    x, hist = h.solve(b, tol=1e-12, max_cycles=400)
    want = oracle.dense_pinv_solve(_dense(g), b)
    assert np.linalg.norm(x - want) <= 1e-8 * np.linalg.norm(want)
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()


def test_elimination_removes_the_one_dimensional_part_of_a_grid():
    # Sec. 3.2: elimination removes what aggregation coarsens badly.  On a 5-point
    # grid every node has degree <= 4, so the first F is a maximal independent set
    # of the whole grid: each node is in F or next to it, hence |F| >= n/5.  Under
    # the parallel handshake with recombination below the finest level only (the
    # earlier readings R9/R15, which coarsen a grid at alpha ~ .8), the work per
    # digit of the whole solve drops well below that without elimination.
    g = W.grid2d(64, 64)
    b = W.zero_sum_rhs(g.n, 1)
    wpd = []
    for e in (0, 1):
        h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=e, agg_rule=0, recomb_finest=0)
        if e:
            assert h.info(0)["nF"] >= g.n / 5
        _, hist = h.solve(b, tol=1e-8, max_cycles=400)
        p = len(hist) - 1
        acf = (hist[-1] / hist[0]) ** (1.0 / p)
        visits, work, nnz0 = 1.0, 0.0, h.info(0)["nnz"]
        for l in range(h.num_levels):
            i = h.info(l)
            work += visits * i["nnz"] / nnz0
            if not i["coarsest"]:
                visits *= i["gamma"]
        wpd.append(work / -math.log10(acf))
    assert wpd[1] <= 0.6 * wpd[0], wpd


def test_standalone_elim_set_reproduces_the_hierarchy():
    # oracle.elim_set applied to a level's own graph with that level's sweep key gives
    # the level's eliminated set (the full-size GPU test relies on this)
    g = W.chung_lu(5000, seed=3)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1, agg_rule=0)   # several elimination levels
    seen = 0
    for l in range(h.num_levels - 1):
        if not h.info(l)["elim"]:
            continue
        rp, col, _ = h.csr(l)
        key = oracle.splitmix64(oracle.splitmix64(1) ^ ((2 * l + 1) << 32) ^ (1 << 63))
        cidx, nF = oracle.elim_set(len(rp) - 1, rp, col, key)
        assert np.array_equal(cidx, h.elim(l)) and nF == h.info(l)["nF"]
        seen += 1
    assert seen >= 2


def test_grid_acf_matches_the_paper():
    # The paper prints an ACF of .216 for the 5-point 1024^2 grid (Sec. 5, grid
    # table).  With the paper's scan (Sec. 3.4.2, in hashed order) and recombination
    # at every level (reading R15), the oracle's ACF on a 256^2 grid lies in that
    # neighbourhood with and without elimination.  Under the earlier readings (the
    # parallel handshake, recombination below the finest level only) only
    # elimination rescued it: aggregation alone stalled (rate above .9 per cycle).
    g = W.grid2d(256, 256)
    b = W.zero_sum_rhs(g.n, 1)
    for kw in ({}, {"elim": 1}, {"elim": 1, "agg_rule": 0, "recomb_finest": 0}):
        h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **kw)
        _, hist = h.solve(b, tol=1e-10, max_cycles=100)
        p = len(hist) - 1
        acf = (hist[-1] / hist[0]) ** (1.0 / p)
        assert 0.15 <= acf <= 0.30 and p <= 25, (kw, acf, p)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, agg_rule=0, recomb_finest=0)
    _, hist = h.solve(b, tol=1e-10, max_cycles=40)
    rate = (hist[-1] / hist[-11]) ** 0.1              # over the last 10 cycles
    assert rate > 0.9, rate


def test_adaptive_cycle_on_the_1024_grid_needs_a_mild_flat_factor():
    # The paper's grid table: 5-point 1024^2 grid, ACF .216.  With elimination, the
    # adaptive cycle with recombination alone (mu = 1, reading R15) stalls on this
    # grid; with a mild flat factor under the recombination (mu_adaptive = 1.2) it
    # converges at about the paper's rate.
    g = W.grid2d(1024, 1024)
    b = W.zero_sum_rhs(g.n, 1)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1, mu_adaptive=1.2)
    _, hist = h.solve(b, tol=1e-10, max_cycles=40)
    p = len(hist) - 1
    acf = (hist[-1] / hist[0]) ** (1.0 / p)
    assert p <= 20 and 0.12 <= acf <= 0.30, (p, acf)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, elim=1)
    _, hist = h.solve(b, tol=1e-10, max_cycles=25)
    assert (hist[-1] / hist[-6]) ** 0.2 > 0.9            # stalled: rate over the last 5 cycles
