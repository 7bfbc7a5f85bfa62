"""Pins of the oracle's block-diagonal union of several graphs (the batched
multi-graph form): it must reduce to the single-graph hierarchy for one graph,
and solve every graph exactly as a dense pseudo-inverse of that graph would."""
import numpy as np
import pytest

import oracle
import workloads as W


def _graphs():
    return [W.grid2d(9, 7), W.chung_lu(700, seed=31), W.path(40), W.star(25), W.erdos_renyi(300, seed=32)]


def test_single_graph_union_equals_plain_setup():
    g = W.chung_lu(1500, seed=33)
    a = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    b = oracle.Hierarchy(g.n, g.rp, g.col, g.w, gptr=[0, g.n])
    assert a.num_levels == b.num_levels
    for l in range(a.num_levels):
        assert a.info(l) == b.info(l)
        for x, y in zip(a.csr(l), b.csr(l)):
            assert np.array_equal(x, y)
    rhs = W.zero_sum_rhs(g.n, 1)
    xa, ha = a.solve(rhs, tol=1e-10)
    xb, hb = b.solve(rhs, tol=1e-10)
    assert np.array_equal(xa, xb) and np.array_equal(ha, hb)


def test_union_validation_codes():
    gs = _graphs()
    u, gptr = W.block_union(gs)
    assert oracle.validate_graphs(u.n, u.rp, u.col, u.w, gptr) == 0
    # the union is disconnected as one graph
    assert oracle.validate(u.n, u.rp, u.col, u.w) == oracle.ERR_DISCONNECTED
    # ranges that split a graph in two: that graph is disconnected... and an edge crosses ranges
    bad = gptr.copy(); bad[1] -= 3
    assert oracle.validate_graphs(u.n, u.rp, u.col, u.w, bad) == oracle.ERR_ARG
    # two graphs declared as one: disconnected
    merged = np.delete(gptr, 1)
    assert oracle.validate_graphs(u.n, u.rp, u.col, u.w, merged) == oracle.ERR_DISCONNECTED
    # empty range
    assert oracle.validate_graphs(u.n, u.rp, u.col, u.w, np.insert(gptr, 1, 0)) == oracle.ERR_ARG


@pytest.mark.parametrize("dense_max", [1024, 8])
def test_union_solves_every_graph(dense_max):
    gs = _graphs()
    u, gptr = W.block_union(gs)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr, dense_max=dense_max)
    b = W.zero_sum_rhs_graphs(gptr, 5)
    x, hist = h.solve(b, tol=1e-10)
    assert len(hist) - 1 < 200
    for k, g in enumerate(gs):
        s, e = gptr[k], gptr[k + 1]
        A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
        xd = np.linalg.lstsq(A, b[s:e], rcond=None)[0]
        xd -= xd.mean()
        # every graph meets the relative residual test on its own
        assert np.linalg.norm(b[s:e] - A @ x[s:e]) <= 1.01e-10 * np.linalg.norm(b[s:e])
        assert abs(x[s:e].sum()) <= 1e-12 * np.abs(x[s:e]).sum()
        assert np.linalg.norm(x[s:e] - xd) <= 1e-7 * np.linalg.norm(xd)


def test_union_rejects_rhs_not_zero_sum_per_graph():
    gs = _graphs()
    u, gptr = W.block_union(gs)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    b = W.zero_sum_rhs(u.n, 6)       # zero-sum on the union, not per graph
    with pytest.raises(oracle.OracleError):
        h.solve(b, tol=1e-8)


def test_union_coarsest_has_several_components():
    gs = _graphs()
    u, gptr = W.block_union(gs)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    L = h.num_levels
    rp, col, w = h.csr(L - 1)
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    A = sp.csr_matrix((w, col, rp), shape=(len(rp) - 1, len(rp) - 1))
    ncomp, _ = cg.connected_components(A, directed=False)
    assert ncomp >= 2   # the direct coarsest solve must treat each component's null space
