"""The seeded synthetic generators (`workloads/`) that feed both the oracle and
the GPU tests.  Every graph they produce must be a valid LAMG input: a
symmetric CSR with strictly increasing columns, positive finite weights, no
self loops, and connected (each graph of a union).  The sizes follow each
recipe, and the same seed gives the same graph."""
import numpy as np
import pytest

import oracle
import workloads as W


def _valid(g):
    assert oracle.validate(g.n, g.rp, g.col, g.w) == 0
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    same_row = rows[1:] == rows[:-1]
    assert np.all(np.diff(g.col.astype(np.int64))[same_row] > 0)     # strictly increasing columns


GENERATORS = {
    "five": W.five_node,
    "path": lambda: W.path(50),
    "star": lambda: W.star(40),
    "complete": lambda: W.complete(30),
    "grid2d": lambda: W.grid2d(12, 9),
    "torus": lambda: W.grid2d_periodic(10),
    "grid3d": lambda: W.grid3d(6, 5, 4, 1.0, 1.0, 0.01),
    "chung_lu": lambda: W.chung_lu(20000, seed=3),
    "rgg": lambda: W.rgg2d(20000, seed=4),
    "er": lambda: W.erdos_renyi(5000, seed=5),
}


@pytest.mark.parametrize("name", list(GENERATORS))
def test_generators_give_valid_deterministic_inputs(name):
    g = GENERATORS[name]()
    _valid(g)
    h = GENERATORS[name]()
    assert np.array_equal(g.rp, h.rp) and np.array_equal(g.col, h.col) and np.array_equal(g.w, h.w)


def test_recipe_sizes():
    g = W.grid2d(12, 9)
    assert (g.n, g.m) == (108, 11 * 9 + 12 * 8)
    g = W.grid3d(6, 5, 4, 1.0, 1.0, 0.01)
    assert (g.n, g.m) == (120, 5 * 5 * 4 + 6 * 4 * 4 + 6 * 5 * 3)
    assert set(np.unique(g.w)) == {0.01, 1.0}
    assert (W.path(50).m, W.star(40).m, W.complete(30).m) == (49, 39, 30 * 29 // 2)
    t = W.grid2d_periodic(10)
    assert (t.n, t.m) == (100, 200) and np.all(np.diff(t.rp) == 4)       # a torus: degree 4 everywhere
    cl = W.chung_lu(20000, seed=3)
    mean = 2 * cl.m / cl.n
    assert 8.0 <= mean <= 12.0
    assert np.diff(cl.rp).max() > 20 * mean                        # heavy tail (power law)
    assert np.all(cl.w == cl.w.astype(np.float32))                  # FP32 weights, exact in FP64
    rgg = W.rgg2d(20000, seed=4)
    assert 10.0 <= 2 * rgg.m / rgg.n <= 13.0
    assert np.all((rgg.w > 0) & (rgg.w <= 1.0))
    er = W.erdos_renyi(5000, seed=5)
    assert 7.0 <= 2 * er.m / er.n <= 9.0


def test_unions_and_right_hand_sides():
    u, gptr = W.er_batch(20, 100, 500, seed=3)
    assert oracle.validate_graphs(u.n, u.rp, u.col, u.w, gptr) == 0
    assert gptr[0] == 0 and gptr[-1] == u.n and np.all(np.diff(gptr) > 0)
    # a subset of the batch is the union of the same graphs
    sub, sptr = W.er_batch(20, 100, 500, seed=3, only=[4, 11])
    for k, (a, e) in enumerate(((gptr[4], gptr[5]), (gptr[11], gptr[12]))):
        s0, s1 = sptr[k], sptr[k + 1]
        assert s1 - s0 == e - a
        assert np.array_equal(sub.rp[s0:s1 + 1] - sub.rp[s0], u.rp[a:e + 1] - u.rp[a])
        assert np.array_equal(sub.w[sub.rp[s0]:sub.rp[s1]], u.w[u.rp[a]:u.rp[e]])
    b = W.zero_sum_rhs_graphs(gptr, 4)
    for k in range(len(gptr) - 1):
        seg = b[gptr[k]:gptr[k + 1]]
        assert abs(seg.sum()) <= 1e-12 * np.abs(seg).sum()
    B = W.zero_sum_rhs(300, 5, count=7)
    assert B.shape == (300, 7) and np.all(np.abs(B.sum(axis=0)) <= 1e-12 * np.abs(B).sum(axis=0))


def test_knn_components_are_a_valid_union():
    pytest.importorskip("torch")
    pytest.importorskip("scipy")
    g, gptr, lab, pts = W.knn_gmm(3000, dim=4, k=5, ncomp=3, seed=1, components=True)
    assert oracle.validate_graphs(g.n, g.rp, g.col, g.w, gptr) == 0
    assert lab.shape == (g.n,) and pts.shape == (g.n, 4)
    assert np.all(g.w > 0) and np.all(g.w <= 1.0)
