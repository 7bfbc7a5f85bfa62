"""Graphs with negative edge weights (Sec. 5, grids with negative weights): the
oracle's option negative_weights and the three stencils of the paper's grid
table, pinned against the paper and against dense linear algebra.

- The generated Laplacians have the paper's stencils in their interior rows and,
  on the 1024^2 grid, exactly the edge counts m the paper's table prints.
- They are positive semi-definite with the constants as their only null vectors.
- The validation rules: negative weights are rejected unless the option is set;
  with it, weights must be nonzero and finite and every row sum positive.
- Solutions equal the dense pseudo-inverse solution.
- The energy-ratio test uses |w| in the nodal energies (reading R22): recomputed
  here in numpy from that definition.
- The 13-point stencil converges at a mesh-independent rate near the paper's.
"""
import numpy as np
import pytest

import oracle
import workloads as W

KINDS = ["13pt", "rot_c", "rot_d"]


def _interior_row(g, nx):
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    u = nx // 2 + nx * (nx // 2)
    return {((v % nx) - (u % nx), (v // nx) - (u // nx)): A[u, v] for v in np.flatnonzero(A[u])}


def test_stencils_are_the_papers():
    # 13-point 4th order: [1 -16 60 -16 1] / 12 along x and y (figure (b))
    r = _interior_row(W.grid2d_stencil(9, "13pt"), 9)
    want = {(0, 0): 60 / 12, (1, 0): -16 / 12, (-1, 0): -16 / 12, (0, 1): -16 / 12, (0, -1): -16 / 12,
            (2, 0): 1 / 12, (-2, 0): 1 / 12, (0, 2): 1 / 12, (0, -2): 1 / 12}
    assert r.keys() == want.keys() and all(abs(r[k] - want[k]) < 1e-15 for k in want)
    # (c): the figure's off-diagonal entries; its centre is garbled (1.5050 would not
    # give zero row sums), Eq. (5.1) gives 2 (cos^2 + eps sin^2) / 2 = 1.01
    r = _interior_row(W.grid2d_stencil(9, "rot_c"), 9)
    want = {(0, 0): 1.01, (1, 0): -.2525, (-1, 0): -.2525, (0, 1): -.2525, (0, -1): -.2525,
            (-1, 1): -.12375, (1, -1): -.12375, (1, 1): .12375, (-1, -1): .12375}
    assert r.keys() == want.keys() and all(abs(r[k] - want[k]) < 1e-12 for k in want)
    # (d): the figure exactly
    r = _interior_row(W.grid2d_stencil(9, "rot_d"), 9)
    want = {(0, 0): 1.505, (1, 0): -.5, (-1, 0): -.5, (0, 1): -.5, (0, -1): -.5, (1, 1): .2475, (-1, -1): .2475}
    assert r.keys() == want.keys() and all(abs(r[k] - want[k]) < 1e-12 for k in want)


def test_edge_counts_match_the_papers_table():
    # the grid table of Sec. 5 prints m for the 1024^2 grids
    assert {k: W.grid2d_stencil(1024, k).m for k in KINDS} == {"13pt": 4188160, "rot_c": 4188162, "rot_d": 3141633}


@pytest.mark.parametrize("kind", KINDS)
def test_positive_semidefinite_with_constant_null_space(kind):
    g = W.grid2d_stencil(24, kind)
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    assert np.allclose(A.sum(axis=1), 0.0, atol=1e-13)
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > -1e-12 and ev[1] > 1e-5, ev[:3]
    assert (g.w < 0).any()


def test_validation_of_signed_weights():
    g = W.grid2d_stencil(10, "13pt")
    assert oracle.validate(g.n, g.rp, g.col, g.w) == oracle.ERR_BAD_WEIGHT
    assert oracle.validate(g.n, g.rp, g.col, g.w, signed=True) == oracle.OK
    with pytest.raises(oracle.OracleError):
        oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    # a zero weight, or a row whose sum is not positive, is rejected
    w = g.w.copy()
    w[0] = 0.0
    assert oracle.validate(g.n, g.rp, g.col, w, signed=True) == oracle.ERR_BAD_WEIGHT
    p = W.from_edges(3, [0, 1, 0], [1, 2, 2], [1.0, 1.0, -1.5])    # row 0: 1 - 1.5 < 0
    assert oracle.validate(p.n, p.rp, p.col, p.w, signed=True) == oracle.ERR_BAD_WEIGHT


# the rotated-anisotropic grids converge only without recombination at the finest
# level (about .94 per cycle at 30^2; with it the cycle stalls near .998)
OPTS = {"13pt": {}, "rot_c": {"recomb_finest": 0}, "rot_d": {"recomb_finest": 0}}


@pytest.mark.parametrize("kind", KINDS)
def test_solution_equals_dense_pseudo_inverse(kind):
    g = W.grid2d_stencil(30, kind)
    b = W.zero_sum_rhs(g.n, 7)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, negative_weights=1, **OPTS[kind])
    assert h.num_levels >= 3
    x, hist = h.solve(b, tol=1e-10, max_cycles=600)
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    xd = np.linalg.lstsq(A, b, rcond=None)[0]
    xd -= xd.mean()
    assert hist[-1] <= 1e-10 * hist[0]
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_energy_ratio_uses_absolute_weights():
    # Eq. (3.12) with the nodal energies of |w| (reading R22): recomputed in numpy
    g = W.grid2d_stencil(12, "rot_d")
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(g.n, 4))
    aff, q, score = oracle.edge_scores(g.n, g.rp, g.col, g.w, X)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    aw = np.abs(g.w)
    a = np.bincount(rows, weights=aw, minlength=g.n)
    for e in rng.choice(g.col.size, 200, replace=False):
        u, s = rows[e], g.col[e]
        nb = slice(g.rp[u], g.rp[u + 1])
        Xv = X[g.col[nb]]
        ystar = (aw[nb, None] * Xv).sum(axis=0) / a[u]
        emin = 0.5 * (aw[nb, None] * (ystar - Xv) ** 2).sum(axis=0)
        es = 0.5 * (aw[nb, None] * (X[s] - Xv) ** 2).sum(axis=0)
        assert q[e] == pytest.approx(np.max(es / emin), rel=1e-10)


def test_thirteen_point_rate_is_mesh_independent():
    # the grid table: ACF .262 on the 1024^2 13-point grid; here 128^2 and 256^2
    acf = []
    for nx in (128, 256):
        g = W.grid2d_stencil(nx, "13pt")
        b = W.zero_sum_rhs(g.n, 2)
        h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, negative_weights=1)
        _, hist = h.solve(b, tol=1e-8, max_cycles=60)
        acf.append((hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1)))
    assert all(0.2 <= r <= 0.4 for r in acf) and abs(acf[1] - acf[0]) <= 0.05, acf
