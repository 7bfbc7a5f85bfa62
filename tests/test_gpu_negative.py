"""Graphs with negative edge weights on the GPU (Sec. 5, grids with negative
weights; option negative_weights) against the CPU oracle: the setup bit for bit,
one cycle element-wise, FP64 and FP32-IR solves against the dense pseudo-inverse,
and the validation codes."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["13pt", "rot_c", "rot_d"]
# the rotated-anisotropic grids converge only without recombination at the finest level
OPTS = {"13pt": {}, "rot_c": {"recomb_finest": 0}, "rot_d": {"recomb_finest": 0}}


@pytest.fixture(scope="module")
def L():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg
    assert torch.cuda.is_available()
    return lamg


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


def _both(L, g, **kw):
    kw = dict(kw, negative_weights=1)
    s = L.Solver.from_graph(g, keep_setup_data=1, **kw)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **kw)
    return s, h


@pytest.mark.parametrize("kind", KINDS)
def test_setup_bit_exact(L, kind):
    g = W.grid2d_stencil(40, kind)
    s, h = _both(L, g, **OPTS[kind])
    assert s._levels() == h.num_levels >= 3
    for l in range(h.num_levels):
        gi, oi = s.level_info(l), h.info(l)
        for k in ("n", "nnz", "ncolours", "K", "nc", "rounds", "sel_round", "coarsest"):
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        rp, col, w = h.csr(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "row_ptr"), rp)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "col"), col)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "w")), _bits(w))
        assert (w < 0).any() or l > 0
        if oi["coarsest"]:
            continue
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "tv")), _bits(h.tv(l)))
        aff, q, score = h.scores(l)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "q")), _bits(q))
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "score")), _bits(score))
        assert np.array_equal(L.lamg_level_copy(s.h, l, "agg"), h.agg(l)[0])
    s.close()


@pytest.mark.parametrize("kind", KINDS)
def test_one_cycle_elementwise(L, kind):
    g = W.grid2d_stencil(40, kind)
    s, h = _both(L, g, **OPTS[kind])
    b = W.zero_sum_rhs(g.n, 3)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    xo = np.zeros(g.n)
    for k in range(2):
        xo = h.cycle(b, xo, adaptive=True)
        L.lamg_cycle(s.h, bt, xt, True)
        assert np.max(np.abs(xt.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo)), k
    s.close()


@pytest.mark.parametrize("kind", KINDS)
def test_solves_match_dense(L, kind):
    g = W.grid2d_stencil(30, kind)
    s, h = _both(L, g, max_cycles=2000, **OPTS[kind])
    b = W.zero_sum_rhs(g.n, 4)
    bt = torch.tensor(b, device="cuda")
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    xd = np.linalg.lstsq(A, b, rcond=None)[0]
    xd -= xd.mean()
    for prec, tol in ((L.LAMG_FP64, 1e-10), (L.LAMG_FP32_IR, 1e-8)):
        x, st = s.solve(bt, tol=tol, precision=prec)
        xg = x.cpu().numpy()
        assert np.linalg.norm(b - A @ xg) <= 1.01 * tol * np.linalg.norm(b)
        assert np.linalg.norm(xg - xd) <= 1e-6 * np.linalg.norm(xd)
    s.close()


def test_validation_codes(L):
    g = W.grid2d_stencil(10, "13pt")

    def status(**kw):
        try:
            s = L.Solver.from_graph(g, **kw)
            s.close()
            return 0
        except L.LamgError as e:
            return e.status

    assert status() == L.LAMG_ERR_BAD_WEIGHT == oracle.validate(g.n, g.rp, g.col, g.w)
    assert status(negative_weights=1) == 0 == oracle.validate(g.n, g.rp, g.col, g.w, signed=True)
    p = W.from_edges(3, [0, 1, 0], [1, 2, 2], [1.0, 1.0, -1.5])    # row 0: 1 - 1.5 < 0
    try:
        s = L.Solver.from_graph(p, negative_weights=1)
        s.close()
        st = 0
    except L.LamgError as e:
        st = e.status
    assert st == L.LAMG_ERR_BAD_WEIGHT == oracle.validate(p.n, p.rp, p.col, p.w, signed=True)
