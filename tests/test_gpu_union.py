"""Many graphs in one hierarchy (block-diagonal union, lamg_setup_graphs) on the
GPU against the oracle's union (oracle.Hierarchy(..., gptr=...)) and dense
per-graph solves."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg
    assert torch.cuda.is_available()
    return lamg


def _mixed():
    return W.block_union([W.grid2d(9, 7), W.chung_lu(700, seed=31), W.path(40), W.star(25),
                          W.erdos_renyi(300, seed=32)])


def _unions():
    return {"mixed": _mixed, "er40": lambda: W.er_batch(40, 200, 3000, seed=9)}


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


@pytest.mark.parametrize("uname", ["mixed", "er40"])
def test_union_setup_bit_exact(L, uname):
    u, gptr = _unions()[uname]()
    s = L.Solver.from_graph(u, gptr=gptr, keep_setup_data=1)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    assert s._levels() == h.num_levels
    for l in range(h.num_levels):
        gi, oi = s.level_info(l), h.info(l)
        for k in ("n", "nnz", "ncolours", "K", "nc", "rounds", "sel_round", "coarsest", "stop_reason", "jp_rounds"):
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        assert gi["alpha"] == oi["alpha"] and gi["gamma"] == oi["gamma"]
        rp, col, w = h.csr(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "row_ptr"), rp)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "col"), col)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "w")), _bits(w))
        if oi["coarsest"]:
            continue
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "tv")), _bits(h.tv(l)))
        agg, state, hub = h.agg(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "agg"), agg)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "state"), state)
    s.close()


@pytest.mark.parametrize("adaptive", [True, False])
def test_union_one_cycle_elementwise(L, adaptive):
    u, gptr = _mixed()
    s = L.Solver.from_graph(u, gptr=gptr)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    b = W.zero_sum_rhs_graphs(gptr, 3)
    xo = h.cycle(b, np.zeros(u.n), adaptive=adaptive)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(u.n, dtype=torch.float64, device="cuda")
    L.lamg_cycle(s.h, bt, xt, adaptive)
    assert np.max(np.abs(xt.cpu().numpy() - xo)) <= 1e-11 * np.max(np.abs(xo))
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_union_solve_every_graph(L, precision):
    u, gptr = W.er_batch(40, 200, 3000, seed=9)
    s = L.Solver.from_graph(u, gptr=gptr)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    b = W.zero_sum_rhs_graphs(gptr, 4)
    tol = 1e-10 if precision == "fp64" else 1e-8
    p = L.LAMG_FP64 if precision == "fp64" else L.LAMG_FP32_IR
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=tol, precision=p)
    xg = x.cpu().numpy()
    assert st.rel_res <= tol
    rel = L.lamg_graph_residuals(s.h, len(gptr) - 1)
    assert rel.max() == st.rel_res and (rel <= tol).all()
    xo, _ = h.solve(b, tol=1e-12)
    for g in range(len(gptr) - 1):
        a, e = gptr[g], gptr[g + 1]
        rp = u.rp[a:e + 1] - u.rp[a]
        A = oracle.laplacian_dense(e - a, rp, u.col[u.rp[a]:u.rp[e]] - a, u.w[u.rp[a]:u.rp[e]])
        assert np.linalg.norm(b[a:e] - A @ xg[a:e]) <= 1.01 * tol * np.linalg.norm(b[a:e])
        assert abs(xg[a:e].sum()) <= 1e-9 * np.abs(xg[a:e]).sum()
        assert np.linalg.norm(xg[a:e] - xo[a:e]) <= 1e-6 * np.linalg.norm(xo[a:e])
    s.close()


def test_union_validation_and_rhs_codes(L):
    u, gptr = _mixed()

    def status(gp):
        try:
            L.Solver.from_graph(u, gptr=gp).close()
            return 0
        except L.LamgError as e:
            return e.status

    assert status(gptr) == 0
    bad = gptr.copy(); bad[1] -= 3
    assert status(bad) == L.LAMG_ERR_ARG == oracle.validate_graphs(u.n, u.rp, u.col, u.w, bad)
    merged = np.delete(gptr, 1)
    assert status(merged) == L.LAMG_ERR_DISCONNECTED == oracle.validate_graphs(u.n, u.rp, u.col, u.w, merged)
    s = L.Solver.from_graph(u, gptr=gptr)
    with pytest.raises(L.LamgError) as e:
        s.solve(torch.tensor(W.zero_sum_rhs(u.n, 6), device="cuda"))   # zero-sum on the union only
    assert e.value.status == L.LAMG_ERR_RHS_NOT_ZERO_SUM
    with pytest.raises(L.LamgError) as e:
        s.solve_batched(torch.zeros(u.n, 4, dtype=torch.float64, device="cuda"))
    assert e.value.status == L.LAMG_ERR_ARG
    s.close()


def test_union_adjoint_matches_oracle(L):
    u, gptr = _mixed()
    s = L.Solver.from_graph(u, gptr=gptr)
    h = oracle.Hierarchy(u.n, u.rp, u.col, u.w, gptr=gptr)
    b = W.zero_sum_rhs_graphs(gptr, 7)
    x, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-12)
    gx = torch.tensor(np.random.default_rng(8).normal(size=u.n), device="cuda")
    eu, ev, _ = u.edges()
    lam = torch.zeros(u.n, dtype=torch.float64, device="cuda")
    dw = torch.zeros(eu.size, dtype=torch.float64, device="cuda")
    L.lamg_adjoint(s.h, x, gx, lam, torch.tensor(eu, device="cuda"), torch.tensor(ev, device="cuda"), dw, tol=1e-12)
    lo, dwo = h.adjoint(x.cpu().numpy(), gx.cpu().numpy(), eu, ev, tol=1e-12)
    assert np.linalg.norm(lam.cpu().numpy() - lo) <= 1e-8 * np.linalg.norm(lo)
    assert np.linalg.norm(dw.cpu().numpy() - dwo) <= 1e-8 * np.linalg.norm(dwo)
    s.close()
