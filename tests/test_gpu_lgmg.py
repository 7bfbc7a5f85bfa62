"""Lean Geometric Multigrid (Sec. 6; option lgmg_nx) on the GPU against the
oracle with the same option.

The geometric mode replaces the algebraic setup by 2x2 aggregates and
red-black colours on a periodic 5-point grid; the Galerkin operators, the
cycle and the solve are the library's own.  The setup agrees bit for bit,
the cycle within the tolerances of the other parity tests, and the solve's
rate per unit of work is the paper's .5 (the oracle's pin of it, on the GPU).
"""
import math

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


def _both(L, nx, **kw):
    g = W.grid2d_periodic(nx)
    kw = dict(lgmg_nx=nx, mu_flat=2.0, **kw)
    s = L.Solver.from_graph(g, keep_setup_data=1, **kw)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **{k: v for k, v in kw.items() if hasattr(oracle.Opts, k)})
    return g, s, h


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


@pytest.mark.parametrize("nx", [16, 64, 256])
def test_lgmg_setup_bit_exact(L, nx):
    g, s, h = _both(L, nx)
    nl = h.num_levels
    assert s._levels() == nl
    side = nx
    for l in range(nl):
        gi, oi = s.level_info(l), h.info(l)
        for k in ("n", "nnz", "ncolours", "K", "nc", "rounds", "sel_round", "coarsest", "stop_reason", "jp_rounds"):
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        assert gi["alpha"] == oi["alpha"] and gi["gamma"] == oi["gamma"]
        assert gi["n"] == side * side
        rp, col, w = h.csr(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "row_ptr"), rp)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "col"), col)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "w")), _bits(w))
        assert np.array_equal(L.lamg_level_copy(s.h, l, "colour"), h.colour(l))
        if not oi["coarsest"]:
            assert oi["ncolours"] == 2
            agg, state, _ = h.agg(l)
            assert np.array_equal(L.lamg_level_copy(s.h, l, "agg"), agg)
            assert np.array_equal(L.lamg_level_copy(s.h, l, "state"), state)
        side //= 2
    s.close()


@pytest.mark.parametrize("adaptive", [False, True])
def test_lgmg_one_cycle_elementwise(L, adaptive):
    g, s, h = _both(L, 64)
    b = W.zero_sum_rhs(g.n, 3)
    xo = h.cycle(b, np.zeros(g.n), adaptive=adaptive)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    L.lamg_cycle(s.h, bt, xt, adaptive)
    assert np.max(np.abs(xt.cpu().numpy() - xo)) <= 1e-11 * np.max(np.abs(xo))
    xo2 = h.cycle(b, xo, adaptive=adaptive)
    L.lamg_cycle(s.h, bt, xt, adaptive)
    assert np.max(np.abs(xt.cpu().numpy() - xo2)) <= 1e-10 * np.max(np.abs(xo2))
    s.close()


def test_lgmg_rate_per_unit_of_work(L):
    # Sec. 6: .5 per unit of work on the periodic Poisson problem.  Run on the GPU
    # cycle by cycle (flat mode, one lamg_cycle per step, the residual norm from the
    # CSR), to a relative residual of 1e-10, and measured over the last 5 cycles
    # like the oracle's pin.
    nx = 128
    g, s, h = _both(L, nx)
    b = W.zero_sum_rhs(g.n, 1)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    rp, col, w = (torch.tensor(a, device="cuda") for a in (g.rp, g.col.astype(np.int64), g.w))
    rows = torch.repeat_interleave(torch.arange(g.n, device="cuda"), torch.diff(rp))
    deg = torch.zeros(g.n, dtype=torch.float64, device="cuda").index_add_(0, rows, w)

    def resnorm(x):
        ax = deg * x - torch.zeros_like(x).index_add_(0, rows, w * x[col])
        return float(torch.linalg.norm(bt - ax))

    hist = [resnorm(xt)]
    while hist[-1] > 1e-10 * hist[0] and len(hist) <= 80:
        L.lamg_cycle(s.h, bt, xt, False)
        hist.append(resnorm(xt))
    assert len(hist) >= 7
    acf = (hist[-1] / hist[-6]) ** 0.2
    nu = h.opts.nu1 + h.opts.nu2
    steps, work = 1, 0.0
    for l in range(h.num_levels - 1):
        work += steps * nu * h.info(l)["n"] / g.n
        steps = math.ceil(steps * h.info(l)["gamma"])
    rate = acf ** (1.0 / work)
    assert 0.45 <= rate <= 0.56, rate
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_lgmg_solve_matches_the_oracle(L, precision):
    g, s, h = _both(L, 256, adaptive=0)
    b = W.zero_sum_rhs(g.n, 5)
    tol = 1e-10 if precision == "fp64" else 1e-8
    p = L.LAMG_FP64 if precision == "fp64" else L.LAMG_FP32_IR
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=tol, precision=p)
    xo, hist = h.solve(b, tol=1e-12, max_cycles=200, adaptive=False)
    assert st.status == 0 and st.rel_res <= tol
    xg = x.cpu().numpy()
    # both solutions have zero mean, so their difference is bounded by the residuals
    # over the smallest non-zero eigenvalue of the periodic grid, 4 sin^2(pi / nx)
    lam_min = 4.0 * math.sin(math.pi / 256) ** 2
    bound = (st.rel_res + 1e-12) * np.linalg.norm(b) / lam_min
    assert np.linalg.norm(xg - xo) <= 1.01 * bound
    assert abs(xg.sum()) <= 1e-9 * np.abs(xg).sum()
    if precision == "fp64":
        _, h10 = h.solve(b, tol=tol, max_cycles=200, adaptive=False)
        assert abs(st.cycles - (len(h10) - 1)) <= 1
    s.close()


def test_lgmg_rejects_a_size_that_is_not_the_square_of_the_side(L):
    g = W.grid2d_periodic(16)
    with pytest.raises(L.LamgError) as e:
        L.Solver.from_graph(g, lgmg_nx=15)
    assert e.value.status == L.LAMG_ERR_ARG
