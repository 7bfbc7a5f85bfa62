"""GPU parity: the CUDA library (through the C-ABI) against the CPU oracle.

Setup (integer work and the FP64 floats that feed it) must agree bit for bit;
the solve floats within the tolerances stated at each test.
"""
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


def _graph(name):
    return {
        "five": W.five_node,
        "path": lambda: W.path(300),
        "star": lambda: W.star(200),
        "grid2d": lambda: W.grid2d(40, 30),
        "grid3d": lambda: W.grid3d(12, 12, 12, 1.0, 1.0, 0.01),
        "chung_lu": lambda: W.chung_lu(6000, seed=13),
        "rgg": lambda: W.rgg2d(5000, seed=14),
        "er": lambda: W.erdos_renyi(3000, seed=16),
        "grid64": lambda: W.grid2d(64, 64),
        # hubs above 4096 entries: block-tier rows in setup and solve
        "hubs": lambda: W.chung_lu(30000, 2.1, 12.0, seed=7, i0=1.0),
        "star6k": lambda: W.star(6000),
        # every node its own colour: tail-colour sweeps and long single-block runs
        "complete": lambda: W.complete(200),
        # the 256^3 workload's family (weights 1/1/0.01) at a size the oracle handles
        "grid3d32": lambda: W.grid3d(32, 32, 32, 1.0, 1.0, 0.01),
    }[name]()


def _both(L, g, **kw):
    s = L.Solver.from_graph(g, keep_setup_data=1, **kw)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, **{k: v for k, v in kw.items() if hasattr(oracle.Opts, k)})
    return s, h


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


SETUP_GRAPHS = ["five", "path", "star", "grid2d", "grid3d", "chung_lu", "rgg", "er", "grid64", "hubs", "star6k",
                "complete", "grid3d32"]

# the other rules of the library (Sec. 3.4.2 and Eq. (2.3)): the parallel handshake
# with recombination below the finest level only, the paper's index-order scan,
# and lexicographic Gauss-Seidel (with either scan order)
RULES = {
    "handshake": {"agg_rule": 0, "recomb_finest": 0},
    "index_scan": {"agg_rule": 1},
    "index_scan_lex": {"agg_rule": 1, "relax_rule": 1},
    "lex": {"relax_rule": 1},
    # the coarse cycle-index cap (Eq. (4.1)) and the restriction factor under
    # recombination (Eq. (3.13)): the per-level gamma is compared exactly
    "cap1": {"gamma_coarse_max": 1.0},
    "mu12": {"mu_adaptive": 1.2},
    # the colouring's priority without the hash: greedy in (degree, index) order
    "colour_greedy": {"colour_rule": 1},
    # the options of the 3-D grid benchmark: fine-level cycle-index cap 1.2 with
    # the coarse cap 1 (Eq. (4.1)) and the greedy colouring
    "grid_bench": {"gamma": 1.2, "gamma_coarse_max": 1.0, "colour_rule": 1},
}


@pytest.mark.parametrize("gname", SETUP_GRAPHS)
def test_setup_bit_exact(L, gname):
    _check_setup_bit_exact(L, _graph(gname))


@pytest.mark.parametrize("rule", list(RULES))
@pytest.mark.parametrize("gname", ["grid2d", "grid3d", "chung_lu", "rgg", "hubs"])
def test_setup_bit_exact_rules(L, gname, rule):
    _check_setup_bit_exact(L, _graph(gname), **RULES[rule])


def _check_setup_bit_exact(L, g, **kw):
    s, h = _both(L, g, **kw)
    nl = h.num_levels
    assert s._levels() == nl
    for l in range(nl):
        gi, oi = s.level_info(l), h.info(l)
        for k in ("n", "nnz", "ncolours", "K", "nc", "rounds", "sel_round", "coarsest", "stop_reason",
                  "jp_rounds"):
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        assert gi["alpha"] == oi["alpha"] and gi["gamma"] == oi["gamma"]
        rp, col, w = h.csr(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "row_ptr"), rp)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "col"), col)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "w")), _bits(w))
        assert np.array_equal(L.lamg_level_copy(s.h, l, "colour"), h.colour(l))
        if oi["coarsest"]:
            continue
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "tv")), _bits(h.tv(l)))
        aff, q, score = h.scores(l)
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "affinity")), _bits(aff))
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "q")), _bits(q))
        assert np.array_equal(_bits(L.lamg_level_copy(s.h, l, "score")), _bits(score))
        agg, state, hub = h.agg(l)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "agg"), agg)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "state"), state)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "hub").astype(bool), hub)
    s.close()


@pytest.mark.parametrize("gname", ["grid2d", "chung_lu", "rgg", "grid3d", "star", "hubs", "complete"])
@pytest.mark.parametrize("adaptive", [True, False])
def test_one_cycle_elementwise(L, gname, adaptive):
    g = _graph(gname)
    s, h = _both(L, g)
    b = W.zero_sum_rhs(g.n, 3)
    x0 = np.zeros(g.n)
    xo = h.cycle(b, x0, adaptive=adaptive)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    L.lamg_cycle(s.h, bt, xt, adaptive)
    xg = xt.cpu().numpy()
    # same hierarchy, FP64; only the summation order inside rows differs
    assert np.max(np.abs(xg - xo)) <= 1e-11 * np.max(np.abs(xo))
    # second cycle from the first iterate
    xo2 = h.cycle(b, xo, adaptive=adaptive)
    L.lamg_cycle(s.h, bt, xt, adaptive)
    assert np.max(np.abs(xt.cpu().numpy() - xo2)) <= 1e-10 * np.max(np.abs(xo2))
    s.close()


@pytest.mark.parametrize("rule", list(RULES))
@pytest.mark.parametrize("gname", ["grid2d", "chung_lu", "grid3d32"])
def test_one_cycle_elementwise_rules(L, gname, rule):
    g = _graph(gname)
    s, h = _both(L, g, **RULES[rule])
    b = W.zero_sum_rhs(g.n, 3)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    xo = np.zeros(g.n)
    for k in range(2):
        xo = h.cycle(b, xo, adaptive=True)
        L.lamg_cycle(s.h, bt, xt, True)
        assert np.max(np.abs(xt.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo)), k
    s.close()


@pytest.mark.parametrize("gname", ["grid64", "chung_lu", "rgg", "five", "path", "star6k", "complete"])
def test_solve_fp64_matches_oracle_and_dense(L, gname):
    g = _graph(gname)
    s, h = _both(L, g)
    b = W.zero_sum_rhs(g.n, 1)
    bt = torch.tensor(b, device="cuda")
    x, st = s.solve(bt, tol=1e-10)
    xg = x.cpu().numpy()
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    res = np.linalg.norm(b - A @ xg) / np.linalg.norm(b)
    assert st.rel_res <= 1e-10 and res <= 1.01e-10
    assert abs(xg.sum()) <= 1e-12 * np.abs(xg).sum()
    xo, hist = h.solve(b, tol=1e-10)
    assert abs(st.cycles - (len(hist) - 1)) <= 1
    xd = np.linalg.lstsq(A, b, rcond=None)[0]
    xd -= xd.mean()
    assert np.linalg.norm(xg - xd) <= 1e-6 * np.linalg.norm(xd)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    s.close()


@pytest.mark.parametrize("opts", [{"gamma_coarse_max": 1.0}, {"mu_adaptive": 1.2}])
@pytest.mark.parametrize("gname", ["chung_lu", "grid64"])
def test_solve_with_cycle_options(L, gname, opts):
    # the cap and the restriction factor change the cycle: FP64 and FP32-IR solves
    # against the oracle with the same options, at the tolerances of the other solves
    g = _graph(gname)
    s, h = _both(L, g, **opts)
    b = W.zero_sum_rhs(g.n, 4)
    bt = torch.tensor(b, device="cuda")
    xo, hist = h.solve(b, tol=1e-12)
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    for prec, tol in ((L.LAMG_FP64, 1e-10), (L.LAMG_FP32_IR, 1e-8)):
        x, st = s.solve(bt, tol=tol, precision=prec)
        xg = x.cpu().numpy()
        assert np.linalg.norm(b - A @ xg) <= 1.01 * tol * np.linalg.norm(b)
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    s.close()


@pytest.mark.parametrize("gname", ["grid64", "chung_lu", "rgg", "hubs", "grid3d32"])
def test_solve_fp32_ir(L, gname):
    g = _graph(gname)
    s, h = _both(L, g)
    b = W.zero_sum_rhs(g.n, 2)
    bt = torch.tensor(b, device="cuda")
    x, st = s.solve(bt, tol=1e-8, precision=L.LAMG_FP32_IR)
    xg = x.cpu().numpy()
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w)
    assert np.linalg.norm(b - A @ xg) <= 1.01e-8 * np.linalg.norm(b)
    xo, _ = h.solve(b, tol=1e-12)
    # relative solution error vs the FP64 oracle (error <= cond * residual; stated per graph)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-6, err
    s.close()


def test_fp32_weights_input(L):
    g = W.chung_lu(4000, seed=40)   # weights are FP32-representable
    s = L.Solver.from_graph(g, w_dtype=torch.float32, keep_setup_data=1)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    assert np.array_equal(L.lamg_level_copy(s.h, 0, "agg"), h.agg(0)[0])
    s.close()


def test_input_validation_codes(L):
    g = W.grid2d(6, 5)

    def status(rp, col, w):
        try:
            s = L.Solver(g.n if rp is g.rp else len(rp) - 1, torch.tensor(rp, device="cuda"),
                         torch.tensor(col, device="cuda"), torch.tensor(w, device="cuda"))
            s.close()
            return 0
        except L.LamgError as e:
            return e.status

    assert status(g.rp, g.col, g.w) == 0
    w = g.w.copy(); w[3] = -1.0
    assert status(g.rp, g.col, w) == L.LAMG_ERR_BAD_WEIGHT == oracle.validate(g.n, g.rp, g.col, w)
    w = g.w.copy(); w[3] = np.nan
    assert status(g.rp, g.col, w) == L.LAMG_ERR_BAD_WEIGHT
    w = g.w.copy(); w[3] = 2.0
    assert status(g.rp, g.col, w) == L.LAMG_ERR_NOT_SYMMETRIC == oracle.validate(g.n, g.rp, g.col, w)
    col = g.col.copy(); col[0] = 0
    assert status(g.rp, col, g.w) == L.LAMG_ERR_ARG
    two = W.from_edges(4, [0, 2], [1, 3], [1.0, 1.0])
    assert status(two.rp, two.col, two.w) == L.LAMG_ERR_DISCONNECTED


def test_rhs_and_convergence_errors(L):
    g = W.grid2d(20, 20)
    s = L.Solver.from_graph(g)
    bad = torch.ones(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LamgError) as e:
        s.solve(bad)
    assert e.value.status == L.LAMG_ERR_RHS_NOT_ZERO_SUM
    s.close()
    s = L.Solver.from_graph(g, max_cycles=1)
    b = torch.tensor(W.zero_sum_rhs(g.n, 5), device="cuda")
    with pytest.raises(L.LamgError) as e:
        s.solve(b, tol=1e-30)
    assert e.value.status == L.LAMG_ERR_NOT_CONVERGED
    x, st = s.solve(b, tol=1e-30, allow_not_converged=True)
    assert st.cycles == 1 and torch.isfinite(x).all()
    s.close()


def test_degenerate_graphs(L):
    # one node, no edges: the only zero-sum b is 0 and x = 0
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.zeros(0, dtype=torch.float64, device="cuda")
    s = L.Solver(1, rp, col, w)
    x, st = s.solve(torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert x.item() == 0.0
    s.close()
    # two nodes
    g = W.path(2)
    s = L.Solver.from_graph(g)
    x, st = s.solve(torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda"), tol=1e-14)
    assert np.allclose(x.cpu().numpy(), [0.5, -0.5], atol=1e-14)
    s.close()


def test_adjoint_matches_oracle(L):
    g = W.rgg2d(3000, seed=41)
    s, h = _both(L, g)
    rng = np.random.default_rng(42)
    b = W.zero_sum_rhs(g.n, 43)
    target = rng.normal(size=g.n)
    x, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-12)
    gx = x - torch.tensor(target, device="cuda")
    eu, ev, _ = g.edges()
    lam = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    dw = torch.zeros(eu.size, dtype=torch.float64, device="cuda")
    L.lamg_adjoint(s.h, x, gx, lam, torch.tensor(eu, device="cuda"), torch.tensor(ev, device="cuda"), dw,
                   tol=1e-12)
    lo, dwo = h.adjoint(x.cpu().numpy(), gx.cpu().numpy(), eu, ev, tol=1e-12)
    assert np.linalg.norm(lam.cpu().numpy() - lo) <= 1e-8 * np.linalg.norm(lo)
    assert np.linalg.norm(dw.cpu().numpy() - dwo) <= 1e-8 * np.linalg.norm(dwo)
    s.close()


def test_host_array_solve(L):
    g = W.chung_lu(5000, seed=44)
    s = L.Solver.from_graph(g)
    b = W.zero_sum_rhs(g.n, 45)
    x = np.zeros(g.n)
    st = L.lamg_solve_host(s.h, b, x, 1e-10)
    xd, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10)
    assert np.array_equal(x, xd.cpu().numpy())
    s.close()


def test_size_limits_rejected_before_any_work(L):
    # nnz must stay below 2^31 (int32 CSR indices on the device); the check reads
    # row_ptr[0] and row_ptr[n] only, so no large arrays are needed
    rp = torch.zeros(3, dtype=torch.int64, device="cuda")
    rp[2] = 2 ** 31
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = torch.ones(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LamgError) as e:
        L.Solver(2, rp, col, w)
    assert e.value.status == L.LAMG_ERR_ARG
    rp[2] = -1
    with pytest.raises(L.LamgError) as e:
        L.Solver(2, rp, col, w)
    assert e.value.status == L.LAMG_ERR_ARG


def test_op_timer(L):
    # the engine's op timer: rows appear after a solve, reading zeroes the table,
    # and stopping frees it (a read then returns nothing)
    g = W.chung_lu(6000, seed=13)
    s = L.Solver.from_graph(g)
    b = torch.tensor(W.zero_sum_rhs(g.n, 3), device="cuda")
    L.lamg_op_times(s.h, 1)
    s.solve(b, tol=1e-8, precision=L.LAMG_FP32_IR)
    rows = L.lamg_op_times(s.h, 0)
    names = {r[1] for r in rows}
    assert {"resid", "restrict", "prolong", "ir_prep", "res64"} <= names, names
    assert all(r[3] > 0 and r[4] >= 0.0 for r in rows)
    assert L.lamg_op_times(s.h, 0) == []
    L.lamg_op_times(s.h, -1)
    s.solve(b, tol=1e-8)
    assert L.lamg_op_times(s.h, 0) == []
    with pytest.raises(L.LamgError):
        L.lamg_op_times(s.h, 2)
    s.close()
