"""Parity at the benchmark's full size (Chung-Lu n = 1M, FP32 weights, FP32
cycles in FP64 refinement, options of bench.py), where the whole-hierarchy
oracle is too slow: the oracle recomputes per-level pieces one by one from the
GPU's own level data (colouring, hubs, per-edge affinities / energy ratios /
scores, aggregates and the Galerkin operator, all bit for bit), SciPy recomputes
P^T A P within rounding, and the solution is checked by its FP64 residual."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg as L
    assert torch.cuda.is_available()
    g = W.config_graph("chung_lu1m")
    s = L.Solver.from_graph(g, w_dtype=torch.float32, keep_setup_data=1, validate=1, max_cycles=2000)
    yield L, g, s
    s.close()


def _colour_key(seed, l):
    return oracle.splitmix64(oracle.splitmix64(seed) ^ ((2 * l + 1) << 32))


def test_fullsize_solve_residual(big):
    L, g, s = big
    b = W.zero_sum_rhs(g.n, 2)
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=1e-8, precision=L.LAMG_FP32_IR)
    xg = x.cpu().numpy()
    A = sp.csr_matrix((g.w, g.col, g.rp), shape=(g.n, g.n))
    r = b - (np.asarray(A.sum(axis=1)).ravel() * xg - A @ xg)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(b)
    assert abs(xg.sum()) <= 1e-9 * np.abs(xg).sum()
    assert st.cycles <= 20


def test_fullsize_levels_against_oracle_pieces(big):
    L, g, s = big
    seed = oracle.default_opts().seed
    nl = s.num_levels
    assert nl >= 5
    for l in range(nl):
        info = s.level_info(l)
        rp = L.lamg_level_copy(s.h, l, "row_ptr")
        col = L.lamg_level_copy(s.h, l, "col")
        w = L.lamg_level_copy(s.h, l, "w")
        n = info["n"]
        # colouring: the oracle's JP colouring of this level's graph, bit for bit
        colour = L.lamg_level_copy(s.h, l, "colour")
        assert np.array_equal(colour, oracle.colour(n, rp, col, _colour_key(seed, l))[0]), l
        if info["coarsest"]:
            continue
        # per-edge affinity, energy ratio and score from the GPU's own TVs
        X = L.lamg_level_copy(s.h, l, "tv")
        aff, q, score = oracle.edge_scores(n, rp, col, w, X)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "affinity").view(np.uint64), aff.view(np.uint64)), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "q").view(np.uint64), q.view(np.uint64)), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "score").view(np.uint64), score.view(np.uint64)), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "hub").astype(bool), oracle.hubs(n, rp, col, w)), l
        # aggregation: the oracle's scan on this level's CSR, scores and hubs, bit for bit
        agg = L.lamg_level_copy(s.h, l, "agg")
        nc = info["nc"]
        agg_o, state_o, ai = oracle.aggregate(n, rp, col, w, score, oracle.hubs(n, rp, col, w), level=l)
        assert np.array_equal(agg, agg_o), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "state"), state_o), l
        assert ai["nc"] == nc and ai["alpha"] == info["alpha"], l
        # Galerkin: the oracle's canonical sums give the next level bit for bit
        rpo, colo, wo = oracle.galerkin(n, rp, col, w, agg, nc)
        # Galerkin: the next level's weights are P^T W P off the diagonal
        A = sp.csr_matrix((w, col, rp), shape=(n, n))
        P = sp.csr_matrix((np.ones(n), agg, np.arange(n + 1)), shape=(n, nc))
        Wc = (P.T @ A @ P).tocsr()
        Wc.setdiag(0.0)
        Wc.eliminate_zeros()
        Wc.sort_indices()
        rpc = L.lamg_level_copy(s.h, l + 1, "row_ptr")
        colc = L.lamg_level_copy(s.h, l + 1, "col")
        wc = L.lamg_level_copy(s.h, l + 1, "w")
        assert np.array_equal(rpo, rpc) and np.array_equal(colo, colc), l
        assert np.array_equal(wo.view(np.uint64), wc.view(np.uint64)), l
        # and SciPy's P^T W P (another summation order) within rounding
        assert np.array_equal(Wc.indptr.astype(np.int64), rpc) and np.array_equal(Wc.indices, colc), l
        assert np.max(np.abs(Wc.data - wc)) <= 1e-12 * np.max(np.abs(wc)), l


# --------------------------------------------------------------------------- #
# The same workload with low-degree elimination levels (Sec. 3.2, elim = 1)
# --------------------------------------------------------------------------- #

@pytest.fixture(scope="module")
def big_elim():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg as L
    g = W.config_graph("chung_lu1m")
    s = L.Solver.from_graph(g, w_dtype=torch.float32, keep_setup_data=1, validate=1, max_cycles=2000, elim=1)
    yield L, g, s
    s.close()


def _elim_key(seed, l):
    return oracle.splitmix64(oracle.splitmix64(seed) ^ ((2 * l + 1) << 32) ^ (1 << 63))


def test_fullsize_elim_levels_against_oracle_pieces(big_elim):
    L, g, s = big_elim
    seed = oracle.default_opts().seed
    nl = s.num_levels
    kinds = ""
    for l in range(nl):
        info = s.level_info(l)
        rp = L.lamg_level_copy(s.h, l, "row_ptr")
        col = L.lamg_level_copy(s.h, l, "col")
        w = L.lamg_level_copy(s.h, l, "w")
        n = info["n"]
        colour = L.lamg_level_copy(s.h, l, "colour")
        if info["elim"]:   # a level followed by elimination never relaxes: one colour
            assert not colour.any() and info["ncolours"] == 1, l
        else:
            assert np.array_equal(colour, oracle.colour(n, rp, col, _colour_key(seed, l))[0]), l
        if info["coarsest"]:
            kinds += "C"
            continue
        if not info["elim"]:
            kinds += "A"
            X = L.lamg_level_copy(s.h, l, "tv")
            aff, q, score = oracle.edge_scores(n, rp, col, w, X)
            assert np.array_equal(L.lamg_level_copy(s.h, l, "score").view(np.uint64), score.view(np.uint64)), l
            continue
        kinds += "E"
        # the eliminated set: the oracle's sweep on this level's own graph
        cidx, nF = oracle.elim_set(n, rp, col, _elim_key(seed, l))
        assert np.array_equal(L.lamg_level_copy(s.h, l, "cidx"), cidx), l
        assert info["nF"] == nF
        # the next level: the Schur complement A_CC - A_CF A_FF^-1 A_FC (SciPy)
        A = sp.csr_matrix((w, col, rp), shape=(n, n))
        d = np.asarray(A.sum(axis=1)).ravel()
        Lap = sp.diags(d) - A
        Cs, Fs = np.flatnonzero(cidx >= 0), np.flatnonzero(cidx < 0)
        S = (Lap[Cs][:, Cs] - Lap[Cs][:, Fs] @ sp.diags(1.0 / d[Fs]) @ Lap[Fs][:, Cs]).tocsr()
        Wc = -S
        Wc.setdiag(0.0)
        Wc.eliminate_zeros()
        Wc.sort_indices()
        rpc = L.lamg_level_copy(s.h, l + 1, "row_ptr")
        colc = L.lamg_level_copy(s.h, l + 1, "col")
        wc = L.lamg_level_copy(s.h, l + 1, "w")
        assert np.array_equal(Wc.indptr.astype(np.int64), rpc) and np.array_equal(Wc.indices, colc), l
        assert np.max(np.abs(Wc.data - wc)) <= 1e-12 * np.max(np.abs(wc)), l
    assert "E" in kinds, kinds


def test_fullsize_elim_solve_residual(big_elim):
    L, g, s = big_elim
    b = W.zero_sum_rhs(g.n, 2)
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=1e-8, precision=L.LAMG_FP32_IR)
    xg = x.cpu().numpy()
    A = sp.csr_matrix((g.w, g.col, g.rp), shape=(g.n, g.n))
    r = b - (np.asarray(A.sum(axis=1)).ravel() * xg - A @ xg)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(b)
    assert abs(xg.sum()) <= 1e-9 * np.abs(xg).sum()
