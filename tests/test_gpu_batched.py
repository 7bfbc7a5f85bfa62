"""Batched solves (many right-hand sides on one hierarchy) against single solves
and the FP64 oracle, through the C-ABI."""
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


def _rhs(n, R, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, R))
    return B - B.mean(axis=0, keepdims=True)


@pytest.mark.parametrize("gname,R", [("chung_lu", 5), ("grid2d", 64), ("rgg", 130)])
def test_batched_fp64_matches_single_and_oracle(L, gname, R):
    g = {"chung_lu": lambda: W.chung_lu(6000, seed=13), "grid2d": lambda: W.grid2d(40, 30),
         "rgg": lambda: W.rgg2d(3000, seed=14)}[gname]()
    s = L.Solver.from_graph(g)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    B = _rhs(g.n, R, 7)
    Bt = torch.tensor(B, device="cuda")
    X, stats = s.solve_batched(Bt, tol=1e-10)
    Xg = X.cpu().numpy()
    A = oracle.laplacian_dense(g.n, g.rp, g.col, g.w) if g.n <= 3000 else None
    for c in sorted({0, R // 2, R - 1}):
        # per column: the same iteration as a single solve of that column
        xs, st1 = s.solve(torch.tensor(np.ascontiguousarray(B[:, c]), device="cuda"), tol=1e-10)
        assert abs(stats[c].cycles - st1.cycles) <= 1, (c, stats[c].cycles, st1.cycles)
        assert stats[c].rel_res <= 1e-10 and stats[c].status == 0
        xo, _ = h.solve(B[:, c], tol=1e-12)
        assert np.linalg.norm(Xg[:, c] - xo) <= 1e-6 * np.linalg.norm(xo)
        assert np.linalg.norm(Xg[:, c] - xs.cpu().numpy()) <= 1e-6 * np.linalg.norm(xo)
        assert abs(Xg[:, c].sum()) <= 1e-12 * np.abs(Xg[:, c]).sum()
        if A is not None:
            assert np.linalg.norm(B[:, c] - A @ Xg[:, c]) <= 1.01e-10 * np.linalg.norm(B[:, c])
    assert all(st.rel_res <= 1e-10 for st in stats)
    s.close()


def test_batched_fp32_ir(L):
    g = W.chung_lu(8000, seed=21)
    s = L.Solver.from_graph(g)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    B = _rhs(g.n, 16, 8)
    X, stats = s.solve_batched(torch.tensor(B, device="cuda"), tol=1e-8, precision=L.LAMG_FP32_IR)
    Xg = X.cpu().numpy()
    assert all(st.rel_res <= 1e-8 and st.status == 0 for st in stats)
    for c in (0, 9, 15):
        xo, _ = h.solve(B[:, c], tol=1e-12)
        assert np.linalg.norm(Xg[:, c] - xo) <= 1e-6 * np.linalg.norm(xo)
    s.close()


def test_batched_strided_initial_guess_and_zero_column(L):
    g = W.grid2d(30, 30)
    s = L.Solver.from_graph(g)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    B = _rhs(g.n, 3, 9)
    B[:, 1] = 0.0
    # columns 0..2 of a wider (n, 8) buffer: ld = 8 > nrhs
    Bw = torch.zeros(g.n, 8, dtype=torch.float64, device="cuda")
    Xw = torch.full((g.n, 8), 7.0, dtype=torch.float64, device="cuda")
    Bw[:, :3] = torch.tensor(B, device="cuda")
    x0 = torch.tensor(np.random.default_rng(3).normal(size=(g.n, 3)), device="cuda")
    x0[:, 1] = 0.0
    Xw[:, :3] = x0
    stats = L.lamg_solve_batched(s.h, Bw[:, :3], Xw[:, :3], tol=1e-10)
    Xg = Xw.cpu().numpy()
    assert np.all(Xg[:, 3:] == 7.0)          # columns outside the view untouched
    assert np.all(Xg[:, 1] == 0.0) and stats[1].cycles == 0
    for c in (0, 2):
        xo, _ = h.solve(B[:, c], tol=1e-12)
        assert np.linalg.norm(Xg[:, c] - xo) <= 1e-6 * np.linalg.norm(xo)
    s.close()


def test_batched_rejects_non_zero_sum_column(L):
    g = W.grid2d(12, 12)
    s = L.Solver.from_graph(g)
    B = _rhs(g.n, 4, 10)
    B[:, 2] += 1.0
    with pytest.raises(L.LamgError) as e:
        s.solve_batched(torch.tensor(B, device="cuda"))
    assert e.value.status == L.LAMG_ERR_RHS_NOT_ZERO_SUM
    assert "column 2" in str(e.value)
    s.close()


def test_autotune_batched_and_cache(L, tmp_path):
    g = W.chung_lu(6000, seed=13)
    s = L.Solver.from_graph(g)
    B = _rhs(g.n, 64, 11)
    cache = str(tmp_path / "tune.json")
    cols = s.autotune_batched(64, precision=L.LAMG_FP32_IR, cache=cache)
    assert cols in (16, 32, 64, 128)
    import json
    table = json.load(open(cache))
    (key, entry), = table.items()
    assert entry["cols"] == cols and all(v > 0 for v in entry["ms"].values())
    X, stats = s.solve_batched(torch.tensor(B, device="cuda"), tol=1e-8, precision=L.LAMG_FP32_IR)
    assert all(st.rel_res <= 1e-8 for st in stats)
    # a second handle takes the cached value without timing
    s2 = L.Solver.from_graph(g)
    assert s2.autotune_batched(64, precision=L.LAMG_FP32_IR, cache=cache) == cols
    # every chunk width gives the same solutions within the solve tolerance
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    for c in (16, 128):
        L.lamg_set_batch_cols(s2.h, c)
        X2, st2 = s2.solve_batched(torch.tensor(B, device="cuda"), tol=1e-10)
        xo, _ = h.solve(B[:, 5], tol=1e-12)
        assert np.linalg.norm(X2.cpu().numpy()[:, 5] - xo) <= 1e-6 * np.linalg.norm(xo)
    with pytest.raises(L.LamgError):
        L.lamg_set_batch_cols(s2.h, 12)
    s.close()
    s2.close()
