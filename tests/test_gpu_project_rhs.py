"""The project_rhs option: a right-hand side that is not zero-sum is replaced by
its compatible part, b minus its mean (per graph of a union, per column of a
batch), instead of being rejected.  Sec. 1 requires a zero-sum b; the
projection makes A x = b solvable in the least-squares sense, and its solution
is the pseudo-inverse solution A^+ b, which the dense oracle gives directly."""
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


def _dense(g, a=0, e=None):
    e = g.n if e is None else e
    rp = g.rp[a:e + 1] - g.rp[a]
    return oracle.laplacian_dense(e - a, rp, g.col[g.rp[a]:g.rp[e]] - a, g.w[g.rp[a]:g.rp[e]])


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_single_graph_projects_instead_of_rejecting(L, precision):
    g = W.chung_lu(3000, seed=41)
    tol = 1e-10 if precision == "fp64" else 1e-8
    p = L.LAMG_FP64 if precision == "fp64" else L.LAMG_FP32_IR
    b = W.zero_sum_rhs(g.n, 42) + 0.37
    bt = torch.tensor(b, device="cuda")
    keep = bt.clone()
    s0 = L.Solver.from_graph(g)
    with pytest.raises(L.LamgError) as e:
        s0.solve(bt, tol=tol, precision=p)
    assert e.value.status == L.LAMG_ERR_RHS_NOT_ZERO_SUM
    s = L.Solver.from_graph(g, project_rhs=1)
    x, st = s.solve(bt, tol=tol, precision=p)
    assert torch.equal(bt, keep)        # the caller's b is not modified
    xg = x.cpu().numpy()
    A = _dense(g)
    bc = b - b.mean()
    assert np.linalg.norm(bc - A @ xg) <= 1.01 * tol * np.linalg.norm(bc)
    assert st.rel_res <= tol
    assert abs(xg.sum()) <= 1e-9 * np.abs(xg).sum()
    xo = oracle.dense_pinv_solve(A, bc)
    assert np.linalg.norm(xg - xo) <= (1e-6 if precision == "fp64" else 1e-5) * np.linalg.norm(xo)
    # a b that is already zero-sum gives the same solution as without the option
    b2 = torch.tensor(W.zero_sum_rhs(g.n, 43), device="cuda")
    x1, _ = s.solve(b2, tol=1e-10)
    x2, _ = s0.solve(b2, tol=1e-10)
    assert torch.linalg.norm(x1 - x2) <= 1e-9 * torch.linalg.norm(x2)
    s.close()
    s0.close()


def test_union_projects_every_graph(L):
    u, gptr = W.er_batch(12, 200, 1500, seed=44)
    b = W.zero_sum_rhs_graphs(gptr, 45)
    G = len(gptr) - 1
    for k in range(G):
        b[gptr[k]:gptr[k + 1]] += 0.1 * (k + 1) * (-1) ** k
    s = L.Solver.from_graph(u, gptr=gptr, project_rhs=1)
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=1e-10)
    xg = x.cpu().numpy()
    assert st.rel_res <= 1e-10
    for k in range(G):
        a, e = gptr[k], gptr[k + 1]
        bc = b[a:e] - b[a:e].mean()
        A = _dense(u, a, e)
        assert np.linalg.norm(bc - A @ xg[a:e]) <= 1.01e-10 * np.linalg.norm(bc)
        assert abs(xg[a:e].sum()) <= 1e-9 * np.abs(xg[a:e]).sum()
    s.close()


def test_batched_projects_every_column(L):
    g = W.grid2d(20, 15)
    rng = np.random.default_rng(46)
    B = rng.normal(size=(g.n, 6))
    B += np.array([0.0, 1.0, -2.0, 0.5, 3.0, 0.0])
    Bt = torch.tensor(B, device="cuda")
    keep = Bt.clone()
    s = L.Solver.from_graph(g, project_rhs=1)
    X, stats = s.solve_batched(Bt, tol=1e-10)
    assert torch.equal(Bt, keep)
    Xg = X.cpu().numpy()
    A = _dense(g)
    for c in range(B.shape[1]):
        bc = B[:, c] - B[:, c].mean()
        assert stats[c].status == 0 and stats[c].rel_res <= 1e-10
        assert np.linalg.norm(bc - A @ Xg[:, c]) <= 1.01e-10 * np.linalg.norm(bc)
        xs, _ = s.solve(torch.tensor(np.ascontiguousarray(B[:, c]), device="cuda"), tol=1e-10)
        assert np.linalg.norm(Xg[:, c] - xs.cpu().numpy()) <= 1e-8 * np.linalg.norm(Xg[:, c])
    s.close()
