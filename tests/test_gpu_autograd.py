"""The differentiable solve (torch.autograd.Function over lamg_setup/solve/adjoint)
against central finite differences and the oracle's adjoint."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def AG():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import autograd
    assert torch.cuda.is_available()
    return autograd


def _problem(n=2000, seed=3):
    """Semi-supervised setting on a kNN graph of Gaussian-mixture points: sources at
    1% labelled nodes (zero-sum), loss on a held-out 5%."""
    g, _, _ = W.knn_gmm(n, dim=16, k=10, seed=seed)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    lab = perm[: max(2, g.n // 100)]
    held = perm[g.n // 100: g.n // 100 + g.n // 20]
    y = rng.integers(0, 2, g.n).astype(np.float64)
    b = np.zeros(g.n)
    b[lab] = y[lab] - y[lab].mean()
    t = y[held] - 0.5
    return g, b, held, t


def _loss(x, held, t):
    return ((x[held] - t) ** 2).sum()


@pytest.mark.parametrize("wdt", [torch.float64, torch.float32])
def test_gradients_match_finite_differences(AG, wdt):
    g, b, held, t = _problem()
    eu, ev, w = g.edges()
    dev = "cuda"
    P = AG.GraphPattern(g.n, torch.tensor(eu, device=dev), torch.tensor(ev, device=dev))
    wt = torch.tensor(w, device=dev, dtype=wdt, requires_grad=True)
    bt = torch.tensor(b, device=dev, requires_grad=True)
    heldt = torch.tensor(held, device=dev)
    tt = torch.tensor(t, device=dev)
    x = AG.laplacian_solve(wt, bt, P, tol=1e-12)
    loss = _loss(x, heldt, tt)
    loss.backward()
    gw = wt.grad.double().cpu().numpy()
    gb = bt.grad.cpu().numpy()
    assert wt.grad.dtype == wdt
    assert abs(gb.sum()) <= 1e-10 * np.abs(gb).sum()     # dL/db lies in the zero-sum subspace

    def L_of(wv, bv):
        with torch.no_grad():
            xv = AG.laplacian_solve(torch.tensor(wv, device=dev, dtype=torch.float64),
                                    torch.tensor(bv, device=dev), P, tol=1e-12)
            return float(_loss(xv, heldt, tt))

    rng = np.random.default_rng(5)
    w64 = wt.detach().double().cpu().numpy()
    # directional derivative along a relative weight perturbation
    d = rng.uniform(-1, 1, w64.size) * w64
    eps = 1e-5
    fd = (L_of(w64 + eps * d, b) - L_of(w64 - eps * d, b)) / (2 * eps)
    assert abs(fd - gw @ d) <= 1e-5 * abs(fd) + 1e-12
    # single edges with the largest gradients
    for e in np.argsort(-np.abs(gw))[:3]:
        de = np.zeros_like(w64)
        de[e] = w64[e]
        fde = (L_of(w64 + eps * de, b) - L_of(w64 - eps * de, b)) / (2 * eps)
        assert abs(fde - gw[e] * w64[e]) <= 1e-5 * abs(fde) + 1e-12
    # zero-sum direction in b
    e_b = rng.normal(size=b.size)
    e_b -= e_b.mean()
    fdb = (L_of(w64, b + eps * e_b) - L_of(w64, b - eps * e_b)) / (2 * eps)
    assert abs(fdb - gb @ e_b) <= 1e-6 * abs(fdb) + 1e-12
    P.close()


def test_gradient_matches_oracle_adjoint(AG):
    g, b, held, t = _problem(1500, seed=4)
    eu, ev, w = g.edges()
    dev = "cuda"
    P = AG.GraphPattern(g.n, torch.tensor(eu, device=dev), torch.tensor(ev, device=dev))
    wt = torch.tensor(w, device=dev, requires_grad=True)
    bt = torch.tensor(b, device=dev, requires_grad=True)
    x = AG.laplacian_solve(wt, bt, P, tol=1e-12)
    loss = _loss(x, torch.tensor(held, device=dev), torch.tensor(t, device=dev))
    loss.backward()
    xn = x.detach().cpu().numpy()
    gx = np.zeros(g.n)
    gx[held] = 2.0 * (xn[held] - t)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    lo, dwo = h.adjoint(xn, gx, eu, ev, tol=1e-12)
    assert np.linalg.norm(bt.grad.cpu().numpy() - lo) <= 1e-8 * np.linalg.norm(lo)
    assert np.linalg.norm(wt.grad.cpu().numpy() - dwo) <= 1e-8 * np.linalg.norm(dwo)
    P.close()
