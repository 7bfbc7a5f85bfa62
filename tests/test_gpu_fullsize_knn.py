"""Parity at the full size of the kNN workload of the adjoint benchmark: 500k
points of a 10-cluster Gaussian mixture in 16-D, k = 10, Gaussian weights in
FP32, every connected component solved as one block-diagonal union.

- The setup, level by level, against the oracle's pieces recomputed from the
  GPU's own level data (colouring, affinities / energy ratios / scores from the
  GPU's test vectors, hubs, the aggregation scan and the Galerkin operator), bit
  for bit.
- The forward solve and the adjoint by their FP64 residuals, per component.
- The gradient of a held-out loss against central finite differences along 16
  random directions of relative weight perturbation and on the 100 edges with
  the largest gradient (the differentiable solve over the Laplacian of
  Eq. (1.1))."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import autograd as AG
    from paper_1108_1310_gb300 import lamg as L
    assert torch.cuda.is_available()
    g, gptr, _, _ = W.knn_gmm(500_000, dim=16, k=10, seed=6, device="cuda", components=True)
    return L, AG, g, gptr


def _colour_key(seed, l):
    return oracle.splitmix64(oracle.splitmix64(seed) ^ ((2 * l + 1) << 32))


def _semi_supervised(g, gptr, seed=6):
    """Zero-sum sources on 1% labelled nodes of every component; loss targets on 5%."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    lab, held = perm[: g.n // 100], perm[g.n // 100: g.n // 100 + g.n // 20]
    y = rng.integers(0, 2, g.n).astype(np.float64)
    labelled = np.zeros(g.n, dtype=bool)
    labelled[lab] = True
    b = np.zeros(g.n)
    for c in range(len(gptr) - 1):
        idx = np.arange(gptr[c], gptr[c + 1])[labelled[gptr[c]:gptr[c + 1]]]
        if idx.size >= 2:
            b[idx] = y[idx] - y[idx].mean()
    return b, held, y[held] - 0.5


def test_knn_levels_against_oracle_pieces(knn):
    L, _, g, gptr = knn
    assert g.n == 500_000 and len(gptr) - 1 >= 2
    s = L.Solver.from_graph(g, w_dtype=torch.float32, gptr=gptr, keep_setup_data=1, validate=1)
    seed = oracle.default_opts().seed
    nl = s.num_levels
    assert nl >= 4
    for l in range(nl):
        info = s.level_info(l)
        rp = L.lamg_level_copy(s.h, l, "row_ptr")
        col = L.lamg_level_copy(s.h, l, "col")
        w = L.lamg_level_copy(s.h, l, "w")
        n = info["n"]
        colour = L.lamg_level_copy(s.h, l, "colour")
        assert np.array_equal(colour, oracle.colour(n, rp, col, _colour_key(seed, l))[0]), l
        if info["coarsest"]:
            continue
        X = L.lamg_level_copy(s.h, l, "tv")
        aff, q, score = oracle.edge_scores(n, rp, col, w, X)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "affinity").view(np.uint64), aff.view(np.uint64)), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "q").view(np.uint64), q.view(np.uint64)), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "score").view(np.uint64), score.view(np.uint64)), l
        hub = oracle.hubs(n, rp, col, w)
        assert np.array_equal(L.lamg_level_copy(s.h, l, "hub").astype(bool), hub), l
        agg = L.lamg_level_copy(s.h, l, "agg")
        agg_o, state_o, ai = oracle.aggregate(n, rp, col, w, score, hub, level=l)
        assert np.array_equal(agg, agg_o), l
        assert np.array_equal(L.lamg_level_copy(s.h, l, "state"), state_o), l
        assert ai["nc"] == info["nc"] and ai["alpha"] == info["alpha"], l
        rpo, colo, wo = oracle.galerkin(n, rp, col, w, agg, info["nc"])
        assert np.array_equal(rpo, L.lamg_level_copy(s.h, l + 1, "row_ptr")), l
        assert np.array_equal(colo, L.lamg_level_copy(s.h, l + 1, "col")), l
        assert np.array_equal(wo.view(np.uint64), L.lamg_level_copy(s.h, l + 1, "w").view(np.uint64)), l
    s.close()


def test_knn_forward_and_adjoint_residuals(knn):
    L, _, g, gptr = knn
    s = L.Solver.from_graph(g, w_dtype=torch.float32, gptr=gptr, max_cycles=2000)
    b, held, t = _semi_supervised(g, gptr)
    A = sp.csr_matrix((g.w.astype(np.float32).astype(np.float64), g.col, g.rp), shape=(g.n, g.n))
    deg = np.asarray(A.sum(axis=1)).ravel()
    x, st = s.solve(torch.tensor(b, device="cuda"), tol=1e-8, precision=L.LAMG_FP32_IR)
    xg = x.cpu().numpy()
    gx = np.zeros(g.n)
    gx[held] = 2.0 * (xg[held] - t)
    lam = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    L.lamg_adjoint(s.h, x, torch.tensor(gx, device="cuda"), lam, None, None, None, tol=1e-8,
                   precision=L.LAMG_FP32_IR)
    lg = lam.cpu().numpy()
    for c in range(len(gptr) - 1):
        sl = slice(gptr[c], gptr[c + 1])
        rx = (b - (deg * xg - A @ xg))[sl]
        gc = gx[sl] - gx[sl].mean()
        rl = gc - (deg * lg - A @ lg)[sl]
        assert np.linalg.norm(rx) <= 1.01e-8 * np.linalg.norm(b[sl]) + 1e-300, c
        assert np.linalg.norm(rl) <= 1.01e-8 * np.linalg.norm(gc) + 1e-300, c
        assert abs(xg[sl].sum()) <= 1e-9 * np.abs(xg[sl]).sum() + 1e-300, c
    s.close()


def test_knn_gradients_match_finite_differences(knn):
    _, AG, g, gptr = knn
    b, held, t = _semi_supervised(g, gptr)
    eu, ev, w = g.edges()
    dev = "cuda"
    P = AG.GraphPattern(g.n, torch.tensor(eu, device=dev), torch.tensor(ev, device=dev), gptr=gptr,
                        max_cycles=2000)
    wt = torch.tensor(w, device=dev, requires_grad=True)
    bt = torch.tensor(b, device=dev)
    heldt = torch.tensor(held, device=dev)
    tt = torch.tensor(t, device=dev)

    def loss(x):
        return ((x[heldt] - tt) ** 2).sum()

    x = AG.laplacian_solve(wt, bt, P, tol=1e-12)
    loss(x).backward()
    gw = wt.grad.cpu().numpy()

    def L_of(wv):
        with torch.no_grad():
            return float(loss(AG.laplacian_solve(torch.tensor(wv, device=dev), bt, P, tol=1e-12)))

    eps = 1e-5
    rng = np.random.default_rng(8)
    # 16 directions of relative weight perturbation: the solves' error is ~1e-7 of
    # these directional derivatives (measured on the oracle at 50k points)
    for k in range(16):
        d = rng.uniform(-1, 1, w.size) * w
        fd = (L_of(w + eps * d) - L_of(w - eps * d)) / (2 * eps)
        assert abs(fd - gw @ d) <= 1e-5 * abs(fd), (k, fd, gw @ d)
    # the 100 edges with the largest |dL/dw_e| w_e: each moves the loss by ~1e-6 of
    # itself, so the finite differences carry more of the solves' error
    for e in np.argsort(-np.abs(gw * w))[:100]:
        de = np.zeros_like(w)
        de[e] = w[e]
        fd = (L_of(w + eps * de) - L_of(w - eps * de)) / (2 * eps)
        assert abs(fd - gw[e] * w[e]) <= 5e-5 * abs(fd), (e, fd, gw[e] * w[e])
    P.close()
