"""Seeded synthetic graphs and right-hand sides for LAMG tests and benchmarks.

This module holds input generators only -- none of the method's arithmetic --
so that both the CUDA library's tests/benchmarks and the CPU oracle can be fed
identical inputs.  Every graph is returned as ``Graph(n, rp, col, w)``: a
symmetric CSR of the off-diagonal pattern of the Laplacian (Eq. (1.2) of the
paper), both directions of every edge, columns strictly increasing per row,
no self loops, int64 row pointers, int32 columns, float64 weights.  Generators
that can produce several components keep the largest connected component.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    rp: np.ndarray   # int64 [n+1]
    col: np.ndarray  # int32 [nnz]
    w: np.ndarray    # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.size)

    @property
    def m(self) -> int:
        return self.nnz // 2

    def edges(self):
        """Undirected edge list (u < v) in CSR order: (eu, ev, w)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rp))
        keep = rows < self.col
        return rows[keep].astype(np.int32), self.col[keep].astype(np.int32), self.w[keep].copy()


def from_edges(n: int, u, v, w, name: str = "") -> Graph:
    """CSR from an undirected edge list with u != v and no repeated pair."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    assert u.shape == v.shape == w.shape
    assert not np.any(u == v), "self loops"
    r = np.concatenate([u, v])
    c = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    order = np.lexsort((c, r))
    r, c, ww = r[order], c[order], ww[order]
    if r.size > 1:
        dup = (r[1:] == r[:-1]) & (c[1:] == c[:-1])
        assert not np.any(dup), "repeated edge"
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, r + 1, 1)
    rp = np.cumsum(rp)
    return Graph(n, rp, c.astype(np.int32), ww, name)


def _dedupe(u, v):
    """Unique undirected pairs (lo, hi) with lo != hi, sorted."""
    lo = np.minimum(u, v).astype(np.int64)
    hi = np.maximum(u, v).astype(np.int64)
    keep = lo != hi
    key = np.unique(lo[keep] * (1 << 32) + hi[keep])
    return (key >> 32).astype(np.int64), (key & 0xFFFFFFFF).astype(np.int64)


def largest_component(g: Graph) -> Graph:
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    A = sp.csr_matrix((np.ones(g.nnz), g.col, g.rp), shape=(g.n, g.n))
    nc, lab = connected_components(A, directed=False)
    if nc == 1:
        return g
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    newid = -np.ones(g.n, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    eu, ev, w = g.edges()
    sel = (newid[eu] >= 0) & (newid[ev] >= 0)
    return from_edges(keep.size, newid[eu[sel]], newid[ev[sel]], w[sel], g.name)


# --------------------------------------------------------------------------- #
# Small graphs
# --------------------------------------------------------------------------- #

def five_node() -> Graph:
    """The paper's 5-node example (Fig. 1.1); nodes renumbered 0..4."""
    eu = [0, 0, 0, 0, 1, 2]
    ev = [1, 2, 3, 4, 3, 3]
    w = [1.0, 1.0, 1.0, 5.0, 1.0, 2.0]
    return from_edges(5, eu, ev, w, "five_node")


def path(n: int, w: float = 1.0) -> Graph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, np.full(n - 1, w), f"path{n}")


def star(n: int) -> Graph:
    return from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), np.ones(n - 1), f"star{n}")


def complete(n: int) -> Graph:
    u, v = np.triu_indices(n, 1)
    return from_edges(n, u, v, np.ones(u.size), f"complete{n}")


def grid2d(nx: int, ny: int, wx: float = 1.0, wy: float = 1.0) -> Graph:
    """5-point grid Laplacian with free (Neumann) boundary; node id = i + nx*j."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    us = [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
    vs = [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    ws = [np.full(us[0].size, wx), np.full(us[1].size, wy)]
    return from_edges(nx * ny, np.concatenate(us), np.concatenate(vs), np.concatenate(ws),
                      f"grid{nx}x{ny}")


def grid2d_stencil(nx: int, kind: str) -> Graph:
    """nx x nx grid Laplacians with negative weights (Sec. 5, grids with negative
    weights), free boundary (Neumann); node (i, j) = i + nx j, i along x.  Edge
    weights w_uv = -a_uv, so A = D - W has zero row sums:
      '13pt':  the 13-point 4th-order stencil [1 -16 60 -16 1] / 12 along x and y:
               w = 16/12 between neighbours at distance 1, w = -1/12 at distance 2;
      'rot_c': Eq. (5.1) with alpha = -pi/4, eps = 1e-2, the 5-point U_xx, U_yy and
               the alignment-agnostic cross term (1/4h^2)[-1 0 1; 0 0 0; 1 0 -1],
               halved: w = .2525 to the four axis neighbours, .12375 to the NW and
               SE neighbours, -.12375 to the NE and SW neighbours (centre 1.01);
      'rot_d': the same with the cross term aligned to the NE/SW neighbours,
               (1/2h^2)[0 -1 1; -1 2 -1; 1 -1 0], halved: w = .5 to the axis
               neighbours and -.2475 to the NE and SW neighbours (centre 1.505)."""
    i, j = np.meshgrid(np.arange(nx), np.arange(nx), indexing="xy")
    i, j = i.ravel(), j.ravel()
    idx = i + nx * j
    if kind == "13pt":
        offs = [((1, 0), 16.0 / 12.0), ((0, 1), 16.0 / 12.0), ((2, 0), -1.0 / 12.0), ((0, 2), -1.0 / 12.0)]
    elif kind == "rot_c":
        a, b, c = 0.505, -0.99, 0.505           # cos^2 + eps sin^2, (1 - eps) sin 2alpha, eps cos^2 + sin^2
        offs = [((1, 0), a / 2), ((0, 1), c / 2), ((-1, 1), -b / 8), ((1, 1), b / 8)]
    elif kind == "rot_d":
        a, b, c = 0.505, -0.99, 0.505
        offs = [((1, 0), (a - b / 2) / 2), ((0, 1), (c - b / 2) / 2), ((1, 1), b / 4)]
    else:
        raise ValueError(kind)
    us, vs, ws = [], [], []
    for (di, dj), wt in offs:
        ok = (i + di >= 0) & (i + di < nx) & (j + dj >= 0) & (j + dj < nx)
        us.append(idx[ok])
        vs.append((i + di + nx * (j + dj))[ok])
        ws.append(np.full(int(ok.sum()), wt))
    u, v, w = np.concatenate(us), np.concatenate(vs), np.concatenate(ws)
    return from_edges(nx * nx, np.minimum(u, v), np.maximum(u, v), w, f"grid{nx}_{kind}")


def grid2d_periodic(nx: int) -> Graph:
    """5-point nx x nx grid Laplacian with periodic boundary (a torus), unit
    weights; node id = i + nx*j; nx >= 3."""
    idx = np.arange(nx * nx).reshape(nx, nx)
    us = [idx.ravel(), idx.ravel()]
    vs = [np.roll(idx, -1, axis=1).ravel(), np.roll(idx, -1, axis=0).ravel()]
    u, v = np.concatenate(us), np.concatenate(vs)
    return from_edges(nx * nx, np.minimum(u, v), np.maximum(u, v), np.ones(u.size), f"torus{nx}")


def grid3d(nx: int, ny: int, nz: int, wx=1.0, wy=1.0, wz=1.0) -> Graph:
    """7-point grid Laplacian with free boundary; node id = i + nx*(j + ny*k).

    Built directly as a CSR (no sort) so that 256^3 stays cheap."""
    n = nx * ny * nz
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    # neighbours in increasing id order: -z, -y, -x, +x, +y, +z
    offs = [(-nx * ny, z > 0, wz), (-nx, y > 0, wy), (-1, x > 0, wx),
            (1, x < nx - 1, wx), (nx, y < ny - 1, wy), (nx * ny, z < nz - 1, wz)]
    deg = np.zeros(n, dtype=np.int64)
    for _, m, _ in offs:
        deg += m
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rp[1:])
    col = np.empty(int(rp[-1]), dtype=np.int32)
    w = np.empty(int(rp[-1]), dtype=np.float64)
    pos = rp[:-1].copy()
    for d, m, wv in offs:
        sel = np.flatnonzero(m)
        col[pos[sel]] = (sel + d).astype(np.int32)
        w[pos[sel]] = wv
        pos[sel] += 1
    return Graph(n, rp, col, w, f"grid{nx}x{ny}x{nz}")


# --------------------------------------------------------------------------- #
# Random graphs of the benchmark configurations
# --------------------------------------------------------------------------- #

def chung_lu(n: int, beta: float = 2.5, mean_deg: float = 10.0, seed: int = 2,
             wlo: float = 0.5, whi: float = 2.0, i0: float | None = None) -> Graph:
    """Power-law expected-degree graph, largest component.

    Expected degrees d_i proportional to (i + i0)^(-1/(beta-1)), scaled to the
    mean; edges are drawn as M ~ Poisson(sum d / 2) independent pairs whose
    endpoints are chosen proportionally to d (the edge-sampling form of the
    Chung-Lu model); self loops and repeats are dropped.  Weights are uniform
    in [wlo, whi], rounded to FP32 (and stored exactly in FP64)."""
    rng = np.random.default_rng(seed)
    if i0 is None:
        i0 = max(1.0, n ** 0.05)
    d = (np.arange(n) + i0) ** (-1.0 / (beta - 1.0))
    d *= mean_deg * n / d.sum()
    M = rng.poisson(d.sum() / 2.0)
    p = d / d.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    u = np.searchsorted(cdf, rng.random(M), side="right")
    v = np.searchsorted(cdf, rng.random(M), side="right")
    lo, hi = _dedupe(u, v)
    perm = rng.permutation(n)               # shuffle ids so degree is not monotone in id
    lo, hi = perm[lo], perm[hi]
    w = rng.uniform(wlo, whi, lo.size).astype(np.float32).astype(np.float64)
    return largest_component(from_edges(n, lo, hi, w, f"chung_lu{n}"))


def rgg2d(n: int, mean_deg: float = 12.0, seed: int = 4) -> Graph:
    """Random geometric graph in the unit square, radius r = sqrt(mean_deg / (pi n)),
    weights exp(-d^2 / sigma^2) with sigma = r; largest component."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = np.sqrt(mean_deg / (np.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    u, v = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    d2 = np.sum((pts[u] - pts[v]) ** 2, axis=1)
    w = np.exp(-d2 / (r * r))
    return largest_component(from_edges(n, u, v, w, f"rgg{n}"))


def erdos_renyi(n: int, mean_deg: float = 8.0, seed: int = 5) -> Graph:
    """G(n, p) with p = mean_deg / (n - 1): M ~ Binomial(n(n-1)/2, p) uniform pairs
    (repeats dropped), unit weights, largest component."""
    rng = np.random.default_rng(seed)
    M = rng.binomial(n * (n - 1) // 2, mean_deg / (n - 1))
    u = rng.integers(0, n, M)
    v = rng.integers(0, n, M)
    lo, hi = _dedupe(u, v)
    return largest_component(from_edges(n, lo, hi, np.ones(lo.size), f"er{n}"))


def knn_gmm(n: int = 500_000, dim: int = 16, k: int = 10, ncomp: int = 10, seed: int = 6,
            device: str = "cpu", block: int = 4096, components: bool = False):
    """k-nearest-neighbour graph (union-symmetrised) on points from a Gaussian
    mixture (means ~ N(0, 3^2 I), unit covariance, equal weights); Gaussian edge
    weights exp(-d^2/sigma^2), sigma = mean k-th neighbour distance, rounded to
    FP32.  Returns (graph of the largest component, labels, points)."""
    import torch

    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, 3.0, (ncomp, dim))
    lab = rng.integers(0, ncomp, n)
    pts = means[lab] + rng.normal(0.0, 1.0, (n, dim))
    P = torch.tensor(pts, dtype=torch.float32, device=device)
    sq = (P * P).sum(1)
    nbr = np.empty((n, k), dtype=np.int64)
    dist = np.empty((n, k), dtype=np.float64)
    for s in range(0, n, block):
        Q = P[s:s + block]
        d2 = sq[s:s + block, None] + sq[None, :] - 2.0 * (Q @ P.T)
        d2[torch.arange(Q.shape[0], device=device), torch.arange(s, s + Q.shape[0], device=device)] = float("inf")
        val, idx = torch.topk(d2, k, dim=1, largest=False)
        nbr[s:s + block] = idx.cpu().numpy()
        dist[s:s + block] = val.clamp_min(0).sqrt().cpu().numpy()
    sigma = float(dist[:, -1].mean())
    u = np.repeat(np.arange(n), k)
    v = nbr.ravel()
    lo, hi = _dedupe(u, v)
    d2 = np.sum((pts[lo] - pts[hi]) ** 2, axis=1)
    w = np.exp(-d2 / (sigma * sigma)).astype(np.float32).astype(np.float64)
    w = np.maximum(w, np.float64(np.finfo(np.float32).tiny))
    g = from_edges(n, lo, hi, w, f"knn{n}")
    if components:
        # every connected component, renumbered so that each is a contiguous
        # node range: (union graph, gptr, labels, points) for lamg_setup_graphs
        import scipy.sparse as sp
        import scipy.sparse.csgraph as cg
        A = sp.csr_matrix((g.w, g.col, g.rp), shape=(n, n))
        nc, comp = cg.connected_components(A, directed=False)
        order = np.argsort(comp, kind="stable")
        inv = np.empty(n, dtype=np.int64)
        inv[order] = np.arange(n)
        gu = from_edges(n, inv[lo], inv[hi], w, f"knn{n}_components")
        gptr = np.zeros(nc + 1, dtype=np.int64)
        gptr[1:] = np.cumsum(np.bincount(comp, minlength=nc))
        return gu, gptr, lab[order], pts[order]
    g2 = largest_component(g)
    return g2, lab, pts


def block_union(graphs) -> tuple[Graph, np.ndarray]:
    """Block-diagonal union of graphs: graph g's nodes are renumbered to
    gptr[g] .. gptr[g+1]-1.  Returns (union graph, gptr int64[G+1])."""
    gptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        gptr[k + 1] = gptr[k] + g.n
    rp = [np.zeros(1, dtype=np.int64)]
    off = 0
    for g in graphs:
        rp.append(g.rp[1:] + off)
        off += int(g.rp[-1])
    col = np.concatenate([g.col.astype(np.int64) + gptr[k] for k, g in enumerate(graphs)]).astype(np.int32)
    w = np.concatenate([g.w for g in graphs])
    return Graph(int(gptr[-1]), np.concatenate(rp), col, w, f"union{len(graphs)}"), gptr


def er_batch_sizes(count: int, n_lo: int, n_hi: int, seed: int = 7) -> np.ndarray:
    """Node counts (before taking the largest component) of the graphs of er_batch."""
    return np.random.default_rng(seed).integers(n_lo, n_hi + 1, count)


def er_batch(count: int, n_lo: int, n_hi: int, mean_deg: float = 8.0, seed: int = 7, only=None):
    """`count` Erdos-Renyi graphs (largest components) with n uniform in [n_lo, n_hi],
    as one block-diagonal union: returns (union graph, gptr).  Every graph has its
    own seed, so `only` (graph indices) builds the union of a subset, in that order."""
    sizes = er_batch_sizes(count, n_lo, n_hi, seed)
    ks = range(count) if only is None else only
    return block_union([erdos_renyi(int(sizes[k]), mean_deg, seed=int(seed * 100003 + k)) for k in ks])


def zero_sum_rhs_graphs(gptr, seed: int) -> np.ndarray:
    """Gaussian right-hand side with the mean removed on every graph's node range."""
    rng = np.random.default_rng(seed)
    b = rng.normal(size=int(gptr[-1]))
    for g in range(len(gptr) - 1):
        b[gptr[g]:gptr[g + 1]] -= b[gptr[g]:gptr[g + 1]].mean()
    return b


def zero_sum_rhs(n: int, seed: int, count: int | None = None) -> np.ndarray:
    """Gaussian right-hand side(s) with the mean removed (Sec. 1: b must be zero-sum)."""
    rng = np.random.default_rng(seed)
    if count is None:
        b = rng.normal(size=n)
        return b - b.mean()
    B = rng.normal(size=(n, count))
    return B - B.mean(axis=0, keepdims=True)


# --------------------------------------------------------------------------- #
# The benchmark configurations
# --------------------------------------------------------------------------- #

def config_graph(name: str) -> Graph:
    """'grid64': 64x64 5-point grid; 'chung_lu1m': Chung-Lu n=1M, beta 2.5, mean degree 10;
    'grid256': 256^3 7-point grid, weights 1/1/0.01 ('grid128': the 128^3 member of that
    family, small enough for an ncu capture); 'rgg2m': 2M-node RGG, mean degree 12;
    'grid1024': 1024x1024 5-point grid, unit weights (the paper's grid table size).
    'torus1024': 1024x1024 periodic 5-point grid."""
    if name == "grid64":
        return grid2d(64, 64)
    if name == "grid1024":
        return grid2d(1024, 1024)
    if name == "chung_lu1m":
        return chung_lu(1_000_000, 2.5, 10.0, seed=2)
    if name == "grid256":
        return grid3d(256, 256, 256, 1.0, 1.0, 0.01)
    if name == "grid128":
        return grid3d(128, 128, 128, 1.0, 1.0, 0.01)
    if name == "rgg2m":
        return rgg2d(2_000_000, 12.0, seed=4)
    if name.startswith("grid1024_"):
        return grid2d_stencil(1024, name.split("_", 1)[1])
    if name == "torus1024":
        return grid2d_periodic(1024)
    raise KeyError(name)
