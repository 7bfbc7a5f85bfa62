"""Plain serial FP64 CPU reference of the LAMG path (Livne & Brandt, arXiv 1108.1310).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by ``bench.py``'s CPU-baseline leg.  The product (``paper_1108_1310_gb300``)
never imports it, and it imports nothing from the product.

The C source is ``lamg_oracle.c`` (compiled with ``-ffp-contract=off``); this
module builds it with gcc and exposes it through ctypes on numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lamg_oracle.c")
_LIB = os.path.join(_HERE, "liblamg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lamg_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("k_finest", C.c_int32), ("k_max", C.c_int32),
                ("k_step", C.c_int32), ("nu_tv", C.c_int32), ("nu1", C.c_int32),
                ("nu2", C.c_int32), ("n_coarsest", C.c_int32), ("q_max", C.c_double),
                ("hub_factor", C.c_double), ("weak_tol", C.c_double),
                ("alpha_stall", C.c_double), ("relax_fast_ratio", C.c_double),
                ("max_rounds", C.c_int32), ("max_levels", C.c_int32),
                ("dense_max", C.c_int32), ("coarse_sweeps", C.c_int32),
                ("mu_flat", C.c_double), ("seed", C.c_uint64), ("agg_rule", C.c_int32),
                ("elim", C.c_int32), ("elim_min_frac", C.c_double), ("lgmg_nx", C.c_int32),
                ("mu_adaptive", C.c_double), ("gamma_coarse_max", C.c_double), ("plain_sums", C.c_int32),
                ("gamma_fine_printed", C.c_int32), ("recomb_finest", C.c_int32),
                ("relax_rule", C.c_int32), ("colour_rule", C.c_int32),
                ("negative_weights", C.c_int32)]


_P = C.c_void_p
_I64, _I32, _D, _U64 = C.c_int64, C.c_int32, C.c_double, C.c_uint64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            sig = {
                "orc_default_opts": (None, [_P]),
                "orc_splitmix64": (_U64, [_U64]),
                "orc_canon_sum": (_D, [_P, _I64]),
                "orc_canon_sum_global": (_D, [_P, _I64]),
                "orc_canon_dot": (_D, [_P, _P, _I64]),
                "orc_validate": (_I32, [_I64, _P, _P, _P]),
                "orc_validate_signed": (_I32, [_I64, _P, _P, _P]),
                "orc_validate_graphs": (_I32, [_I64, _P, _P, _P, _I32, _P]),
                "orc_laplacian_dense": (None, [_I64, _P, _P, _P, _P]),
                "orc_colour": (_I32, [_I64, _P, _P, _U64, _P]),
                "orc_colour_lex": (_I32, [_I64, _P, _P, _P]),
                "orc_gs_sweep_lex": (None, [_I64, _P, _P, _P, _P, _P]),
                "orc_gs_sweep_colour": (None, [_I64, _P, _P, _P, _P, _I32, _P, _P]),
                "orc_edge_scores": (None, [_I64, _P, _P, _P, _I32, _P, _D, _D, _P, _P, _P]),
                "orc_hubs": (None, [_I64, _P, _P, _P, _D, _P]),
                "orc_dense_pinv_solve": (_I32, [_I64, _P, _P, _P]),
                "orc_setup": (_I32, [_I64, _P, _P, _P, _P, _P]),
                "orc_setup_graphs": (_I32, [_I64, _P, _P, _P, _I32, _P, _P, _P]),
                "orc_free": (None, [_P]),
                "orc_num_levels": (_I32, [_P]),
                "orc_level_info": (None, [_P, _I32, _P]),
                "orc_level_csr": (None, [_P, _I32, _P, _P, _P]),
                "orc_level_colour": (None, [_P, _I32, _P]),
                "orc_level_tv": (None, [_P, _I32, _P]),
                "orc_level_scores": (None, [_P, _I32, _P, _P, _P]),
                "orc_level_agg": (None, [_P, _I32, _P, _P, _P]),
                "orc_level_elim": (None, [_P, _I32, _P]),
                "orc_elim_set": (_I64, [_I64, _P, _P, _U64, _P]),
                "orc_aggregate": (None, [_I64, _P, _P, _P, _P, _P, _P, _I32, _P, _P, _P]),
                "orc_galerkin": (_I64, [_I64, _P, _P, _P, _P, _I64, _P, _P, _P]),
                "orc_solve": (_I32, [_P, _P, _P, _D, _I32, _I32, _P, _P]),
                "orc_cycle": (_I32, [_P, _P, _P, _I32]),
                "orc_adjoint": (_I32, [_P, _P, _P, _P, _P, _P, _I64, _P, _D, _I32, _I32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _csr(rp, col, w):
    return (np.ascontiguousarray(rp, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(w, dtype=np.float64))


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().orc_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def splitmix64(key: int) -> int:
    return int(lib().orc_splitmix64(key & 0xFFFFFFFFFFFFFFFF))


def canon_sum(t) -> float:
    t = np.ascontiguousarray(t, dtype=np.float64)
    return float(lib().orc_canon_sum(_p(t), t.size))


def canon_dot(a, b) -> float:
    """Canonical sum of the products a_i b_i, each lane advanced by a fused multiply-add."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert a.size == b.size
    return float(lib().orc_canon_dot(_p(a), _p(b), a.size))


def canon_sum_global(t) -> float:
    t = np.ascontiguousarray(t, dtype=np.float64)
    return float(lib().orc_canon_sum_global(_p(t), t.size))


def validate_graphs(n, rp, col, w, gptr) -> int:
    """Status of a block-diagonal union of graphs (node ranges gptr)."""
    rp, col, w = _csr(rp, col, w)
    gp = np.ascontiguousarray(gptr, dtype=np.int64)
    return int(lib().orc_validate_graphs(n, _p(rp), _p(col), _p(w), len(gp) - 1, _p(gp)))


def validate(n, rp, col, w, signed=False) -> int:
    rp, col, w = _csr(rp, col, w)
    f = lib().orc_validate_signed if signed else lib().orc_validate
    return int(f(n, _p(rp), _p(col), _p(w)))


def laplacian_dense(n, rp, col, w):
    rp, col, w = _csr(rp, col, w)
    A = np.zeros((n, n))
    lib().orc_laplacian_dense(n, _p(rp), _p(col), _p(w), _p(A))
    return A


def colour(n, rp, col, key):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    c = np.zeros(n, dtype=np.int32)
    nc = lib().orc_colour(n, _p(rp), _p(col), key & 0xFFFFFFFFFFFFFFFF, _p(c))
    return c, int(nc)


def colour_lex(n, rp, col):
    """Level sets of the lower-triangular dependency graph (relax_rule 1)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    c = np.zeros(n, dtype=np.int32)
    nc = lib().orc_colour_lex(n, _p(rp), _p(col), _p(c))
    return c, int(nc)


def elim_set(n, rp, col, key):
    """Eliminated set of a graph (Sec. 3.2): coarse index of each node, -1 in F."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    cidx = np.zeros(n, np.int32)
    nF = lib().orc_elim_set(n, _p(rp), _p(col), key & 0xFFFFFFFFFFFFFFFF, _p(cidx))
    return cidx, int(nF)


def aggregate(n, rp, col, w, score, hub, level=0, opts: Opts | None = None, **kw):
    """One level's aggregation (Sec. 3.4.1-3.4.2, the setup's rule) from its CSR,
    edge scores and hub flags: (agg, state, info) with info = nc, rounds,
    selected round, alpha."""
    o = opts if opts is not None else default_opts(**kw)
    rp, col, w = _csr(rp, col, w)
    score = np.ascontiguousarray(score, dtype=np.float64)
    hub = np.ascontiguousarray(hub, dtype=np.uint8)
    agg, state = np.zeros(n, np.int32), np.zeros(n, np.int32)
    info = np.zeros(4, np.int64)
    lib().orc_aggregate(n, _p(rp), _p(col), _p(w), _p(score), _p(hub), C.byref(o), level, _p(agg), _p(state), _p(info))
    return agg, state, dict(nc=int(info[0]), rounds=int(info[1]), sel_round=int(info[2]),
                            alpha=float(info[3:4].view(np.float64)[0]))


def galerkin(n, rp, col, w, agg, nc):
    """One level's Galerkin operator P^T A P (Eq. (2.5)) as a CSR (rp, col, w)."""
    rp, col, w = _csr(rp, col, w)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    rpc = np.zeros(nc + 1, np.int64)
    colc = np.zeros(max(col.size, 1), np.int32)
    wc = np.zeros(max(col.size, 1))
    nnz = lib().orc_galerkin(n, _p(rp), _p(col), _p(w), _p(agg), nc, _p(rpc), _p(colc), _p(wc))
    return rpc, colc[:nnz].copy(), wc[:nnz].copy()


def gs_sweep_lex(n, rp, col, w, b, x):
    rp, col, w = _csr(rp, col, w)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    lib().orc_gs_sweep_lex(n, _p(rp), _p(col), _p(w), _p(b), _p(x))


def gs_sweep_colour(n, rp, col, w, colours, ncolours, b, x):
    rp, col, w = _csr(rp, col, w)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(colours, dtype=np.int32)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    lib().orc_gs_sweep_colour(n, _p(rp), _p(col), _p(w), _p(c), ncolours, _p(b), _p(x))


def edge_scores(n, rp, col, w, X, q_max=2.5, weak_tol=1e-8):
    rp, col, w = _csr(rp, col, w)
    X = np.ascontiguousarray(X, dtype=np.float64)
    K = X.shape[1]
    nnz = col.size
    aff, q, score = np.zeros(nnz), np.zeros(nnz), np.zeros(nnz)
    lib().orc_edge_scores(n, _p(rp), _p(col), _p(w), K, _p(X), q_max, weak_tol,
                          _p(aff), _p(q), _p(score))
    return aff, q, score


def hubs(n, rp, col, w, hub_factor=8.0):
    rp, col, w = _csr(rp, col, w)
    h = np.zeros(n, dtype=np.uint8)
    lib().orc_hubs(n, _p(rp), _p(col), _p(w), hub_factor, _p(h))
    return h.astype(bool)


def dense_pinv_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    st = lib().orc_dense_pinv_solve(A.shape[0], _p(A), _p(b), _p(x))
    if st:
        raise RuntimeError("dense solve failed")
    return x


# status codes of oracle/lamg_oracle.h
OK, ERR_ARG, ERR_NOT_SYMMETRIC, ERR_BAD_WEIGHT, ERR_DISCONNECTED, ERR_RHS_NOT_ZERO_SUM = 0, 1, 2, 3, 4, 5


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


class Hierarchy:
    """The oracle's LAMG hierarchy (setup phase, Sec. 4.1) with its solve (Sec. 4.2)."""

    def __init__(self, n, rp, col, w, opts: Opts | None = None, gptr=None, **kw):
        self.opts = opts if opts is not None else default_opts(**kw)
        rp, col, w = _csr(rp, col, w)
        self.n = int(n)
        self._rp, self._col, self._w = rp, col, w
        h = C.c_void_p()
        if gptr is None:
            st = lib().orc_setup(self.n, _p(rp), _p(col), _p(w), C.byref(self.opts), C.byref(h))
        else:
            # block-diagonal union of graphs: graph g owns nodes gptr[g]..gptr[g+1]-1
            self._gptr = np.ascontiguousarray(gptr, dtype=np.int64)
            st = lib().orc_setup_graphs(self.n, _p(rp), _p(col), _p(w), len(self._gptr) - 1, _p(self._gptr),
                                        C.byref(self.opts), C.byref(h))
        if st:
            raise OracleError(st)
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_free(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return int(lib().orc_num_levels(self._h))

    def info(self, l):
        a = np.zeros(16, dtype=np.int64)
        lib().orc_level_info(self._h, l, _p(a))
        f = a.view(np.float64)
        return dict(n=int(a[0]), nnz=int(a[1]), ncolours=int(a[2]), K=int(a[3]), nc=int(a[4]),
                    rounds=int(a[5]), sel_round=int(a[6]), coarsest=bool(a[7]),
                    stop_reason=int(a[8]), alpha=float(f[9]), gamma=float(f[10]),
                    tv_ratio=float(f[11]), jp_rounds=int(a[12]), elim=bool(a[13]), nF=int(a[14]))

    def csr(self, l):
        i = self.info(l)
        rp = np.zeros(i["n"] + 1, dtype=np.int64)
        col = np.zeros(i["nnz"], dtype=np.int32)
        w = np.zeros(i["nnz"])
        lib().orc_level_csr(self._h, l, _p(rp), _p(col), _p(w))
        return rp, col, w

    def colour(self, l):
        c = np.zeros(self.info(l)["n"], dtype=np.int32)
        lib().orc_level_colour(self._h, l, _p(c))
        return c

    def tv(self, l):
        i = self.info(l)
        X = np.zeros((i["n"], i["K"]))
        lib().orc_level_tv(self._h, l, _p(X))
        return X

    def scores(self, l):
        nnz = self.info(l)["nnz"]
        aff, q, s = np.zeros(nnz), np.zeros(nnz), np.zeros(nnz)
        lib().orc_level_scores(self._h, l, _p(aff), _p(q), _p(s))
        return aff, q, s

    def elim(self, l):
        """Level l followed by its Schur complement: coarse index of each node, -1 in F."""
        cidx = np.zeros(self.info(l)["n"], np.int32)
        lib().orc_level_elim(self._h, l, _p(cidx))
        return cidx

    def agg(self, l):
        n = self.info(l)["n"]
        agg, state, hub = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.uint8)
        lib().orc_level_agg(self._h, l, _p(agg), _p(state), _p(hub))
        return agg, state, hub.astype(bool)

    def solve(self, b, x0=None, tol=1e-10, max_cycles=200, adaptive=True):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        hist = np.zeros(max_cycles + 1)
        cyc = C.c_int32(0)
        st = lib().orc_solve(self._h, _p(b), _p(x), tol, max_cycles, int(adaptive), _p(hist),
                             C.byref(cyc))
        if st:
            raise OracleError(st)
        return x, hist[:cyc.value + 1].copy()

    def cycle(self, b, x, adaptive=True):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.array(x, dtype=np.float64)
        lib().orc_cycle(self._h, _p(b), _p(x), int(adaptive))
        return x

    def adjoint(self, x, g, eu, ev, tol=1e-10, max_cycles=200, adaptive=True):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        eu = np.ascontiguousarray(eu, dtype=np.int32)
        ev = np.ascontiguousarray(ev, dtype=np.int32)
        lam = np.zeros(self.n)
        dw = np.zeros(eu.size)
        st = lib().orc_adjoint(self._h, _p(x), _p(g), _p(lam), _p(eu), _p(ev), eu.size, _p(dw),
                               tol, max_cycles, int(adaptive))
        if st:
            raise OracleError(st)
        return lam, dw
