"""Python binding of the LAMG C-ABI (``include/lamg.h``).

Argument marshalling only: every computation runs in the CUDA library
``liblamg.so``.  PyTorch supplies device memory (tensors' data pointers) and
streams.  The functions keep the C names (``lamg_setup``, ``lamg_solve``,
``lamg_solve_batched``, ``lamg_adjoint``, ``lamg_free``); ``Solver`` wraps a
handle for convenience.  Importing this module loads the library and fails
loudly when it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblamg.so")

LAMG_OK = 0
LAMG_ERR_ARG = 1
LAMG_ERR_NOT_SYMMETRIC = 2
LAMG_ERR_BAD_WEIGHT = 3
LAMG_ERR_DISCONNECTED = 4
LAMG_ERR_RHS_NOT_ZERO_SUM = 5
LAMG_ERR_OOM = 6
LAMG_ERR_CUDA = 7
LAMG_ERR_NOT_CONVERGED = 8
LAMG_ERR_TIMEOUT = 9
LAMG_FP64 = 0
LAMG_FP32_IR = 1

FIELD = {"row_ptr": 0, "col": 1, "w": 2, "colour": 3, "agg": 4, "state": 5, "hub": 6, "tv": 7,
         "affinity": 8, "q": 9, "score": 10, "cidx": 11}


class lamg_options(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("gamma", C.c_double), ("k_finest", C.c_int32), ("k_max", C.c_int32),
                ("k_step", C.c_int32), ("nu_tv", C.c_int32), ("nu1", C.c_int32),
                ("nu2", C.c_int32), ("n_coarsest", C.c_int32), ("q_max", C.c_double),
                ("hub_factor", C.c_double), ("weak_tol", C.c_double),
                ("alpha_stall", C.c_double), ("relax_fast_ratio", C.c_double),
                ("max_rounds", C.c_int32), ("max_levels", C.c_int32),
                ("dense_max", C.c_int32), ("coarse_sweeps", C.c_int32),
                ("mu_flat", C.c_double), ("seed", C.c_uint64), ("adaptive", C.c_int32),
                ("max_cycles", C.c_int32), ("ir_inner", C.c_int32), ("validate", C.c_int32),
                ("keep_setup_data", C.c_int32), ("project_rhs", C.c_int32), ("mu_adaptive", C.c_double),
                ("gamma_coarse_max", C.c_double), ("elim", C.c_int32), ("elim_min_frac", C.c_double),
                ("lgmg_nx", C.c_int32), ("agg_rule", C.c_int32), ("recomb_finest", C.c_int32),
                ("relax_rule", C.c_int32), ("sb_work32", C.c_int32), ("sb_work64", C.c_int32),
                ("tail_work32", C.c_int32), ("tail_work64", C.c_int32), ("colour_rule", C.c_int32),
                ("negative_weights", C.c_int32)]


class lamg_stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("cycles", C.c_int32), ("outer_steps", C.c_int32),
                ("status", C.c_int32), ("rel_res", C.c_double), ("acf", C.c_double),
                ("t_setup_s", C.c_double), ("t_solve_s", C.c_double), ("nnz_total", C.c_int64),
                ("bytes_per_cycle", C.c_int64), ("bytes_per_cycle32", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1108_1310_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "lamg_default_options": (None, [P]),
        "lamg_op_times": (I32, [P, I32, I32, P, P, P, P, P, P]),
        "lamg_last_error": (C.c_char_p, []),
        "lamg_setup": (I32, [I64, P, P, P, I32, P, P, P]),
        "lamg_setup_graphs": (I32, [I32, P, I64, P, P, P, I32, P, P, P]),
        "lamg_solve": (I32, [P, P, P, D, I32, P, P]),
        "lamg_solve_host": (I32, [P, P, P, D, I32, P, P]),
        "lamg_solve_batched": (I32, [P, I32, P, P, I64, D, I32, P, P]),
        "lamg_adjoint": (I32, [P, P, P, P, P, P, I64, P, I32, D, I32, P, P]),
        "lamg_free": (None, [P]),
        "lamg_level_info": (I32, [P, I32, P]),
        "lamg_level_copy": (I32, [P, I32, I32, P, I64]),
        "lamg_cycle": (I32, [P, P, P, I32, P]),
        "lamg_cycle_noalloc": (I32, [P, P, P, I32, P]),
        "lamg_autotune_batched": (I32, [P, I32, I32, P, P, P]),
        "lamg_set_batch_cols": (I32, [P, I32]),
        "lamg_barrier_selftest": (I32, [I32, P]),
        "lamg_graph_residuals": (I32, [P, P]),
        "lamg_profile": (I32, [P, I32, P, P, P]),
        "lamg_launch_count": (I32, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()


class LamgError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.lamg_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(st: int, where: str, allow=()):
    if st != LAMG_OK and st not in allow:
        raise LamgError(st, where)
    return st


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    raise TypeError(type(t))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t


def lamg_default_options(**kw) -> lamg_options:
    o = lamg_options()
    _lib.lamg_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


# --------------------------------------------------------------------------- #
# The C-ABI, one function each
# --------------------------------------------------------------------------- #

def lamg_setup(n: int, row_ptr, col, w, opt: lamg_options | None = None, stream=None):
    """Build the hierarchy from a device CSR (int64 row_ptr, int32 col, FP64/FP32 w)."""
    _dev(row_ptr, torch.int64, "row_ptr")
    _dev(col, torch.int32, "col")
    if w.dtype not in (torch.float64, torch.float32):
        raise TypeError("w must be float64 or float32")
    _dev(w, w.dtype, "w")
    h = C.c_void_p()
    st = _lib.lamg_setup(int(n), _ptr(row_ptr), _ptr(col), _ptr(w), int(w.dtype == torch.float32),
                         C.byref(opt) if opt is not None else None, _stream(stream), C.byref(h))
    _check(st, "lamg_setup")
    return h


def lamg_setup_graphs(gptr, row_ptr, col, w, opt: lamg_options | None = None, stream=None):
    """Hierarchy of a block-diagonal union of graphs; gptr: host int64 node ranges."""
    _dev(row_ptr, torch.int64, "row_ptr")
    _dev(col, torch.int32, "col")
    if w.dtype not in (torch.float64, torch.float32):
        raise TypeError("w must be float64 or float32")
    _dev(w, w.dtype, "w")
    gp = np.ascontiguousarray(gptr, dtype=np.int64)
    h = C.c_void_p()
    st = _lib.lamg_setup_graphs(int(len(gp) - 1), _ptr(gp), int(gp[-1]), _ptr(row_ptr), _ptr(col), _ptr(w),
                                int(w.dtype == torch.float32), C.byref(opt) if opt is not None else None,
                                _stream(stream), C.byref(h))
    _check(st, "lamg_setup_graphs")
    return h


def lamg_solve(h, b, x, tol: float = 1e-8, precision: int = LAMG_FP64, stream=None,
               allow_not_converged: bool = False) -> lamg_stats:
    _dev(b, torch.float64, "b")
    _dev(x, torch.float64, "x")
    s = lamg_stats()
    st = _lib.lamg_solve(h, _ptr(b), _ptr(x), float(tol), int(precision), _stream(stream), C.byref(s))
    _check(st, "lamg_solve", (LAMG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return s


def lamg_solve_host(h, b: np.ndarray, x: np.ndarray, tol: float = 1e-8, precision: int = LAMG_FP64,
                    stream=None, allow_not_converged: bool = False) -> lamg_stats:
    assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
    s = lamg_stats()
    st = _lib.lamg_solve_host(h, _ptr(b), _ptr(x), float(tol), int(precision), _stream(stream), C.byref(s))
    _check(st, "lamg_solve_host", (LAMG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return s


def lamg_solve_batched(h, B, X, tol: float = 1e-8, precision: int = LAMG_FP64, stream=None,
                       allow_not_converged: bool = False):
    """B, X: (n, nrhs) FP64 device tensors with unit column stride (row-interleaved,
    ld = stride(0) >= nrhs).  Returns one lamg_stats per column."""
    for t, name in ((B, "B"), (X, "X")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
                and t.stride(1) == 1):
            raise TypeError(f"{name} must be a CUDA float64 (n, nrhs) tensor with unit column stride")
    if B.shape != X.shape or B.stride(0) != X.stride(0):
        raise TypeError("B and X must have the same shape and row stride")
    nrhs = B.shape[1]
    stats = (lamg_stats * nrhs)()
    st = _lib.lamg_solve_batched(h, int(nrhs), _ptr(B), _ptr(X), int(B.stride(0)), float(tol),
                                 int(precision), _stream(stream), stats)
    _check(st, "lamg_solve_batched", (LAMG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return list(stats)


def lamg_autotune_batched(h, nrhs: int, precision: int = LAMG_FP32_IR, stream=None):
    """Times one refinement step of nrhs columns at column chunks 16/32/64/128 and keeps
    the fastest in the handle.  Returns (chosen chunk, [ms at 16, 32, 64, 128])."""
    chosen = C.c_int32(0)
    ms = (C.c_double * 4)()
    _check(_lib.lamg_autotune_batched(h, int(nrhs), int(precision), _stream(stream), C.byref(chosen), ms),
           "lamg_autotune_batched")
    return chosen.value, list(ms)


def lamg_set_batch_cols(h, cols: int):
    _check(_lib.lamg_set_batch_cols(h, int(cols)), "lamg_set_batch_cols")


def lamg_adjoint(h, x, g, lam, eu=None, ev=None, dw=None, tol: float = 1e-8,
                 precision: int = LAMG_FP64, stream=None) -> lamg_stats:
    _dev(x, torch.float64, "x")
    _dev(g, torch.float64, "g")
    _dev(lam, torch.float64, "lambda")
    m = 0
    if dw is not None:
        _dev(eu, torch.int32, "eu")
        _dev(ev, torch.int32, "ev")
        m = eu.numel()
    s = lamg_stats()
    st = _lib.lamg_adjoint(h, _ptr(x), _ptr(g), _ptr(lam), _ptr(eu), _ptr(ev), int(m), _ptr(dw),
                           int(dw is not None and dw.dtype == torch.float32), float(tol),
                           int(precision), _stream(stream), C.byref(s))
    _check(st, "lamg_adjoint")
    return s


def lamg_free(h):
    if h is not None and getattr(h, "value", None):
        _lib.lamg_free(h)


def lamg_level_info(h, level: int) -> dict:
    a = np.zeros(16, dtype=np.int64)
    _check(_lib.lamg_level_info(h, int(level), _ptr(a)), "lamg_level_info")
    f = a.view(np.float64)
    return dict(n=int(a[0]), nnz=int(a[1]), ncolours=int(a[2]), K=int(a[3]), nc=int(a[4]),
                rounds=int(a[5]), sel_round=int(a[6]), coarsest=bool(a[7]), stop_reason=int(a[8]),
                alpha=float(f[9]), gamma=float(f[10]), tv_ratio=float(f[11]), jp_rounds=int(a[12]),
                dense=bool(a[13]), elim=bool(a[14]), nF=int(a[15]))


def lamg_level_copy(h, level: int, field: str) -> np.ndarray:
    info = lamg_level_info(h, level)
    n, nnz, K = info["n"], info["nnz"], info["K"]
    shape, dtype = {
        "row_ptr": (n + 1, np.int64), "col": (nnz, np.int32), "w": (nnz, np.float64),
        "colour": (n, np.int32), "agg": (n, np.int32), "state": (n, np.int32), "hub": (n, np.uint8),
        "tv": (n * K, np.float64), "affinity": (nnz, np.float64), "q": (nnz, np.float64),
        "score": (nnz, np.float64), "cidx": (n, np.int32)}[field]
    out = np.zeros(shape, dtype=dtype)
    _check(_lib.lamg_level_copy(h, int(level), FIELD[field], _ptr(out), out.nbytes), "lamg_level_copy")
    return out.reshape(n, K) if field == "tv" else out


def lamg_cycle(h, b, x, adaptive: bool = True, stream=None):
    _dev(b, torch.float64, "b")
    _dev(x, torch.float64, "x")
    _check(_lib.lamg_cycle(h, _ptr(b), _ptr(x), int(adaptive), _stream(stream)), "lamg_cycle")


def lamg_cycle_noalloc(h, b, x, adaptive: bool = True, stream=None):
    """lamg_cycle without allocation; the handle must have run lamg_cycle once."""
    _dev(b, torch.float64, "b")
    _dev(x, torch.float64, "x")
    _check(_lib.lamg_cycle_noalloc(h, _ptr(b), _ptr(x), int(adaptive), _stream(stream)), "lamg_cycle_noalloc")


def lamg_graph_residuals(h, ngraphs: int) -> np.ndarray:
    """Per-graph relative residuals of the last solve on a many-graphs handle."""
    out = np.zeros(int(ngraphs))
    _check(_lib.lamg_graph_residuals(h, _ptr(out)), "lamg_graph_residuals")
    return out


def lamg_barrier_selftest(hold_one_block: bool, stream=None) -> int:
    """Status of the grid barrier's bounded wait (LAMG_ERR_TIMEOUT when a block is held back)."""
    return int(_lib.lamg_barrier_selftest(int(bool(hold_one_block)), _stream(stream)))


def lamg_profile(h, enable: bool):
    avg = C.c_double(0.0)
    cnt = C.c_int64(0)
    byt = C.c_int64(0)
    _check(_lib.lamg_profile(h, int(enable), C.byref(avg), C.byref(cnt), C.byref(byt)), "lamg_profile")
    return avg.value, cnt.value, byt.value


OP_NAMES = ["sweep", "sweep_run", "resid", "restrict", "zero", "coarse", "prolong", "recomb_dots",
            "recomb_apply", "mean_part", "mean_apply", "ir_prep", "ir_update", "mean64_part", "mean64_apply",
            "res64", "norm64", "sweep_smem", "gmean_part", "gmean_apply", "gmean64_part", "gmean64_apply",
            "gnorm64", "tail_pre", "tail_run", "elim_restrict", "elim_prolong", "elim_back"]


def lamg_op_times(h, mode: int, cap: int = 8192):
    """The engine's op timer: mode 1 starts it, -1 stops it, 0 returns the rows
    (level, op name, single_block, count, total_ms) recorded since the last read."""
    lv = np.zeros(cap, np.int32)
    op = np.zeros(cap, np.int32)
    sb = np.zeros(cap, np.int32)
    cnt = np.zeros(cap, np.int64)
    ns = np.zeros(cap, np.float64)
    nr = C.c_int32(0)
    _check(_lib.lamg_op_times(h, int(mode), cap, lv.ctypes.data, op.ctypes.data, sb.ctypes.data,
                              cnt.ctypes.data, ns.ctypes.data, C.byref(nr)), "lamg_op_times")
    k = min(nr.value, cap)
    return [(int(lv[i]), OP_NAMES[op[i]] if op[i] < len(OP_NAMES) else str(op[i]), int(sb[i]), int(cnt[i]),
             ns[i] * 1e-6) for i in range(k)]


def lamg_launch_count() -> int:
    c = C.c_int64(0)
    _check(_lib.lamg_launch_count(C.byref(c)), "lamg_launch_count")
    return c.value


# --------------------------------------------------------------------------- #
# Convenience wrapper
# --------------------------------------------------------------------------- #

class Solver:
    """Owns one hierarchy.  ``Solver(graph_csr_on_device)`` then ``solve(b)``."""

    def __init__(self, n, row_ptr, col, w, stream=None, gptr=None, **opts):
        self.n = int(n)
        self.opt = lamg_default_options(**opts)
        if gptr is None:
            self.h = lamg_setup(n, row_ptr, col, w, self.opt, stream)
        else:
            self.h = lamg_setup_graphs(gptr, row_ptr, col, w, self.opt, stream)
        self.device = row_ptr.device

    @classmethod
    def from_graph(cls, g, device="cuda", w_dtype=torch.float64, gptr=None, **opts):
        rp = torch.as_tensor(g.rp, dtype=torch.int64, device=device)
        col = torch.as_tensor(g.col, dtype=torch.int32, device=device)
        w = torch.as_tensor(g.w, device=device).to(w_dtype)
        return cls(g.n, rp, col, w, gptr=gptr, **opts)

    def solve(self, b, x0=None, tol=1e-8, precision=LAMG_FP64, stream=None, allow_not_converged=False):
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        st = lamg_solve(self.h, b, x, tol, precision, stream, allow_not_converged)
        return x, st

    def solve_batched(self, B, X0=None, tol=1e-8, precision=LAMG_FP64, stream=None, allow_not_converged=False):
        X = torch.zeros_like(B) if X0 is None else X0.clone()
        st = lamg_solve_batched(self.h, B, X, tol, precision, stream, allow_not_converged)
        return X, st

    def autotune_batched(self, nrhs, precision=LAMG_FP32_IR, cache=None, stream=None):
        """Column chunk for batched solves of nrhs right-hand sides: looked up in the JSON
        file `cache` (key: n, level-1 nnz, nrhs, precision), else timed on this handle and
        stored there.  Returns the chunk in use."""
        import json
        info = self.level_info(0)
        key = f"{self.n}:{info['nnz']}:{int(nrhs)}:{'fp64' if precision == LAMG_FP64 else 'fp32ir'}"
        table = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if key in table:
            lamg_set_batch_cols(self.h, int(table[key]["cols"]))
            return int(table[key]["cols"])
        cols, ms = lamg_autotune_batched(self.h, nrhs, precision, stream)
        if cache is not None:
            table[key] = {"cols": cols, "ms": dict(zip(["16", "32", "64", "128"], ms))}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return cols

    def level_info(self, level):
        return lamg_level_info(self.h, level)

    @property
    def num_levels(self):
        return self._levels()

    def _levels(self):
        l = 0
        while True:
            i = lamg_level_info(self.h, l)
            if i["coarsest"]:
                return l + 1
            l += 1

    def close(self):
        lamg_free(self.h)
        self.h = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass
