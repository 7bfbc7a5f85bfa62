"""Pin of the oracle's solve cycle (Sec. 4.2) as the composition of its steps.

The oracle's cycle is one C routine: relaxation, restriction with the factor
mu, the fractional cycle index, recursion, prolongation, iterate recombination
(Eq. (3.13)) and the final mean subtraction.  Here a second cycle is assembled
in numpy from the oracle's hierarchy (level matrices, colours, aggregates),
with each step taken from its definition in matrix form:

- multicolour Gauss-Seidel: each colour class is an independent set, so its
  Gauss-Seidel update equals a Jacobi update of that class, x_S += (b - Ax)_S / diag_S;
- restriction mu P^T r and prolongation x += P x^c with P the 0/1 aggregate matrix;
- the coarsest level: the minimum-norm least-squares solution (numpy lstsq),
  which for a consistent Laplacian system is the component-wise mean-zero solution;
- recombination: y = x + sum_i alpha_i (x_i - x) with alpha from numpy lstsq on
  min ||b - A y||_2 (the oracle solves the 2x2 normal equations instead);
- an elimination level (Sec. 3.2): the coarse right-hand side
  r_C - A_CF A_FF^-1 r_F and the back-substitution x_F = A_FF^-1 (b_F - A_FC x_C).

The iterates recombined are those of this build's reading of Sec. 3.5: the
iterate after the pre-relaxation of each two-level step, recombined with the
iterate at the end of the visit, at every level (reading R15; with the option
recomb_finest = 0, at every level but the finest).  The cycle index
of level l with gamma_l gives its k-th coarse correction ceil((k+1) gamma_l) -
ceil(k gamma_l) coarse visits, kept in [1, 2].  A wrong operand, sign, index
or order in the C cycle changes its result well beyond rounding.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _dense(n, rp, col, w):
    Wm = np.zeros((n, n))
    Wm[np.repeat(np.arange(n), np.diff(rp)), col] = w
    return np.diag(Wm.sum(axis=1)) - Wm


class _NumpyCycle:
    def __init__(self, h, adaptive, gptr=None):
        o = h.opts
        self.nu1, self.nu2 = o.nu1, o.nu2
        self.mu = o.mu_adaptive if adaptive else o.mu_flat
        self.adaptive = adaptive
        self.recomb_finest = bool(o.recomb_finest)
        self.gptr = gptr
        self.lv = []
        for l in range(h.num_levels):
            i = h.info(l)
            rp, col, w = h.csr(l)
            d = dict(n=i["n"], A=_dense(i["n"], rp, col, w), coarsest=i["coarsest"],
                     elim=i["elim"], gamma=i["gamma"], colour=h.colour(l), ncol=i["ncolours"])
            d["diag"] = np.diag(d["A"]).copy()
            if not d["coarsest"]:
                if d["elim"]:
                    d["cidx"] = h.elim(l)
                else:
                    d["agg"] = h.agg(l)[0]
            self.lv.append(d)

    def relax(self, F, b, x):
        for c in range(F["ncol"]):
            S = F["colour"] == c
            x[S] += (b[S] - F["A"][S] @ x) / F["diag"][S]

    def coarsest(self, F, b):
        return np.linalg.lstsq(F["A"], b, rcond=None)[0]

    def coarse_visit(self, l, theta, b):
        """theta visits of level l from a zero initial guess; returns x."""
        F = self.lv[l]
        if F["coarsest"]:
            return self.coarsest(F, b)
        x = np.zeros(F["n"])
        if not F["elim"]:
            return self.visit(l, b, x, theta)
        for _ in range(theta):
            x = self.elim_step(l, b, x)
        return x

    def elim_step(self, l, b, x):
        F, C = self.lv[l], self.lv[l + 1]
        A, cidx = F["A"], F["cidx"]
        Fs, Cs = np.flatnonzero(cidx < 0), np.flatnonzero(cidx >= 0)
        assert np.array_equal(cidx[Cs], np.arange(Cs.size))
        r = b - A @ x
        AFF = A[np.ix_(Fs, Fs)]
        assert np.count_nonzero(AFF - np.diag(np.diag(AFF))) == 0       # F is independent
        bc = r[Cs] - A[np.ix_(Cs, Fs)] @ np.linalg.solve(AFF, r[Fs])
        xc = self.coarse_visit(l + 1, 1, bc)
        x = x.copy()
        x[Cs] += xc
        x[Fs] = np.linalg.solve(AFF, b[Fs] - A[np.ix_(Fs, Cs)] @ x[Cs])
        return x

    def visit(self, l, b, x, theta):
        F, C = self.lv[l], self.lv[l + 1]
        A, agg = F["A"], F["agg"]
        x = x.copy()
        recomb = self.adaptive and (l >= 1 or self.recomb_finest)
        saved = []
        for _ in range(theta):
            for _ in range(self.nu1):
                self.relax(F, b, x)
            r = b - A @ x
            if recomb:
                saved.append(x.copy())
            bc = self.mu * np.bincount(agg, weights=r, minlength=C["n"])
            if C["coarsest"]:
                xc = self.coarsest(C, bc)
            else:
                k = self.visits[l]
                self.visits[l] += 1
                g = F["gamma"]
                th = min(max(math.ceil((k + 1) * g) - math.ceil(k * g), 1), 2)
                xc = self.coarse_visit(l + 1, th, bc)
            x += xc[agg]
            for _ in range(self.nu2):
                self.relax(F, b, x)
        if recomb:
            r = b - A @ x
            D = np.column_stack([A @ (xi - x) for xi in saved])
            alpha = np.linalg.lstsq(D, r, rcond=None)[0]
            x = x + sum(a * (xi - x) for a, xi in zip(alpha, saved))
        return x

    def cycle(self, b, x):
        self.visits = [0] * len(self.lv)
        F = self.lv[0]
        if F["coarsest"]:
            return self.coarsest(F, b)
        x = self.elim_step(0, b, x) if F["elim"] else self.visit(0, b, x, 1)
        gptr = self.gptr if self.gptr is not None else [0, F["n"]]
        for a, e in zip(gptr[:-1], gptr[1:]):
            x[a:e] -= x[a:e].mean()
        return x


def _graphs():
    return {
        "chung_lu": (W.chung_lu(2500, seed=31), None, {}),
        "grid": (W.grid2d(36, 30), None, {}),
        "rgg": (W.rgg2d(1500, seed=32), None, {}),
        "grid_elim": (W.grid2d(36, 30), None, {"elim": 1}),
        "chung_lu_elim": (W.chung_lu(2500, seed=33), None, {"elim": 1}),
        "union": (*W.er_batch(12, 60, 400, seed=34), {}),
        # the restriction factor under recombination, and the coarse cycle-index cap
        "chung_lu_mu": (W.chung_lu(2500, seed=35), None, {"mu_adaptive": 1.2}),
        "rgg_cap1": (W.rgg2d(1500, seed=36), None, {"gamma_coarse_max": 1.0}),
        # the earlier readings: the parallel handshake, recombination below the finest level
        "grid_handshake": (W.grid2d(36, 30), None, {"agg_rule": 0, "recomb_finest": 0}),
        # the paper's sequential forms: index-order scan, lexicographic GS
        "rgg_lex": (W.rgg2d(1500, seed=37), None, {"agg_rule": 1, "relax_rule": 1}),
    }


@pytest.mark.parametrize("adaptive", [True, False])
@pytest.mark.parametrize("gname", list(_graphs()))
def test_cycle_is_the_composition_of_its_steps(gname, adaptive):
    g, gptr, kw = _graphs()[gname]
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w, gptr=gptr, **kw)
    assert h.num_levels >= 3
    if kw.get("elim"):
        assert any(h.info(l)["elim"] for l in range(h.num_levels))
    ref = _NumpyCycle(h, adaptive, gptr=gptr)
    b = W.zero_sum_rhs(g.n, 5) if gptr is None else W.zero_sum_rhs_graphs(gptr, 5)
    x = np.zeros(g.n)
    for _ in range(3):                       # three cycles, each from the last result
        want = ref.cycle(b, x)
        got = h.cycle(b, x, adaptive=adaptive)
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want)), gname
        x = got


def test_composition_detects_the_recombination():
    # the pin has teeth: the same composition without recombination, or with the
    # restriction factor of the other mode, differs from the oracle's adaptive cycle
    g = W.chung_lu(2500, seed=31)
    h = oracle.Hierarchy(g.n, g.rp, g.col, g.w)
    b = W.zero_sum_rhs(g.n, 5)
    got = h.cycle(b, np.zeros(g.n), adaptive=True)
    scale = np.max(np.abs(got))
    ref = _NumpyCycle(h, True)
    ref.adaptive = False                     # recombination off, mu of the adaptive mode
    assert np.max(np.abs(ref.cycle(b, np.zeros(g.n)) - got)) > 1e-6 * scale
    ref = _NumpyCycle(h, True)
    ref.mu = h.opts.mu_flat
    assert np.max(np.abs(ref.cycle(b, np.zeros(g.n)) - got)) > 1e-6 * scale
    ref = _NumpyCycle(h, True)
    ref.recomb_finest = False                # no recombination at the finest level
    assert np.max(np.abs(ref.cycle(b, np.zeros(g.n)) - got)) > 1e-6 * scale
