"""lamg_cycle_noalloc (the allocation-free one-cycle entry point) against lamg_cycle.

Collected last on purpose: it must pass both alone in a fresh process and
after every other test has used the library on the same device.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("gname", ["chung_lu", "grid2d"])
@pytest.mark.parametrize("adaptive", [True, False])
def test_noalloc_matches_cycle_two_calls(L, gname, adaptive):
    g = W.chung_lu(6000, seed=13) if gname == "chung_lu" else W.grid2d(40, 30)
    s = L.Solver.from_graph(g)
    b = torch.tensor(W.zero_sum_rhs(g.n, 3), device="cuda")
    # reference: two lamg_cycle calls in a row (the first also prepares the handle)
    xr = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    L.lamg_cycle(s.h, b, xr, adaptive)
    xr1 = xr.clone()
    L.lamg_cycle(s.h, b, xr, adaptive)
    xr2 = xr.clone()
    # the allocation-free path: two calls in a row from the same start
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    x1 = torch.empty_like(x)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    L.lamg_cycle_noalloc(s.h, b, x, adaptive)
    x1.copy_(x)
    L.lamg_cycle_noalloc(s.h, b, x, adaptive)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # no device memory was taken by the two calls
    assert free1 >= free0
    # same program, same arithmetic: equal within the cycle tests' tolerance
    for a, r in ((x1, xr1), (x, xr2)):
        a, r = a.cpu().numpy(), r.cpu().numpy()
        assert np.max(np.abs(a - r)) <= 1e-11 * np.max(np.abs(r))
    s.close()


def test_noalloc_rejects_unprepared_handle(L):
    g = W.grid2d(20, 20)
    s = L.Solver.from_graph(g)
    b = torch.tensor(W.zero_sum_rhs(g.n, 5), device="cuda")
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LamgError) as e:
        L.lamg_cycle_noalloc(s.h, b, x, True)
    assert e.value.status == L.LAMG_ERR_ARG
    assert torch.count_nonzero(x).item() == 0
    # prepared for adaptive cycles only: the flat program is still missing
    L.lamg_cycle(s.h, b, torch.zeros_like(x), True)
    with pytest.raises(L.LamgError) as e:
        L.lamg_cycle_noalloc(s.h, b, x, False)
    assert e.value.status == L.LAMG_ERR_ARG
    L.lamg_cycle_noalloc(s.h, b, x, True)
    assert torch.isfinite(x).all() and torch.count_nonzero(x).item() > 0
    s.close()
