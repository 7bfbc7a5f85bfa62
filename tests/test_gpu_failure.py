"""Failure detection of the cycle engine's grid barrier, without a GPU fault:
one block is held back, the others' bounded wait runs out, the kernel returns
and reports it, and the context stays usable."""
import time

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


def test_barrier_wait_runs_out_and_context_stays_usable(L):
    assert L.lamg_barrier_selftest(False) == L.LAMG_OK
    t0 = time.time()
    assert L.lamg_barrier_selftest(True) == L.LAMG_ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    # the device is still usable: a full setup and solve afterwards
    g = W.grid2d(30, 30)
    s = L.Solver.from_graph(g)
    b = torch.tensor(W.zero_sum_rhs(g.n, 3), device="cuda")
    x, st = s.solve(b, tol=1e-10)
    assert st.rel_res <= 1e-10 and np.isfinite(x.cpu().numpy()).all()
    s.close()
    assert L.lamg_barrier_selftest(False) == L.LAMG_OK
