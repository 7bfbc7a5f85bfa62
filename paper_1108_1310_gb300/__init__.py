"""GB300 (sm_103a) Lean Algebraic Multigrid: a graph-Laplacian solver after
Livne & Brandt, "Lean Algebraic Multigrid (LAMG)", arXiv 1108.1310.

The compute path is the CUDA library ``liblamg.so`` (C-ABI in
``include/lamg.h``); ``paper_1108_1310_gb300.lamg`` is its Python binding and
``paper_1108_1310_gb300.autograd`` the differentiable solve.  Build the
library with ``paper_1108_1310_gb300.build.build()``.

Typical use (graph as a symmetric CSR with both directions of every edge)::

    import torch
    from paper_1108_1310_gb300 import build, lamg
    build.build()
    s = lamg.Solver(n, row_ptr_i64_cuda, col_i32_cuda, w_cuda)   # setup (Sec. 4.1)
    x, st = s.solve(b_cuda, tol=1e-8, precision=lamg.LAMG_FP32_IR)   # b zero-sum
    X, sts = s.solve_batched(B_cuda)                             # many right-hand sides
    s.close()
"""

__all__ = ["lamg", "build", "autograd"]
