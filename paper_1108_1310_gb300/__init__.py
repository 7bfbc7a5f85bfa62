"""GB300 (sm_103a) Lean Algebraic Multigrid: a graph-Laplacian solver after
Livne & Brandt, "Lean Algebraic Multigrid (LAMG)", arXiv 1108.1310.

The compute path is the CUDA library ``liblamg.so`` (C-ABI in
``include/lamg.h``); ``paper_1108_1310_gb300.lamg`` is its Python binding and
``paper_1108_1310_gb300.autograd`` the differentiable solve.  Build the
library with ``paper_1108_1310_gb300.build.build()``.
"""

__all__ = ["lamg", "build", "autograd"]
