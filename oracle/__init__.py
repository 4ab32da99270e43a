"""CPU oracle for the structure-preserving spectral divide-and-conquer of
definite pseudosymmetric matrices (Benner, Nakatsukasa, Penke, arXiv 2203.08900).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports, links or calls it, and it shares no code with the library.

Layout:
  pssd_oracle.c   scalar-loop FP64 kernels (Cholesky, pivoted elimination,
                  Jacobi eigensolver, pivoted low-rank Cholesky, Jacobi
                  elliptic functions and Zolotarev coefficients)
  oracle.py       the paper's algorithms, step by step, in FP64 (numpy matmul
                  is the only library primitive used as a step, except the
                  general non-definite layer: numpy eig and scipy's
                  Bunch-Kaufman ldl, as Alg. 5 prescribes)

Parity status of each function is stated in its docstring; all are pinned by
the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from .oracle import *  # noqa: F401,F403
