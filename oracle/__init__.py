"""FP64 CPU oracle for the Local Exponential Method (Bonaventura, arXiv 1505.02248).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously-correct statement
of what the GPU hot path computes. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it. The product path (the C-ABI library
and its Python binding) never imports, links or calls anything here, and this package
imports nothing from the product.

Modules
-------
``lem_oracle``   operator assembly (Eq. spacedisc), decomposition (Sec. 3), Pade-13
                 scaling-and-squaring expm, phi_1 and phi_k (Sec. 2 / Sec. 4), the LEM step
                 (Eq. lem, Sec. 3 steps 1-3), a third-order exponential Rosenbrock LEM step
                 (Sec. 4.2) and the global steps they approximate; real or complex inputs
                 (the Schroedinger test of Sec. 4.1); the porous-medium nonlinearity and its
                 Barenblatt solution (Sec. 4.2); truncated propagators (the off-band decay
                 of Sec. 2, Theorem 1).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms, invariants,
an independent library (scipy), arbitrary precision (mpmath) or brute force.
Parity status per function is listed in the module docstring of ``lem_oracle``.
"""
from .lem_oracle import *  # noqa: F401,F403
