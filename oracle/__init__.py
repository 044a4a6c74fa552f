"""Plain FP64 CPU oracle for the stochastic-Galerkin domain-decomposition wave solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its Python
binding) imports, links or runs this package.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may use it.

Each function follows a passage of the paper "A Domain Decomposition-based Solver for
Acoustic Wave Propagation in Two-Dimensional Random Media" (arXiv 2512.23027), cited by
section and equation label.  The code favours obviousness over speed: library
primitives (sparse LU, dense Cholesky, root brackets) serve as steps, with no blocking
or fusion beyond what the equations state.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against closed
forms, invariants, special cases or brute force (see tests/test_oracle_*.py), except
where a docstring says "parity unpinned".
"""
