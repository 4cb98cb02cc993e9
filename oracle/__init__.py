"""CPU oracle for Chebyshev-basis s-step CG with Forward Gauss-Seidel Gram solves
(Thomas and D'Ambra, "Inexact Gauss-Seidel Coarse Solvers for AMG and s-step CG",
arXiv 2512.09642).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, FP64 restatement of the method used
to check the CUDA library. Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import it. The library and its Python binding never import or call it,
and it shares no code with them (inputs come from the separate `workloads` package).

Every routine follows the paper's steps in its order and notation; a library primitive
(scipy's CSR mat-vec, numpy's matrix product) serves as a step where the paper uses a plain
product. Pinned by tests/test_oracle_pins.py against closed forms, textbook special cases and
the paper's propositions. The claim kappa(G) = O(s^2) (Theorem "Polynomial Growth") is parity
unpinned: it is recorded, not asserted.
"""
from . import sstep_cg, spectral, adjoint, conjugated, coarse  # noqa: F401
from .sstep_cg import (  # noqa: F401
    Operator, chebyshev_basis, monomial_basis, gram, column_scaling, fgs, fgs_iterates,
    cholesky, cholesky_solve, solve, SolveResult,
)
from .conjugated import solve_conjugated, scaled_solve  # noqa: F401
