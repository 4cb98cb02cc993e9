"""Seeded synthetic inputs for the s-step CG solver and its CPU oracle.

This package is the only code that both the CUDA path's tests/bench and the oracle use. It
draws random numbers and assembles the linear systems of the synthetic workloads (the
SPD matrix A, the exact solution x*, the right-hand side b = A x*). It holds none of the
solver's arithmetic: no Krylov basis, Gram matrix, Gauss-Seidel sweep or update lives here.
"""
from . import rng, problems  # noqa: F401
