"""Oracle: gradient of L = ||x - x_target||^2 with respect to the per-cell coefficient kappa
of the cell-centred diffusion matrix A(kappa), x = A(kappa)^-1 b.

Test infrastructure only. The paper has no adjoint; this is the differentiable form of the
solve built on it. With A symmetric the adjoint system is A lambda = g, g = dL/dx =
2 (x - x_target), and

    dL/dkappa_c = -lambda^T (dA/dkappa_c) x,    dL/db = lambda.

A is a sum of rank-one face terms: an interior face f = (a, b) contributes
w_f (e_a - e_b)(e_a - e_b)^T with w_f = 2 ka kb / (ka + kb), and each boundary face of cell c
contributes 2 kappa_c e_c e_c^T. Hence

    dL/dkappa_c = - sum_{f = (c, o)} (dw_f / dkappa_c) (lambda_c - lambda_o)(x_c - x_o)
                  - 2 * nbf_c * lambda_c x_c,
    dw_f / dkappa_a = 2 kb^2 / (ka + kb)^2,

where nbf_c is the number of boundary faces of cell c.
"""
from __future__ import annotations

import numpy as np


def _shape(dims):
    """The (nz, ny, nx) array shape of a grid and its dimension (no arithmetic of the method)."""
    nx, ny, nz = (tuple(dims) + (1, 1))[:3]
    return (nz, ny, nx), (3 if len(dims) == 3 else 2)


def grad_kappa(dims, kappa, x, lam):
    """dL/dkappa from the forward solution x and the adjoint solution lambda. The paper has
    no adjoint: this differentiates the solve of Section 2 through the diffusion operator
    (the module docstring gives the formula)."""
    shape, d = _shape(dims)
    K = np.asarray(kappa, np.float64).reshape(shape)
    X = np.asarray(x, np.float64).reshape(shape)
    Lm = np.asarray(lam, np.float64).reshape(shape)
    grad = np.zeros(shape)
    for ax in [2, 1, 0][:d]:
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        ka, kb = K[lo], K[hi]
        prod = (Lm[lo] - Lm[hi]) * (X[lo] - X[hi])
        den = (ka + kb) ** 2
        grad[lo] -= 2.0 * kb * kb / den * prod
        grad[hi] -= 2.0 * ka * ka / den * prod
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = slice(0, 1)
        last[ax] = slice(-1, None)
        first, last = tuple(first), tuple(last)
        grad[first] -= 2.0 * Lm[first] * X[first]
        grad[last] -= 2.0 * Lm[last] * X[last]
    return grad.reshape(-1)


def loss_and_grad(dims, kappa, b, x_target, solve_fn):
    """L, dL/dkappa, dL/db with `solve_fn(rhs) -> A(kappa)^-1 rhs` (forward and adjoint
    solves of Section 2's method; the paper has no adjoint)."""
    x = solve_fn(b)
    g = 2.0 * (x - x_target)
    lam = solve_fn(g)
    loss = float(np.sum((x - x_target) ** 2))
    return loss, grad_kappa(dims, kappa, x, lam), lam, x
