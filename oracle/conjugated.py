"""Oracle: block-conjugated s-step CG (the Chronopoulos-Gear s-step CG cited in Section 1).

Test infrastructure only (see the package docstring). Paper: arXiv 2512.09642.

The outer iteration of Section 2 (`sstep_cg.solve`) projects onto the new basis P_k alone
(a restarted s-dimensional Galerkin step). The s-step CG of Chronopoulos and Gear, which
Section 1 names as the origin of the method, additionally makes each block A-conjugate to
the previous one:

  1. P_k: the Chebyshev basis of K_s(M^-1 A, r_k) (Section 2, Definition), and A P_k;
  2. k = 0: Q_0 = P_0, AQ_0 = A P_0. k > 0: C_k = (A Q_(k-1))^T P_k, B_k = W_(k-1)^-1 C_k,
     Q_k = P_k - Q_(k-1) B_k, A Q_k = A P_k - A Q_(k-1) B_k;
  3. W_k = Q_k^T A Q_k (lower triangle, mirrored), g_k = Q_k^T r_k;
  4. alpha_k = W_k^-1 g_k by column scaling + nu FGS sweeps (or Cholesky), exactly as for
     the Gram system of Section 2; the s right-hand sides of B_k use the same scaled solve
     with W_(k-1);
  5. x_(k+1) = x_k + Q_k alpha_k, r_(k+1) = r_k - A Q_k alpha_k.

Every quantity is formed from its definition (explicit products with A, no change-of-basis
algebra). Readings (recorded in the design notes): B_k is solved with the same scaled FGS as
alpha_k; a true-residual replacement at recursive convergence restarts the conjugation
(the next block is Q = P); stopping as in Section 8.
"""
from __future__ import annotations

import numpy as np

from .sstep_cg import (Operator, OuterRecord, SolveResult, _gram_solve_scaled, chebyshev_basis,
                       column_scaling)


def scaled_solve(W, rhs, nu: int, solver: str = "fgs"):
    """x = W^-1 rhs by the Section 2 procedure: column scaling of W, then nu FGS sweeps on
    the scaled system (or Cholesky); rhs may hold several columns."""
    rhs = np.asarray(rhs, np.float64)
    cols = rhs.reshape(rhs.shape[0], -1)
    out = np.zeros_like(cols)
    for j in range(cols.shape[1]):
        d, Wt, ct = column_scaling(W, cols[:, j])
        out[:, j] = d * _gram_solve_scaled(Wt, ct, nu, solver)
    return out.reshape(rhs.shape)


def solve_conjugated(op: Operator, b, x0=None, *, s: int, nu: int, lam_min: float, lam_max: float,
                     tol: float = 1e-8, max_outer: int = 100000, gram_solver: str = "fgs",
                     max_refresh: int = 3, history: int = 0) -> SolveResult:
    """Block-conjugated s-step CG (Chronopoulos and Gear, the method Section 1 cites) with
    the Chebyshev basis of Section 2 (steps 1-5 of the module docstring)."""
    b = np.asarray(b, np.float64)
    x = np.zeros(op.n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - op.matvec(x)
    r0 = float(np.linalg.norm(r))
    hist = []
    if r0 == 0.0:
        return SolveResult(x, 0, True, 0.0, 0.0, 0, r0, hist)
    k = 0
    refreshes = 0
    converged = False
    Q_prev = AQ_prev = W_prev = None
    while True:
        rel = float(np.linalg.norm(r)) / r0
        if rel < tol:
            rt = b - op.matvec(x)
            if float(np.linalg.norm(rt)) / r0 < tol or refreshes >= max_refresh:
                converged = float(np.linalg.norm(rt)) / r0 < tol
                break
            r = rt
            refreshes += 1
            Q_prev = AQ_prev = W_prev = None
            continue
        if k >= max_outer:
            break
        P = chebyshev_basis(op, r, s, lam_min, lam_max)
        AP = np.column_stack([op.matvec(P[:, j]) for j in range(s)])
        if Q_prev is None:
            Q, AQ = P, AP
        else:
            C = AQ_prev.T @ P
            B = scaled_solve(W_prev, C, nu, gram_solver)
            Q = P - Q_prev @ B
            AQ = AP - AQ_prev @ B
        Wfull = Q.T @ AQ
        W = np.tril(Wfull) + np.tril(Wfull, -1).T
        g = Q.T @ r
        d, Wt, gt = column_scaling(W, g)
        if not np.any(d > 0.0):
            break
        a = _gram_solve_scaled(Wt, gt, nu, gram_solver)
        alpha = d * a
        x = x + Q @ alpha
        r = r - AQ @ alpha
        Q_prev, AQ_prev, W_prev = Q, AQ, W
        k += 1
        if k <= history:
            ng = float(np.linalg.norm(gt))
            delta = float(np.linalg.norm(gt - Wt @ a)) / ng if ng > 0 else 0.0
            hist.append(OuterRecord(k, rel, d, Wt, gt, alpha, x.copy(), r.copy(), delta))
    rel_true = float(np.linalg.norm(b - op.matvec(x))) / r0
    return SolveResult(x, k, converged, float(np.linalg.norm(r)) / r0, rel_true, refreshes, r0, hist)
