"""Oracle: spectral bounds [lam_min, lam_max] of M^-1 A for the Chebyshev basis.

Test infrastructure only. Section 8 of arXiv 2512.09642 estimates the extreme eigenvalues
with 10 Lanczos iterations and a 10% safety margin. Readings (paper silent on details):
  * Lanczos runs on the symmetric D^-1/2 A D^-1/2 (same spectrum as D^-1 A), without
    reorthogonalisation, from a seeded U(-1, 1) start vector;
  * "lanczos10":  lam_min = 0.9 * theta_min(T_10), lam_max = 1.1 * theta_max(T_10);
  * "gersh_lanczos10": lam_min = 0.9 * theta_min(T_10), lam_max = Gershgorin bound of
    D^-1 A, max_i sum_j |a_ij| / a_ii (already an upper bound, so no margin; exactly 2 for
    the Jacobi-scaled Laplacian).
Eigenvalues of the tridiagonal T come from Sturm-sequence bisection.
"""
from __future__ import annotations

import numpy as np

from .sstep_cg import Operator


def lanczos(op: Operator, v0, k: int = 10):
    """k steps of Lanczos on B = D^-1/2 A D^-1/2 (Section 8's eigenvalue estimate): returns
    (alpha[0:m], beta[0:m-1])."""
    dh = np.sqrt(op.minv)                  # D^-1/2
    q = np.asarray(v0, np.float64) / np.linalg.norm(v0)
    q_prev = np.zeros_like(q)
    beta_prev = 0.0
    alphas, betas = [], []
    for j in range(k):
        w = dh * op.matvec(dh * q) - beta_prev * q_prev
        a = float(q @ w)
        w = w - a * q
        alphas.append(a)
        bnorm = float(np.linalg.norm(w))
        if j == k - 1 or bnorm == 0.0:
            break
        betas.append(bnorm)
        q_prev, q = q, w / bnorm
        beta_prev = bnorm
    return np.array(alphas), np.array(betas)


def sturm_count(alpha, beta, x: float) -> int:
    """Number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x (the Sturm
    count behind the Ritz values of Section 8's Lanczos estimate)."""
    count = 0
    q = 1.0
    for i in range(len(alpha)):
        b2 = beta[i - 1] ** 2 if i > 0 else 0.0
        q = alpha[i] - x - (b2 / q if i > 0 else 0.0)
        if q == 0.0:
            q = -1e-300
        if q < 0.0:
            count += 1
    return count


def tridiag_eigvals(alpha, beta):
    """All eigenvalues (ascending) of a symmetric tridiagonal matrix by bisection: the Ritz
    values of Section 8's Lanczos estimate."""
    m = len(alpha)
    if m == 0:
        return np.array([])
    rad = np.zeros(m)
    rad[:-1] += np.abs(beta)
    rad[1:] += np.abs(beta)
    lo0, hi0 = float(np.min(alpha - rad)), float(np.max(alpha + rad))
    out = []
    for i in range(m):
        lo, hi = lo0, hi0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid == lo or mid == hi:
                break
            if sturm_count(alpha, beta, mid) > i:
                hi = mid
            else:
                lo = mid
        out.append(0.5 * (lo + hi))
    return np.array(out)


def gershgorin_upper(op: Operator) -> float:
    """max_i sum_j |(M^-1 A)_ij|: Gershgorin upper bound on the spectrum of M^-1 A (the
    upper end of the workloads' "Gershgorin/10-step Lanczos" bounds, a reading of Section 8)."""
    absrow = np.asarray(abs(op.A).sum(axis=1)).ravel()
    return float(np.max(np.abs(op.minv) * absrow))


def bounds(op: Operator, mode: str, v0, k: int = 10):
    """(lam_min, lam_max) of Section 8 under the two readings above."""
    a, b = lanczos(op, v0, k)
    ev = tridiag_eigvals(a, b)
    if mode == "lanczos10":
        return 0.9 * ev[0], 1.1 * ev[-1]
    if mode == "gersh_lanczos10":
        return 0.9 * ev[0], gershgorin_upper(op)
    raise ValueError(mode)
