"""Oracle: the s-step CG outer iteration with a Chebyshev basis and FGS Gram solves.

Test infrastructure only (see the package docstring). Paper: arXiv 2512.09642.

One outer iteration k (Section 2, "Preliminaries"):
  1. basis P in K_s(M^-1 A, r_k) by the Chebyshev recurrence (Section 2, Definition
     "Chebyshev Polynomial Basis");
  2. Gram system G alpha = P^T r_k with G = P^T A P (Section 1, Section 2);
  3. column scaling d_i = (p_i^T A p_i)^-1/2, G~ = S G S, c~ = S P^T r_k, so diag(G~) = I
     and G~ = I + L + L^T (Section 2, "Column scaling");
  4. nu FGS sweeps (I + L) a^(l+1) = c~ - L^T a^(l), a^(0) = 0 (Section 2), or a Cholesky
     solve, the O(s^3) baseline FGS replaces (Section 1);
  5. alpha = S a; x_(k+1) = x_k + P alpha; r_(k+1) = r_k - (A P) alpha.
Stopping: ||r_k|| / ||r_0|| < tol with r_0 = b - A x_0 (Section 8).

Readings where the paper is silent (all recorded in the design notes):
  * literal update x += P alpha, no conjugation against the previous block;
  * p_0 = r_k as written (option: p_0 = M^-1 r_k);
  * G is formed from its lower triangle (i >= j) and mirrored;
  * a column with G_ii <= 0 or non-finite G_ii is dropped (d_i = 0, alpha_i = 0);
  * at recursive convergence the true residual b - A x is recomputed; if it is above tol
    it replaces r and the iteration continues, at most `max_refresh` times.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp


class Operator:
    """A sparse SPD matrix with its Jacobi preconditioner M = diag(A) (or M = I)."""

    def __init__(self, rowptr, colind, vals, n: Optional[int] = None, precond: str = "jacobi"):
        n = len(rowptr) - 1 if n is None else n
        self.A = sp.csr_matrix((np.asarray(vals, np.float64), np.asarray(colind), np.asarray(rowptr)),
                               shape=(n, n))
        self.n = n
        diag = self.A.diagonal()
        if precond == "jacobi":
            self.minv = 1.0 / diag
        elif precond == "none":
            self.minv = np.ones(n)
        else:
            raise ValueError(precond)
        self.precond = precond

    @classmethod
    def from_dense(cls, A, precond="jacobi"):
        S = sp.csr_matrix(np.asarray(A, np.float64))
        return cls(S.indptr, S.indices, S.data, S.shape[0], precond)

    def matvec(self, v):
        return self.A @ v


def chebyshev_basis(op: Operator, r, s: int, lam_min: float, lam_max: float, ncols: Optional[int] = None):
    """Columns p_0 .. p_(ncols-1) of the Chebyshev basis (Section 2, Definition):

        p_0 = r,  p_1 = theta (M^-1 A - sigma I) p_0,
        p_(j+1) = 2 theta (M^-1 A - sigma I) p_j - p_(j-1),   j >= 1,
        theta = 2 / (lam_max - lam_min),  sigma = (lam_max + lam_min) / 2.
    """
    ncols = s if ncols is None else ncols
    theta = 2.0 / (lam_max - lam_min)
    sigma = (lam_max + lam_min) / 2.0
    P = np.empty((op.n, ncols))
    P[:, 0] = r
    if ncols > 1:
        P[:, 1] = theta * (op.minv * op.matvec(P[:, 0]) - sigma * P[:, 0])
    for j in range(1, ncols - 1):
        P[:, j + 1] = 2.0 * theta * (op.minv * op.matvec(P[:, j]) - sigma * P[:, j]) - P[:, j - 1]
    return P


def monomial_basis(op: Operator, r, s: int):
    """p_j = (M^-1 A)^j r: the basis the paper contrasts with (Section 2, Section 4)."""
    P = np.empty((op.n, s))
    P[:, 0] = r
    for j in range(1, s):
        P[:, j] = op.minv * op.matvec(P[:, j - 1])
    return P


def gram(op: Operator, P, r):
    """G = P^T A P (lower triangle, mirrored) and c = P^T r (Section 1, Section 2)."""
    AP = np.column_stack([op.matvec(P[:, j]) for j in range(P.shape[1])])
    Gfull = P.T @ AP
    G = np.tril(Gfull) + np.tril(Gfull, -1).T
    c = P.T @ r
    return G, c, AP


def column_scaling(G, c):
    """Ruhe column scaling (Section 2): d_i = G_ii^-1/2, G~ = S G S, c~ = S c.

    A column whose G_ii is not a positive finite number is dropped (d_i = 0).
    """
    g = np.diag(G)
    ok = np.isfinite(g) & (g > 0.0)
    d = np.zeros_like(g)
    d[ok] = 1.0 / np.sqrt(g[ok])
    Gt = d[:, None] * G * d[None, :]
    ct = d * c
    return d, Gt, ct


def fgs(G, rhs, nu: int, alpha0=None):
    """nu Forward Gauss-Seidel sweeps on G a = rhs (Section 2; Section 3, Proposition
    "FGS Residual Structure", in its general form with D = diag(G)):

        (D + L) a^(l+1) = rhs - L^T a^(l),   a^(0) = 0 (or alpha0),

    swept forward j = 0 .. s-1 in place. With column scaling D = I. A zero diagonal entry
    (dropped column) keeps a_j = 0.
    """
    return fgs_iterates(G, rhs, nu, alpha0)[-1]


def fgs_iterates(G, rhs, nu: int, alpha0=None):
    """All sweep iterates a^(0) .. a^(nu) of `fgs` (Section 2's sweep; Section 3 states its
    residual structure in terms of them)."""
    s = G.shape[0]
    a = np.zeros(s) if alpha0 is None else np.array(alpha0, dtype=np.float64)
    out = [a.copy()]
    for _ in range(nu):
        for j in range(s):
            if G[j, j] == 0.0:
                a[j] = 0.0
                continue
            acc = rhs[j]
            for i in range(s):
                if i != j:
                    acc -= G[j, i] * a[i]
            a[j] = acc / G[j, j]
        out.append(a.copy())
    return out


def cholesky(G):
    """Plain Cholesky G = R^T R (R upper triangular), the direct Gram factorisation that
    Sections 1 and 8 compare FGS against; raises on a non-positive pivot."""
    s = G.shape[0]
    R = np.zeros_like(G)
    for j in range(s):
        acc = G[j, j] - sum(R[k, j] * R[k, j] for k in range(j))
        if not acc > 0.0:
            raise np.linalg.LinAlgError(f"non-positive pivot {acc} at {j}")
        R[j, j] = np.sqrt(acc)
        for i in range(j + 1, s):
            R[j, i] = (G[j, i] - sum(R[k, j] * R[k, i] for k in range(j))) / R[j, j]
    return R


def cholesky_solve(G, rhs):
    """Direct Gram solve by Cholesky and two triangular solves (the O(s^3) baseline of
    Sections 1 and 8)."""
    R = cholesky(G)
    s = G.shape[0]
    y = np.zeros(s)
    for i in range(s):
        y[i] = (rhs[i] - sum(R[k, i] * y[k] for k in range(i))) / R[i, i]
    a = np.zeros(s)
    for i in reversed(range(s)):
        a[i] = (y[i] - sum(R[i, k] * a[k] for k in range(i + 1, s))) / R[i, i]
    return a


def _gram_solve_scaled(Gt, ct, nu, solver):
    """a from the scaled Gram system G~ a = c~ of Section 2: nu FGS sweeps, or Cholesky on the
    kept (non-dropped) columns for the direct comparison of Sections 1 and 8."""
    if solver == "fgs":
        return fgs(Gt, ct, nu)
    if solver == "cholesky":
        keep = np.diag(Gt) > 0.0
        a = np.zeros_like(ct)
        if keep.any():
            a[keep] = cholesky_solve(Gt[np.ix_(keep, keep)], ct[keep])
        return a
    raise ValueError(solver)


@dataclass
class OuterRecord:
    """What one outer iteration computed (inputs r_k, outputs x_(k+1), r_(k+1))."""
    k: int
    res_norm: float
    d: np.ndarray
    Gt: np.ndarray
    ct: np.ndarray
    alpha: np.ndarray
    x: Optional[np.ndarray] = None
    r: Optional[np.ndarray] = None
    delta: float = 0.0   # ||c~ - G~ a|| / ||c~||: inexactness of the Gram solve (Section 7)


@dataclass
class SolveResult:
    x: np.ndarray
    outer_iters: int
    converged: bool
    rel_res_recursive: float
    rel_res_true: float
    refreshes: int
    r0_norm: float
    history: list = field(default_factory=list)


def solve(op: Operator, b, x0=None, *, s: int, nu: int, lam_min: float, lam_max: float,
          tol: float = 1e-8, max_outer: int = 100000, gram_solver: str = "fgs",
          basis_start: str = "r", max_refresh: int = 3, history: int = 0) -> SolveResult:
    """s-step CG (Section 2) with the Chebyshev basis, column scaling and FGS/Cholesky.

    `history` = number of leading outer iterations whose iterates (x, r) are kept.
    """
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
    while True:
        rel = float(np.linalg.norm(r)) / r0
        if rel < tol:
            rt = b - op.matvec(x)
            if float(np.linalg.norm(rt)) / r0 < tol or refreshes >= max_refresh:
                converged = float(np.linalg.norm(rt)) / r0 < tol
                break
            r = rt
            refreshes += 1
            continue
        if k >= max_outer:
            break
        p0 = r if basis_start == "r" else op.minv * r
        P = chebyshev_basis(op, p0, s, lam_min, lam_max)
        G, c, AP = gram(op, P, r)
        d, Gt, ct = column_scaling(G, c)
        if not np.any(d > 0.0):
            break
        a = _gram_solve_scaled(Gt, ct, nu, gram_solver)
        alpha = d * a
        x = x + P @ alpha
        r = r - AP @ alpha
        k += 1
        if k <= history:
            nct = float(np.linalg.norm(ct))
            delta = float(np.linalg.norm(ct - Gt @ a)) / nct if nct > 0 else 0.0
            hist.append(OuterRecord(k, rel, d, Gt, ct, alpha, x.copy(), r.copy(), delta))
    rel_true = float(np.linalg.norm(b - op.matvec(x))) / r0
    return SolveResult(x, k, converged, float(np.linalg.norm(r)) / r0, rel_true, refreshes, r0, hist)
