"""Oracle: FGS as the AMG coarse-grid solver (Section 6, "AMG Coarse-Grid Extension").

Test infrastructure only (see the package docstring). Paper: arXiv 2512.09642.

At a coarse level with prolongation P (n_f x n_c) the coarse operator is A_c = P^T A_f P.
Section 6 replaces the direct coarse solve by nu Forward Gauss-Seidel sweeps on A_c y = g
(Proposition "AMG Convergence": kappa(A_c) stays bounded, so a fixed nu of 10-30 suffices),
and notes that the sweeps can stream A_f instead of forming A_c. Here P is an aggregation
prolongation (column i is the indicator of aggregate i, a stand-in for an AMG hierarchy's P):

  * `coarse_operator` forms A_c = P^T A_f P by its definition (sparse products);
  * `coarse_fgs` runs nu sweeps of Section 2's FGS in its general form (D = diag(A_c),
    y^(0) = y0, rows in increasing order) on the formed A_c;
  * `coarse_fgs_streaming` runs the same sweeps without A_c: it keeps z = P y on the fine
    level, and row i of A_c y is p_i^T A_f z, the sum of (A_f z) over aggregate i; after
    y_i changes by delta, z changes by delta on aggregate i. In exact arithmetic both give
    the same iterates.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .sstep_cg import Operator, fgs


def box_aggregates(dims, block):
    """Aggregate id of every fine point for aggregates that are block[0] x block[1] (x
    block[2]) boxes of the grid (the last box along an axis may be smaller), ids ordered
    x fastest over the coarse grid; returns (agg, n_c, coarse dims). Section 6 takes P from
    an AMG hierarchy; box aggregation stands in for it (a reading)."""
    nx, ny, nz = (tuple(dims) + (1, 1))[:3]
    bx, by, bz = (tuple(block) + (1, 1))[:3]
    cx, cy, cz = -(-nx // bx), -(-ny // by), -(-nz // bz)
    idx = np.arange(nx * ny * nz, dtype=np.int64)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    agg = (i // bx) + cx * ((j // by) + cy * (k // bz))
    return agg.astype(np.int64), cx * cy * cz, (cx, cy, cz)


def prolongation(agg, n_c):
    """The aggregation prolongation P (n_f x n_c, column i the indicator of aggregate i) that
    stands in for the P of Section 6."""
    n_f = len(agg)
    return sp.csr_matrix((np.ones(n_f), (np.arange(n_f), agg)), shape=(n_f, n_c))


def coarse_operator(op: Operator, agg, n_c):
    """A_c = P^T A_f P (dense), the coarse operator of Section 6."""
    P = prolongation(agg, n_c)
    return (P.T @ (op.A @ P)).toarray()


def coarse_fgs(Ac, g, nu: int, y0=None):
    """nu FGS sweeps on the formed A_c (general D = diag(A_c) form of Section 2's sweep)."""
    return fgs(np.asarray(Ac, np.float64), np.asarray(g, np.float64), nu, y0)


def coarse_fgs_streaming(op: Operator, agg, n_c: int, g, nu: int, y0=None):
    """The same sweeps with A_c never formed (Section 6's streaming form): rows of A_c y
    from the fine level."""
    agg = np.asarray(agg)
    g = np.asarray(g, np.float64)
    y = np.zeros(n_c) if y0 is None else np.array(y0, dtype=np.float64)
    members = [np.flatnonzero(agg == i) for i in range(n_c)]
    A = op.A.tocsr()
    # diag(A_c)_i = p_i^T A_f p_i: the sum of A_f over rows and columns of aggregate i
    dc = np.array([A[m][:, m].sum() for m in members])
    z = y[agg].astype(np.float64)
    for _ in range(nu):
        for i in range(n_c):
            m = members[i]
            if dc[i] == 0.0:
                continue
            s = float((A[m] @ z).sum())          # (A_c y)_i = p_i^T A_f (P y)
            delta = (g[i] - s) / dc[i]
            y[i] += delta
            z[m] += delta
    return y
