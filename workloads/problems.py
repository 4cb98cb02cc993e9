"""Synthetic SPD systems of the s-step CG workloads (seeded, reproducible).

Two discretisations on a structured grid with homogeneous Dirichlet boundaries. Unknown
(i, j, k) has linear index i + nx * (j + ny * k); 2D grids have nz = 1.

* Poisson (vertex-centred finite differences, unscaled): diagonal 2*dim, -1 for every
  neighbour that lies inside the grid. This is the 5-point (2D) / 7-point (3D) Laplacian;
  the h**-2 factor is dropped because the relative residual and the Jacobi-preconditioned
  iteration do not depend on it.
* Box-stencil Poisson (stencil="box"): every one of the 3**dim - 1 grid points of the unit
  box around a point (faces, edges and corners) is a neighbour with weight -1, and the
  diagonal is 3**dim - 1: the 27-point finite-difference Laplacian of the paper's experiments
  (Section 8) in 3D, the 9-point one in 2D, again without the h**-2 factor.
* Diffusion -div(kappa grad u) (cell-centred finite volumes): an interior face between cells
  a and b has coefficient w = 2 ka kb / (ka + kb) (harmonic mean); it adds w to both
  diagonals and -w to the two off-diagonal entries. A face on the domain boundary (Dirichlet
  value 0 half a cell away) adds 2 * k_cell to that cell's diagonal. With kappa > 0 the matrix
  is symmetric positive definite.

Seeds follow one scheme: exact solution x* = 1000 + config, coefficient field
kappa = 2000 + config, batch sides = 3000, finite-difference cells = 4000, Lanczos start
vector = 5000, adjoint target = 6005. Per-system streams of the batch use (base << 20) + index.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import rng

SEED_XSTAR = 1000
SEED_KAPPA = 2000
SEED_SIDES = 3000
SEED_FD_CELLS = 4000
SEED_LANCZOS = 5000
SEED_TARGET = 6005


def grid_shape(dims):
    nx, ny, nz = (tuple(dims) + (1, 1))[:3]
    return int(nx), int(ny), int(nz)


def grid_dim(dims) -> int:
    return 3 if grid_shape(dims)[2] > 1 or len(dims) == 3 else 2


def lognormal_kappa(dims, sigma: float, seed: int) -> np.ndarray:
    """Per-cell coefficient exp(sigma * N(0, 1))."""
    nx, ny, nz = grid_shape(dims)
    return np.exp(sigma * rng.normal(seed, nx * ny * nz))


def _axes(dims):
    """(stride, extent) per axis, i fastest."""
    nx, ny, nz = grid_shape(dims)
    out = [(1, nx), (nx, ny)]
    if grid_dim(dims) == 3:
        out.append((nx * ny, nz))
    return out


def _face_weight(ka, kb):
    return 2.0 * ka * kb / (ka + kb)


def csr(dims, kappa: Optional[np.ndarray] = None, index_dtype=np.int32):
    """CSR arrays (rowptr, colind, vals) of the Poisson (kappa None) or diffusion matrix.

    Columns are in ascending order inside each row. Assembled one k-plane slab at a time to
    bound temporaries.
    """
    nx, ny, nz = grid_shape(dims)
    n = nx * ny * nz
    axes = _axes(dims)
    d = len(axes)
    nslots = 2 * d + 1
    # (offset, axis) per slot in ascending order of the offset: -stride(last) ... -1, 0, +1 ...
    # +stride(last); the axis is carried with the slot (two axes share a stride when one of them
    # has extent 1, e.g. the y and z strides of an nx x 1 x nz grid)
    slots = [(-a[0], ax) for ax, a in reversed(list(enumerate(axes)))] + [(0, None)] + \
            [(a[0], ax) for ax, a in enumerate(axes)]
    counts = np.empty(n, dtype=np.int64)
    plane = nx * ny
    slab = max(1, (1 << 22) // plane)
    cols_parts, vals_parts = [], []
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        idx = np.arange(k0 * plane, k1 * plane, dtype=np.int64)
        coord = [idx % nx, (idx // nx) % ny, idx // plane]
        cols = np.empty((idx.size, nslots), dtype=np.int64)
        vals = np.zeros((idx.size, nslots), dtype=np.float64)
        valid = np.zeros((idx.size, nslots), dtype=bool)
        diag = np.zeros(idx.size, dtype=np.float64)
        kc = None if kappa is None else kappa[idx]
        for slot, (off, ax) in enumerate(slots):
            if off == 0:
                continue
            ext = axes[ax][1]
            inside = (coord[ax] > 0) if off < 0 else (coord[ax] < ext - 1)
            nb = idx + off
            cols[:, slot] = nb
            valid[:, slot] = inside
            if kappa is None:
                vals[inside, slot] = -1.0
            else:
                w = np.where(inside, _face_weight(kc, kappa[np.where(inside, nb, idx)]), 0.0)
                vals[:, slot] = -w
                diag += np.where(inside, w, 2.0 * kc)
        cslot = d
        cols[:, cslot] = idx
        valid[:, cslot] = True
        vals[:, cslot] = 2.0 * d if kappa is None else diag
        counts[idx] = valid.sum(axis=1)
        cols_parts.append(cols[valid].astype(index_dtype))
        vals_parts.append(vals[valid])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(index_dtype), np.concatenate(cols_parts), np.concatenate(vals_parts)


def apply(dims, x: np.ndarray, kappa: Optional[np.ndarray] = None) -> np.ndarray:
    """Matrix-free y = A x for the same matrices as `csr` (used to form b = A x*)."""
    nx, ny, nz = grid_shape(dims)
    shape = (nz, ny, nx)
    X = x.reshape(shape)
    Y = np.zeros(shape, dtype=np.result_type(x, np.float64 if kappa is None else kappa))
    d = grid_dim(dims)
    # numpy axis for grid axis 0 (i) is 2, for 1 (j) is 1, for 2 (k) is 0
    np_axes = [2, 1, 0][:d]
    if kappa is None:
        Y += 2.0 * d * X
        for ax in np_axes:
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            Y[tuple(lo)] -= X[tuple(hi)]
            Y[tuple(hi)] -= X[tuple(lo)]
        return Y.reshape(-1)
    K = kappa.reshape(shape)
    for ax in np_axes:
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        w = _face_weight(K[lo], K[hi])
        flux = w * (X[lo] - X[hi])
        Y[lo] += flux
        Y[hi] -= flux
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = slice(0, 1)
        last[ax] = slice(-1, None)
        first, last = tuple(first), tuple(last)
        Y[first] += 2.0 * K[first] * X[first]
        Y[last] += 2.0 * K[last] * X[last]
    return Y.reshape(-1)


def box_csr(dims, index_dtype=np.int32):
    """CSR arrays of the box-stencil Poisson matrix (columns ascending in each row)."""
    nx, ny, nz = grid_shape(dims)
    d = grid_dim(dims)
    n = nx * ny * nz
    rng_z = (-1, 0, 1) if d == 3 else (0,)
    # offsets (dz, dy, dx) in ascending order of the linear column index
    offs = [(dz, dy, dx) for dz in rng_z for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    plane = nx * ny
    slab = max(1, (1 << 21) // plane)
    counts = np.empty(n, dtype=np.int64)
    cols_parts, vals_parts = [], []
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        idx = np.arange(k0 * plane, k1 * plane, dtype=np.int64)
        ci, cj, ck = idx % nx, (idx // nx) % ny, idx // plane
        cols = np.empty((idx.size, len(offs)), dtype=np.int64)
        vals = np.empty((idx.size, len(offs)), dtype=np.float64)
        valid = np.empty((idx.size, len(offs)), dtype=bool)
        for slot, (dz, dy, dx) in enumerate(offs):
            inside = ((ci + dx >= 0) & (ci + dx < nx) & (cj + dy >= 0) & (cj + dy < ny) &
                      (ck + dz >= 0) & (ck + dz < nz))
            cols[:, slot] = idx + dx + nx * dy + plane * dz
            valid[:, slot] = inside
            vals[:, slot] = float(3 ** d - 1) if (dz, dy, dx) == (0, 0, 0) else -1.0
        counts[idx] = valid.sum(axis=1)
        cols_parts.append(cols[valid].astype(index_dtype))
        vals_parts.append(vals[valid])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(index_dtype), np.concatenate(cols_parts), np.concatenate(vals_parts)


def box_apply(dims, x: np.ndarray) -> np.ndarray:
    """Matrix-free y = A x of the box-stencil Poisson matrix (used to form b = A x*)."""
    nx, ny, nz = grid_shape(dims)
    d = grid_dim(dims)
    X = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.result_type(x, np.float64))
    X[1:-1, 1:-1, 1:-1] = x.reshape(nz, ny, nx)
    Y = float(3 ** d - 1) * X[1:-1, 1:-1, 1:-1]
    rng_z = (-1, 0, 1) if d == 3 else (0,)
    for dz in rng_z:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) != (0, 0, 0):
                    Y = Y - X[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return Y.reshape(-1)


@dataclass
class Problem:
    """One synthetic system A x = b with b = A x*, x0 = 0."""
    name: str
    dims: tuple
    kappa: Optional[np.ndarray]
    x_star: np.ndarray
    b: np.ndarray
    s: int
    nu: int
    tol: float = 1e-8
    meta: dict = field(default_factory=dict)
    stencil: str = "star"     # "star": 2 dim + 1 points (or diffusion); "box": 3**dim points

    @property
    def n(self) -> int:
        nx, ny, nz = grid_shape(self.dims)
        return nx * ny * nz

    def csr(self, index_dtype=np.int32):
        if self.stencil == "box":
            return box_csr(self.dims, index_dtype)
        return csr(self.dims, self.kappa, index_dtype)


def make(name: str, dims, *, kappa_sigma: Optional[float] = None, config: int = 0,
         s: int = 8, nu: int = 25, tol: float = 1e-8, xstar_seed: Optional[int] = None,
         kappa_seed: Optional[int] = None, stencil: str = "star", **meta) -> Problem:
    dims = tuple(int(v) for v in dims)
    nx, ny, nz = grid_shape(dims)
    n = nx * ny * nz
    if stencil not in ("star", "box") or (stencil == "box" and kappa_sigma is not None):
        raise ValueError("stencil is 'star' or 'box' (box: Poisson only)")
    kappa = None
    if kappa_sigma is not None:
        kappa = lognormal_kappa(dims, kappa_sigma, SEED_KAPPA + config if kappa_seed is None else kappa_seed)
    xs = rng.uniform(SEED_XSTAR + config if xstar_seed is None else xstar_seed, n)
    b = box_apply(dims, xs) if stencil == "box" else apply(dims, xs, kappa)
    return Problem(name, dims, kappa, xs, b, s, nu, tol, dict(meta, config=config), stencil)


# --- the workloads ------------------------------------------------------------------------

def poisson2d_64() -> Problem:
    """2D 5-point Poisson 64 x 64 (n = 4096), s = 4, nu = 20 (CSR)."""
    return make("poisson2d_64", (64, 64), config=1, s=4, nu=20)


def poisson3d(side: int = 256, s: int = 8, nu: int = 25, xstar_seed: Optional[int] = None) -> Problem:
    """3D 7-point Poisson side**3 (256**3 = 16.8M unknowns), s = 8, nu = 25; x* from seed
    1002 unless xstar_seed is given."""
    return make(f"poisson3d_{side}", (side, side, side), config=2, s=s, nu=nu, xstar_seed=xstar_seed)


def diffusion3d(side: int = 384, s: int = 12, nu: int = 30, sigma: float = 1.0) -> Problem:
    """3D 7-point variable-coefficient diffusion, log-normal kappa (sigma = 1)."""
    return make(f"diffusion3d_{side}", (side, side, side), kappa_sigma=sigma, config=3, s=s, nu=nu)


def poisson27(side: int = 230, s: int = 8, nu: int = 25) -> Problem:
    """3D 27-point Poisson side**3 (230**3 = 12.2M unknowns, the per-GPU size of the paper's
    experiments), s = 8, nu = 25."""
    return make(f"poisson27_{side}", (side, side, side), config=6, s=s, nu=nu, stencil="box")


def batch_sides(count: int = 512, lo: int = 32, hi: int = 512, seed: int = SEED_SIDES) -> np.ndarray:
    return rng.integers(seed, count, lo, hi)


def diffusion2d_batch(count: int = 512, lo: int = 32, hi: int = 512, sigma: float = 0.5,
                      s: int = 8, nu: int = 20, sides: Optional[np.ndarray] = None):
    """Independent square 2D diffusion systems with seeded sides U{lo..hi}."""
    if sides is None:
        sides = batch_sides(count, lo, hi)
    out = []
    for k, side in enumerate(sides):
        out.append(make(f"batch_{k}", (int(side), int(side)), kappa_sigma=sigma, config=4, s=s, nu=nu,
                        xstar_seed=((SEED_XSTAR + 4) << 20) + k, kappa_seed=((SEED_KAPPA + 4) << 20) + k))
    return out


def diffusion2d_adjoint(side: int = 1024, sigma: float = 0.5, s: int = 8, nu: int = 25):
    """2D diffusion with kappa = exp(N(0, sigma^2)); returns (problem, x_target)."""
    p = make(f"adjoint2d_{side}", (side, side), kappa_sigma=sigma, config=5, s=s, nu=nu, tol=1e-10)
    return p, rng.uniform(SEED_TARGET, p.n)


def fd_cells(n: int, count: int = 64, seed: int = SEED_FD_CELLS) -> np.ndarray:
    """`count` distinct seeded cell indices in [0, n) (first occurrences of a seeded stream)."""
    draws = rng.integers(seed, 8 * count + 64, 0, n - 1)
    _, first = np.unique(draws, return_index=True)
    return draws[np.sort(first)][:count].astype(np.int64)


def lanczos_start(n: int, seed: int = SEED_LANCZOS) -> np.ndarray:
    return rng.uniform(seed, n)
