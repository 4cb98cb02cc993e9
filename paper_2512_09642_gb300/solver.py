"""SStepCG: one solver handle over a device-resident SPD system (torch tensors).

A thin owner of the C handle: it keeps the borrowed device arrays alive, allocates the
output vector and turns options into the C struct. The work is done by libsstep_cg.so.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import abi


def check_array(t, name: str, numel: int, dtype, device=None):
    """Refuses what the C ABI cannot check: it takes plain pointers with the lengths the
    handle implies, so a tensor with another element type, fewer elements or on another
    device would be read or written out of bounds."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if device is not None and t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got {t.device}")


class SStepCG:
    """Chebyshev-basis s-step CG (arXiv 2512.09642, Section 2) on one CUDA device.

    Exactly one of `csr=(rowptr, colind, vals)` (int32, int32, float64 CUDA tensors) or
    `grid=(nx, ny[, nz])` (matrix-free Poisson, or diffusion with `kappa`; stencil="box" gives
    the 9-/27-point box Poisson operator of Section 8) is given.
    Options are the fields of sstep_cg_opts (s, nu, tol, bounds_mode, lambda_min, ...);
    `bounds=(lmin, lmax)` is shorthand for bounds_mode="given".
    """

    def __init__(self, *, csr=None, grid=None, kappa: Optional[torch.Tensor] = None, bounds=None, stream=None,
                 stencil: str = "star", **opts):
        if (csr is None) == (grid is None):
            raise ValueError("give exactly one of csr= or grid=")
        if stencil not in ("star", "box") or (stencil == "box" and kappa is not None):
            raise ValueError("stencil is 'star' (5/7-point or diffusion) or 'box' (9/27-point Poisson)")
        if bounds is not None:
            opts.update(bounds_mode="given", lambda_min=float(bounds[0]), lambda_max=float(bounds[1]))
        self.opts = abi.sstep_cg_default_opts(**opts)
        self._keep = []
        self.stream = stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        if csr is not None:
            rowptr, colind, vals = csr
            self.n = rowptr.numel() - 1
            check_array(rowptr, "rowptr", self.n + 1, torch.int32, self.device)
            check_array(colind, "colind", colind.numel(), torch.int32, self.device)
            check_array(vals, "vals", colind.numel(), torch.float64, self.device)
            self._keep += [rowptr, colind, vals]
            self.h = abi.sstep_cg_create_csr(self.n, rowptr, colind, vals, self.opts, stream)
        else:
            dims = tuple(int(v) for v in grid)
            dim = len(dims)
            nx, ny, nz = (dims + (1, 1))[:3]
            self.n = nx * ny * nz
            if kappa is not None:
                check_array(kappa, "kappa", self.n, torch.float64, self.device)
                self._keep.append(kappa)
            if stencil == "box":
                self.h = abi.sstep_cg_create_box_stencil(dim, nx, ny, nz, self.opts, stream)
            else:
                self.h = abi.sstep_cg_create_stencil(dim, nx, ny, nz, kappa, self.opts, stream)

    def _vec(self, t, name: str, ncols: int = 1):
        check_array(t, name, ncols * self.n, torch.float64, self.device)
        return t

    @property
    def s(self) -> int:
        return self.opts.s

    def solve(self, b: torch.Tensor, x0: Optional[torch.Tensor] = None, allow_no_convergence: bool = True):
        """Returns (x, info dict); x0 defaults to zeros. x is a new tensor: with use_graph the
        handle captures its outer-loop graph again for each new (b, x) pair, so loops of solves
        that want the graph reused call solve_into with the same buffers."""
        self._vec(b, "b")
        x = torch.zeros_like(b) if x0 is None else self._vec(x0, "x0").clone()
        info = abi.sstep_cg_solve(self.h, b, x, allow=(5,) if allow_no_convergence else ())
        return x, info.as_dict()

    def solve_into(self, b: torch.Tensor, x: torch.Tensor):
        return abi.sstep_cg_solve(self.h, self._vec(b, "b"), self._vec(x, "x")).as_dict()

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        self._vec(x, "x")
        y = torch.empty_like(x)
        abi.sstep_cg_apply(self.h, x, y)
        return y

    def basis(self, r: torch.Tensor, ncols: int) -> torch.Tensor:
        """Chebyshev basis columns p_0 .. p_(ncols-1), returned as an (ncols, n) tensor."""
        self._vec(r, "r")
        P = torch.empty((ncols, self.n), dtype=torch.float64, device=r.device)
        abi.sstep_cg_basis(self.h, r, P, self.n, ncols)
        return P

    def gram_solve(self, P: torch.Tensor):
        """Gram reduction + scaling + Gram solve on a given basis P ((s+1, n), row j = p_j)."""
        abi.sstep_cg_load_basis(self.h, self._vec(P, "P", self.s + 1).contiguous(), self.n)
        return abi.sstep_cg_gram_solve(self.h, self.s)

    def residual(self) -> torch.Tensor:
        r = torch.empty(self.n, dtype=torch.float64, device=self.device)
        abi.sstep_cg_get_residual(self.h, r)
        return r

    @property
    def bounds(self):
        return abi.sstep_cg_get_bounds(self.h)

    def lanczos(self, k: int, seed: int):
        return abi.sstep_cg_lanczos(self.h, k, seed)

    def close(self):
        if getattr(self, "h", None):
            abi.sstep_cg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
