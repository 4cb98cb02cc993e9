"""Autotuner for the batched form: picks s, nu, the Gram form and the launch shapes (unknowns
per Gram/update work item, resident blocks per SM of the stencil kernels) for a given batch,
in two stages: (s, nu, Gram form) over DEFAULT_CANDIDATES at the default shapes, then the
launch shapes over SHAPE_CANDIDATES at the chosen (s, nu, form).

For each candidate it solves a subsample of the batch to the tolerance with the library's
batched solve (the largest systems, which set the batch's critical path, plus a spread of
smaller ones). From that run it takes
  * each sampled system's outer-iteration count N_i, fitted as N = a n^b over system size n
    (outer counts of these solves grow as a power of the grid size), and
  * the device time per unknown and outer iteration, c = t / sum_i n_i N_i,
and predicts the batch's time as c * sum_j n_j N(n_j) (a converged system leaves the batch,
so each costs only its own outer iterations). The candidate with the smallest prediction
wins. Short probes of a few outer iterations are not used: the contraction of the early
outer iterations is much faster than the asymptotic one and mispredicts the count by
orders of magnitude. All solves run in libsstep_cg.so.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import abi

DEFAULT_CANDIDATES = [
    {"s": s, "nu": nu, "gram_form": form, "batch_chunk": 8192, "batch_ctas_per_sm": 6}
    for (s, nu) in ((6, 20), (8, 20), (8, 30), (10, 25), (12, 30))
    for form in ("direct", "moments")
]


SHAPE_CANDIDATES = [{"batch_chunk": chunk, "batch_ctas_per_sm": ctas}
                    for chunk in (4096, 8192, 16384) for ctas in (4, 6, 8)]


@dataclass
class TuneResult:
    best: dict
    predicted_s: float
    table: List[dict] = field(default_factory=list)
    sample: List[int] = field(default_factory=list)


def pick_sample(sizes: Sequence[int], k: int = 12) -> List[int]:
    """The k//2 largest systems and k - k//2 others spread evenly over the remaining sizes."""
    order = list(np.argsort(-np.asarray(sizes), kind="stable"))
    chosen = order[: k // 2]
    rest = order[k // 2:]
    m = k - len(chosen)
    if m > 0 and rest:
        idx = np.linspace(0, len(rest) - 1, num=min(m, len(rest))).round().astype(int)
        chosen += [rest[i] for i in idx]
    return sorted(set(int(i) for i in chosen))


def _solve_sample(grids, kappas, bs, cand: dict, tol: float, max_outer: int, stream=None):
    opts = abi.sstep_cg_default_opts(tol=tol, max_outer=max_outer, use_graph=1, **cand)
    h = abi.sstep_cg_batch_create(grids, kappas, opts, stream)
    try:
        offs, total, _ = abi.sstep_cg_batch_layout(h, len(grids))
        b = torch.zeros(total, dtype=torch.float64, device="cuda")
        for bi, o in zip(bs, offs):
            b[o:o + bi.numel()] = bi
        x = torch.zeros_like(b)
        infos, summary = abi.sstep_cg_batch_solve(h, b, x, len(grids))
    finally:
        abi.sstep_cg_batch_destroy(h)
    return summary["ms"], [i["outer_iters"] for i in infos], [i["status"] for i in infos]


def tune(grids, kappas, bs, tol: float = 1e-8, candidates: Optional[list] = None, sample: int = 12,
         max_outer: int = 40000, stream=None, shapes: Optional[list] = None) -> TuneResult:
    """grids: list of (nx, ny[, nz]); kappas: CUDA tensors or None; bs: CUDA right-hand sides.
    shapes: launch shapes of the second stage (SHAPE_CANDIDATES by default; [] skips it)."""
    candidates = candidates or DEFAULT_CANDIDATES
    shapes = SHAPE_CANDIDATES if shapes is None else shapes
    sizes = np.array([int(np.prod(g)) for g in grids], dtype=np.float64)
    idx = pick_sample(list(sizes), sample)
    sg = [grids[i] for i in idx]
    sk = [kappas[i] for i in idx]
    sb = [bs[i] for i in idx]
    n_s = sizes[idx]
    table = []

    def run(cand, stage):
        ms, outers, status = _solve_sample(sg, sk, sb, cand, tol, max_outer, stream)
        N = np.maximum(np.asarray(outers, dtype=np.float64), 1.0)
        ok = all(st == "SSTEP_OK" for st in status)
        # N = a n^b by least squares in log-log
        b_, a_ = np.polyfit(np.log(n_s), np.log(N), 1) if len(set(n_s)) > 1 else (0.0, np.log(N.mean()))
        N_all = np.exp(a_) * sizes ** b_
        c = ms / float(np.sum(n_s * N))                      # ms per unknown-outer on the sample
        pred = c * float(np.sum(sizes * N_all)) / 1e3
        row = dict(cand, stage=stage, sample_ms=ms, fit_exponent=float(b_),
                   predicted_s=pred if ok else float("inf"), sample_max_outer=int(N.max()),
                   ns_per_unknown_outer=c * 1e6)
        table.append(row)
        return row

    for cand in candidates:
        run(cand, "basis")
    best = min(table, key=lambda r: r["predicted_s"])
    keys = ("s", "nu", "gram_form", "batch_chunk", "batch_ctas_per_sm")
    for shape in shapes:
        cand = dict({k: best[k] for k in keys}, **shape)
        if any(all(r[k] == cand[k] for k in keys) for r in table):
            continue   # this shape was measured in the first stage
        run(cand, "shape")
    best = min(table, key=lambda r: r["predicted_s"])
    params = {k: best[k] for k in keys}
    return TuneResult(best=params, predicted_s=best["predicted_s"], table=table, sample=idx)
