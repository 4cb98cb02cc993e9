"""Autotuner for the batched form: picks s, nu and the launch shapes (unknowns per Gram/update
work item, resident blocks per SM of the stencil kernels) for a given batch.

For each candidate it runs two short probes on a subsample of the batch (the largest systems,
which set the batch's time, plus a spread of smaller ones): K1 and K2 > K1 outer iterations
with tolerance 0, through the library's batched solve. From them it takes
  * the device time per unknown and outer iteration, c = (t(K2) - t(K1)) / (sum_i n_i (K2 - K1)),
  * each system's contraction per outer iteration, rho_i = (r_i(K2) / r_i(K1))^(1 / (K2 - K1)),
    measured after the first K1 outer iterations, where the smooth error modes dominate,
and predicts the time to tol as c * sum_i n_i N_i with N_i = K1 + log(tol / r_i(K1)) / log(rho_i)
(converged systems leave the batch, so each costs only its own outer iterations). The
candidate with the smallest prediction wins. All solves run in libsstep_cg.so.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import abi

DEFAULT_CANDIDATES = [
    {"s": s, "nu": nu, "batch_chunk": chunk, "batch_ctas_per_sm": ctas}
    for (s, nu) in ((4, 20), (8, 20), (8, 30), (12, 30), (16, 30))
    for chunk in (8192, 32768)
    for ctas in (4, 6)
]


@dataclass
class TuneResult:
    best: dict
    predicted_s: float
    table: List[dict] = field(default_factory=list)
    sample: List[int] = field(default_factory=list)


def pick_sample(sizes: Sequence[int], k: int = 16) -> List[int]:
    """The k//2 largest systems and k - k//2 others spread evenly over the remaining sizes."""
    order = list(np.argsort(-np.asarray(sizes), kind="stable"))
    big = order[: k // 2]
    rest = order[k // 2:]
    m = k - len(big)
    if m > 0 and rest:
        idx = np.linspace(0, len(rest) - 1, num=min(m, len(rest))).round().astype(int)
        big += [rest[i] for i in idx]
    return sorted(set(int(i) for i in big))


def _probe(grids, kappas, bs, cand: dict, outers: int, stream=None):
    opts = abi.sstep_cg_default_opts(tol=1e-30, max_outer=outers, use_graph=1, **cand)
    h = abi.sstep_cg_batch_create(grids, kappas, opts, stream)
    try:
        offs, total, _ = abi.sstep_cg_batch_layout(h, len(grids))
        b = torch.zeros(total, dtype=torch.float64, device="cuda")
        for bi, o in zip(bs, offs):
            b[o:o + bi.numel()] = bi
        x = torch.zeros_like(b)
        abi.sstep_cg_batch_solve(h, b, x, len(grids))          # warm (graph capture, lazy loading)
        x.zero_()
        infos, summary = abi.sstep_cg_batch_solve(h, b, x, len(grids))
    finally:
        abi.sstep_cg_batch_destroy(h)
    return summary["ms"], [i["rel_res_true"] for i in infos]


def tune(grids, kappas, bs, tol: float = 1e-8, candidates: Optional[list] = None, sample: int = 16,
         k1: int = 20, k2: int = 60, stream=None) -> TuneResult:
    """grids: list of (nx, ny[, nz]); kappas: CUDA tensors or None; bs: CUDA right-hand sides."""
    candidates = candidates or DEFAULT_CANDIDATES
    sizes = [int(np.prod(g)) for g in grids]
    idx = pick_sample(sizes, sample)
    sg = [grids[i] for i in idx]
    sk = [kappas[i] for i in idx]
    sb = [bs[i] for i in idx]
    # the sample stands for the whole batch: scale by unknowns
    scale = sum(sizes) / sum(sizes[i] for i in idx)
    table = []
    for cand in candidates:
        t1, r1 = _probe(sg, sk, sb, cand, k1, stream)
        t2, r2 = _probe(sg, sk, sb, cand, k2, stream)
        n_s = [sizes[i] for i in idx]
        c = max(t2 - t1, 1e-6) / (sum(n_s) * (k2 - k1))          # ms per unknown-outer
        work = 0.0
        for n, a, b in zip(n_s, r1, r2):
            if b <= tol or a <= 0.0:
                N = k2
            else:
                rho = (b / a) ** (1.0 / (k2 - k1)) if b < a else 1.0 - 1e-9
                N = k1 + math.log(tol / a) / math.log(rho) if rho < 1.0 else 1e9
            work += n * N
        pred_ms = c * work * scale
        table.append(dict(cand, ms_per_unknown_outer=c, predicted_s=pred_ms / 1e3))
    best = min(table, key=lambda r: r["predicted_s"])
    params = {k: best[k] for k in ("s", "nu", "batch_chunk", "batch_ctas_per_sm")}
    return TuneResult(best=params, predicted_s=best["predicted_s"], table=table, sample=idx)
