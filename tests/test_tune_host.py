"""Host logic of the batched-form autotuner (paper_2512_09642_gb300/tune.py), on the CPU: the
sample it solves, and its prediction of the batch time from the sample's outer-iteration
counts and device time, with the GPU solve of the sample replaced by a model whose answer is
known in closed form."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def tune():
    from paper_2512_09642_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2512_09642_gb300 import tune as mod
    return mod


def test_pick_sample_takes_the_largest_and_a_spread(tune):
    sizes = [5, 90, 12, 300, 7, 41, 300, 64, 2, 150, 18, 77, 33, 250, 9, 120]
    idx = tune.pick_sample(sizes, 6)
    assert idx == sorted(set(idx)) and len(idx) == 6
    largest = np.argsort(-np.asarray(sizes), kind="stable")[:3]
    assert set(int(i) for i in largest) <= set(idx)
    rest = [i for i in idx if i not in set(int(j) for j in largest)]
    # the others spread from the largest remaining size down to the smallest
    assert sizes.index(2) in rest and sizes.index(150) in rest
    assert tune.pick_sample(sizes[:4], 12) == [0, 1, 2, 3]


def test_prediction_and_choice_follow_the_fitted_model(tune, monkeypatch):
    sides = [32, 40, 57, 64, 80, 96, 111, 128, 150, 181, 200, 256, 300, 333, 400, 512]
    grids = [(s, s) for s in sides]
    sizes = np.array([s * s for s in sides], dtype=np.float64)
    # per candidate: outer count N = a n^b and device time c ms per unknown-outer; one fails
    model = {6: (3.0, 0.52, 2e-6, "SSTEP_OK"), 8: (2.0, 0.50, 2.5e-6, "SSTEP_OK"),
             10: (1.2, 0.55, 3e-6, "SSTEP_OK"), 12: (0.5, 0.40, 1e-6, "SSTEP_ERR_NO_CONVERGENCE")}

    def fake_solve(sg, sk, sb, cand, tol, max_outer, stream=None):
        a, b, c, st = model[cand["s"]]
        n = np.array([g[0] * g[1] for g in sg], dtype=np.float64)
        N = a * n ** b
        return c * float(np.sum(n * N)), list(N), [st] * len(sg)

    monkeypatch.setattr(tune, "_solve_sample", fake_solve)
    cands = [{"s": s, "nu": 20, "gram_form": "moments", "batch_chunk": 8192, "batch_ctas_per_sm": 6} for s in model]
    res = tune.tune(grids, [None] * len(grids), [None] * len(grids), candidates=cands, sample=8)
    want = {s: (c * float(np.sum(sizes * a * sizes ** b)) / 1e3 if st == "SSTEP_OK" else float("inf"))
            for s, (a, b, c, st) in model.items()}
    for row in res.table:
        a, b, c, st = model[row["s"]]
        if st == "SSTEP_OK":
            assert row["predicted_s"] == pytest.approx(want[row["s"]], rel=1e-9)
            assert row["fit_exponent"] == pytest.approx(b, rel=1e-9)
        else:
            assert row["predicted_s"] == float("inf")
    best_s = min((s for s in model if model[s][3] == "SSTEP_OK"), key=lambda s: want[s])
    assert res.best["s"] == best_s and res.predicted_s == pytest.approx(want[best_s], rel=1e-9)
    assert set(res.best) == {"s", "nu", "gram_form", "batch_chunk", "batch_ctas_per_sm"}
    assert len(res.sample) == 8


def test_second_stage_picks_the_fastest_launch_shape(tune, monkeypatch):
    """The shape stage re-solves the sample at the first stage's (s, nu, form) for every launch
    shape (unknowns per Gram/update item x resident stencil blocks per SM) and keeps the one
    with the smallest predicted batch time; shapes do not change the outer counts here."""
    grids = [(s, s) for s in (32, 64, 96, 128, 160, 192, 224, 256)]
    speed = {(4096, 4): 1.30, (4096, 6): 1.10, (4096, 8): 1.20, (8192, 4): 1.05, (8192, 6): 1.00,
             (8192, 8): 0.97, (16384, 4): 1.15, (16384, 6): 0.91, (16384, 8): 0.99}
    calls = []

    def fake_solve(sg, sk, sb, cand, tol, max_outer, stream=None):
        calls.append(dict(cand))
        n = np.array([g[0] * g[1] for g in sg], dtype=np.float64)
        N = (2.0 if cand["s"] == 8 else 3.0) * n ** 0.5
        c = 1e-6 * speed[(cand["batch_chunk"], cand["batch_ctas_per_sm"])]
        return c * float(np.sum(n * N)), list(N), ["SSTEP_OK"] * len(sg)

    monkeypatch.setattr(tune, "_solve_sample", fake_solve)
    cands = [{"s": s, "nu": 20, "gram_form": "moments", "batch_chunk": 8192, "batch_ctas_per_sm": 6} for s in (6, 8)]
    res = tune.tune(grids, [None] * len(grids), [None] * len(grids), candidates=cands, sample=6)
    assert res.best == {"s": 8, "nu": 20, "gram_form": "moments", "batch_chunk": 16384, "batch_ctas_per_sm": 6}
    shape_rows = [r for r in res.table if r["stage"] == "shape"]
    assert len(shape_rows) == 8 and all(r["s"] == 8 for r in shape_rows)   # 9 shapes, one already measured
    assert len(calls) == 2 + 8
    # without the second stage the first stage's choice stands
    res1 = tune.tune(grids, [None] * len(grids), [None] * len(grids), candidates=cands, sample=6, shapes=[])
    assert res1.best["batch_chunk"] == 8192 and res1.best["batch_ctas_per_sm"] == 6
