"""bench.py's JSON line on the CPU: run_ours on a small 3D Poisson grid with the CUDA calls and the
library's solve replaced by stand-ins (fixed event times, fixed solve records), so that the
line's keys and their arithmetic (value, ms_per_step, e2e bytes, roofline, launch count,
speedups) are checked without a GPU. The CPU baseline leg runs the oracle for real."""
import json
import os
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SIDE, STEPS, WARMUP = 8, 2, 1
EVENT_MS = 1500.0        # every timed region: 1.5 s over STEPS solves
OUTERS, LAUNCHES = 12, 150


@pytest.fixture
def fake_gpu(monkeypatch):
    import paper_2512_09642_gb300 as pkg
    from paper_2512_09642_gb300 import abi

    class Event:
        def __init__(self, **kw):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return EVENT_MS

    zeros = torch.zeros
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(torch, "zeros", lambda *a, device=None, **k: zeros(*a, **k))

    calls = {"device": [], "host": 0}

    class Info:
        def __init__(self, mixed):
            self.mixed = mixed

        def as_dict(self):
            return {"outer_iters": OUTERS, "status": "SSTEP_OK", "rel_res_true": 5e-9, "kernel_launches": LAUNCHES,
                    "prof_ms": [0.8, 0.3, 0.2, 0.1], "prof_launches": [8, 1, 1, 1], "refreshes": 0,
                    "step_tma": 1 if self.mixed else 0, "ms": EVENT_MS / STEPS}

    class Solver:
        def __init__(self, **kw):
            self.h = object()
            self.mixed = kw.get("precision") == "mixed"

        def close(self):
            pass

    handles = {}

    def make(**kw):
        sv = Solver(**kw)
        handles[id(sv.h)] = sv
        return sv

    def solve(h, b, x, allow=(5,)):
        calls["device"].append(x.data_ptr())
        x.copy_(b)
        return Info(handles[id(h)].mixed)

    def solve_host(h, b, x, allow=(5,)):
        calls["host"] += 1
        return Info(handles[id(h)].mixed)

    monkeypatch.setattr(pkg, "SStepCG", make, raising=False)
    monkeypatch.setattr(abi, "sstep_cg_solve", solve)
    monkeypatch.setattr(abi, "sstep_cg_solve_host", solve_host)
    return calls


def test_bench_line_carries_every_contract_key(fake_gpu, monkeypatch, capsys):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--side", str(SIDE), "--steps", str(STEPS), "--warmup",
                                      str(WARMUP), "--no-spread", "--cpu-outers", "1",
                                      "--forms", "fp64+mom,mixed+fused+r8"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_ours(bench.parse())
    out = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(out) == 1
    d = json.loads(out[0])

    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"):
        assert k in d, k
    assert d["value"] == pytest.approx(EVENT_MS / STEPS / 1e3) and d["ms_per_step"] == pytest.approx(EVENT_MS / STEPS)
    assert (d["n_gpus"], d["steps"], d["warmup"], d["unit"]) == (1, STEPS, WARMUP, "s")
    assert d["higher_is_better"] is False and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["config"]["workload"].startswith(f"poisson3d_7pt_{SIDE}")

    n = SIDE ** 3
    assert d["e2e"]["unit"] == "s" and d["e2e"]["value"] is not None
    assert (d["e2e"]["h2d_bytes_per_step"], d["e2e"]["d2h_bytes_per_step"]) == (16 * n, 8 * n)
    assert d["gpu_launches"] == STEPS * LAUNCHES

    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel"):
        assert k in roof, k
    assert roof["bound"] in ("alu", "hbm") and roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    # 8 step launches at 0.1 ms against one Gram at 0.3 and one update at 0.2: the step dominates
    assert roof["kernel"] == "cheb_step" and roof["avg_launch_ms"] == pytest.approx(0.1)

    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0 and cpu["sample"]
    assert cpu["all_cores"]["cores"] >= 1

    forms = d["forms"]
    assert set(forms) == {"fp64+mom", "mixed+fused+r8"}
    assert forms["mixed+fused+r8"]["fp32_step"] == "tma" and forms["fp64+mom"]["fp32_step"] is None
    assert forms["mixed+fused+r8"]["speedup_vs"] == "fp64+mom"
    assert forms["fp64+mom"]["ms_per_outer"] == pytest.approx(EVENT_MS / STEPS / OUTERS)

    # one output vector per form: every device solve of a form writes the same address, and the
    # end-to-end leg runs the warm-up and the timed host solves of the headline form
    ptrs = fake_gpu["device"]
    per_form = WARMUP + STEPS + 2           # + the two host-loop solves that sample the kernels
    assert len(ptrs) == 2 * per_form
    assert len(set(ptrs[:per_form])) == 1 and len(set(ptrs[per_form:])) == 1
    assert fake_gpu["host"] == WARMUP + STEPS


def test_sweep_line_reports_every_s_and_form(fake_gpu, monkeypatch, capsys):
    """--workload sweep: one row per s in {4, 8, 12, 16} and form (FP64 moments, mixed fused
    refresh every 8), each from its own solve's record, in one JSON line."""
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "sweep", "--side", str(SIDE), "--sweep-outers", "2",
                                      "--steps", "1", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_sweep(bench.parse())
    out = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(out) == 1
    d = json.loads(out[0])
    rows = d["sweep"]
    assert [(r["s"], r["form"]) for r in rows] == [(s, f) for s in (4, 8, 12, 16) for f in ("fp64+mom", "mixed+fused+r8")]
    for r in rows:
        assert r["fp32_step"] == ("tma" if r["form"].startswith("mixed") else None)
        assert r["ms_per_outer"] == pytest.approx(EVENT_MS / 1 / 1e3 / OUTERS * 1e3)
        assert r["dominant"]["kernel"] == "cheb_step" and r["outer_iters"] == OUTERS
    assert d["config"]["workload"] == f"poisson3d_7pt_{SIDE}^3_s_sweep"


@pytest.mark.parametrize("extra,workload", [
    (["--workload", "poisson27"], "poisson3d_27pt_8^3"),
    (["--workload", "poisson2d_64"], "poisson2d_5pt_64^2"),
    (["--workload", "diffusion3d", "--no-cpu-baseline"], "diffusion3d_7pt_8^3_lognormal1"),
    (["--csr"], "poisson3d_7pt_8^3_csr"),
])
def test_other_workload_lines(fake_gpu, monkeypatch, capsys, extra, workload):
    """The other workloads' lines (27-point box stencil, 2D CSR, 3D diffusion, 3D Poisson as
    CSR) carry the same keys; the CSR lines count the matrix bytes in their roofline."""
    monkeypatch.setattr(sys, "argv", ["bench.py", "--side", str(SIDE), "--steps", "1", "--warmup", "1", "--no-spread",
                                      "--cpu-outers", "1", "--forms", "fp64+mom,mixed+mom"] + extra)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_ours(bench.parse())
    out = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["config"]["workload"].startswith(workload), d["config"]
    for k in ("metric", "value", "unit", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline", "forms"):
        assert k in d, k
    assert set(d["forms"]) == {"fp64+mom", "mixed+mom"}
    if "csr" in workload or "2d" in workload:
        by = d["roofline"]["bytes_per_launch"]
        n = 64 * 64 if "2d" in workload else SIDE ** 3
        assert by > 24 * n   # the step reads the matrix: 12 nnz/n + 4 bytes per row on top of the vectors


def test_a_failing_secondary_form_is_reported_not_fatal(fake_gpu, monkeypatch, capsys):
    """A secondary form whose solve raises is recorded as an error in `forms`; the headline line
    is still printed (a failing headline form ends the run)."""
    from paper_2512_09642_gb300 import abi
    good = abi.sstep_cg_solve

    def solve(h, b, x, allow=(5,)):
        info = good(h, b, x, allow)
        if info.mixed:
            raise abi.SStepError(4, "out of memory (stand-in)")
        return info

    monkeypatch.setattr(abi, "sstep_cg_solve", solve)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--side", str(SIDE), "--steps", "1", "--warmup", "1", "--no-spread",
                                      "--no-cpu-baseline", "--forms", "fp64+mom,mixed+fused+r8"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_ours(bench.parse())
    out = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["form"] == "fp64+mom" and d["value"] > 0
    assert "out of memory" in d["forms"]["mixed+fused+r8"]["error"]
    assert "speedup_vs" not in d["forms"]["fp64+mom"]

    # the headline form failing is fatal
    monkeypatch.setattr(sys, "argv", ["bench.py", "--side", str(SIDE), "--steps", "1", "--warmup", "1", "--no-spread",
                                      "--no-cpu-baseline", "--forms", "mixed+fused+r8,fp64+mom"])
    with pytest.raises(abi.SStepError):
        bench.run_ours(bench.parse())


def test_xstar_spread_and_its_failure(fake_gpu, monkeypatch, capsys):
    """The headline line's `xstar_spread` (five seeded x*), and an error entry in its place when
    it fails."""
    argv = ["bench.py", "--side", str(SIDE), "--steps", "1", "--warmup", "1", "--no-cpu-baseline", "--forms", "fp64+mom"]
    monkeypatch.setattr(sys, "argv", argv)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_ours(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    sp = d["xstar_spread"]
    assert [r["xstar_seed"] for r in sp["runs"]] == list(bench.SPREAD_SEEDS)
    assert sp["outer_min"] <= sp["outer_median"] <= sp["outer_max"] and sp["form"] == "fp64+mom"

    def broken(*a, **k):
        raise RuntimeError("stand-in failure")

    monkeypatch.setattr(bench, "xstar_spread", broken)
    bench.run_ours(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    assert d["xstar_spread"] == {"form": "fp64+mom", "error": "RuntimeError: stand-in failure"}


def test_coarse_line(fake_gpu, monkeypatch, capsys):
    """--workload coarse: both modes timed (streaming the headline), their memory footprints
    (n_c^2 doubles formed, n_f + n_c streaming) and the line's keys."""
    from paper_2512_09642_gb300 import abi
    calls = []

    def coarse(h, block, g, y, nu, mode):
        calls.append((tuple(block), nu, mode))
        y.fill_(1.0)

    monkeypatch.setattr(abi, "sstep_coarse_fgs", coarse)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "coarse", "--steps", "2", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_coarse(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    nc, nf = 16 ** 3, 128 ** 3
    assert d["config"]["n_coarse"] == nc and d["config"]["n_fine"] == nf
    assert d["modes"]["formed"]["extra_device_bytes"] == nc * nc * 8
    assert d["modes"]["streaming"]["extra_device_bytes"] == (nf + nc) * 8
    assert d["value"] == pytest.approx(EVENT_MS / 2 / 1e3) == d["modes"]["streaming"]["time_s"]
    assert calls == [((8, 8, 8), 20, "streaming")] * 3 + [((8, 8, 8), 20, "formed")] * 3


def test_adjoint_line(fake_gpu, monkeypatch, capsys):
    """--workload adjoint: forward + backward timed, the directional gradient check against the
    assembled dL/dkappa, and the line's keys (solves and the assembly replaced by stand-ins:
    x = b, lambda = the adjoint right-hand side, dL/dkappa = lambda)."""
    import paper_2512_09642_gb300 as pkg
    from paper_2512_09642_gb300 import abi, autograd

    class Solver:
        def __init__(self, **kw):
            self.h = object()
            self.opts = abi.sstep_cg_default_opts()

        def solve(self, b, x0=None, allow_no_convergence=True):
            return b.detach().clone(), {"outer_iters": 40, "lambda_min_used": 0.01, "lambda_max_used": 2.0,
                                        "status": "SSTEP_OK"}

        def close(self):
            pass

    def grad_kappa(h, x, lam, gk):
        gk.copy_(lam)

    monkeypatch.setattr(pkg, "SStepCG", Solver, raising=False)
    monkeypatch.setattr(autograd, "SStepCG", Solver)
    monkeypatch.setattr(abi, "sstep_cg_grad_kappa", grad_kappa)
    monkeypatch.setattr(abi, "sstep_cg_set_tolerance", lambda *a: None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "adjoint", "--steps", "2", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_adjoint(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    assert d["config"]["workload"] == "adjoint_diffusion2d_1024^2" and d["config"]["n"] == 1024 ** 2
    assert d["value"] == pytest.approx(EVENT_MS / 2 / 1e3) and d["forward_outer_iters"] == 40
    gc = d["gradient_check"]
    assert set(gc) >= {"kind", "fd", "adjoint", "rel_err", "note"} and gc["rel_err"] >= 0
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "dtype", "clocks"):
        assert k in d, k


def test_batch_line(fake_gpu, monkeypatch, capsys):
    """--workload batch (4 systems, no tuning): the batched solve over the concatenated vectors,
    the plain loop of single-system solves, and the line's keys."""
    import numpy as np
    import paper_2512_09642_gb300 as pkg
    from paper_2512_09642_gb300 import abi
    seen = {}

    def create(grids, kappas, opts, stream=None):
        seen["grids"] = [tuple(g) for g in grids]
        return object()

    def layout(h, count):
        sizes = [int(np.prod(g)) for g in seen["grids"]]
        offs = np.concatenate([[0], np.cumsum([(n + 31) // 32 * 32 for n in sizes])[:-1]]).astype(np.int64)
        return offs, int(offs[-1] + sizes[-1]), np.tile([0.01, 2.0], (count, 1))

    def solve(h, b, x, count, allow=(5,)):
        x.copy_(b)
        info = {"status": "SSTEP_OK", "outer_iters": 30, "rel_res_true": 5e-9}
        return [dict(info) for _ in range(count)], dict(info)

    class Solver:
        def __init__(self, **kw):
            self.h = object()

        def solve_into(self, b, x):
            x.copy_(b)
            return {"outer_iters": 25, "status": "SSTEP_OK"}

        def close(self):
            pass

    monkeypatch.setattr(abi, "sstep_cg_batch_create", create)
    monkeypatch.setattr(abi, "sstep_cg_batch_layout", layout)
    monkeypatch.setattr(abi, "sstep_cg_batch_solve", solve)
    monkeypatch.setattr(abi, "sstep_cg_batch_destroy", lambda h: None)
    monkeypatch.setattr(pkg, "SStepCG", Solver, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "batch", "--batch-count", "4", "--no-tune",
                                      "--steps", "2", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_batch(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    assert len(seen["grids"]) == 4 and d["config"]["workload"] == "batch_4_diffusion2d_sides32-512"
    assert d["config"]["n_total"] == sum(int(np.prod(g)) for g in seen["grids"])
    assert d["value"] == pytest.approx(EVENT_MS / 2 / 1e3)
    assert d["batch"]["systems_ok"] == 4 and d["batch"]["max_outer_iters"] == 30 and d["batch"]["tuned"] is None
    assert d["plain_fp64_loop"]["max_outer_iters"] == 25 and d["plain_fp64_loop"]["graph"] is True


def test_spread_line(fake_gpu, monkeypatch, capsys):
    """--workload spread: every form on the five seeded x* at both sizes (the grids shrunk to 8^3
    here), the median time per outer iteration of the headline form at the larger size as the
    value, and the oracle's stored counts beside the 128^3 runs."""
    from workloads import problems as W
    real = W.poisson3d
    monkeypatch.setattr(W, "poisson3d", lambda side, xstar_seed=None, **kw: real(8, xstar_seed=xstar_seed))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "spread", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_spread(bench.parse())
    d = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][0])
    rows = d["spread"]
    forms = ["fp64+mom", "fp64", "mixed+mom", "mixed"]
    assert [(r["side"], r["form"]) for r in rows] == [(s, f) for s in (128, 256) for f in forms]
    for r in rows:
        assert [x["xstar_seed"] for x in r["runs"]] == list(bench.SPREAD_SEEDS)
        assert r["outer_min"] <= r["outer_median"] <= r["outer_max"]
    assert all(x["oracle_outer_iters"] for x in rows[0]["runs"])   # stored oracle counts at 128^3
    assert d["value"] == pytest.approx(rows[4]["ms_per_outer_median"] / 1e3)
