"""bench.py's reference arm (`--impl reference`) times the CPU oracle on a bounded sample of
the 3D Poisson solve and prints one JSON line with the same metric and config keys as the
GPU arm; under torchrun only rank 0 prints. Run here on the 64^3 problem (the oracle's
stored outer-iteration count for it is 60), on the CPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--side", "64", "--steps", "1", "--warmup", "0"]


def _json_lines(text):
    return [json.loads(ln) for ln in text.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + ARGS, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["config"]["workload"] == "poisson3d_7pt_64^3" and d["config"]["n"] == 64 ** 3
    # the GPU arm's line carries the same workload description
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.poisson3d_config(64, 8, 25)
    assert d["cpu_baseline"]["cores"] == os.cpu_count() and "cores" in d["cpu_baseline"]["cpu"]
    # time to tolerance = seconds per oracle outer iteration x the oracle's stored 60 outer iterations
    assert abs(d["value"] - d["ms_per_step"] / 1e3 * 60) <= 1e-9 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--gpus", "2"] + ARGS
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
