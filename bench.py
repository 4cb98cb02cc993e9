"""Benchmark: time to a 1e-8 relative residual of Chebyshev-basis s-step CG with FGS Gram
solves on the 3D 7-point Poisson problem, 256^3 unknowns (16.8M), s = 8, nu = 25, Jacobi,
spectral bounds from Gershgorin + 10 Lanczos steps, b = A x*, x* ~ U(-1, 1), x_0 = 0.

One step = one full solve on inputs resident in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--side 256]

With N > 1 (torchrun) each rank solves its own copy of the system on its own GPU (replicas:
no collective on the data path); the time is the max over ranks. `--impl reference` times
the CPU oracle (numpy/scipy, one thread) instead, on a bounded sample of outer iterations.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual & HBM GB/s, 3D Poisson 256³: FP64 vs mixed s-step CG"
GOLDEN_COUNTS = os.path.join(ROOT, "tests", "golden", "oracle_outer_counts.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--s", type=int, default=8)
    ap.add_argument("--nu", type=int, default=25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-outers", type=int, default=2)
    return ap.parse_args()


# ---- distributed plumbing (replicas) --------------------------------------------------------

def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ---------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- roofline model --------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 pipe rate derived from the nominal 1.25 TFLOP/s FP64 of GB300 (152 SMs, 2070 MHz):
# 1.25e12 / 2 flops per FMA = 0.625e12 FP64 instructions per second (152 x 2.06 per clock x
# 2.07 GHz); an FP64 add, multiply or FMA each occupies one of them.
FP64_OPS_PEAK = 0.625e12


def kernel_model(side, s, dim=3):
    """Algorithmic FP64 operations and HBM bytes per unknown, per launch, for the 7-point
    Poisson stencil path with the change-of-basis Gram (see the design notes)."""
    nbr = 2 * dim
    return {
        # 5 adds of the neighbour sum (2 dim - 1) + 2 FMAs; reads p_j, p_(j-1), writes p_(j+1)
        "cheb_step": {"ops": (nbr - 1) + 2, "bytes": 24},
        # s(s+1)/2 + s FMAs; reads s+1 basis vectors
        "gram_fgs": {"ops": s * (s + 1) // 2 + s, "bytes": 8 * (s + 1)},
        # s FMAs for x, s+1 for r; reads s+1 vectors and x, writes x and r
        "update": {"ops": 2 * s + 1, "bytes": 8 * (s + 1) + 24},
        # 2 dim adds/FMAs for A x, one subtract, one FMA for the norm; reads x, b, writes r
        "residual": {"ops": nbr + 2, "bytes": 24},
    }


def outer_bytes(s, dim=3):
    m = kernel_model(0, s, dim)
    return (m["cheb_step"]["bytes"] * s - 8) + m["gram_fgs"]["bytes"] + m["update"]["bytes"]


# ---- CPU oracle timing -----------------------------------------------------------------------

CPU_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import oracle as O
from oracle import spectral as OS
from workloads import problems as W
p = W.poisson3d({side}, s={s}, nu={nu})
op = O.Operator(*p.csr())
lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
out = []
for rep in range({reps}):
    t0 = time.perf_counter()
    O.solve(op, p.b, s={s}, nu={nu}, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer={outers})
    out.append(time.perf_counter() - t0)
print(json.dumps(out))
"""


def oracle_outer_times(side, s, nu, outers, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = CPU_SNIPPET.format(root=ROOT, side=side, s=s, nu=nu, reps=reps, outers=outers)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def stored_oracle_outers(side):
    if not os.path.exists(GOLDEN_COUNTS):
        return None
    for line in open(GOLDEN_COUNTS):
        if line.startswith(f"poisson3d_{side} "):
            for tok in line.split():
                if tok.startswith("outer="):
                    return int(tok.split("=")[1])
    return None


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---- arms ------------------------------------------------------------------------------------

def run_reference(args):
    world, rank, _ = dist_init(args)
    if rank != 0:
        return
    outers_needed = stored_oracle_outers(args.side)
    times = oracle_outer_times(args.side, args.s, args.nu, 1, args.warmup + args.steps)[args.warmup:]
    per_outer = statistics.mean(times)
    if outers_needed is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle outer-iteration count for this size not stored "
                          "(run tests/golden/make_oracle_outer_counts.py)"}))
        return
    value = per_outer * outers_needed
    sample = (f"each step = 1 outer iteration of the {args.side}^3 solve on the oracle (numpy/scipy, 1 thread); "
              f"time to 1e-8 = seconds per outer x {outers_needed} outer iterations the oracle needs "
              f"(tests/golden/oracle_outer_counts.txt)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_outer * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"poisson3d_7pt_{args.side}^3", "n": args.side ** 3, "s": args.s, "nu": args.nu,
                   "precond": "jacobi", "tol": 1e-8},
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_2512_09642_gb300 import SStepCG, abi
    from workloads import problems as W

    side, s, nu = args.side, args.s, args.nu
    p = W.poisson3d(side, s=s, nu=nu)
    n = p.n
    b = torch.as_tensor(p.b).cuda()
    sv = SStepCG(grid=p.dims, s=s, nu=nu, tol=1e-8, check_every=8, profile_every=4)
    stream = torch.cuda.current_stream()

    def one_solve():
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = abi.sstep_cg_solve(sv.h, b, x)
        return x, info.as_dict()

    for _ in range(args.warmup):
        x, info = one_solve()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        x, info = one_solve()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    t_solve = max_over_ranks(ms / 1e3, world)
    info = infos[-1]
    statuses = {i["status"] for i in infos}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    bh = torch.as_tensor(p.b).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(max(1, args.steps)):
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        abi.sstep_cg_solve_host(sv.h, bh.numpy(), xh.numpy())
        e2e_times.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(statistics.mean(e2e_times), world)

    # per-kernel durations sampled inside the timed solves (CUDA events on the solve stream)
    names = ["cheb_step", "gram_fgs", "update", "residual"]
    per_launch = {}
    for k, nm in enumerate(names):
        cnt = sum(i["prof_launches"][k] for i in infos)
        tot = sum(i["prof_ms"][k] for i in infos)
        per_launch[nm] = tot / cnt if cnt else None
    outers = info["outer_iters"]
    launches_per_solve = {"cheb_step": s * outers, "gram_fgs": outers, "update": outers,
                          "residual": 1 + 1 + info["refreshes"]}
    share = {nm: (per_launch[nm] or 0.0) * launches_per_solve[nm] for nm in names}
    dom = max(share, key=share.get)
    model = kernel_model(side, s)
    hbm_peak, peak_kind = measured_peaks()
    dl = per_launch[dom] / 1e3
    ops = model[dom]["ops"] * n
    by = model[dom]["bytes"] * n
    roofline = {"bound": "alu", "kernel": dom, "achieved": ops / dl / 1e9, "peak": FP64_OPS_PEAK / 1e9,
                "unit": "G FP64-op/s", "frac": ops / dl / FP64_OPS_PEAK, "traffic": None,
                "peak_kind": "derived from nominal 1.25 TFLOP/s FP64 (152 SMs x 2.07 GHz)",
                "ops_per_launch": ops, "bytes_per_launch": by, "avg_launch_ms": per_launch[dom],
                "hbm_gbs": by / dl / 1e9, "hbm_frac": by / dl / 1e9 / hbm_peak,
                "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind}
    kernel_table = {nm: {"avg_launch_ms": per_launch[nm], "launches_per_solve": launches_per_solve[nm],
                         "share": share[nm] / max(sum(share.values()), 1e-30),
                         "fp64_ops_per_s": (model[nm]["ops"] * n / (per_launch[nm] / 1e3)) if per_launch[nm] else None,
                         "hbm_gbs": (model[nm]["bytes"] * n / (per_launch[nm] / 1e3) / 1e9) if per_launch[nm] else None}
                    for nm in names}
    bytes_solve = outer_bytes(s) * n * outers
    hbm_gbs_solve = bytes_solve / t_solve / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            per = statistics.mean(oracle_outer_times(side, s, nu, args.cpu_outers, 1)) / args.cpu_outers
            cpu = {"value": per * outers, "unit": "s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                   "sample": f"{args.cpu_outers} outer iterations of the same {side}^3 solve on the oracle "
                             f"(numpy/scipy, 1 thread), seconds per outer x the {outers} outer iterations "
                             "of the measured solve", "s_per_outer": per}
        except Exception as ex:  # the CPU leg must not hide the GPU result
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": t_solve * world / world, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (b = A x*, x* ~ U(-1,1) splitmix64 seed 1002)",
            "config": {"workload": f"poisson3d_7pt_{side}^3", "n": n, "operator": "matrix-free stencil",
                       "s": s, "nu": nu, "precond": "jacobi", "bounds": "gershgorin + lanczos10",
                       "tol": 1e-8, "form": "fp64", "l2": "inputs larger than L2 (P_+ = 1.2 GB)",
                       "parallelism": f"replicas x{world}"},
            "outer_iters": outers, "status": sorted(statuses), "rel_res_true": info["rel_res_true"],
            "outer_per_s": outers / t_solve, "hbm_gbs_model": hbm_gbs_solve,
            "model_bytes_per_outer": outer_bytes(s) * n,
            "roofline": roofline, "kernels": kernel_table,
            "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
            "clocks": clk, "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    sv.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
