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
import re
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
GOLDEN_COUNTS_BOX = os.path.join(ROOT, "tests", "golden", "oracle_outer_counts_box.txt")


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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--forms", default=parse_default_forms(),
                    help="comma list of fp64, mixed, fp64+mom, mixed+mom, fp64+mom+conj (+mom: Gram from "
                         "Chebyshev moments; +conj: block-conjugated s-step CG); the first is the headline")
    ap.add_argument("--host-loop", action="store_true",
                    help="time the host-driven outer loop (convergence read every 8 outer iterations) instead of "
                         "the CUDA-graph loop; the per-kernel sampling then runs inside the timed solves")
    ap.add_argument("--workload", default="poisson3d",
                    choices=["poisson3d", "poisson27", "poisson2d_64", "diffusion3d", "batch", "coarse", "sweep",
                             "spread", "adjoint"],
                    help="poisson3d: the headline 3D Poisson solve (--side); poisson27: 3D 27-point Poisson "
                         "--side (230, 12.2M unknowns), Lanczos-10 bounds; poisson2d_64: 2D Poisson 64^2 CSR, "
                         "s = 4, nu = 20; diffusion3d: 3D diffusion --side (384), log-normal kappa, s = 12, "
                         "nu = 30; batch: 512 uneven 2D diffusion systems; coarse: AMG coarse-grid FGS, "
                         "3D diffusion 128^3 aggregated into 8^3 boxes (n_c = 4096), nu = 20; sweep: 3D Poisson "
                         "--side (512, 134M unknowns), s in 4, 8, 12, 16, --sweep-outers outer iterations per "
                         "solve, per-kernel bandwidth and FP64 rate; spread: outer-iteration counts and ms per "
                         "outer iteration of 3D Poisson 128^3 and 256^3 for five seeded x* (1002 .. 1402), "
                         "FP64 and mixed, direct and moments Gram; adjoint: the differentiable solve of 2D "
                         "diffusion 1024^2 (forward to 1e-10, adjoint solve and dL/dkappa), with a directional "
                         "finite-difference check of the gradient")
    ap.add_argument("--sweep-outers", type=int, default=16)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-plain-loop", action="store_true")
    ap.add_argument("--cpu-outers", type=int, default=2)
    ap.add_argument("--no-spread", action="store_true",
                    help="poisson3d: skip the headline form's solves of four more seeded x*")
    ap.add_argument("--csr", action="store_true",
                    help="poisson3d: give the operator as a CSR matrix (int32 indices, FP64 values) instead of the "
                         "matrix-free stencil")
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
    """The largest value over the ranks (the slowest replica sets the time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
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


TRAFFIC = os.path.join(ROOT, "profiles", "traffic.txt")


def kernel_source_sha(path, kernel):
    """sha256 of a kernel's __global__ definition (up to its closing brace at column 0)."""
    import hashlib
    src = open(os.path.join(ROOT, path)).read()
    # the launch bounds may hold one level of parentheses (a constexpr call)
    m = re.search(r"__global__ void __launch_bounds__\((?:[^()]|\([^()]*\))*\) " + re.escape(kernel) + r"\(", src)
    if not m:
        return None
    end = src.find("\n}\n", m.start())
    return hashlib.sha256(src[m.start():end + 3].encode()).hexdigest() if end >= 0 else None


def measured_traffic(workload, form, logical):
    """ncu DRAM bytes per launch for this bench line's dominant kernel, or None when no capture
    exists or the kernel changed since it was taken."""
    if not os.path.exists(TRAFFIC):
        return None
    for line in open(TRAFFIC):
        tok = line.split()
        if len(tok) < 7 or line.startswith("#"):
            continue
        if tok[0] == workload and tok[1] == form and tok[2] == logical:
            return {"bytes": int(tok[5]), "kernel": tok[3], "profile": tok[7] if len(tok) > 7 else None} \
                if kernel_source_sha(tok[4], tok[3]) == tok[6] else None
    return None


# FP64 issue rate measured on GB300 by paper_2512_09642_gb300/microbench/fp64_rate.cu: FMAs at
# 627.9 G lane-operations/s (2 per SM per clock at 2070 MHz, 152 SMs); adds and multiplies
# issue at only 528 G, which is why the FP64 stencils write their additions as FMAs.
FP64_OPS_PEAK = 0.6279e12
FP64_PEAK_KIND = ("measured: FP64 FMA issue rate, 627.9 G lane-ops/s at 2070 MHz "
                  "(paper_2512_09642_gb300/microbench/fp64_rate.cu)")


def form_gram(form):
    """Gram form of a bench form name: fp64 / mixed, +mom (moments), +fused (moments reduced
    by the step kernels), +conj (block-conjugated), +rN (mixed: FP64 refresh every N outers)."""
    parts = form.split("+")
    return "fused" if "fused" in parts else ("moments" if "mom" in parts else "direct")


def form_refresh(form):
    for part in form.split("+"):
        if re.fullmatch(r"r\d+", part):
            return int(part[1:])
    return 1


def kernel_model(s, mixed=False, dim=3, mom=False, diffusion=False, box=False, conj=False, fused=False,
                 write_r=False, csr=None):
    """Algorithmic FP64-pipe operations and HBM bytes per unknown per launch of the stencil
    path (change-of-basis Gram; the derivation is in the design notes). fused: the step
    kernels reduce the moments (2 FMAs per unknown and step in FP64) and the Gram launch only
    sums per-block partials; write_r: the mixed update also writes the recursive FP32
    residual (reads p_s, writes p_0)."""
    nbr = 2 * dim
    gram_fma = (2 * s if mom else s * (s + 1) // 2 + s) + (s if diffusion else 0)
    # box stencil: the 3^dim box sum by separable row / plane / z sums, 2 adds each
    box_sum = 2 * dim
    if csr is not None:
        # CSR with nnz/n = csr entries per row and the Jacobi diagonal as a vector M: the Gram
        # and update are those of a vector M; the step reads the row's values (8 B, FP32 copy
        # 4 B) and columns (4 B), its row pointer (4 B), p_j once (ideal caching of the
        # gathers), p_(j-1), writes p_(j+1), and reads 2 theta / diag; nnz/n FMAs + 2 per row
        m = kernel_model(s, mixed, dim, mom, True, False, conj, fused, write_r)
        vb, wb = (4, 4) if mixed else (8, 8)
        m["cheb_step"] = {"ops": 0 if mixed else csr + 2, "bytes": (vb + 4) * csr + 4 + 3 * wb + wb}
        m["residual"] = {"ops": csr + 2, "bytes": 12 * csr + 4 + 16 + (4 if mixed else 8)}
        return m
    if fused:
        m = kernel_model(s, mixed, dim, True, diffusion, box, conj, False, write_r)
        m["cheb_step"] = dict(m["cheb_step"], ops=m["cheb_step"]["ops"] + (0 if mixed else 2))
        m["gram_fgs"] = {"ops": 0, "bytes": 0}
        return m
    if not mixed:
        return {
            # Poisson: 2 dim - 1 adds of the neighbour sum + 2 FMAs; box: the box sum + 2 FMAs;
            # diffusion: 2 dim products of face weight and neighbour + 2 FMAs; reads p_j,
            # p_(j-1), writes p_(j+1) (+ the face weights and 2 theta / diag for diffusion)
            "cheb_step": {"ops": box_sum + 2 if box else ((nbr + 2) if diffusion else (nbr - 1) + 2),
                          "bytes": 24 + (8 * (dim + 1) if diffusion else 0)},
            # s(s+1)/2 + s FMAs (moments form: 2s), + s for c and s scalings with a vector M;
            # reads the s+1 basis vectors (+ diag M)
            # (+ conj: C = (A Q)^T P and d = Q^T r, s^2 + s FMAs reading P, Q, A Q again)
            "gram_fgs": {"ops": gram_fma + (s if diffusion else 0) + (s * s + s if conj else 0),
                         "bytes": 8 * (s + 1) + (8 if diffusion else 0) + (8 * 3 * s if conj else 0)},
            # s FMAs for x, s+1 for r (+1 with a vector M); reads s+1 vectors and x, writes x, r.
            # Block-conjugated form: A P through the change of basis (4 s), Q and A Q (2 s^2),
            # x and r (2 s); reads P_+, Q, A Q, x, writes Q, A Q, x, r
            "update": ({"ops": 2 * s * s + 6 * s, "bytes": 8 * (s + 1) + 8 * 4 * s + 24 + (8 if diffusion else 0)}
                       if conj else
                       {"ops": 2 * s + 1 + (1 if diffusion else 0), "bytes": 8 * (s + 1) + 24 + (8 if diffusion else 0)}),
            # A x, b - A x, the norm FMA; reads x, b (+ faces), writes r
            "residual": {"ops": (box_sum + 3) if box else nbr + 2, "bytes": 24 + (8 * (dim + 1) if diffusion else 0)},
        }
    return {
        # FP32: no FP64 operations; reads p_j, p_(j-1), writes p_(j+1) in 4-byte words
        "cheb_step": {"ops": 0, "bytes": 12 + (4 * (dim + 1) if diffusion else 0)},
        # products and compensated sums on the FP32 pipe; reads s+1 FP32 vectors
        "gram_fgs": {"ops": 0, "bytes": 4 * (s + 1) + (4 if diffusion else 0)},
        # one add + one FMA in FP64; reads s FP32 vectors and x, writes x (write_r: reads p_s
        # and writes the FP32 residual too)
        "update": {"ops": 2, "bytes": 4 * s + 16 + (8 if write_r else 0)},
        # FP64 residual and its norm (scaling and FP32 rounding use integer instructions);
        # reads x, b (+ faces), writes the FP32 p_0
        "residual": {"ops": (box_sum + 3) if box else nbr + 2, "bytes": 20 + (8 * (dim + 1) if diffusion else 0)},
    }


def outer_bytes(s, mixed=False, dim=3, diffusion=False, conj=False, fused=False, refresh=1, csr=None):
    """Algorithmic bytes per unknown of one outer iteration (mixed with refresh period N: the
    FP64 refresh in one outer iteration of N, the recursive residual written in the others
    but the last of each group)."""
    m = kernel_model(s, mixed, dim, diffusion=diffusion, conj=conj, fused=fused, csr=csr)
    # the first step reads no p_(j-1)
    first = m["cheb_step"]["bytes"] - (4 if mixed else 8) if csr is not None else (16 if not mixed else 8)
    steps = m["cheb_step"]["bytes"] * (s - 1) + first
    extra = m["residual"]["bytes"] / refresh if mixed else 0
    upd = m["update"]["bytes"] + (8 * (refresh - 1) / refresh if mixed else 0)
    return steps + m["gram_fgs"]["bytes"] + upd + extra


# ---- CPU oracle timing -----------------------------------------------------------------------

CPU_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import oracle as O
from oracle import spectral as OS
from workloads import problems as W
p = W.{maker}({side}, s={s}, nu={nu})
op = O.Operator(*p.csr())
lam = OS.bounds(op, {bounds!r}, W.lanczos_start(p.n))
out = []
for rep in range({reps}):
    t0 = time.perf_counter()
    O.solve(op, p.b, s={s}, nu={nu}, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer={outers})
    out.append(time.perf_counter() - t0)
print(json.dumps(out))
"""


def oracle_outer_times(side, s, nu, outers, reps, box=False, threads=1, maker=None):
    """Seconds per solve of `outers` outer iterations of the oracle (numpy/scipy), `reps` times,
    in a fresh process whose BLAS may use `threads` threads."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = CPU_SNIPPET.format(root=ROOT, side=side, s=s, nu=nu, reps=reps, outers=outers,
                              maker=maker or ("poisson27" if box else "poisson3d"),
                              bounds="lanczos10" if box else "gersh_lanczos10")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


ORACLE_SOLUTION_SNIPPET = r"""
import sys, time, json
import numpy as np
sys.path.insert(0, {root!r})
import oracle as O
from oracle import spectral as OS
from workloads import problems as W
p = W.diffusion3d({side}, s={s}, nu={nu})
op = O.Operator(*p.csr())
lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
t0 = time.perf_counter()
res = O.solve(op, p.b, s={s}, nu={nu}, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
np.save({out!r}, res.x)
print(json.dumps({{"seconds": time.perf_counter() - t0, "outer_iters": res.outer_iters,
                  "rel_res_true": res.rel_res_true, "lam": [float(lam[0]), float(lam[1])]}}))
"""


def diffusion_error_vs_oracle(forms, side, s, nu):
    """The CPU-baseline leg's check of the diffusion forms against the oracle: the oracle solves
    the same log-normal diffusion problem at a size it finishes in under a minute (side^3) to
    1e-8, and each GPU form solves it with the oracle's bounds; returns ||x - x_oracle|| /
    ||x_oracle|| per form with both outer counts."""
    import numpy as np
    import torch
    from paper_2512_09642_gb300 import SStepCG
    from workloads import problems as W
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", ORACLE_SOLUTION_SNIPPET.format(root=ROOT, side=side, s=s, nu=nu, out=path)],
                       capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    meta = json.loads(r.stdout.strip().splitlines()[-1])
    xo = np.load(path)
    os.unlink(path)
    p = W.diffusion3d(side, s=s, nu=nu)
    kappa = torch.as_tensor(p.kappa).cuda()
    b = torch.as_tensor(p.b).cuda()
    out = {"workload": f"diffusion3d_7pt_{side}^3_lognormal1", "oracle_outer_iters": meta["outer_iters"],
           "oracle_rel_res_true": meta["rel_res_true"], "oracle_seconds_1_thread": meta["seconds"], "forms": {}}
    for form in forms:
        sv = SStepCG(grid=p.dims, kappa=kappa, bounds=tuple(meta["lam"]), s=s, nu=nu, tol=1e-8,
                     precision=form.split("+")[0], gram_form=form_gram(form),
                     refresh_period=form_refresh(form) if form.startswith("mixed") else 1)
        x, info = sv.solve(b)
        sv.close()
        xg = x.cpu().numpy()
        out["forms"][form] = {"rel_err_vs_oracle_x": float(np.linalg.norm(xg - xo) / np.linalg.norm(xo)),
                              "outer_iters": info["outer_iters"], "rel_res_true": info["rel_res_true"],
                              "status": info["status"]}
    return out


def stored_oracle_outers(side, box=False):
    path, prefix = (GOLDEN_COUNTS_BOX, "poisson27") if box else (GOLDEN_COUNTS, "poisson3d")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith(f"{prefix}_{side} "):
            for tok in line.split():
                if tok.startswith("outer="):
                    return int(tok.split("=")[1])
    return None


def cpu_model():
    """CPU model name (lscpu's "Model name", else /proc/cpuinfo's) and the host's core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        fields = {}
        try:
            for line in open("/proc/cpuinfo"):
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
        except OSError:
            pass
        name = fields.get("model name") or (f"implementer {fields.get('cpu implementer')} part {fields.get('cpu part')}"
                                            if "cpu part" in fields else "unknown")
    return f"{name}, {os.cpu_count()} cores"


def poisson3d_config(side, s, nu, box=False):
    """The workload description shared by both arms (the GPU line and the CPU oracle's)."""
    return {"workload": f"poisson3d_27pt_{side}^3" if box else f"poisson3d_7pt_{side}^3", "n": side ** 3,
            "operator": "3D 27-point Poisson" if box else "3D 7-point Poisson", "s": s, "nu": nu,
            "precond": "jacobi", "bounds": "lanczos10 (both ends, 10% margins)" if box else "gershgorin + lanczos10",
            "tol": 1e-8, "l2": "inputs larger than L2" if side ** 3 * 8 * (s + 1) > 129e6 else "inputs fit in L2",
            "x0": "zero", "b": "A x*, x* ~ U(-1,1)"}


# ---- arms ------------------------------------------------------------------------------------

def run_reference(args):
    world, rank, _ = dist_init(args)
    if rank != 0:
        return
    outers_needed = stored_oracle_outers(args.side)
    if outers_needed is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle outer-iteration count for this size not stored "
                          "(run tests/golden/make_oracle_outer_counts.py)"}))
        return
    cores = os.cpu_count() or 1
    times = oracle_outer_times(args.side, args.s, args.nu, 1, args.warmup + args.steps, threads=cores)[args.warmup:]
    per_outer = statistics.mean(times)
    value = per_outer * outers_needed
    sample = (f"each step = 1 outer iteration of the {args.side}^3 solve on the oracle (numpy/scipy; BLAS on "
              f"{cores} threads, the rest single-threaded); time to 1e-8 = seconds per outer x {outers_needed} outer "
              f"iterations the oracle needs (tests/golden/oracle_outer_counts.txt)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_outer * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (b = A x*, x* ~ U(-1,1) splitmix64 seed 1002)",
        "config": poisson3d_config(args.side, args.s, args.nu),
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def measure_form(args, p, b, world, local, precision, csr=None, fixed_outers=None, e2e=True):
    """Warm-up + K timed solves of one form, the outer loop as one CUDA graph (the library's
    fastest way to run it; --host-loop times the host-driven loop instead); then one more
    solve with the host loop and CUDA events around every kernel of sampled outer iterations,
    for the per-kernel durations (kernels cannot be timed one by one inside a graph).
    fixed_outers: run exactly that many outer iterations per solve (tol 1e-30) with the host
    loop, sampling the kernels in every chunk of 8, and skip the end-to-end leg."""
    import torch
    from paper_2512_09642_gb300 import SStepCG, abi

    n, s = p.n, args.s
    parts = precision.split("+")
    prec = parts[0]
    graph = not args.host_loop and not fixed_outers
    kw = dict(s=s, nu=args.nu, tol=1e-8, check_every=8, profile_every=0 if graph else 4, precision=prec,
              gram_form=form_gram(precision), use_graph=1 if graph else 0,
              block_conjugate=1 if "conj" in parts else 0, refresh_period=form_refresh(precision))
    if fixed_outers:
        kw.update(tol=1e-30, max_outer=int(fixed_outers), profile_every=1)
    if p.stencil == "box":
        kw["bounds_mode"] = "lanczos10"   # Section 8: Lanczos-10 estimates of both ends, 10% margins
    kappa = None if p.kappa is None else torch.as_tensor(p.kappa).cuda()

    def make(**extra):
        o = dict(kw, **extra)
        if csr is not None:
            return SStepCG(csr=csr, **o)
        return SStepCG(grid=p.dims, kappa=kappa, stencil=p.stencil, **o)

    sv = make()
    stream = torch.cuda.current_stream()

    # one output vector for every solve, zeroed in place (x_0 = 0): the handle keeps the CUDA
    # graph of its last (b, x) pair, so a new x address per solve would capture and instantiate
    # the graph again inside the timed region
    xbuf = torch.zeros(n, dtype=torch.float64, device="cuda")

    def one_solve(h=None):
        xbuf.zero_()
        info = abi.sstep_cg_solve((h or sv).h, b, xbuf)
        return xbuf, info.as_dict()

    for _ in range(args.warmup):
        one_solve()
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
    t_solve = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, world)
    x = xbuf.clone()   # the last timed solve's result (the buffer is reused below)

    t_e2e = None
    if e2e and not args.no_e2e and not fixed_outers:
        # end to end through the C ABI with pinned host buffers, copies inside the timed region
        bh = torch.as_tensor(p.b).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        for _ in range(args.warmup):   # the same warm-up as the device-resident solves
            xh.zero_()
            abi.sstep_cg_solve_host(sv.h, bh.numpy(), xh.numpy())
        times = []
        for _ in range(max(1, args.steps)):
            xh.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            abi.sstep_cg_solve_host(sv.h, bh.numpy(), xh.numpy())
            times.append(time.perf_counter() - t0)
        t_e2e = max_over_ranks(statistics.mean(times), world)
    sv.close()
    prof_infos = infos
    if graph:
        # per-kernel durations: one host-loop solve with every chunk's second outer iteration sampled
        sp = make(use_graph=0, profile_every=1)
        one_solve(sp)
        prof_infos = [one_solve(sp)[1]]
        sp.close()
    return {"t": t_solve, "e2e": t_e2e, "infos": infos, "prof_infos": prof_infos, "clocks": clk, "x": x,
            "graph": graph}


def kernel_report(args, n, infos, precision, dim=3, diffusion=False, box=False, csr=None):
    s = args.s
    names = ["cheb_step", "gram_fgs", "update", "residual"]
    info = infos[-1]
    per_launch = {}
    for k, nm in enumerate(names):
        cnt = sum(i["prof_launches"][k] for i in infos)
        tot = sum(i["prof_ms"][k] for i in infos)
        per_launch[nm] = tot / cnt if cnt else None
    outers = info["outer_iters"]
    mixed = precision.startswith("mixed")
    mom = "+mom" in precision
    conj = "+conj" in precision
    fused = form_gram(precision) == "fused"
    per = form_refresh(precision) if mixed else 1
    launches = {"cheb_step": s * outers, "gram_fgs": outers, "update": outers,
                "residual": (-(-outers // per) + 1 if mixed else 0) + 2 + info["refreshes"]}
    share = {nm: (per_launch[nm] or 0.0) * launches[nm] for nm in names}
    # the sampled outer iteration (the chunk's first with a refresh period above 1) writes the
    # recursive residual in its update
    model = kernel_model(s, mixed, dim=dim, mom=mom, diffusion=diffusion, box=box, conj=conj, fused=fused,
                         write_r=mixed and per > 1, csr=csr)
    hbm_peak, peak_kind = measured_peaks()
    table = {}
    for nm in names:
        d = per_launch[nm]
        table[nm] = {"avg_launch_ms": d, "launches_per_solve": launches[nm],
                     "share": share[nm] / max(sum(share.values()), 1e-30),
                     "fp64_ops_per_launch": model[nm]["ops"] * n, "bytes_per_launch": model[nm]["bytes"] * n,
                     "fp64_gops": model[nm]["ops"] * n / (d / 1e3) / 1e9 if d else None,
                     "hbm_gbs": model[nm]["bytes"] * n / (d / 1e3) / 1e9 if d else None}
    dom = max(share, key=share.get)
    d = per_launch[dom] / 1e3
    ops, by = model[dom]["ops"] * n, model[dom]["bytes"] * n
    alu_frac = ops / d / FP64_OPS_PEAK
    hbm_frac = by / d / 1e9 / hbm_peak
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": ops / d / 1e9, "peak": FP64_OPS_PEAK / 1e9, "unit": "G FP64-op/s",
                "frac": alu_frac, "peak_kind": FP64_PEAK_KIND}
    else:
        roof = {"bound": "hbm", "achieved": by / d / 1e9, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    roof.update({"kernel": dom, "traffic": None, "avg_launch_ms": per_launch[dom], "fp64_ops_per_launch": ops,
                 "bytes_per_launch": by, "alu_frac": alu_frac, "hbm_frac": hbm_frac})
    return roof, table


def xstar_spread(args, p, b, side, head):
    """The headline form on the five seeded x* (the first is the workload's): the outer count
    to 1e-8 of this restarted iteration moves with rounding, the time per outer iteration does
    not."""
    import torch
    from paper_2512_09642_gb300 import SStepCG, abi
    from workloads import problems as W
    s, nu, n = args.s, args.nu, p.n
    parts = head.split("+")
    sv = SStepCG(grid=p.dims, s=s, nu=nu, tol=1e-8, check_every=8, precision=parts[0], gram_form=form_gram(head),
                 block_conjugate=1 if "conj" in parts else 0, use_graph=0 if args.host_loop else 1,
                 refresh_period=form_refresh(head) if parts[0] == "mixed" else 1)
    runs = []
    for sd in SPREAD_SEEDS:
        bq = b if sd == SPREAD_SEEDS[0] else torch.as_tensor(W.poisson3d(side, xstar_seed=sd).b).cuda()
        xq = torch.zeros(n, dtype=torch.float64, device="cuda")
        inf = abi.sstep_cg_solve(sv.h, bq, xq).as_dict()
        runs.append({"xstar_seed": sd, "outer_iters": inf["outer_iters"], "time_s": inf["ms"] / 1e3,
                     "ms_per_outer": inf["ms"] / max(inf["outer_iters"], 1), "rel_res_true": inf["rel_res_true"]})
    sv.close()
    cnt = sorted(r["outer_iters"] for r in runs)
    tms = sorted(r["time_s"] for r in runs)
    return {"form": head, "outer_min": cnt[0], "outer_median": cnt[2], "outer_max": cnt[-1],
            "time_median_s": tms[2], "runs": runs}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    from workloads import problems as W

    csr = None
    if args.workload == "poisson2d_64":
        args.s, args.nu = 4, 20
        p = W.poisson2d_64()
        csr = tuple(torch.as_tensor(a).cuda() for a in p.csr())
        side = 64
        wname, opname = "poisson2d_5pt_64^2", "CSR"
    elif args.workload == "diffusion3d":
        side = args.side if args.side != 256 else 384
        args.s, args.nu = 12, 30
        if args.forms == parse_default_forms():
            args.forms = "fp64+mom,mixed+mom,mixed+mom+r4"   # a vector M: no fused moments
        p = W.diffusion3d(side)
        wname, opname = f"diffusion3d_7pt_{side}^3_lognormal1", "matrix-free stencil"
    elif args.workload == "poisson27":
        side = args.side if args.side != 256 else 230
        p = W.poisson27(side, s=args.s, nu=args.nu)
        wname, opname = f"poisson3d_27pt_{side}^3", "matrix-free 27-point stencil"
    else:
        side = args.side
        p = W.poisson3d(side, s=args.s, nu=args.nu)
        wname, opname = f"poisson3d_7pt_{side}^3", "matrix-free stencil"
        if args.csr:
            csr = tuple(torch.as_tensor(a).cuda() for a in p.csr())
            wname, opname = f"poisson3d_7pt_{side}^3_csr", "CSR (int32 indices, FP64 values)"
    box = p.stencil == "box"
    s, nu = args.s, args.nu
    n = p.n
    b = torch.as_tensor(p.b).cuda()
    forms = {}
    res = {}
    for prec in args.forms.split(","):
        # the end-to-end leg (host buffers, copies timed) for the headline form only
        headline = prec == args.forms.split(",")[0]
        try:
            r = measure_form(args, p, b, world, local, prec, csr, e2e=headline)
        except Exception as ex:   # a failing secondary form is reported, not allowed to hide the line
            if headline:
                raise
            forms[prec] = {"error": f"{type(ex).__name__}: {ex}"}
            torch.cuda.empty_cache()
            continue
        dim = len(p.dims)
        diff = p.kappa is not None
        nnz_row = None if csr is None else float(csr[0][-1].item()) / n
        roof, table = kernel_report(args, n, r["prof_infos"], prec, dim, diff, box, nnz_row)
        info = r["infos"][-1]
        outers = info["outer_iters"]
        cj = "+conj" in prec
        fz = form_gram(prec) == "fused"
        rp = form_refresh(prec) if prec.startswith("mixed") else 1
        ob = outer_bytes(s, prec.startswith("mixed"), dim, diff, cj, fz, rp, nnz_row)
        bytes_solve = ob * n * outers
        forms[prec] = {"time_s": r["t"], "outer_iters": outers, "status": sorted({i["status"] for i in r["infos"]}),
                       "rel_res_true": info["rel_res_true"], "outer_per_s": outers / r["t"],
                       "hbm_gbs_model": bytes_solve / r["t"] / 1e9,
                       "model_bytes_per_outer": ob * n,
                       "ms_per_outer": r["t"] / max(outers, 1) * 1e3,
                       "e2e_s": r["e2e"], "roofline": roof, "kernels": table, "clocks": r["clocks"],
                       "gpu_launches": int(sum(i["kernel_launches"] for i in r["infos"])),
                       # the mixed forms' FP32 step: through TMA tiles or plain loads (opts.step_kernel AUTO)
                       "fp32_step": ("tma" if info.get("step_tma") else "plain") if prec.startswith("mixed") else None}
        res[prec] = r
    # speedups and differences are against the first FP64 form listed (the headline, FP64
    # with the moments Gram, by default)
    ref = next((f for f in res if f.startswith("fp64")), None)
    xs = torch.as_tensor(p.x_star).cuda()
    for prec in res:
        forms[prec]["rel_err_vs_xstar"] = float(torch.linalg.norm(res[prec]["x"] - xs) / torch.linalg.norm(xs))
        if ref is not None and prec != ref:
            x64 = res[ref]["x"]
            forms[prec]["speedup_vs"] = ref
            forms[prec]["speedup_vs_fp64"] = res[ref]["t"] / res[prec]["t"]
            forms[prec]["rel_diff_vs_fp64_x"] = float(torch.linalg.norm(res[prec]["x"] - x64) / torch.linalg.norm(x64))
    head = args.forms.split(",")[0]
    h = forms[head]
    for prec, f in forms.items():   # ncu DRAM bytes per launch where a capture of this kernel exists
        tr = measured_traffic(wname, prec, f["roofline"].get("kernel")) if f.get("roofline") else None
        if tr:
            f["roofline"]["traffic"] = tr["bytes"]
            f["roofline"]["traffic_source"] = f"ncu capture of {tr['kernel']}, profiles/{tr['profile']}"

    spread = None
    if args.workload == "poisson3d" and csr is None and not args.no_spread:
        try:
            spread = xstar_spread(args, p, b, side, head)
        except Exception as ex:   # the spread is context: it must not hide the headline line
            spread = {"form": head, "error": f"{type(ex).__name__}: {ex}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ("poisson3d", "poisson27"):
        stored = stored_oracle_outers(side, box)
        outers = stored if stored else h["outer_iters"]
        src = (f"the oracle's own converged run (tests/golden/{os.path.basename(GOLDEN_COUNTS_BOX if box else GOLDEN_COUNTS)})"
               if stored else "the measured GPU solve")
        try:
            per = statistics.mean(oracle_outer_times(side, s, nu, args.cpu_outers, 1, box)) / args.cpu_outers
            cores = os.cpu_count() or 1
            per_all = statistics.mean(oracle_outer_times(side, s, nu, args.cpu_outers, 1, box, threads=cores)) \
                / args.cpu_outers
            cpu = {"value": per * outers, "unit": "s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                   "sample": f"{args.cpu_outers} outer iterations of the same {side}^3 solve on the oracle "
                             f"(numpy/scipy FP64, 1 thread), seconds per outer x {outers} outer iterations "
                             f"to 1e-8 from {src}", "s_per_outer": per, "outer_iters": outers,
                   "all_cores": {"value": per_all * outers, "unit": "s", "cores": cores, "s_per_outer": per_all,
                                 "sample": f"the same, BLAS on {cores} threads (the rest of the oracle is "
                                           f"single-threaded numpy/scipy)"}}
        except Exception as ex:  # the CPU leg must not hide the GPU result
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "diffusion3d":
        try:
            outers = h["outer_iters"]
            per = statistics.mean(oracle_outer_times(side, s, nu, 1, 1, maker="diffusion3d"))
            cpu = {"value": per * outers, "unit": "s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                   "sample": f"1 outer iteration of the same {side}^3 diffusion solve on the oracle (numpy/scipy "
                             f"FP64, 1 thread), seconds per outer x the {outers} outer iterations of the GPU's "
                             f"{head} solve", "s_per_outer": per, "outer_iters": outers,
                   "error_vs_oracle": diffusion_error_vs_oracle(list(forms), 48, s, nu)}
        except Exception as ex:  # the CPU leg must not hide the GPU result
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        metric = METRIC if args.workload == "poisson3d" else f"time-to-1e-8 residual, {wname}: s-step CG"
        if args.workload in ("poisson3d", "poisson27") and csr is None:
            cfg = poisson3d_config(side, s, nu, box)
        else:
            cfg = {"workload": wname, "n": n, "operator": opname, "s": s, "nu": nu, "precond": "jacobi",
                   "bounds": "gershgorin + lanczos10", "tol": 1e-8,
                   "l2": "inputs larger than L2" if n * 8 * (s + 1) > 129e6 else "inputs fit in L2"}
        line = {
            "metric": metric, "value": h["time_s"], "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["time_s"] * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head.startswith("fp64") else "f32 basis + f64 Gram/x/residual",
            "data": f"synthetic (b = A x*, x* ~ U(-1,1) splitmix64 seed {1000 + p.meta['config']})",
            "config": cfg,
            "form": head, "graph": not args.host_loop, "parallelism": f"replicas x{world}",
            "outer_iters": h["outer_iters"], "rel_res_true": h["rel_res_true"], "outer_per_s": h["outer_per_s"],
            "hbm_gbs_model": h["hbm_gbs_model"], "roofline": h["roofline"],
            "e2e": {"value": h["e2e_s"], "unit": "s", "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
            "gpu_launches": h["gpu_launches"], "clocks": h["clocks"], "cpu_baseline": cpu,
            "ms_per_outer": h["ms_per_outer"], "xstar_spread": spread, "forms": forms,
        }
        print(json.dumps(line))


def run_batch(args):
    """Batched form: 512 2D diffusion systems, sides U{32..512} (seed 3000), kappa =
    exp(0.5 N(0,1)), FP64, tol 1e-8; autotuned s, nu and launch shapes; graph-driven loop.
    Compared with the plain FP64 solver run system by system on the same GPU."""
    import torch
    from paper_2512_09642_gb300 import SStepCG, abi, tune
    from workloads import problems as W

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    probs = W.diffusion2d_batch(count=args.batch_count)
    grids = [p.dims for p in probs]
    kap = [torch.as_tensor(p.kappa).cuda() for p in probs]
    bs = [torch.as_tensor(p.b).cuda() for p in probs]
    n_total = sum(p.n for p in probs)
    params = {"s": 8, "nu": 20, "gram_form": "moments", "batch_chunk": 8192, "batch_ctas_per_sm": 6}
    tuned = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tr = tune.tune(grids, kap, bs)
        params = tr.best
        tuned = {"chosen": tr.best, "predicted_s": tr.predicted_s, "tune_wall_s": time.perf_counter() - t0,
                 "candidates": len(tr.table), "sample_systems": len(tr.sample),
                 "table": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in tr.table]}
    opts = abi.sstep_cg_default_opts(tol=1e-8, use_graph=1, **params)
    h = abi.sstep_cg_batch_create(grids, kap, opts)
    offs, total, lam = abi.sstep_cg_batch_layout(h, len(probs))
    b = torch.zeros(total, dtype=torch.float64, device="cuda")
    for bi, o in zip(bs, offs):
        b[o:o + bi.numel()] = bi
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        x = torch.zeros_like(b)
        abi.sstep_cg_batch_solve(h, b, x, len(probs))
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x = torch.zeros_like(b)
        infos, summary = abi.sstep_cg_batch_solve(h, b, x, len(probs))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_batch = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, world)
    abi.sstep_cg_batch_destroy(h)
    plain = None
    if not args.no_plain_loop:
        # the plain single-system solver with the same s, nu and Gram form, graph-driven (its
        # fastest mode for small systems), one system after the other
        handles = [SStepCG(grid=p.dims, kappa=k, s=params["s"], nu=params["nu"], gram_form=params["gram_form"],
                           tol=1e-8, use_graph=1) for p, k in zip(probs, kap)]
        xs = [torch.zeros_like(bi) for bi in bs]
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        outers = []
        for sv, bi, xi in zip(handles, bs, xs):
            outers.append(sv.solve_into(bi, xi)["outer_iters"])
        p1.record(stream)
        torch.cuda.synchronize()
        plain = {"time_s": p0.elapsed_time(p1) / 1e3, "s": params["s"], "nu": params["nu"],
                 "gram_form": params["gram_form"], "graph": True, "max_outer_iters": max(outers),
                 "sum_outer_iters": sum(outers)}
        for sv in handles:
            sv.close()
    if rank == 0:
        line = {
            "metric": f"time to 1e-8 residual in every system, {len(probs)} 2D diffusion systems (batched form)",
            "value": t_batch, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded sides, kappa, x*)",
            "config": {"workload": f"batch_{len(probs)}_diffusion2d_sides32-512", "n_total": n_total,
                       "params": params, "tol": 1e-8, "graph": True},
            "batch": {"status": summary["status"], "max_outer_iters": summary["outer_iters"],
                      "worst_rel_res_true": summary["rel_res_true"],
                      "systems_ok": sum(1 for i in infos if i["status"] == "SSTEP_OK"), "tuned": tuned},
            "plain_fp64_loop": plain,
            "speedup_vs_plain_fp64_loop": (plain["time_s"] / t_batch) if plain else None,
            "clocks": clk,
        }
        print(json.dumps(line))


def run_coarse(args):
    """AMG coarse-grid FGS (Section 6): nu = 20 sweeps on A_c y = g, A_c = P^T A_f P, with A_f the
    3D diffusion operator on 128^3 (kappa = exp(N(0,1))) and P the aggregation into 8^3 boxes
    (n_c = 4096, the size of the paper's coarse level), formed and streaming."""
    import numpy as np
    import torch
    from paper_2512_09642_gb300 import SStepCG, abi
    from workloads import problems as W
    from workloads import rng

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    side, blk, nu = 128, 8, 20
    p = W.make("coarse_diffusion3d", (side,) * 3, kappa_sigma=1.0, config=7)
    sv = SStepCG(grid=p.dims, kappa=torch.as_tensor(p.kappa).cuda(), bounds=(0.05, 2.0), s=2)
    nc = (side // blk) ** 3
    g = torch.as_tensor(rng.normal(7001, nc)).cuda()
    stream = torch.cuda.current_stream()
    res = {}
    for mode in ("streaming", "formed"):
        for _ in range(args.warmup):
            y = torch.zeros(nc, dtype=torch.float64, device="cuda")
            abi.sstep_coarse_fgs(sv.h, (blk,) * 3, g, y, nu, mode)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            y = torch.zeros(nc, dtype=torch.float64, device="cuda")
            abi.sstep_coarse_fgs(sv.h, (blk,) * 3, g, y, nu, mode)
        e1.record(stream)
        torch.cuda.synchronize()
        res[mode] = {"time_s": max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, world),
                     "extra_device_bytes": nc * nc * 8 if mode == "formed" else (p.n + nc) * 8,
                     "y_norm": float(torch.linalg.norm(y))}
    sv.close()
    if rank == 0:
        t = res["streaming"]["time_s"]
        print(json.dumps({
            "metric": "time for nu = 20 coarse-grid FGS sweeps (AMG coarse level, n_c = 4096)", "value": t,
            "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (kappa = exp(N(0,1)) seed 2007, g ~ N(0,1) seed 7001)",
            "config": {"workload": "coarse_fgs_diffusion3d_128^3_agg8^3", "n_fine": p.n, "n_coarse": nc,
                       "nu": nu, "headline_mode": "streaming"},
            "modes": res,
            "note": "Gauss-Seidel is sequential over the coarse rows: one block walks them; the work "
                    "within a row is parallel"}))


def run_sweep(args):
    """Bandwidth sweep on 3D Poisson (7-point, 512^3 = 134M unknowns by default) over s in
    {4, 8, 12, 16}, FP64 (moments Gram) and mixed (fused moments, FP64 refresh every 8) forms,
    host-driven loop: each solve runs a fixed number of
    outer iterations, and every kernel's CUDA-event time, sampled inside them, gives its
    algorithmic GB/s and FP64 rate against the HBM and FP64-pipe roofs."""
    import torch
    from workloads import problems as W

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    side = args.side if args.side != 256 else 512
    p = W.poisson3d(side)
    n = p.n
    b = torch.as_tensor(p.b).cuda()
    rows = []
    for s in (4, 8, 12, 16):
        args.s = s
        for prec in ("fp64+mom", "mixed+fused+r8"):
            r = measure_form(args, p, b, world, local, prec, fixed_outers=args.sweep_outers)
            roof, table = kernel_report(args, n, r["infos"], prec)
            outers = r["infos"][-1]["outer_iters"]
            per_outer = r["t"] / outers
            ob = outer_bytes(s, prec.startswith("mixed"), 3, fused=form_gram(prec) == "fused",
                             refresh=form_refresh(prec) if prec.startswith("mixed") else 1) * n
            rows.append({"s": s, "form": prec, "outer_iters": outers, "ms_per_outer": per_outer * 1e3,
                         "model_bytes_per_outer": ob, "hbm_gbs_model": ob / per_outer / 1e9,
                         "dominant": {k: roof[k] for k in ("kernel", "bound", "frac", "alu_frac", "hbm_frac")},
                         "kernels": {k: {f: v[f] for f in ("avg_launch_ms", "share", "hbm_gbs", "fp64_gops")}
                                     for k, v in table.items() if v["avg_launch_ms"]},
                         "clocks": r["clocks"],
                         "gpu_launches": int(sum(i["kernel_launches"] for i in r["infos"])),
                       # the mixed forms' FP32 step: through TMA tiles or plain loads (opts.step_kernel AUTO)
                       "fp32_step": (("tma" if r["infos"][-1].get("step_tma") else "plain")
                                     if prec.startswith("mixed") else None)})
            torch.cuda.empty_cache()
    if rank == 0:
        head = next(rw for rw in rows if rw["s"] == 8 and rw["form"] == "fp64+mom")
        hbm_peak, _ = measured_peaks()
        print(json.dumps({
            "metric": f"time per outer iteration, 3D Poisson {side}^3, s = 8 (sweep over s)",
            "value": head["ms_per_outer"] / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_outer"] * head["outer_iters"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic (b = A x*, x* ~ U(-1,1) splitmix64 seed {1000 + p.meta['config']})",
            "config": {"workload": f"poisson3d_7pt_{side}^3_s_sweep", "n": n, "nu": args.nu, "precond": "jacobi",
                       "outer_iters_per_solve": args.sweep_outers, "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{world}"},
            "peaks": {"hbm_gbs": hbm_peak, "fp64_gops": FP64_OPS_PEAK / 1e9},
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "sweep": rows}))


SPREAD_SEEDS = (1002, 1102, 1202, 1302, 1402)
GOLDEN_SEEDS = os.path.join(ROOT, "tests", "golden", "oracle_outer_counts_seeds.txt")


def run_spread(args):
    """Outer-iteration counts to 1e-8 of the restarted iteration over five seeded exact
    solutions x* (b = A x*), at 128^3 and 256^3, for each form: the count moves with rounding
    over hundreds of outer iterations, the time per outer iteration does not. The oracle's own
    counts at 128^3 for the same seeds are read from tests/golden/oracle_outer_counts_seeds.txt."""
    import torch
    from paper_2512_09642_gb300 import SStepCG, abi
    from workloads import problems as W

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    forms = args.forms.split(",") if args.forms != parse_default_forms() else \
        ["fp64+mom", "fp64", "mixed+mom", "mixed"]
    stored = {}
    if os.path.exists(GOLDEN_SEEDS):
        for line in open(GOLDEN_SEEDS):
            if line.startswith("poisson3d_"):
                name = line.split()[0]
                tok = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                stored[name] = int(tok["outer"])
    rows = []
    clk = None
    for side in (128, 256):
        probs = [W.poisson3d(side, xstar_seed=sd) for sd in SPREAD_SEEDS]
        bs = [torch.as_tensor(p.b).cuda() for p in probs]
        for form in forms:
            parts = form.split("+")
            sv = SStepCG(grid=probs[0].dims, s=8, nu=25, tol=1e-8, check_every=8, precision=parts[0],
                         gram_form=form_gram(form), refresh_period=form_refresh(form) if parts[0] == "mixed" else 1,
                         use_graph=0 if args.host_loop else 1)
            x = torch.zeros(probs[0].n, dtype=torch.float64, device="cuda")
            for _ in range(max(args.warmup, 1)):
                x.zero_()
                abi.sstep_cg_solve(sv.h, bs[0], x)
            if side == 256 and form == forms[0]:
                clocks = ClockSampler(local)
                clocks.start()
            per = []
            for sd, b in zip(SPREAD_SEEDS, bs):
                x.zero_()
                torch.cuda.synchronize()
                inf = abi.sstep_cg_solve(sv.h, b, x).as_dict()
                per.append({"xstar_seed": sd, "outer_iters": inf["outer_iters"], "time_s": inf["ms"] / 1e3,
                            "ms_per_outer": inf["ms"] / max(inf["outer_iters"], 1), "status": inf["status"],
                            "rel_res_true": inf["rel_res_true"],
                            "oracle_outer_iters": stored.get(f"poisson3d_{side}_xstar{sd}")})
            if side == 256 and form == forms[0]:
                clk = clocks.stop()
            sv.close()
            cnt = sorted(r["outer_iters"] for r in per)
            mso = sorted(r["ms_per_outer"] for r in per)
            rows.append({"side": side, "form": form, "outer_min": cnt[0], "outer_median": cnt[len(cnt) // 2],
                         "outer_max": cnt[-1], "ms_per_outer_median": mso[len(mso) // 2],
                         "ms_per_outer_min": mso[0], "ms_per_outer_max": mso[-1], "runs": per})
            torch.cuda.empty_cache()
    if rank == 0:
        head = next(r for r in rows if r["side"] == 256 and r["form"] == forms[0])
        print(json.dumps({
            "metric": "median time per outer iteration over five x* seeds, 3D Poisson 256^3, s = 8, nu = 25",
            "value": head["ms_per_outer_median"] / 1e3, "unit": "s", "n_gpus": world, "steps": len(SPREAD_SEEDS),
            "warmup": max(args.warmup, 1), "ms_per_step": head["ms_per_outer_median"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (b = A x*, x* ~ U(-1,1) splitmix64 seeds 1002, 1102, 1202, 1302, 1402)",
            "config": {"workload": "poisson3d_7pt_128^3_and_256^3_xstar_spread", "s": 8, "nu": 25,
                       "precond": "jacobi", "bounds": "gershgorin + lanczos10", "tol": 1e-8,
                       "l2": "inputs larger than L2 at 256^3"},
            "clocks": clk, "spread": rows}))


def run_adjoint(args):
    """Differentiable solve (the adjoint form): 2D diffusion 1024^2, kappa =
    exp(N(0, 0.5^2)), L = ||x - x_target||^2; forward s-step CG (s = 8, nu = 25) to 1e-10, the
    backward adjoint solve (A lambda = 2 (x - x_target), to 1e-9: the attainable accuracy of
    this white-noise right-hand side is about 5e-10) and the dL/dkappa assembly. One step =
    forward + backward. After the timed steps the gradient is checked by a central difference
    along a seeded direction v (+-kappa_c, h = 1e-4), both sides run with the forward solve's
    bounds and outer count; per-cell differences at h = 1e-6 measure the solver's rounding
    noise at this size, so the 1e-6 cell-by-cell check runs at 32^2 in the test suite."""
    import numpy as np
    import torch
    from paper_2512_09642_gb300 import SStepCG
    from paper_2512_09642_gb300.autograd import solve_diffusion
    from workloads import problems as W
    from workloads import rng

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    p, xt = W.diffusion2d_adjoint(1024)
    xt_d = torch.as_tensor(xt).cuda()
    b = torch.as_tensor(p.b).cuda()
    k0 = torch.as_tensor(p.kappa).cuda()
    opts = dict(s=8, nu=25, tol=1e-10, adjoint_tol=1e-9)
    stream = torch.cuda.current_stream()

    def step():
        kappa = k0.clone().requires_grad_(True)
        x = solve_diffusion(kappa, b, p.dims, **opts)
        f1 = torch.cuda.Event(enable_timing=True)
        f1.record(stream)
        torch.sum((x - xt_d) ** 2).backward()
        return x, kappa.grad, f1

    for _ in range(max(args.warmup, 1)):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd = []
    e0.record(stream)
    s0 = e0
    for _ in range(args.steps):
        x, g, f1 = step()
        fwd.append((s0, f1))
        s1 = torch.cuda.Event(enable_timing=True)
        s1.record(stream)
        s0 = s1
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_step = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, world)
    t_fwd = statistics.mean(a.elapsed_time(bb) for a, bb in fwd) / 1e3
    # outer counts and bounds of the forward solve, then the directional check
    sv = SStepCG(grid=p.dims, kappa=k0, s=8, nu=25, tol=1e-10)
    _, info = sv.solve(b)
    sv.close()

    def loss_at(kv):
        s2 = SStepCG(grid=p.dims, kappa=kv, s=8, nu=25, tol=1e-30, max_outer=info["outer_iters"],
                     bounds=(info["lambda_min_used"], info["lambda_max_used"]))
        xx, _ = s2.solve(b)
        s2.close()
        return float(torch.sum((xx - xt_d) ** 2))

    v = np.sign(rng.uniform(4100, p.n)) * p.kappa
    h = 1e-4
    fd = (loss_at(torch.as_tensor(p.kappa + h * v).cuda()) - loss_at(torch.as_tensor(p.kappa - h * v).cuda())) / (2 * h)
    ad = float(g.cpu().numpy() @ v)
    if rank == 0:
        print(json.dumps({
            "metric": "time of one differentiable solve (forward to 1e-10 + adjoint solve + dL/dkappa), 2D diffusion 1024^2",
            "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (kappa = exp(N(0, 0.5^2)) seed 2005, x* seed 1005, x_target seed 6005)",
            "config": {"workload": "adjoint_diffusion2d_1024^2", "n": p.n, "s": 8, "nu": 25, "forward_tol": 1e-10,
                       "adjoint_tol": 1e-9, "loss": "||x - x_target||^2"},
            "forward_s": t_fwd, "backward_s": t_step - t_fwd, "forward_outer_iters": info["outer_iters"],
            "gradient_check": {"kind": "central difference along a seeded direction v = +-kappa_c, h = 1e-4",
                               "fd": fd, "adjoint": ad, "rel_err": abs(fd - ad) / abs(ad),
                               "note": "per-cell differences at h = 1e-6 measure the solves' rounding noise at "
                                       "1024^2; the 1e-6 per-cell and dense-reference checks run at 32^2 "
                                       "(tests/test_gpu_adjoint.py)"},
            "clocks": clk}))


def parse_default_forms():
    return "fp64+mom,mixed+fused+r8,mixed+fused+r4,fp64,fp64+fused,mixed+mom,fp64+mom+conj"


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "coarse":
        run_coarse(args)
    elif args.workload == "spread":
        run_spread(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
