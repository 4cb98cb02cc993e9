"""Writes tests/golden/oracle_outer_counts.txt (7-point Poisson, bounds gersh_lanczos10) and,
with `box` as first argument, tests/golden/oracle_outer_counts_box.txt (27-point Poisson,
the Lanczos-10 bounds with 10% margins of Section 8): outer-iteration counts, final relative
residuals and per-outer CPU time of the oracle on the benchmark workloads, run to
convergence (tol 1e-8). Calls only oracle/ and workloads/. Slow: the 256^3 and 230^3 cases
take hours on one CPU core, which is why their results are stored.

    python tests/golden/make_oracle_outer_counts.py [sides...]
    python tests/golden/make_oracle_outer_counts.py box [sides...]
    python tests/golden/make_oracle_outer_counts.py seeds [side]

`seeds` writes tests/golden/oracle_outer_counts_seeds.txt: the 7-point Poisson problem at one
side (default 128) for the five exact solutions x* of seeds 1002, 1102, 1202, 1302 and 1402
(1002 is the benchmark's), solved in parallel worker processes. It measures how much the
literal restarted iteration's outer-iteration count depends on the right-hand side.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle as O  # noqa: E402
from oracle import spectral as OS  # noqa: E402
from workloads import problems as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "oracle_outer_counts.txt")
OUT_BOX = os.path.join(HERE, "oracle_outer_counts_box.txt")
OUT_SEEDS = os.path.join(HERE, "oracle_outer_counts_seeds.txt")
SPREAD_SEEDS = (1002, 1102, 1202, 1302, 1402)


def run(name, p, s, nu, bounds="gersh_lanczos10"):
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, bounds, W.lanczos_start(p.n))
    t0 = time.time()
    res = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    dt = time.time() - t0
    line = (f"{name} n={p.n} s={s} nu={nu} lam_min={lam[0]!r} lam_max={lam[1]!r} outer={res.outer_iters} "
            f"refreshes={res.refreshes} converged={res.converged} rel_res_true={res.rel_res_true:.6e} "
            f"cpu_s_per_outer={dt / max(res.outer_iters, 1):.4f}")
    print(line, flush=True)
    return line


def main_box(sides):
    lines = ["# oracle (FP64, 1 thread) to ||r||/||r0|| < 1e-8; 27-point Poisson, Jacobi, bounds lanczos10 "
             "(seed 5000)", "# written by tests/golden/make_oracle_outer_counts.py box"]
    for side in sides:
        lines.append(run(f"poisson27_{side}", W.poisson27(side), 8, 25, bounds="lanczos10"))
        with open(OUT_BOX, "w") as f:
            f.write("\n".join(lines) + "\n")


def _seed_line(args):
    side, seed = args
    return run(f"poisson3d_{side}_xstar{seed}", W.poisson3d(side, xstar_seed=seed), 8, 25)


def main_seeds(side):
    import multiprocessing as mp
    lines = [f"# oracle (FP64, 1 thread per run) to ||r||/||r0|| < 1e-8; 7-point Poisson {side}^3, s = 8, "
             "nu = 25, Jacobi, bounds gersh_lanczos10 (seed 5000); x* ~ U(-1,1) from the seed in the name",
             "# written by tests/golden/make_oracle_outer_counts.py seeds"]
    with mp.get_context("spawn").Pool(len(SPREAD_SEEDS)) as pool:
        lines += pool.map(_seed_line, [(side, sd) for sd in SPREAD_SEEDS])
    with open(OUT_SEEDS, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__" and sys.argv[1:2] == ["seeds"]:
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    main_seeds(int(sys.argv[2]) if len(sys.argv) > 2 else 128)
elif __name__ == "__main__" and sys.argv[1:2] == ["box"]:
    main_box([int(v) for v in sys.argv[2:]] or [64, 128, 230])
elif __name__ == "__main__":
    sides = [int(v) for v in sys.argv[1:]] or [64, 128, 256]
    lines = ["# oracle (FP64, 1 thread) to ||r||/||r0|| < 1e-8; Jacobi, bounds gersh_lanczos10 (seed 5000)",
             "# written by tests/golden/make_oracle_outer_counts.py"]
    lines.append(run("config1_poisson2d_64", W.poisson2d_64(), 4, 20))
    for side in sides:
        lines.append(run(f"poisson3d_{side}", W.poisson3d(side), 8, 25))
        with open(OUT, "w") as f:
            f.write("\n".join(lines) + "\n")
