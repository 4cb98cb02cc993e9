"""Writes tests/golden/oracle_outer_counts.txt: outer-iteration counts, final relative
residuals and per-outer CPU time of the oracle on the benchmark workloads, run to
convergence (tol 1e-8). Calls only oracle/ and workloads/. Slow: the 256^3 case takes
hours on one CPU core, which is why its result is stored.

    python tests/golden/make_oracle_outer_counts.py [sides...]
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle as O  # noqa: E402
from oracle import spectral as OS  # noqa: E402
from workloads import problems as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_outer_counts.txt")


def run(name, p, s, nu):
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    t0 = time.time()
    res = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    dt = time.time() - t0
    line = (f"{name} n={p.n} s={s} nu={nu} lam_min={lam[0]!r} lam_max={lam[1]!r} outer={res.outer_iters} "
            f"refreshes={res.refreshes} converged={res.converged} rel_res_true={res.rel_res_true:.6e} "
            f"cpu_s_per_outer={dt / max(res.outer_iters, 1):.4f}")
    print(line, flush=True)
    return line


if __name__ == "__main__":
    sides = [int(v) for v in sys.argv[1:]] or [64, 128, 256]
    lines = ["# oracle (FP64, 1 thread) to ||r||/||r0|| < 1e-8; Jacobi, bounds gersh_lanczos10 (seed 5000)",
             "# written by tests/golden/make_oracle_outer_counts.py"]
    lines.append(run("config1_poisson2d_64", W.poisson2d_64(), 4, 20))
    for side in sides:
        lines.append(run(f"poisson3d_{side}", W.poisson3d(side), 8, 25))
        with open(OUT, "w") as f:
            f.write("\n".join(lines) + "\n")
