"""The algorithmic work model behind bench.py's roofline fractions, on the CPU: FP64 operations
and HBM bytes per unknown of each kernel, counted from the arithmetic of each step (7-point
Chebyshev step: 5 adds of the neighbour sum + 2 FMAs, reading p_j, p_(j-1) and writing
p_(j+1); moments Gram: 2s FMAs over the s + 1 basis vectors; update: s FMAs for x and s + 1
for r, reading the s + 1 vectors and x, writing x and r), and the rule that a stored ncu
traffic figure is reported only while the kernel's source is unchanged."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fp64_poisson_model_per_unknown():
    for s in (4, 8, 12, 16):
        m = bench.kernel_model(s, mom=True)
        assert m["cheb_step"] == {"ops": 7, "bytes": 24}
        assert m["gram_fgs"] == {"ops": 2 * s, "bytes": 8 * (s + 1)}
        assert m["update"] == {"ops": 2 * s + 1, "bytes": 8 * (s + 1) + 24}
        assert m["residual"] == {"ops": 8, "bytes": 24}
        # direct Gram: the s(s+1)/2 symmetric entries and the s entries against p_s
        assert bench.kernel_model(s)["gram_fgs"]["ops"] == s * (s + 1) // 2 + s
    # 2D: 3 adds + 2 FMAs
    assert bench.kernel_model(8, dim=2)["cheb_step"]["ops"] == 5
    # 27-point box step: separable box sum (2 adds per axis) + 2 FMAs
    assert bench.kernel_model(8, box=True)["cheb_step"] == {"ops": 8, "bytes": 24}


def test_outer_iteration_bytes():
    # FP64, s = 8: first step 16 B (no p_(j-1)), 7 more at 24 B, Gram 72 B, update 96 B
    assert bench.outer_bytes(8) == 16 + 7 * 24 + 72 + 96 == 352
    # mixed: FP32 steps (8 + 7 x 12 B), FP32 Gram 36 B, update 48 B, FP64 refresh 20 B
    assert bench.outer_bytes(8, mixed=True) == 8 + 7 * 12 + 36 + 48 + 20
    mixed = bench.kernel_model(8, mixed=True)
    assert mixed["cheb_step"]["ops"] == 0 and mixed["gram_fgs"]["ops"] == 0


def test_stored_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    """A traffic row is reported while the kernel's definition hashes to the stored sha256, and
    not after any edit of it. The rule is checked on a table written here for the current
    source of the FP64 Chebyshev step; the committed table's rows follow the same rule."""
    src, kernel = "paper_2512_09642_gb300/csrc/k_operator.cu", "k_cheb_poisson_pair"
    sha = bench.kernel_source_sha(src, kernel)
    assert sha is not None
    table = tmp_path / "traffic.txt"
    table.write_text("# test table\n"
                     f"poisson3d_7pt_256^3 fp64+mom cheb_step {kernel} {src} 123456 {sha} capture.md\n")
    monkeypatch.setattr(bench, "TRAFFIC", str(table))
    got = bench.measured_traffic("poisson3d_7pt_256^3", "fp64+mom", "cheb_step")
    assert got is not None and got["bytes"] == 123456 and got["kernel"] == kernel
    # committed rows: reported exactly when their source is unchanged
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        tok = line.split()
        if line.startswith("#") or len(tok) < 7:
            continue
        # every named kernel's definition is found (launch bounds may hold a constexpr call)
        assert bench.kernel_source_sha(tok[4], tok[3]) is not None, tok[3]
        current = bench.kernel_source_sha(tok[4], tok[3]) == tok[6]
        monkeypatch.setattr(bench, "TRAFFIC", os.path.join(ROOT, "profiles", "traffic.txt"))
        assert (bench.measured_traffic(tok[0], tok[1], tok[2]) is not None) == current
        monkeypatch.setattr(bench, "TRAFFIC", str(table))
    # the same table against an edited kernel definition: no traffic figure
    fake_root = tmp_path / "root"
    shutil.copytree(os.path.join(ROOT, os.path.dirname(src)), fake_root / os.path.dirname(src))
    path = fake_root / src
    text = path.read_text()
    i = text.index(kernel + "(")
    j = text.index("{", i)
    path.write_text(text[:j + 1] + "\n    // edited\n" + text[j + 1:])
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.kernel_source_sha(src, kernel) not in (None, sha)
    assert bench.measured_traffic("poisson3d_7pt_256^3", "fp64+mom", "cheb_step") is None


def test_fused_csr_and_refresh_models():
    """The fused moments move the Gram's FMAs into the steps (2 per unknown and step in FP64)
    and leave the finish no streaming bytes; the mixed update writes the recursive residual
    (reads p_s, writes p_0: 8 B more) in refresh_period - 1 of every refresh_period outer
    iterations, and the FP64 refresh runs once per period; a CSR step reads 12 B per nonzero
    (8 B in the mixed form) plus the row pointer and four vectors."""
    f = bench.kernel_model(8, fused=True)
    assert f["cheb_step"] == {"ops": 9, "bytes": 24} and f["gram_fgs"] == {"ops": 0, "bytes": 0}
    fm = bench.kernel_model(8, mixed=True, fused=True)
    assert fm["cheb_step"] == {"ops": 0, "bytes": 12} and fm["gram_fgs"]["bytes"] == 0
    assert bench.kernel_model(8, mixed=True, write_r=True)["update"]["bytes"] == 4 * 8 + 16 + 8
    # mixed, fused, refresh every 4: steps 8 + 7 x 12, update 48 + 8 x 3/4, refresh 20 / 4
    assert bench.outer_bytes(8, mixed=True, fused=True, refresh=4) == 8 + 7 * 12 + 48 + 6 + 5
    assert bench.outer_bytes(8, mixed=True, fused=True, refresh=1) == 8 + 7 * 12 + 48 + 20
    c = bench.kernel_model(8, csr=7.0)
    assert c["cheb_step"] == {"ops": 9.0, "bytes": 12 * 7.0 + 4 + 24 + 8}
    cm = bench.kernel_model(8, mixed=True, csr=7.0)
    assert cm["cheb_step"] == {"ops": 0, "bytes": 8 * 7.0 + 4 + 12 + 4}
    assert bench.form_gram("mixed+fused+r8") == "fused" and bench.form_refresh("mixed+fused+r8") == 8
    assert bench.form_gram("fp64+mom") == "moments" and bench.form_refresh("fp64") == 1


def test_kernel_report_dominant_kernel_and_roof():
    """The line's roofline comes from the kernel with the largest share of solve time: its
    average sampled launch time times its launches per solve (s steps, one Gram and one update
    per outer iteration, the residuals at start, exit and each refresh). The FP64 step is
    measured against the FP64 FMA rate, the mixed form's FP32 step against the HBM rate."""
    import types
    args = types.SimpleNamespace(s=8)
    n = 256 ** 3

    def info(ms, launches, outers=170, refreshes=0):
        return {"prof_ms": list(ms), "prof_launches": list(launches), "outer_iters": outers,
                "refreshes": refreshes}

    # FP64 moments: 8 step launches at 0.2 ms, one Gram at 0.3 ms, one update at 0.4 ms,
    # residual 0.5 ms; two sampled solves with the same averages
    infos = [info([1.6, 0.3, 0.4, 0.5], [8, 1, 1, 1]), info([3.2, 0.6, 0.8, 1.0], [16, 2, 2, 2])]
    roof, table = bench.kernel_report(args, n, infos, "fp64+mom")
    assert abs(table["cheb_step"]["avg_launch_ms"] - 0.2) < 1e-15
    assert table["cheb_step"]["launches_per_solve"] == 8 * 170
    assert table["gram_fgs"]["launches_per_solve"] == table["update"]["launches_per_solve"] == 170
    assert table["residual"]["launches_per_solve"] == 2
    assert abs(sum(v["share"] for v in table.values()) - 1.0) < 1e-12
    assert roof["kernel"] == "cheb_step" and roof["bound"] == "alu"
    ops = 7 * n
    assert roof["fp64_ops_per_launch"] == ops and roof["bytes_per_launch"] == 24 * n
    assert abs(roof["frac"] - ops / 0.2e-3 / bench.FP64_OPS_PEAK) < 1e-9
    assert abs(roof["hbm_frac"] * bench.measured_peaks()[0] * 1e9 - 24 * n / 0.2e-3) < 1e-3 * 24 * n / 0.2e-3

    # mixed, fused, refresh every 8: no FP64 work in the FP32 step, so its roof is HBM; the
    # refreshes add one residual per group of 8 outer iterations
    infos = [info([0.32, 0.05, 0.06, 0.09], [8, 1, 1, 1], outers=262, refreshes=1)]
    roof, table = bench.kernel_report(args, n, infos, "mixed+fused+r8")
    assert table["residual"]["launches_per_solve"] == -(-262 // 8) + 1 + 2 + 1
    assert roof["kernel"] == "cheb_step" and roof["bound"] == "hbm"
    by = bench.kernel_model(8, mixed=True, fused=True, write_r=True)["cheb_step"]["bytes"] * n
    assert abs(roof["achieved"] - by / 0.04e-3 / 1e9) < 1e-6 * by / 0.04e-3 / 1e9
    assert roof["peak"] == bench.measured_peaks()[0]

    # a kernel never sampled has no time and no share
    infos = [info([1.6, 0.3, 0.4, 0.0], [8, 1, 1, 0])]
    roof, table = bench.kernel_report(args, n, infos, "fp64+mom")
    assert table["residual"]["avg_launch_ms"] is None and table["residual"]["share"] == 0.0


def test_every_profile_summary_gives_its_command():
    """Each summary under profiles/ names the command that produced its figures (a bench.py or
    ncu line, the build-and-run line of a microbenchmark, or the capture it shares), and runs
    committed files only."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(f).read()
        assert any(k in text for k in ("python bench.py", "ncu ", "nvcc ", "Same capture as")), f
        assert "_work" not in text, f
