"""The C ABI without a GPU: the library loads, exports every entry point the header declares,
the ctypes structs match the C layout (checked by compiling the header with gcc), and
invalid arguments are rejected on the host before any CUDA call."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def abi():
    from paper_2512_09642_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2512_09642_gb300 import abi as mod
    return mod


def _declared():
    names = set()
    for h in HEADERS:
        names |= set(re.findall(r"SSTEP_API\s+[\w\s\*]+?\b(sstep_\w+)\s*\(", open(h).read()))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    assert "sstep_cg_solve" in names and "sstep_cg_create_csr" in names and len(names) >= 10


def test_library_exports_every_declared_symbol(abi):
    for name in _declared():
        assert hasattr(abi.lib, name), name


def test_binding_covers_every_declared_symbol(abi):
    missing = [n for n in _declared() if n not in abi.exported_names()]
    assert not missing, missing


def test_struct_layout_matches_c(abi):
    import ctypes
    fields = {"sstep_cg_opts": abi.Opts, "sstep_cg_info": abi.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sstep_cg.h"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for cname, cls in fields.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_default_options(abi):
    o = abi.sstep_cg_default_opts()
    assert (o.s, o.nu, o.tol, o.max_outer) == (8, 25, 1e-8, 100000)
    assert o.bounds_mode == abi.BOUNDS["gersh_lanczos10"] and o.precond == abi.PRECOND["jacobi"]
    assert o.gram_solver == abi.GRAM_SOLVER["fgs"] and o.precision == abi.PRECISION["fp64"]
    assert o.step_kernel == abi.STEP_KERNEL["auto"] and o.history == 0


@pytest.mark.parametrize("bad", [dict(s=0), dict(s=33), dict(nu=0), dict(tol=0.0), dict(tol=-1.0),
                                 dict(bounds_mode=0, lambda_min=1.0, lambda_max=0.5),
                                 dict(bounds_mode=0, lambda_min=-1.0, lambda_max=2.0), dict(bounds_mode=7),
                                 dict(gram_solver=5), dict(precond=3), dict(max_outer=-1), dict(check_every=0)])
def test_invalid_options_rejected_on_host(abi, bad):
    o = abi.sstep_cg_default_opts(**bad)
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_stencil(2, 8, 8, 1, None, o, stream=0)
    assert ei.value.status == 1
    assert abi.sstep_cg_last_error(None)


@pytest.mark.parametrize("grid", [(4, 8, 8, 1), (2, 8, 8, 2), (3, 0, 8, 8), (2, -1, 4, 1)])
def test_invalid_grid_rejected_on_host(abi, grid):
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_stencil(*grid, None, abi.sstep_cg_default_opts(), stream=0)
    assert ei.value.status == 1
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_box_stencil(*grid, abi.sstep_cg_default_opts(), stream=0)
    assert ei.value.status == 1


@pytest.mark.parametrize("create,grid", [("stencil", (3, 4, 524281, 4)), ("stencil", (2, 4, 524281, 1)),
                                         ("stencil", (3, 4, 4, 524281)), ("box", (3, 4, 524281, 4)),
                                         ("box", (3, 4, 4, 1048561))])
def test_grid_extents_beyond_launch_limits_rejected_on_host(abi, create, grid):
    """A stencil grid whose y or z extent would need more than 65535 blocks of 8 rows or 8
    planes (16 for the box stencil's z) is refused at create, before any CUDA call."""
    with pytest.raises(abi.SStepError) as ei:
        if create == "stencil":
            abi.sstep_cg_create_stencil(*grid, None, abi.sstep_cg_default_opts(), stream=0)
        else:
            abi.sstep_cg_create_box_stencil(*grid, abi.sstep_cg_default_opts(), stream=0)
    assert ei.value.status == 1 and "bad grid" in abi.sstep_cg_last_error(None)


def test_block_conjugate_options_checked_on_host(abi):
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_stencil(2, 8, 8, 1, None, abi.sstep_cg_default_opts(block_conjugate=2), stream=0)
    assert ei.value.status == 1
    for bad in (dict(precision="mixed"), dict(s=17)):
        with pytest.raises(abi.SStepError) as ei:
            abi.sstep_cg_create_stencil(2, 8, 8, 1, None, abi.sstep_cg_default_opts(block_conjugate=1, **bad), stream=0)
        assert ei.value.status == 7


def test_box_stencil_invalid_options_rejected_on_host(abi):
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_box_stencil(3, 8, 8, 8, abi.sstep_cg_default_opts(s=0), stream=0)
    assert ei.value.status == 1


def test_invalid_csr_rejected_on_host(abi):
    import ctypes
    h = ctypes.c_void_p()
    o = abi.sstep_cg_default_opts()
    assert abi.lib.sstep_cg_create_csr(ctypes.byref(h), 0, 16, 16, 16, ctypes.byref(o), None) == 1
    assert abi.lib.sstep_cg_create_csr(ctypes.byref(h), 10, None, 16, 16, ctypes.byref(o), None) == 1
    assert abi.lib.sstep_cg_create_csr(ctypes.byref(h), 10, 8, 16, 16, ctypes.byref(o), None) == 1  # misaligned
    assert not h.value


def test_status_strings(abi):
    for code, name in abi.STATUS.items():
        assert abi.sstep_cg_status_string(code) == name


@pytest.mark.parametrize("bad", [dict(gram_form=3), dict(gram_form=2, block_conjugate=1), dict(refresh_period=0),
                                 dict(step_kernel=3), dict(step_kernel=-1)])
def test_gram_form_and_refresh_options_checked_on_host(abi, bad):
    """FUSED (the moments reduced by the step kernels) does not combine with the block
    conjugation (SSTEP_ERR_UNSUPPORTED); an unknown form, a refresh period below 1 or an unknown
    step_kernel is an invalid argument. All rejected before any CUDA call."""
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_create_stencil(3, 8, 8, 8, None, abi.sstep_cg_default_opts(**bad), stream=0)
    assert ei.value.status == (7 if bad.get("block_conjugate") else 1)
    assert abi.sstep_cg_last_error(None)


def test_noalloc_arguments_checked_on_host(abi):
    """sstep_gram_fgs_noalloc validates every argument before its first CUDA call: sizes, the
    static scratch's limit s <= 16, bounds, the preconditioner and the pointers (the fake
    device addresses below are never dereferenced)."""
    lib = abi.lib
    P, out, md = 4096, 8192, 12288
    good = dict(n=64, s=4, nu=10, solver=0, P=P, ldp=64, md=None, mc=4.0, lo=0.1, hi=2.0, out=out)

    def call(**kw):
        a = dict(good, **kw)
        return lib.sstep_gram_fgs_noalloc(a["n"], a["s"], a["nu"], a["solver"], a["P"], a["ldp"], a["md"], a["mc"],
                                          a["lo"], a["hi"], a["out"], None)

    for bad in (dict(P=None), dict(out=None), dict(s=0), dict(s=17), dict(n=0), dict(ldp=63), dict(nu=0),
                dict(nu=10001), dict(solver=2), dict(lo=2.0, hi=2.0), dict(lo=3.0), dict(lo=-0.5),
                dict(md=None, mc=0.0), dict(md=None, mc=-1.0)):
        assert call(**bad) == 1, bad
        msg = lib.sstep_cg_last_error(None).decode()
        assert msg.startswith("sstep_gram_fgs_noalloc:"), (bad, msg)
        if bad.get("s") in (0, 17):
            assert "16" in msg
    # mdiag given: mconst is not used
    assert call(md=md, mc=0.0, s=17) == 1


@pytest.mark.parametrize("grids,bad,status", [
    ([], {}, 1),                                                   # no systems
    ([(8, 8)], dict(s=17), 1), ([(8, 8)], dict(s=0), 1), ([(8, 8)], dict(nu=0), 1),
    ([(8, 8)], dict(tol=0.0), 1), ([(8, 8)], dict(tol=float("inf")), 1),
    ([(8, 8)], dict(max_outer=-1), 1), ([(8, 8)], dict(check_every=0), 1),
    ([(8, 8)], dict(gram_solver=5), 1),
    ([(8, 8)], dict(bounds_mode=0, lambda_min=1.0, lambda_max=0.5), 1),
    ([(8, 8)], dict(bounds_mode=0, lambda_min=0.1, lambda_max=float("inf")), 1),
    ([(8, 8)], dict(bounds_mode=7), 1),
    ([(8, 8)], dict(batch_chunk=100), 1), ([(8, 8)], dict(batch_ctas_per_sm=9), 1),
    ([(8, 8), (0, 8)], {}, 1), ([(8, 8, 0)], {}, 1),              # an empty grid
    ([(8, 8)], dict(precision=1), 7), ([(8, 8)], dict(precond=0), 7),   # FP64 Jacobi only
    ([(8, 8)], dict(gram_form=2), 7), ([(8, 8)], dict(block_conjugate=1), 7),
])
def test_batch_create_checked_on_host(abi, grids, bad, status):
    """The batched form's options and grids are checked before its first CUDA call:
    INVALID_ARG (1) for values outside their ranges, UNSUPPORTED (7) for the forms it does not
    run (mixed precision, no preconditioner, the fused Gram, block conjugation)."""
    o = abi.sstep_cg_default_opts(**bad)
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_cg_batch_create(grids, [None] * len(grids), o, stream=0)
    assert ei.value.status == status, str(ei.value)
    assert str(ei.value).split(": ", 1)[1]


def test_solver_refuses_arrays_the_abi_cannot_check():
    """The C ABI takes plain pointers whose lengths the handle implies, so SStepCG refuses, before
    any call, a tensor that is not on the GPU, has another element type, another number of
    elements or lives on another device (stand-in objects with the tensor attributes it reads)."""
    import torch
    from paper_2512_09642_gb300.solver import check_array

    class Fake:
        def __init__(self, dtype=torch.float64, n=10, dev="cuda:0", cuda=True):
            self.dtype, self._n, self.device, self.is_cuda = dtype, n, torch.device(dev), cuda

        def numel(self):
            return self._n

    dev = torch.device("cuda", 0)
    check_array(Fake(), "b", 10, torch.float64, dev)
    check_array(Fake(torch.int32, 11), "rowptr", 11, torch.int32, dev)
    for bad, what in ((Fake(cuda=False, dev="cpu"), "CUDA"), (Fake(torch.float32), "float64"),
                      (Fake(n=9), "10 elements"), (Fake(dev="cuda:1"), "cuda:0")):
        with pytest.raises(ValueError, match=what):
            check_array(bad, "b", 10, torch.float64, dev)
    with pytest.raises(ValueError, match="CUDA"):
        check_array(torch.zeros(10, dtype=torch.float64), "b", 10, torch.float64, dev)


def test_microbenchmarks_compile(tmp_path):
    """The standalone programs behind the FP64 roof and the one-warp latency figures keep
    compiling for sm_103a against the library's current headers (no GPU needed)."""
    import glob
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    srcs = sorted(glob.glob(os.path.join(ROOT, "paper_2512_09642_gb300", "microbench", "*.cu")))
    assert {os.path.basename(s) for s in srcs} >= {"fp64_rate.cu", "warp_fp64_latency.cu", "fgs_sweep_forms.cu"}
    for src in srcs:
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                            "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-c", src,
                            "-o", str(tmp_path / (os.path.basename(src) + ".o"))], capture_output=True, text=True)
        assert r.returncode == 0, (src, r.stderr[-2000:])


def test_every_declaration_is_documented_and_cited():
    """Each entry point of the C ABI has its own comment block; those that compute part of the
    method cite the section of the paper that defines it (status, lifetime and self-test calls
    excepted)."""
    plumbing = {"sstep_cg_default_opts", "sstep_cg_destroy", "sstep_cg_status_string", "sstep_cg_last_error",
                "sstep_cg_batch_destroy", "sstep_cg_batch_last_error", "sstep_selftest_tma_timeout"}
    for h in HEADERS:
        src = open(h).read()
        for m in re.finditer(r"SSTEP_API\s+[\w\s\*]+?\b(sstep_\w+)\s*\(", src):
            before = src[:m.start()].rstrip()
            assert before.endswith("*/"), f"{m.group(1)} has no comment"
            comment = before[before.rfind("/*"):]
            if m.group(1) not in plumbing:
                assert "Section" in comment or "paper" in comment, f"{m.group(1)} cites no passage"


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With no built library next to it, importing the binding (and so SStepCG) raises: there is
    no CPU fallback on the product path. Checked on a copy of the package's Python files."""
    import shutil
    import sys
    pkg = os.path.join(ROOT, "paper_2512_09642_gb300")
    dst = tmp_path / "paper_2512_09642_gb300"
    dst.mkdir()
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            shutil.copy(os.path.join(pkg, f), dst / f)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    from paper_2512_09642_gb300 import SStepCG\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n"
            "else:\n"
            "    print('imported')\n") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("raised") and "libsstep_cg.so is missing" in r.stdout, r.stdout + r.stderr
