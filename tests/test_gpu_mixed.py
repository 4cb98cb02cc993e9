"""Mixed-precision form (FP32 basis and SpMV; FP64 Gram accumulation, FGS, x and the refreshed
true residual) against the FP64 oracle.

There is no FP32 oracle: the checks are that the solve reaches the same FP64 true relative
residual (<= 1e-8), that its solution differs from the FP64 oracle's by no more than the
residual tolerance allows (||x - x_o|| / ||x_o|| <= 2 kappa(A) tol, measured and printed),
that the outer-iteration count stays close to the FP64 one, and that the first iterate agrees
with the oracle's at FP32 level.
"""
import numpy as np
import pytest

import oracle as O
from oracle import spectral as OS
from workloads import problems as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _solver(p, mode, **opts):
    from paper_2512_09642_gb300 import SStepCG
    if mode == "csr":
        rp, ci, v = p.csr()
        return SStepCG(csr=(_dev(rp), _dev(ci), _dev(v)), **opts)
    return SStepCG(grid=p.dims, kappa=None if p.kappa is None else _dev(p.kappa), **opts)


CASES = [
    ("config1_poisson2d_64_csr", W.poisson2d_64, "csr", 4, 20),
    ("config1_poisson2d_64_stencil", W.poisson2d_64, "stencil", 4, 20),
    ("poisson3d_32_s8", lambda: W.poisson3d(32), "stencil", 8, 25),
    ("diffusion3d_ragged_s12", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "stencil", 12, 30),
    ("diffusion3d_csr_s8", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "csr", 8, 25),
    ("diffusion2d_stencil_s8", lambda: W.make("d2", (45, 33), kappa_sigma=0.5, config=13), "stencil", 8, 20),
]


@pytest.mark.parametrize("name,make,mode,s,nu", CASES, ids=[c[0] for c in CASES])
def test_mixed_solve_reaches_fp64_tolerance(name, make, mode, s, nu):
    p = make()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-8, precision="mixed")
    x, info = sv.solve(_dev(p.b))
    x = x.cpu().numpy()
    assert info["status"] == "SSTEP_OK", info
    true_rel = np.linalg.norm(p.b - op.matvec(x)) / np.linalg.norm(p.b)
    assert true_rel <= 1e-8 and info["rel_res_true"] <= 1e-8
    kA = np.linalg.cond(op.A.toarray()) if p.n <= 4096 else None
    err = _rel(x, ref.x)
    print(f"{name}: mixed outers {info['outer_iters']} vs fp64 oracle {ref.outer_iters}; "
          f"|x_mixed - x_oracle| / |x_oracle| = {err:.3e}")
    if kA is not None:
        assert err <= 2 * kA * 1e-8
    assert err <= 1e-4
    assert info["outer_iters"] <= int(1.25 * ref.outer_iters) + 2


@pytest.mark.parametrize("name,make,mode,s,nu", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_mixed_first_iterate_at_fp32_level(name, make, mode, s, nu):
    p = make()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=1, history=1)
    sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-30, max_outer=1, precision="mixed", check_every=1)
    x, info = sv.solve(_dev(p.b))
    assert info["outer_iters"] == 1
    assert _rel(x.cpu().numpy(), ref.history[0].x) <= 1e-5


def test_mixed_is_scale_invariant():
    """The FP32 basis is scaled by a power of two: b * 2^-120 (far below FP32's normal range
    when unscaled) gives the same iterates times 2^-120."""
    p = W.poisson3d(16)
    sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, precision="mixed")
    x1, i1 = sv.solve(_dev(p.b))
    x2, i2 = sv.solve(_dev(p.b * 2.0 ** -120))
    assert i1["status"] == i2["status"] == "SSTEP_OK"
    assert i1["outer_iters"] == i2["outer_iters"]
    assert torch.equal(x2 * 2.0 ** 120, x1)


def test_mixed_matches_fp64_library_solution():
    p = W.poisson3d(48)
    sv64 = _solver(p, "stencil", s=8, nu=25, tol=1e-8)
    sv32 = _solver(p, "stencil", s=8, nu=25, tol=1e-8, precision="mixed")
    b = _dev(p.b)
    x64, i64 = sv64.solve(b)
    x32, i32 = sv32.solve(b)
    assert i64["status"] == i32["status"] == "SSTEP_OK"
    err = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
    print(f"48^3: fp64 {i64['outer_iters']} outers, mixed {i32['outer_iters']}, |x32 - x64|/|x64| = {err:.2e}")
    assert err <= 1e-5


def test_mixed_conversions_round_to_nearest_even_and_back_exactly():
    """The refresh's float(r * 2^k) is built from the IEEE fields with integer operations and
    the update's float -> double likewise: compare with torch's conversions."""
    from paper_2512_09642_gb300 import abi
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(200000, generator=g, dtype=torch.float64)
    x = torch.cat([x, x * 1e-30, x * 1e30, torch.tensor([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 3.0 * 2 ** -150,
                                                         float("inf"), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24])])
    # halfway cases: mantissas ending exactly at the FP32 rounding boundary
    ties = torch.tensor([1.0 + (2 * k + 1) * 2.0 ** -24 for k in range(64)], dtype=torch.float64)
    x = torch.cat([x, ties, -ties]).cuda()
    for k in (0, 5, -7, 40):
        out = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
        back = torch.empty(x.numel(), dtype=torch.float64, device="cuda")
        abi.sstep_convert_check(x, k, out, back)
        ref = (x * 2.0 ** k).float()
        assert torch.equal(out, ref) or bool(torch.all((out == ref) | (torch.isnan(out) & torch.isnan(ref))))
        assert torch.equal(back, out.double())


REFRESH_CASES = [
    ("poisson3d_48_fused", lambda: W.poisson3d(48), 8, 25, "fused"),
    ("poisson3d_odd_ragged_fused", lambda: W.make("p3", (19, 13, 11), config=12), 8, 25, "fused"),
    ("diffusion3d_ragged_moments", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), 12, 30, "moments"),
    ("diffusion2d_direct", lambda: W.make("d2", (45, 33), kappa_sigma=0.5, config=13), 8, 20, "direct"),
]


@pytest.mark.parametrize("name,make,s,nu,form", REFRESH_CASES, ids=[c[0] for c in REFRESH_CASES])
@pytest.mark.parametrize("period", [1, 2, 3, 4])
def test_mixed_refresh_period_reaches_fp64_tolerance(name, make, s, nu, form, period):
    """The mixed form with the FP64 residual refreshed every `period` outer iterations (the
    others update the FP32 residual recursively and test convergence on it): every form of the
    Gram reaches the FP64 true relative residual 1e-8, with a solution within 1e-5 of the FP64
    oracle's and an outer count close to the oracle's; the graph-driven loop equals the host
    loop bit for bit (period 3 does not divide the host loop's 8 outer iterations per check)."""
    p = make()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    b = _dev(p.b)
    kw = dict(bounds=lam, s=s, nu=nu, tol=1e-8, precision="mixed", gram_form=form, refresh_period=period)
    sv = _solver(p, "stencil", **kw)
    x, info = sv.solve(b)
    assert info["status"] == "SSTEP_OK", info
    xn = x.cpu().numpy()
    true_rel = np.linalg.norm(p.b - op.matvec(xn)) / np.linalg.norm(p.b)
    assert true_rel <= 1e-8 and info["rel_res_true"] <= 1e-8
    err = _rel(xn, ref.x)
    print(f"{name} period {period}: mixed outers {info['outer_iters']} (refreshes {info['refreshes']}) vs fp64 "
          f"oracle {ref.outer_iters}; |x_mixed - x_oracle| / |x_oracle| = {err:.3e}")
    assert err <= 1e-5
    assert info["outer_iters"] <= int(1.25 * ref.outer_iters) + period + 2
    sg = _solver(p, "stencil", use_graph=1, **kw)
    xg, ig = sg.solve(b)
    assert ig["outer_iters"] == info["outer_iters"] and torch.equal(xg, x)


def test_mixed_fused_first_iterate_at_fp32_level():
    p = W.poisson3d(32)
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=8, nu=25, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=2, history=2)
    for k in (1, 2):
        sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=k, precision="mixed",
                     gram_form="fused", check_every=1, refresh_period=2)
        x, info = sv.solve(_dev(p.b))
        assert info["outer_iters"] == k
        assert _rel(x.cpu().numpy(), ref.history[k - 1].x) <= 1e-5, k


# The FP32 Chebyshev step through tensor-map (TMA) tiles (3D Poisson, nx a multiple of 4) against
# the same step with plain loads: the same sums in the same order, so with the separate Gram pass
# (moments form) the solves agree bit for bit. With the fused moments the per-block partial sums
# follow each kernel's blocks (32-plane slabs against 16), so there the iterates agree to FP32
# rounding. Grids: 64 x 13 x 11 (one x tile, ragged y and z tiles against 64 x 8 x 32), 4 x 3 x 70
# (a 4-point-wide grid inside one 64-wide tile, three 32-plane slabs), 132 x 37 x 35 (a 4-point x
# tile at the end, both x faces inside boxes that start 4 points before the tile).
TMA_GRIDS = [((64, 13, 11), 41), ((4, 3, 70), 42), ((132, 37, 35), 43)]


@pytest.mark.parametrize("dims,cfg", TMA_GRIDS, ids=["x".join(map(str, d)) for d, _ in TMA_GRIDS])
@pytest.mark.parametrize("form,period", [("moments", 1), ("moments", 3), ("fused", 1), ("fused", 4)])
def test_fp32_step_through_tma_tiles_equals_plain_loads(dims, cfg, form, period):
    p = W.make("p3t", dims, config=cfg)
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "lanczos10", W.lanczos_start(p.n))
    b = _dev(p.b)
    for k, tol in ((1, 1e-30), (3, 1e-30), (100000, 1e-8)):
        out = {}
        for path in ("tma", "plain"):
            sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=tol, max_outer=k, check_every=1,
                         precision="mixed", gram_form=form, refresh_period=period, step_kernel=path)
            x, info = sv.solve(b)
            out[path] = (x.cpu().numpy(), info)
            sv.close()
        (xt, it), (xp, ip) = out["tma"], out["plain"]
        assert it["step_tma"] == 1 and ip["step_tma"] == 0
        if form == "moments":
            assert it["outer_iters"] == ip["outer_iters"], (k, it["outer_iters"], ip["outer_iters"])
            assert np.array_equal(xt, xp), (k, _rel(xt, xp))
        elif tol < 1e-20:
            assert _rel(xt, xp) <= 1e-5, (k, _rel(xt, xp))
        if tol == 1e-8:
            assert it["status"] == "SSTEP_OK" and it["rel_res_true"] <= 1e-8


def test_fp32_step_tma_falls_back_where_the_shape_does_not_allow_it():
    """nx not a multiple of 4 (a TMA row stride must be a multiple of 16 bytes), and 2D: plain
    loads, the same solve."""
    for dims, cfg in (((70, 13, 11), 44), ((64, 45), 45)):
        p = W.make("p3t", dims, config=cfg)
        op = O.Operator(*p.csr())
        lam = OS.bounds(op, "lanczos10", W.lanczos_start(p.n))
        xs = {}
        for path in ("tma", "plain"):
            sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-8, precision="mixed", gram_form="moments",
                         step_kernel=path)
            x, info = sv.solve(_dev(p.b))
            assert info["step_tma"] == 0 and info["status"] == "SSTEP_OK"
            xs[path] = x.cpu().numpy()
            sv.close()
        assert np.array_equal(xs["tma"], xs["plain"])


def test_fp32_step_auto_uses_tma_only_when_the_step_exceeds_l2():
    """AUTO: plain loads at 64^3 (3 x 1 MB of FP32 vectors), TMA tiles at 256^3 (3 x 67 MB > L2)."""
    for side, want in ((64, 0), (256, 1)):
        p = W.poisson3d(side)
        sv = _solver(p, "stencil", bounds=(0.003, 2.0), s=8, nu=25, tol=1e-30, max_outer=1, precision="mixed",
                     gram_form="fused")
        _, info = sv.solve(_dev(p.b))
        assert info["step_tma"] == want, side
        sv.close()
