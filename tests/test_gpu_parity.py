"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances (FP64): operator and basis 1e-12 relative (the kernels sum in a different order
than scipy/numpy, and the Chebyshev recurrence amplifies rounding by at most a small factor
for bounds that contain the spectrum); Gram quantities 1e-10; whole-solve iterates 1e-10
relative per iterate over the first five outer iterations and a final true relative residual
<= 1e-8, as the target of this method states.
"""
import numpy as np
import pytest

import oracle as O
from oracle import spectral as OS
from workloads import problems as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _solver(p, mode, **opts):
    from paper_2512_09642_gb300 import SStepCG
    if mode == "csr":
        rp, ci, v = p.csr()
        return SStepCG(csr=(_dev(rp), _dev(ci), _dev(v)), **opts)
    kappa = None if p.kappa is None else _dev(p.kappa)
    return SStepCG(grid=p.dims, kappa=kappa, **opts)


CASES = [
    ("poisson2d_csr", lambda: W.make("p2", (37, 29), config=11), "csr"),
    ("poisson2d_stencil", lambda: W.make("p2", (37, 29), config=11), "stencil"),
    ("poisson3d_stencil", lambda: W.make("p3", (19, 13, 11), config=12), "stencil"),
    ("poisson3d_csr", lambda: W.make("p3", (19, 13, 11), config=12), "csr"),
    ("diffusion2d_stencil", lambda: W.make("d2", (45, 33), kappa_sigma=1.0, config=13), "stencil"),
    ("diffusion3d_stencil", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "stencil"),
    ("diffusion3d_csr", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "csr"),
    # even nx: the two-points-per-thread Poisson kernels (ragged in every direction); in 3D the
    # FP64 step's register-blocked persistent march (warp columns of 32 lanes over (row pair,
    # x pair): 70 x 13 straddles row pairs and leaves a partial last column; 2 x 9 is one pair
    # with both x faces; 4 x 3 x 70 splits one column over many warps mid-column; 130 x 37 x 35
    # has 65 pairs, an odd ny and ragged planes)
    ("poisson3d_even_ragged", lambda: W.make("p3e", (70, 13, 11), config=17), "stencil"),
    ("poisson2d_even_ragged", lambda: W.make("p2e", (130, 33), config=18), "stencil"),
    ("poisson3d_even_pair", lambda: W.make("p3e", (2, 9, 5), config=19), "stencil"),
    ("poisson3d_even_deep", lambda: W.make("p3e", (4, 3, 70), config=20), "stencil"),
    ("poisson3d_even_wide", lambda: W.make("p3e", (130, 37, 35), config=21), "stencil"),
]


@pytest.mark.parametrize("name,make,mode", CASES, ids=[c[0] for c in CASES])
def test_apply_matches_oracle(name, make, mode):
    p = make()
    op = O.Operator(*p.csr())
    sv = _solver(p, mode, bounds=(0.05, 2.0), s=4)
    x = np.random.default_rng(0).uniform(-1, 1, p.n)
    y = sv.apply(_dev(x)).cpu().numpy()
    assert _rel(y, op.matvec(x)) <= 1e-14


@pytest.mark.parametrize("name,make,mode", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_chebyshev_basis_matches_oracle(name, make, mode, precond):
    p = make()
    op = O.Operator(*p.csr(), precond=precond)
    lam = (0.03, 2.05) if precond == "jacobi" else (0.1, 8.5 * (1 + (p.kappa is not None) * 8))
    s = 9
    sv = _solver(p, mode, bounds=lam, s=s, precond=precond)
    r = p.b.copy()
    P = sv.basis(_dev(r), s + 1).cpu().numpy()
    ref = O.chebyshev_basis(op, r, s, lam[0], lam[1], ncols=s + 1)
    for j in range(s + 1):
        assert _rel(P[j], ref[:, j]) <= 1e-12, j


@pytest.mark.parametrize("name,make,mode", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("s", [1, 4, 8, 12])
@pytest.mark.parametrize("form", ["direct", "moments"])
def test_gram_solve_matches_oracle(name, make, mode, s, form):
    p = make()
    op = O.Operator(*p.csr())
    lam = (0.04, 2.0)
    sv = _solver(p, mode, bounds=lam, s=s, nu=20, gram_form=form)
    r = p.b.copy()
    Pp = O.chebyshev_basis(op, r, s, lam[0], lam[1], ncols=s + 1)
    alpha, d, ct, Gt = sv.gram_solve(_dev(Pp.T))
    G, c, _ = O.gram(op, Pp[:, :s], r)
    d0, Gt0, ct0 = O.column_scaling(G, c)
    a0 = O.fgs(Gt0, ct0, 20)
    assert _rel(Gt, Gt0) <= 1e-10
    assert _rel(ct, ct0) <= 1e-10
    assert _rel(d, d0) <= 1e-10
    assert _rel(alpha, d0 * a0) <= 1e-9


def test_gram_solve_cholesky_matches_oracle():
    p = W.make("d2", (45, 33), kappa_sigma=1.0, config=13)
    op = O.Operator(*p.csr())
    s, lam = 6, (0.04, 2.0)
    sv = _solver(p, "stencil", bounds=lam, s=s, gram_solver="cholesky")
    Pp = O.chebyshev_basis(op, p.b, s, lam[0], lam[1], ncols=s + 1)
    alpha, d, ct, Gt = sv.gram_solve(_dev(Pp.T))
    G, c, _ = O.gram(op, Pp[:, :s], p.b)
    d0, Gt0, ct0 = O.column_scaling(G, c)
    assert _rel(alpha, d0 * O.cholesky_solve(Gt0, ct0)) <= 1e-9


def _iterates(p, mode, s, nu, lam, k, **kw):
    sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-30, max_outer=k, check_every=1, **kw)
    b = _dev(p.b)
    x, info = sv.solve(b)
    return x.cpu().numpy(), sv.residual().cpu().numpy(), info


SOLVE_CASES = [
    ("config1_poisson2d_64_csr", W.poisson2d_64, "csr", 4, 20),
    ("config1_poisson2d_64_stencil", W.poisson2d_64, "stencil", 4, 20),
    ("poisson3d_32_stencil_s8", lambda: W.poisson3d(32), "stencil", 8, 25),
    ("diffusion3d_ragged_s12", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "stencil", 12, 30),
    ("diffusion2d_csr_s8", lambda: W.make("d2", (45, 33), kappa_sigma=0.5, config=13), "csr", 8, 20),
    ("poisson3d_even_ragged_s8", lambda: W.make("p3e", (70, 13, 11), config=17), "stencil", 8, 25),
    ("poisson3d_even_wide_s8", lambda: W.make("p3e", (130, 37, 35), config=21), "stencil", 8, 25),
]


# cases whose operator admits the fused moments (stencil, constant M): the pair kernel (nx
# even), the one-point kernel (nx odd), 2D and 3D
FUSED_CASES = [
    ("config1_poisson2d_64_stencil", W.poisson2d_64, "stencil", 4, 20),
    ("poisson3d_32_stencil_s8", lambda: W.poisson3d(32), "stencil", 8, 25),
    ("poisson3d_even_ragged_s8", lambda: W.make("p3e", (70, 13, 11), config=17), "stencil", 8, 25),
    ("poisson3d_even_wide_s8", lambda: W.make("p3e", (130, 37, 35), config=21), "stencil", 8, 25),
    ("poisson3d_odd_ragged_s12", lambda: W.make("p3", (19, 13, 11), config=12), "stencil", 12, 30),
    ("poisson2d_odd_s1", lambda: W.make("p2", (37, 29), config=11), "stencil", 1, 5),
]


@pytest.mark.parametrize("name,make,mode,s,nu", SOLVE_CASES + FUSED_CASES[4:],
                         ids=[c[0] for c in SOLVE_CASES + FUSED_CASES[4:]])
@pytest.mark.parametrize("form", ["direct", "moments", "fused"])
def test_per_iterate_parity_first_five_outer_iterations(name, make, mode, s, nu, form):
    """x_k and r_k, k = 1..5, within 1e-10 of the oracle (which forms G = P^T A P directly)
    for every way of forming G on the GPU (fused: the moments reduced by the step kernels,
    where the operator allows it)."""
    if form == "fused" and name not in [c[0] for c in FUSED_CASES]:
        pytest.skip("fused moments need a stencil operator with a constant M")
    p = make()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=5, history=5)
    for k in range(1, 6):
        x, r, info = _iterates(p, mode, s, nu, lam, k, gram_form=form)
        assert info["outer_iters"] == k
        h = ref.history[k - 1]
        assert _rel(x, h.x) <= 1e-10, (k, _rel(x, h.x))
        assert _rel(r, h.r) <= 1e-10, (k, _rel(r, h.r))


@pytest.mark.parametrize("name,make,mode,s,nu", SOLVE_CASES[:3] + SOLVE_CASES[4:], ids=[c[0] for c in SOLVE_CASES[:3] + SOLVE_CASES[4:]])
def test_full_solve_reaches_tolerance_like_oracle(name, make, mode, s, nu):
    p = make()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-8)
    x, info = sv.solve(_dev(p.b))
    x = x.cpu().numpy()
    assert info["status"] == "SSTEP_OK", info
    assert info["rel_res_true"] <= 1e-8
    assert np.linalg.norm(p.b - op.matvec(x)) / np.linalg.norm(p.b) <= 1e-8
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    assert _rel(x, ref.x) <= 1e-7


@pytest.mark.parametrize("mode", ["csr", "stencil"])
@pytest.mark.parametrize("which", ["gersh_lanczos10", "lanczos10"])
def test_spectral_bounds_match_oracle(mode, which):
    p = W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14) if mode == "stencil" else W.poisson2d_64()
    op = O.Operator(*p.csr())
    sv = _solver(p, mode, s=4, bounds_mode=which, seed=5000)
    a, b = sv.lanczos(10, 5000)
    a0, b0 = OS.lanczos(op, W.lanczos_start(p.n), 10)
    assert np.allclose(a, a0, rtol=1e-10, atol=1e-12) and np.allclose(b, b0, rtol=1e-10, atol=1e-12)
    lo, hi = sv.bounds
    lo0, hi0 = OS.bounds(op, which, W.lanczos_start(p.n))
    assert lo == pytest.approx(lo0, rel=1e-10) and hi == pytest.approx(hi0, rel=1e-10)


def test_solve_is_deterministic():
    p = W.poisson3d(24)
    sv = _solver(p, "stencil", s=8, nu=25)
    b = _dev(p.b)
    x1, i1 = sv.solve(b)
    x2, i2 = sv.solve(b)
    assert torch.equal(x1, x2) and i1["outer_iters"] == i2["outer_iters"]


def test_edge_cases():
    # 1 x 1 grid: A = [4]; one outer iteration solves it
    p = W.make("tiny", (1, 1), config=15)
    sv = _solver(p, "stencil", bounds=(0.5, 1.5), s=1, nu=1)
    x, info = sv.solve(_dev(p.b))
    assert info["status"] == "SSTEP_OK" and abs(x.item() - p.x_star[0]) <= 1e-14 * abs(p.x_star[0])
    # b = 0 converges at once with x = 0
    p = W.make("z", (8, 8), config=15)
    sv = _solver(p, "stencil", bounds=(0.1, 2.0), s=4)
    x, info = sv.solve(torch.zeros(64, dtype=torch.float64, device="cuda"))
    assert info["status"] == "SSTEP_OK" and info["outer_iters"] == 0 and torch.count_nonzero(x) == 0
    # max_outer = 0 returns x0 unchanged with NO_CONVERGENCE
    sv = _solver(p, "stencil", bounds=(0.1, 2.0), s=4, max_outer=0)
    x0 = _dev(np.full(64, 0.25))
    x, info = sv.solve(_dev(p.b), x0)
    assert info["status"] == "SSTEP_ERR_NO_CONVERGENCE" and torch.equal(x, x0)
    # s = 32 on a small 2D problem, and odd sizes
    for dims, s in [((33, 31), 32), ((2, 2), 3), ((9, 7, 5), 16)]:
        q = W.make("e", dims, kappa_sigma=0.3, config=16)
        op = O.Operator(*q.csr())
        lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(q.n))
        ref = O.solve(op, q.b, s=s, nu=30, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=2, history=2)
        sv = _solver(q, "stencil", bounds=lam, s=s, nu=30, tol=1e-30, max_outer=2)
        x, info = sv.solve(_dev(q.b))
        assert _rel(x.cpu().numpy(), ref.history[-1].x) <= 1e-9, dims


def test_resume_from_a_saved_iterate():
    """Checkpoint and resume: the restarted iteration's state is x, so a solve started from a
    saved iterate (the oracle's x_3, nx even: the register-blocked steps) continues as the
    oracle continues from it: its two resumed iterates agree to 1e-10 for both Gram forms, and
    the resumed solve reaches 1e-8 relative to its own starting residual."""
    p = W.make("p3", (20, 13, 11), config=12)
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    kw = dict(s=8, nu=25, lam_min=lam[0], lam_max=lam[1], tol=1e-30)
    x3 = O.solve(op, p.b, max_outer=3, **kw).x
    ref = O.solve(op, p.b, x3, max_outer=2, history=2, **kw)
    for form in ("direct", "moments"):
        sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=2, gram_form=form, check_every=1)
        x, info = sv.solve(_dev(p.b), _dev(x3))
        sv.close()
        assert info["outer_iters"] == 2, info
        assert _rel(x.cpu().numpy(), ref.history[-1].x) <= 1e-10, form
    sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-8)
    x, info = sv.solve(_dev(p.b), _dev(x3))
    sv.close()
    assert info["status"] == "SSTEP_OK" and info["rel_res_true"] <= 1e-8, info


def test_host_buffer_solve_matches_device_solve():
    from paper_2512_09642_gb300 import abi
    p = W.poisson2d_64()
    sv = _solver(p, "stencil", s=4, nu=20)
    xd, _ = sv.solve(_dev(p.b))
    xh = np.zeros(p.n)
    info = abi.sstep_cg_solve_host(sv.h, np.ascontiguousarray(p.b), xh)
    assert info.status == 0
    assert np.array_equal(xh, xd.cpu().numpy())


@pytest.mark.parametrize("form", ["direct", "moments", "fused"])
def test_full_solve_outer_counts_match_stored_oracle_runs(form):
    """64^3, 128^3 and 256^3 Poisson (s = 8, nu = 25) to 1e-8 against the outer-iteration
    counts of the oracle's own converged runs (tests/golden/oracle_outer_counts.txt). The
    first iterates agree to 1e-10, but the literal restarted method's count over hundreds of
    outer iterations is sensitive to rounding: at 256^3 changing only the summation order of
    the stencil's neighbour sum moved the GPU count from 227 to 320 (direct Gram) and from
    219 to 170, and a different Gram grid size then gave 166 (moments);
    the oracle needs 269, and the same change-of-basis arithmetic in numpy already needs 116
    instead of 112 at 128^3. So the count must lie between half and 1.5 times the oracle's
    (the observed spread, 166 to 320 against 269, is 0.62x to 1.19x), and the true residual
    must reach the tolerance."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_outer_counts.txt")
    stored = {}
    for line in open(path):
        if line.startswith("poisson3d_"):
            tok = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            stored[int(line.split()[0].split("_")[1])] = int(tok["outer"])
    for side in (64, 128, 256):
        p = W.poisson3d(side)
        sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, gram_form=form)
        x, info = sv.solve(_dev(p.b))
        sv.close()
        assert info["status"] == "SSTEP_OK" and info["rel_res_true"] <= 1e-8
        assert stored[side] / 2 <= info["outer_iters"] <= 1.5 * stored[side], \
            (side, info["outer_iters"], stored[side])


_REF_256 = {}


def _oracle_256():
    """The oracle's first five iterates at 256^3 (computed once per test session)."""
    if not _REF_256:
        p = W.poisson3d(256)
        op = O.Operator(*p.csr())
        lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
        ref = O.solve(op, p.b, s=8, nu=25, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=5, history=5)
        _REF_256.update(p=p, lam=lam, ref=ref)
    return _REF_256["p"], _REF_256["lam"], _REF_256["ref"]


@pytest.mark.slow
@pytest.mark.parametrize("form", ["moments", "direct", "fused"])
def test_full_size_poisson3d_256_first_five_iterates(form):
    """256^3 (16.8M unknowns), s = 8, nu = 25, stencil operator as the benchmark runs it, with
    both ways of forming G (moments: the benchmark's headline form): every entry of x_k and
    r_k for k = 1, 3, 5 against the oracle."""
    p, lam, ref = _oracle_256()
    sv = _solver(p, "stencil", s=8, nu=25, gram_form=form)
    lo, hi = sv.bounds
    assert lo == pytest.approx(lam[0], rel=1e-9) and hi == lam[1]
    sv.close()
    b = _dev(p.b)
    for k in (1, 3, 5):
        sv2 = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=k, gram_form=form)
        x, info = sv2.solve(b)
        assert info["outer_iters"] == k
        h = ref.history[k - 1]
        assert _rel(x.cpu().numpy(), h.x) <= 1e-10, (form, k, _rel(x.cpu().numpy(), h.x))
        assert _rel(sv2.residual().cpu().numpy(), h.r) <= 1e-10, (form, k)
        sv2.close()


@pytest.mark.slow
def test_full_size_poisson3d_256_mixed_tma_first_iterates():
    """The mixed form at 256^3 as the benchmark runs it (fused moments, refresh every 8): its
    FP32 steps go through TMA tiles (the three FP32 vectors exceed L2), and x_1, x_3 agree with
    the FP64 oracle's to FP32 level."""
    p, lam, ref = _oracle_256()
    b = _dev(p.b)
    for k, tol in ((1, 1e-5), (3, 1e-4)):
        sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=k, check_every=1,
                     precision="mixed", gram_form="fused", refresh_period=8)
        x, info = sv.solve(b)
        assert info["outer_iters"] == k and info["step_tma"] == 1
        assert _rel(x.cpu().numpy(), ref.history[k - 1].x) <= tol, (k, _rel(x.cpu().numpy(), ref.history[k - 1].x))
        sv.close()


def test_fused_form_reaches_tolerance_like_oracle_and_graph_equals_host_loop():
    """Full solves with the fused moments (FP64) on a 2D and a 3D Poisson problem: true
    residual <= 1e-8, outer count within one of the oracle's, the solution within 1e-7; the
    CUDA-graph loop gives the host loop's result bit for bit."""
    for p, s, nu in ((W.poisson2d_64(), 4, 20), (W.poisson3d(40), 8, 25)):
        op = O.Operator(*p.csr())
        lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
        ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
        b = _dev(p.b)
        sv = _solver(p, "stencil", bounds=lam, s=s, nu=nu, tol=1e-8, gram_form="fused")
        x, info = sv.solve(b)
        assert info["status"] == "SSTEP_OK" and info["rel_res_true"] <= 1e-8, info
        assert abs(info["outer_iters"] - ref.outer_iters) <= 1, (info["outer_iters"], ref.outer_iters)
        assert _rel(x.cpu().numpy(), ref.x) <= 1e-7
        sg = _solver(p, "stencil", bounds=lam, s=s, nu=nu, tol=1e-8, gram_form="fused", use_graph=1)
        xg, ig = sg.solve(b)
        assert torch.equal(x, xg) and ig["outer_iters"] == info["outer_iters"]


def test_fused_form_rejects_operators_without_constant_m():
    from paper_2512_09642_gb300 import abi
    p = W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14)
    for mode in ("stencil", "csr"):
        with pytest.raises(abi.SStepError) as ex:
            _solver(p, mode, bounds=(0.04, 2.0), s=4, gram_form="fused")
        assert ex.value.status == 7   # SSTEP_ERR_UNSUPPORTED
    # diffusion without a preconditioner has M = I: allowed, and per-iterate equal to the oracle
    op = O.Operator(*p.csr(), precond="none")
    lam = (0.1, 8.5 * 9)
    ref = O.solve(op, p.b, s=4, nu=20, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=3, history=3)
    sv = _solver(p, "stencil", bounds=lam, s=4, nu=20, tol=1e-30, max_outer=3, precond="none",
                 gram_form="fused", check_every=1)
    x, info = sv.solve(_dev(p.b))
    assert info["outer_iters"] == 3
    assert _rel(x.cpu().numpy(), ref.history[2].x) <= 1e-10


@pytest.mark.parametrize("form,precision", [("moments", "fp64"), ("fused", "fp64"), ("direct", "fp64"),
                                            ("fused", "mixed")])
def test_per_outer_history_records(form, precision):
    """opts.history keeps, per outer iteration, ||r_(k-1)||^2 / ||r_0||^2 of the residual the
    iteration starts from, the Gram solve's inexactness delta_k and the smallest G_ii: the
    residual norms match the oracle's iterates (FP64: 1e-9 relative; mixed: the FP32 level),
    delta_k matches the oracle's ||c~ - G~ a|| / ||c~|| of its own FGS solve, and a ring smaller
    than the solve keeps its newest records."""
    from paper_2512_09642_gb300 import abi
    p = W.poisson3d(24)
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    ref = O.solve(op, p.b, s=8, nu=25, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=6, history=6)
    r0 = np.linalg.norm(p.b)
    sv = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=6, check_every=1, gram_form=form,
                 precision=precision, history=64)
    x, info = sv.solve(_dev(p.b))
    recs = abi.sstep_cg_history(sv.h, 64)
    assert [r["outer"] for r in recs] == list(range(1, 7))
    tol = 1e-9 if precision == "fp64" else 1e-4   # mixed: its iterates differ from FP64's at the FP32 level
    for k, rec in enumerate(recs):
        r_prev = p.b if k == 0 else ref.history[k - 1].r
        want = (np.linalg.norm(r_prev) / r0) ** 2
        assert abs(rec["rel_res_sq"] - want) <= tol * want, (k, rec, want)
        assert 0.0 <= rec["delta"] < 1.0 and rec["min_gii"] > 0.0
    # the oracle's inexactness of its own Gram solve at the first outer iteration
    Pp = O.chebyshev_basis(op, p.b, 8, lam[0], lam[1])
    G, c, _ = O.gram(op, Pp, p.b)
    d, Gt, ct = O.column_scaling(G, c)
    a = O.fgs(Gt, ct, 25)
    delta0 = np.linalg.norm(ct - Gt @ a) / np.linalg.norm(ct)
    assert abs(recs[0]["delta"] - delta0) <= (1e-6 if precision == "fp64" else 5e-2) * delta0
    sv.close()
    small = _solver(p, "stencil", bounds=lam, s=8, nu=25, tol=1e-30, max_outer=6, check_every=1, gram_form=form,
                    precision=precision, history=4)
    small.solve(_dev(p.b))
    assert [r["outer"] for r in abi.sstep_cg_history(small.h, 10)] == [3, 4, 5, 6]
    assert [r["outer"] for r in abi.sstep_cg_history(small.h, 2)] == [5, 6]
    plain = _solver(p, "stencil", bounds=lam, s=8)
    with pytest.raises(abi.SStepError):
        abi.sstep_cg_history(plain.h, 4)


# Degenerate 3D grids with nx even (a line or a single plane): the register-blocked persistent
# steps and residuals (7-point and 27-point) with ny = 1 or nz = 1, against the oracle's basis
# and residual; the mixed form through TMA tiles (nx a multiple of 4) bitwise equal to plain
# loads.
DEGENERATE = [(6, 1, 3), (4, 5, 1), (8, 1, 1)]


@pytest.mark.parametrize("dims", DEGENERATE, ids=["x".join(map(str, d)) for d in DEGENERATE])
@pytest.mark.parametrize("stencil", ["star", "box"])
def test_degenerate_even_grids_basis_and_residual(dims, stencil):
    from paper_2512_09642_gb300 import SStepCG
    p = W.make("deg", dims, config=47, stencil=stencil)
    op = O.Operator(*p.csr())
    lam = (0.03, 2.05)
    s = 4
    sv = SStepCG(grid=p.dims, stencil=stencil, bounds=lam, s=s)
    P = sv.basis(_dev(p.b), s + 1).cpu().numpy()
    ref = O.chebyshev_basis(op, p.b, s, lam[0], lam[1], ncols=s + 1)
    for j in range(s + 1):
        assert _rel(P[j], ref[:, j]) <= 1e-12, j
    x = np.random.default_rng(3).uniform(-1, 1, p.n)
    assert _rel(sv.apply(_dev(x)).cpu().numpy(), op.matvec(x)) <= 1e-14
    sv2 = SStepCG(grid=p.dims, stencil=stencil, bounds=lam, s=2, tol=1e-30, max_outer=1)
    xg, info = sv2.solve(_dev(p.b))
    r_true = p.b - op.matvec(xg.cpu().numpy())
    assert info["rel_res_true"] == pytest.approx(np.linalg.norm(r_true) / np.linalg.norm(p.b), rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("dims", [(4, 5, 1), (8, 1, 1)], ids=["4x5x1", "8x1x1"])
def test_degenerate_grids_tma_step_equals_plain(dims):
    from paper_2512_09642_gb300 import SStepCG
    p = W.make("deg", dims, config=48)
    xs = {}
    for path in ("tma", "plain"):
        sv = SStepCG(grid=p.dims, bounds=(0.03, 2.05), s=4, nu=10, tol=1e-30, max_outer=2, check_every=1,
                     precision="mixed", gram_form="moments", step_kernel=path)
        x, info = sv.solve(_dev(p.b))
        assert info["step_tma"] == (path == "tma")
        xs[path] = x.cpu().numpy()
        sv.close()
    assert np.array_equal(xs["tma"], xs["plain"])
