"""GPU parity of the block-conjugated s-step CG (`block_conjugate = 1`, the Chronopoulos-Gear
method cited in Section 1) against the oracle's `solve_conjugated`, which forms every block
quantity from its definition (explicit products with A, W = Q^T A Q), while the GPU uses the
Chebyshev change of basis for A P and W_k = G - C^T B - B^T C + B^T W_(k-1) B.

Tolerances as in test_gpu_parity.py: iterates 1e-10 for k = 1..5, final true relative
residual <= 1e-8.
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _solver(p, mode, **opts):
    from paper_2512_09642_gb300 import SStepCG
    if mode == "csr":
        return SStepCG(csr=tuple(_dev(a) for a in p.csr()), **opts)
    kappa = None if p.kappa is None else _dev(p.kappa)
    return SStepCG(grid=p.dims, kappa=kappa, stencil=p.stencil, **opts)


CASES = [
    ("poisson3d_ragged", lambda: W.make("p3", (19, 13, 11), config=12), "stencil", 8, 25),
    ("diffusion2d", lambda: W.make("d2", (45, 33), kappa_sigma=1.0, config=13), "stencil", 6, 25),
    ("diffusion3d_csr", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "csr", 4, 20),
    ("box27", lambda: W.make("q3", (37, 19, 21), config=31, stencil="box"), "stencil", 8, 25),
    ("config1_csr_s16", W.poisson2d_64, "csr", 16, 30),
]


def _bounds(op, p):
    return OS.bounds(op, "lanczos10" if p.stencil == "box" else "gersh_lanczos10", W.lanczos_start(p.n))


@pytest.mark.parametrize("name,make,mode,s,nu", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("form", ["direct", "moments"])
def test_conj_per_iterate_parity_first_five_outer_iterations(name, make, mode, s, nu, form):
    p = make()
    op = O.Operator(*p.csr())
    lam = _bounds(op, p)
    ref = O.solve_conjugated(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=5,
                             history=5)
    for k in range(1, 6):
        sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-30, max_outer=k, check_every=1, gram_form=form,
                     block_conjugate=1)
        x, info = sv.solve(_dev(p.b))
        assert info["outer_iters"] == k
        h = ref.history[k - 1]
        assert _rel(x.cpu().numpy(), h.x) <= 1e-10, (k, _rel(x.cpu().numpy(), h.x))
        assert _rel(sv.residual().cpu().numpy(), h.r) <= 1e-10, k
        sv.close()


def test_conj_cholesky_per_iterate_parity():
    p = W.make("d2", (45, 33), kappa_sigma=1.0, config=13)
    op = O.Operator(*p.csr())
    lam = _bounds(op, p)
    ref = O.solve_conjugated(op, p.b, s=6, nu=1, lam_min=lam[0], lam_max=lam[1], tol=1e-30, max_outer=4,
                             history=4, gram_solver="cholesky")
    for k in (1, 2, 4):
        sv = _solver(p, "stencil", bounds=lam, s=6, tol=1e-30, max_outer=k, gram_solver="cholesky",
                     block_conjugate=1)
        x, info = sv.solve(_dev(p.b))
        assert _rel(x.cpu().numpy(), ref.history[k - 1].x) <= 1e-10, k
        sv.close()


@pytest.mark.parametrize("name,make,mode,s,nu", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_conj_full_solve_matches_oracle(name, make, mode, s, nu):
    p = make()
    op = O.Operator(*p.csr())
    lam = _bounds(op, p)
    ref = O.solve_conjugated(op, p.b, s=s, nu=nu, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    sv = _solver(p, mode, bounds=lam, s=s, nu=nu, tol=1e-8, gram_form="moments", block_conjugate=1)
    x, info = sv.solve(_dev(p.b))
    x = x.cpu().numpy()
    assert info["status"] == "SSTEP_OK" and info["rel_res_true"] <= 1e-8
    assert np.linalg.norm(p.b - op.matvec(x)) / np.linalg.norm(p.b) <= 1e-8
    assert abs(info["outer_iters"] - ref.outer_iters) <= 2, (info["outer_iters"], ref.outer_iters)
    assert _rel(x, ref.x) <= 1e-7


def test_conj_graph_equals_host_loop():
    p = W.poisson3d(40)
    out = []
    for g in (0, 1):
        sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, gram_form="moments", block_conjugate=1, use_graph=g)
        x, info = sv.solve(_dev(p.b))
        out.append((x, info["outer_iters"]))
        sv.close()
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])


def test_conj_solve_twice_restarts_the_recurrence():
    """A second solve on the same handle starts a fresh block recurrence (same result)."""
    p = W.make("d2", (45, 33), kappa_sigma=1.0, config=13)
    sv = _solver(p, "stencil", s=6, nu=25, tol=1e-8, block_conjugate=1)
    b = _dev(p.b)
    x1, i1 = sv.solve(b)
    x2, i2 = sv.solve(b)
    assert torch.equal(x1, x2) and i1["outer_iters"] == i2["outer_iters"]


def test_conj_128_cube_converges_in_fewer_outer_iterations():
    p = W.poisson3d(128)
    b = _dev(p.b)
    res = {}
    for conj in (0, 1):
        sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, gram_form="moments", block_conjugate=conj)
        x, info = sv.solve(b)
        assert info["status"] == "SSTEP_OK" and info["rel_res_true"] <= 1e-8
        res[conj] = info["outer_iters"]
        sv.close()
    assert 2 * res[1] < res[0], res


def test_conj_rejects_unsupported_combinations():
    from paper_2512_09642_gb300 import abi
    p = W.make("p2", (16, 16), config=11)
    for bad in (dict(precision="mixed"), dict(s=17)):
        with pytest.raises(abi.SStepError, match="UNSUPPORTED"):
            _solver(p, "stencil", block_conjugate=1, **bad)
