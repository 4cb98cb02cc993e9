"""sstep_gram_fgs_noalloc, the allocation-free Gram + FGS entry point (for callers that must
not allocate device memory, e.g. because a caching allocator owns it or because cudaMalloc
would synchronise a latency-bound loop), against the handle-based entry point that runs the
same kernel with handle-owned scratch (sstep_cg_load_basis + sstep_cg_gram_solve).

Two calls in a row with different systems check that the shared static scratch is
re-initialised between calls. The file is named to be collected last."""
import numpy as np
import pytest

import oracle as O
from workloads import problems as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12   # same kernel on the same basis: agreement to rounding of the block order


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _case(kind):
    if kind == "diffusion3d_s8":
        p = W.make("na1", (21, 17, 9), kappa_sigma=1.0, config=14)
        return p, "csr", 8, 25, (0.04, 2.0)
    if kind == "poisson3d_s16":   # s = 16: the largest basis the static scratch holds
        p = W.make("na3", (24, 20, 12), config=19)
        return p, "stencil", 16, 30, (0.04, 2.0)
    p = W.make("na2", (45, 33), config=11)
    return p, "stencil", 4, 20, (0.05, 2.0)


def _reference_and_inputs(kind, solver="fgs"):
    from paper_2512_09642_gb300 import SStepCG
    p, mode, s, nu, lam = _case(kind)
    op = O.Operator(*p.csr())
    Pp = O.chebyshev_basis(op, p.b, s, lam[0], lam[1], ncols=s + 1)   # the basis both calls see
    P = _dev(Pp.T)                                                    # (s+1, n): column j at j*n
    if mode == "csr":
        rp, ci, v = p.csr()
        sv = SStepCG(csr=(_dev(rp), _dev(ci), _dev(v)), bounds=lam, s=s, nu=nu, gram_solver=solver)
        mdiag, mconst = _dev(op.A.diagonal()), 0.0    # diag(A), as the handle extracts it
    else:
        sv = SStepCG(grid=p.dims, bounds=lam, s=s, nu=nu, gram_solver=solver)
        mdiag, mconst = None, 2.0 * len(p.dims)
    alpha, d, ct, Gt = sv.gram_solve(P)
    sv.close()
    return dict(n=p.n, s=s, nu=nu, lam=lam, P=P, mdiag=mdiag, mconst=mconst, ref=(alpha, d, ct, Gt),
                solver=solver)


def _noalloc(c):
    from paper_2512_09642_gb300 import abi
    s = c["s"]
    out = torch.full((3 * s + s * s + 1,), float("nan"), dtype=torch.float64, device="cuda")
    abi.sstep_gram_fgs_noalloc(c["n"], s, c["nu"], c.get("solver", "fgs"), c["P"], c["n"], c["mdiag"], c["mconst"],
                               c["lam"][0], c["lam"][1], out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return o[:s], o[s:2 * s], o[2 * s:3 * s], o[3 * s:3 * s + s * s].reshape(s, s), o[-1]


def test_noalloc_matches_handle_entry_point_on_two_calls_in_a_row():
    cases = [_reference_and_inputs("diffusion3d_s8"), _reference_and_inputs("poisson2d_s4")]
    for c in cases:   # two calls in a row on the shared static scratch
        alpha, d, ct, Gt, status = _noalloc(c)
        ra, rd, rct, rGt = c["ref"]
        assert status == 0.0
        assert _rel(alpha, ra) <= TOL
        assert _rel(d, rd) <= TOL
        assert _rel(ct, rct) <= TOL
        assert _rel(Gt, rGt) <= TOL


def test_noalloc_at_its_largest_basis_and_with_cholesky():
    """s = 16 (the scratch's limit) with FGS, then Cholesky Gram solves on two systems, all in a
    row on the shared scratch, against the handle entry point with the same solver."""
    cases = [_reference_and_inputs("poisson3d_s16"), _reference_and_inputs("diffusion3d_s8", "cholesky"),
             _reference_and_inputs("poisson3d_s16", "cholesky")]
    for c in cases:
        alpha, d, ct, Gt, status = _noalloc(c)
        ra, rd, rct, rGt = c["ref"]
        assert status == 0.0
        assert _rel(alpha, ra) <= TOL, (c["s"], c["solver"])
        assert _rel(d, rd) <= TOL
        assert _rel(ct, rct) <= TOL
        assert _rel(Gt, rGt) <= TOL


def test_noalloc_breakdown_reports_nan_not_an_earlier_calls_values():
    """A good call, then a call on an all-zero basis (every column dropped: numerical
    breakdown): the second call's state is 3 and its outputs are NaN, not the first call's."""
    c = _reference_and_inputs("poisson2d_s4")
    alpha, _, _, _, status = _noalloc(c)
    assert status == 0.0 and np.all(np.isfinite(alpha))
    z = dict(c, P=torch.zeros_like(c["P"]))
    alpha, d, ct, Gt, status = _noalloc(z)
    assert status == 3.0
    assert np.all(np.isnan(alpha)) and np.all(np.isnan(d)) and np.all(np.isnan(ct)) and np.all(np.isnan(Gt))


def test_noalloc_rejects_s_beyond_its_static_scratch():
    from paper_2512_09642_gb300 import abi
    P = torch.zeros((18, 64), dtype=torch.float64, device="cuda")
    out = torch.zeros(3 * 17 + 17 * 17 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.SStepError) as ei:
        abi.sstep_gram_fgs_noalloc(64, 17, 10, "fgs", P, 64, None, 4.0, 0.1, 2.0, out)
    assert ei.value.status == 1
    assert "s = 17" in abi.sstep_cg_last_error(None)
