"""Failure detection on the host-visible paths: every failure is made on the host (a bad input
array, an option that forbids the recovery), never by faulting the GPU, and must come back as
the documented status code.

  * NaN in b: the first Gram system (FP64 form) or the first FP64 refresh (mixed form) is not
    finite -> SSTEP_ERR_NUMERICAL, with x left finite.
  * a non-positive or non-finite kappa in a diffusion stencil, and a CSR matrix whose diagonal
    has a zero or negative entry -> SSTEP_ERR_INVALID_ARG at create time.
  * a recursive residual that converges while the true residual b - A x does not, with no
    restart allowed (max_refresh = 0) -> SSTEP_ERR_NO_CONVERGENCE; with restarts allowed the
    same solve replaces the residual and reaches the tolerance.
  * a bounded device-side wait that runs out (the TMA step's self-test: its stages expect more
    bytes than their copies deliver, so no wait completes) -> the TIMED_OUT state (4) instead
    of a hang, with the context usable afterwards.
"""
import numpy as np
import pytest

from workloads import problems as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _solver(p, mode, **opts):
    from paper_2512_09642_gb300 import SStepCG
    if mode == "csr":
        rp, ci, v = p.csr()
        return SStepCG(csr=(_dev(rp), _dev(ci), _dev(v)), **opts)
    return SStepCG(grid=p.dims, kappa=None if p.kappa is None else _dev(p.kappa), **opts)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("form", ["direct", "moments", "fused"])
@pytest.mark.parametrize("mode", ["stencil", "csr"])
def test_nan_in_b_gives_numerical(precision, form, mode):
    if form == "fused" and mode == "csr":
        pytest.skip("fused moments need a stencil operator")
    p = W.make("p3", (19, 13, 11), config=12)
    b = p.b.copy()
    b[100] = np.nan
    from paper_2512_09642_gb300 import abi
    sv = _solver(p, mode, bounds=(0.05, 2.0), s=4, nu=10, precision=precision, gram_form=form)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    info = abi.sstep_cg_solve(sv.h, _dev(b), x, allow=(4,)).as_dict()
    assert info["status"] == "SSTEP_ERR_NUMERICAL", info
    assert info["outer_iters"] == 0
    assert bool(torch.isfinite(x).all())
    assert "SSTEP_ERR_NUMERICAL" in abi.sstep_cg_last_error(sv.h)


@pytest.mark.parametrize("bad", [0.0, -1.0, np.inf, np.nan])
def test_bad_kappa_rejected_at_create(bad):
    from paper_2512_09642_gb300 import abi
    p = W.make("d3", (12, 10, 8), kappa_sigma=1.0, config=14)
    kappa = p.kappa.copy()
    kappa[37] = bad
    with pytest.raises(abi.SStepError) as ei:
        _solver(W.Problem(p.name, p.dims, kappa, p.x_star, p.b, 4, 10), "stencil", s=4)
    assert ei.value.status == 1   # SSTEP_ERR_INVALID_ARG
    assert "kappa" in str(ei.value)


@pytest.mark.parametrize("bad", [0.0, -4.0, np.nan])
def test_csr_with_bad_diagonal_rejected_at_create(bad):
    from paper_2512_09642_gb300 import abi
    p = W.make("p2", (9, 7), config=11)
    rp, ci, v = p.csr()
    v = v.copy()
    row = 20
    k = [t for t in range(rp[row], rp[row + 1]) if ci[t] == row][0]
    v[k] = bad
    with pytest.raises(abi.SStepError) as ei:
        from paper_2512_09642_gb300 import SStepCG
        SStepCG(csr=(_dev(rp), _dev(ci), _dev(v)), s=4)
    assert ei.value.status == 1
    assert "diagonal" in str(ei.value)


def test_true_residual_check_without_restarts_gives_no_convergence():
    """Mixed form with the FP64 refresh only every 1000 outer iterations: the FP32 recursive
    residual drifts from b - A x by about the FP32 rounding of the first residual, so it
    reaches 1e-10 long before the true residual does. max_refresh = 0 forbids replacing it:
    NO_CONVERGENCE with the true residual above the tolerance. max_refresh = 3 replaces it and
    converges."""
    p = W.poisson3d(24)
    kw = dict(s=8, nu=25, tol=1e-10, precision="mixed", gram_form="fused", refresh_period=1000)
    sv = _solver(p, "stencil", max_refresh=0, **kw)
    x, info = sv.solve(_dev(p.b))
    assert info["status"] == "SSTEP_ERR_NO_CONVERGENCE", info
    assert info["refreshes"] == 0
    assert info["rel_res_recursive"] < 1e-10 < info["rel_res_true"]
    sv2 = _solver(p, "stencil", max_refresh=3, **kw)
    x2, info2 = sv2.solve(_dev(p.b))
    assert info2["status"] == "SSTEP_OK", info2
    assert info2["refreshes"] >= 1 and info2["rel_res_true"] < 1e-10


def test_max_outer_gives_no_convergence_with_last_iterate():
    p = W.poisson3d(24)
    sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, max_outer=3, check_every=1, gram_form="fused")
    x, info = sv.solve(_dev(p.b))
    assert info["status"] == "SSTEP_ERR_NO_CONVERGENCE" and info["outer_iters"] == 3
    assert 1e-8 < info["rel_res_true"] < 1.0


def test_tma_step_bounded_waits_time_out_and_leave_the_context_usable():
    from paper_2512_09642_gb300 import abi
    assert abi.sstep_selftest_tma_timeout() == 4
    assert torch.cuda.synchronize() is None   # no sticky error
    p = W.make("p3t", (64, 13, 11), config=41)
    sv = _solver(p, "stencil", s=8, nu=25, tol=1e-8, precision="mixed", gram_form="fused", step_kernel="tma")
    _, info = sv.solve(_dev(p.b))
    assert info["status"] == "SSTEP_OK" and info["step_tma"] == 1 and info["rel_res_true"] <= 1e-8
    sv.close()
