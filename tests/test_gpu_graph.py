"""Graph mode: the outer loop as one CUDA graph with a device-side while node gives the same
iterates as the host-driven loop (same kernels, same order: bitwise equal), for both forms,
re-captures when the vectors change, and honours max_outer."""
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


CASES = [("poisson2d_64_csr", W.poisson2d_64, "csr", 4, 20),
         ("diffusion3d_stencil", lambda: W.make("d3", (21, 17, 9), kappa_sigma=1.0, config=14), "stencil", 8, 25)]


@pytest.mark.parametrize("name,make,mode,s,nu", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_mode_equals_host_loop(name, make, mode, s, nu, precision):
    p = make()
    b = _dev(p.b)
    host = _solver(p, mode, s=s, nu=nu, precision=precision)
    graph = _solver(p, mode, s=s, nu=nu, precision=precision, use_graph=1)
    x1, i1 = host.solve(b)
    x2, i2 = graph.solve(b)
    assert i1["status"] == i2["status"] == "SSTEP_OK"
    assert i1["outer_iters"] == i2["outer_iters"]
    assert torch.equal(x1, x2)
    # a second solve with new vectors re-captures the graph
    x3, i3 = graph.solve(b.clone())
    assert torch.equal(x3, x1) and i3["outer_iters"] == i1["outer_iters"]


def test_graph_mode_honours_max_outer():
    p = W.poisson3d(20)
    b = _dev(p.b)
    host = _solver(p, "stencil", s=8, nu=25, tol=1e-30, max_outer=3)
    graph = _solver(p, "stencil", s=8, nu=25, tol=1e-30, max_outer=3, use_graph=1)
    x1, i1 = host.solve(b)
    x2, i2 = graph.solve(b)
    assert i1["outer_iters"] == i2["outer_iters"] == 3
    assert i2["status"] == "SSTEP_ERR_NO_CONVERGENCE"
    assert torch.equal(x1, x2)
