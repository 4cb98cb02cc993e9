"""Batched form: each system of a batch (uneven sizes, 2D/3D, Poisson and diffusion, solved
together with one launch per phase) equals its own single-system oracle solve under the same
s, nu and bounds; host-driven and graph-driven batch loops agree bitwise."""
import numpy as np
import pytest

import oracle as O
from oracle import spectral as OS
from workloads import problems as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch_problems():
    return [W.make("b0", (33, 29), kappa_sigma=0.5, config=21),
            W.make("b1", (16, 16), config=22),
            W.make("b2", (9, 7, 5), kappa_sigma=1.0, config=23),
            W.make("b3", (64, 48), kappa_sigma=0.5, config=24),
            W.make("b4", (1, 1), config=25),
            W.make("b5", (12, 10, 8), config=26),
            W.make("b6", (40, 3), kappa_sigma=0.3, config=27)]


def _make_batch(probs, **opts):
    from paper_2512_09642_gb300 import abi
    kap = [None if p.kappa is None else torch.as_tensor(p.kappa).cuda() for p in probs]
    o = abi.sstep_cg_default_opts(**opts)
    h = abi.sstep_cg_batch_create([p.dims for p in probs], kap, o)
    offs, total, lam = abi.sstep_cg_batch_layout(h, len(probs))
    b = torch.zeros(total, dtype=torch.float64, device="cuda")
    for p, o_ in zip(probs, offs):
        b[o_:o_ + p.n] = torch.as_tensor(p.b)
    return h, kap, offs, total, lam, b


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def test_batch_bounds_match_single_system_estimates():
    from paper_2512_09642_gb300 import abi
    probs = _batch_problems()
    h, kap, offs, total, lam, b = _make_batch(probs, s=8, nu=20)
    for p, (lo, hi) in zip(probs, lam):
        op = O.Operator(*p.csr())
        lo0, hi0 = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
        if p.n > 1:
            assert lo == pytest.approx(lo0, rel=1e-9) and hi == pytest.approx(hi0, rel=1e-12)
    abi.sstep_cg_batch_destroy(h)


@pytest.mark.parametrize("gram_form", ["direct", "moments"])
@pytest.mark.parametrize("s,nu", [(4, 20), (8, 20)])
def test_batch_first_iterates_match_oracle_per_system(s, nu, gram_form):
    from paper_2512_09642_gb300 import abi
    probs = _batch_problems()
    h, kap, offs, total, lam, b = _make_batch(probs, s=s, nu=nu, tol=1e-30, max_outer=3, gram_form=gram_form)
    x = torch.zeros(total, dtype=torch.float64, device="cuda")
    infos, summary = abi.sstep_cg_batch_solve(h, b, x, len(probs))
    xs = x.cpu().numpy()
    for p, o_, (lo, hi), inf in zip(probs, offs, lam, infos):
        op = O.Operator(*p.csr())
        ref = O.solve(op, p.b, s=s, nu=nu, lam_min=lo, lam_max=hi, tol=1e-30, max_outer=3, history=3)
        if ref.rel_res_recursive > 0.0:
            # (a 1 x 1 system's residual is exactly 0 after one outer in the oracle and a few
            # ulps on the GPU, which then runs the remaining outers without changing x)
            assert inf["outer_iters"] == ref.outer_iters
        assert _rel(xs[o_:o_ + p.n], ref.x) <= 1e-10, (p.name, _rel(xs[o_:o_ + p.n], ref.x))
    abi.sstep_cg_batch_destroy(h)


@pytest.mark.parametrize("use_graph,gram_form", [(0, "direct"), (1, "direct"), (1, "moments")])
def test_batch_full_solve_matches_oracle_per_system(use_graph, gram_form):
    from paper_2512_09642_gb300 import abi
    probs = _batch_problems()
    h, kap, offs, total, lam, b = _make_batch(probs, s=8, nu=20, tol=1e-8, use_graph=use_graph, gram_form=gram_form)
    x = torch.zeros(total, dtype=torch.float64, device="cuda")
    infos, summary = abi.sstep_cg_batch_solve(h, b, x, len(probs))
    assert summary["status"] == "SSTEP_OK", [i["status"] for i in infos]
    xs = x.cpu().numpy()
    for p, o_, (lo, hi), inf in zip(probs, offs, lam, infos):
        op = O.Operator(*p.csr())
        ref = O.solve(op, p.b, s=8, nu=20, lam_min=lo, lam_max=hi, tol=1e-8)
        xi = xs[o_:o_ + p.n]
        assert np.linalg.norm(p.b - op.matvec(xi)) <= 1e-8 * np.linalg.norm(p.b)
        if p.n > 1:
            assert abs(inf["outer_iters"] - ref.outer_iters) <= 1, (p.name, inf["outer_iters"], ref.outer_iters)
        assert _rel(xi, ref.x) <= 1e-7
    abi.sstep_cg_batch_destroy(h)


@pytest.mark.parametrize("gram_form", ["direct", "moments"])
def test_batch_graph_equals_host_loop(gram_form):
    from paper_2512_09642_gb300 import abi
    probs = _batch_problems()
    out = []
    for g in (0, 1):
        h, kap, offs, total, lam, b = _make_batch(probs, s=8, nu=20, tol=1e-8, use_graph=g, gram_form=gram_form)
        x = torch.zeros(total, dtype=torch.float64, device="cuda")
        infos, _ = abi.sstep_cg_batch_solve(h, b, x, len(probs))
        out.append((x, [i["outer_iters"] for i in infos]))
        abi.sstep_cg_batch_destroy(h)
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])


def test_batch_rejects_unsupported_options():
    from paper_2512_09642_gb300 import abi
    probs = _batch_problems()[:2]
    with pytest.raises(abi.SStepError, match="UNSUPPORTED"):
        _make_batch(probs, s=8, nu=20, precision="mixed")
