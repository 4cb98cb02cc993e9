"""GPU parity of the AMG coarse-grid FGS (Section 6) against the oracle: nu sweeps on
A_c y = g with A_c = P^T A_f P for box aggregation, in the formed and the streaming mode,
on Poisson, diffusion and 27-point operators with ragged aggregates. FP64; the sweeps are
the same sequence of row updates on both sides, so the tolerance is that of rounding order
(1e-12 relative)."""
import numpy as np
import pytest

import oracle as O
from oracle import coarse as OC
from workloads import problems as W
from workloads import rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _solver(p):
    from paper_2512_09642_gb300 import SStepCG
    kappa = None if p.kappa is None else _dev(p.kappa)
    return SStepCG(grid=p.dims, kappa=kappa, stencil=p.stencil, bounds=(0.05, 2.0), s=2)


CASES = [
    ("poisson3d", lambda: W.make("c3", (16, 12, 10), config=61), (4, 4, 3)),
    ("diffusion2d", lambda: W.make("c2", (45, 33), kappa_sigma=1.0, config=62), (3, 4)),
    ("diffusion3d", lambda: W.make("c3d", (13, 11, 9), kappa_sigma=0.5, config=63), (2, 3, 2)),
    ("box27", lambda: W.make("cq", (13, 11, 9), config=64, stencil="box"), (2, 2, 2)),
    ("unit_aggregates", lambda: W.make("cu", (9, 7), kappa_sigma=0.7, config=65), (1, 1)),
]


@pytest.mark.parametrize("name,make,block", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", ["formed", "streaming"])
def test_coarse_fgs_matches_oracle(name, make, block, mode):
    from paper_2512_09642_gb300 import abi
    p = make()
    op = O.Operator(*p.csr())
    agg, nc, _ = OC.box_aggregates(p.dims, block)
    Ac = OC.coarse_operator(op, agg, nc)
    sv = _solver(p)
    g = rng.normal(66, nc)
    y0 = rng.uniform(67, nc)
    for nu in (1, 3, 20):
        y = _dev(y0)
        abi.sstep_coarse_fgs(sv.h, block, _dev(g), y, nu, mode)
        ref = OC.coarse_fgs(Ac, g, nu, y0)
        got = y.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), (nu, np.linalg.norm(got - ref))
    sv.close()


def test_coarse_fgs_converges_to_the_coarse_solution():
    """Proposition "AMG Convergence": with kappa(A_c) bounded, 30 sweeps on the 3D Poisson
    coarse level reduce the error by orders of magnitude (towards A_c^-1 g)."""
    from paper_2512_09642_gb300 import abi
    p = W.make("c3", (32, 32, 32), config=68)
    op = O.Operator(*p.csr())
    agg, nc, _ = OC.box_aggregates(p.dims, (4, 4, 4))
    Ac = OC.coarse_operator(op, agg, nc)
    g = rng.normal(69, nc)
    ys = np.linalg.solve(Ac, g)
    sv = _solver(p)
    for mode in ("formed", "streaming"):
        y = torch.zeros(nc, dtype=torch.float64, device="cuda")
        abi.sstep_coarse_fgs(sv.h, (4, 4, 4), _dev(g), y, 30, mode)
        assert np.linalg.norm(y.cpu().numpy() - ys) <= 0.01 * np.linalg.norm(ys), mode
    sv.close()


def test_coarse_fgs_rejects_bad_arguments():
    from paper_2512_09642_gb300 import SStepCG, abi
    p = W.make("c2", (16, 16), config=61)
    sv = _solver(p)
    g = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros(16, dtype=torch.float64, device="cuda")
    for block, nu, mode in (((0, 4), 1, "formed"), ((4, 4, 2), 1, "formed"), ((4, 4), 0, "streaming")):
        with pytest.raises(abi.SStepError):
            abi.sstep_coarse_fgs(sv.h, block, g, y, nu, mode)
    sv.close()
    rp, ci, v = (_dev(a) for a in p.csr())
    csr = SStepCG(csr=(rp, ci, v), bounds=(0.05, 2.0), s=2)
    with pytest.raises(abi.SStepError, match="UNSUPPORTED"):
        abi.sstep_coarse_fgs(csr.h, (4, 4), g, y, 1, "formed")
    csr.close()
