"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed operand, a missing mirror) fails at least one of them:
closed-form spectra, the Chebyshev polynomials evaluated through an eigendecomposition,
library routines for special cases (Cholesky, dense solves, tridiagonal eigenvalues), exact
rational arithmetic for the backward-error bound, and the propositions and theorems of
arXiv 2512.09642 (Sections 3-5).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from oracle import spectral as OS
from workloads import problems as W
from workloads import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def _claims():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_claims.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def _dense(op):
    return op.A.toarray()


def _cheb_T(j, t):
    """T_j(t) by its trigonometric / hyperbolic closed form."""
    t = np.asarray(t, np.float64)
    out = np.empty_like(t)
    m = np.abs(t) <= 1.0
    out[m] = np.cos(j * np.arccos(t[m]))
    hi = t > 1.0
    out[hi] = np.cosh(j * np.arccosh(t[hi]))
    lo = t < -1.0
    out[lo] = (-1.0) ** j * np.cosh(j * np.arccosh(-t[lo]))
    return out


# --- inputs -----------------------------------------------------------------------------

def test_splitmix64_reference_vectors():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *vals = [int(v) for v in line.split()]
        got = [int(v) for v in rng.draws(seed, len(vals))]
        assert got == vals


def test_rng_streams_are_counter_based():
    a = rng.draws(77, 100)
    b = rng.draws(77, 40, offset=60)
    assert np.array_equal(a[60:], b)
    u = rng.uniform(5, 200000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    z = rng.normal(6, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    k = rng.integers(7, 50000, 32, 512)
    assert k.min() == 32 and k.max() == 512


@pytest.mark.parametrize("dims", [(7, 5), (4, 3, 5)])
def test_poisson_generator_structure(dims):
    op = O.Operator(*W.csr(dims))
    A = _dense(op)
    assert np.array_equal(A, A.T)
    d = 2 * len(dims)
    assert np.all(np.diag(A) == d)
    rows = A.sum(axis=1)
    nx, ny, nz = W.grid_shape(dims)
    idx = np.arange(A.shape[0])
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    interior = (i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1)
    if len(dims) == 3:
        interior &= (k > 0) & (k < nz - 1)
    assert np.all(rows[interior] == 0) and np.all(rows[~interior] > 0)


@pytest.mark.parametrize("dims", [(6, 1, 3), (1, 5, 4), (1, 13, 1), (8, 1, 1), (4, 5, 1), (1, 7), (5, 1)])
@pytest.mark.parametrize("diffusion", [False, True])
def test_star_generator_on_grids_with_unit_extents(dims, diffusion):
    """Grids with an axis of extent 1, where two axes share a stride (nx x 1 x nz: the y and z
    strides are both nx): each row couples exactly the in-grid face neighbours by grid
    coordinates, and the CSR agrees with the matrix-free form."""
    kappa = W.lognormal_kappa(dims, 0.5, 81) if diffusion else None
    op = O.Operator(*W.csr(dims, kappa))
    A = _dense(op)
    assert np.allclose(A, A.T, rtol=0, atol=1e-14)
    nx, ny, nz = W.grid_shape(dims)
    idx = np.arange(A.shape[0])
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    for r in range(A.shape[0]):
        nb = [c for c in range(A.shape[0]) if abs(i[c] - i[r]) + abs(j[c] - j[r]) + abs(k[c] - k[r]) == 1]
        off = [c for c in np.flatnonzero(A[r]) if c != r]
        assert sorted(off) == sorted(nb), (r, off, nb)
    x = rng.uniform(9, A.shape[0])
    assert np.allclose(A @ x, W.apply(dims, x, kappa), rtol=0, atol=1e-12)


@pytest.mark.parametrize("dims", [(8, 6), (4, 3, 5)])
def test_jacobi_poisson_spectrum_closed_form(dims):
    """Eigenvalues of D^-1 A for the Dirichlet Laplacian: 1 - (1/d) sum_i cos(k_i pi / (N_i + 1))."""
    op = O.Operator(*W.csr(dims))
    got = np.sort(np.linalg.eigvals(np.diag(op.minv) @ _dense(op)).real)
    d = len(dims)
    grids = np.meshgrid(*[np.arange(1, N + 1) for N in dims], indexing="ij")
    lam = 1.0 - sum(np.cos(g * np.pi / (N + 1)) for g, N in zip(grids, dims)) / d
    assert np.allclose(got, np.sort(lam.ravel()), atol=1e-12)


@pytest.mark.parametrize("dims", [(7, 5), (5, 4, 3), (3, 1, 2)])
def test_box_stencil_generator_structure(dims):
    """27-point (3D) / 9-point (2D) box stencil: diagonal 3^d - 1, -1 for every in-grid point
    of the unit box; zero row sums inside, positive at the boundary; matrix-free form agrees."""
    op = O.Operator(*W.box_csr(dims))
    A = _dense(op)
    d = len(dims)
    assert np.array_equal(A, A.T) and np.all(np.diag(A) == 3 ** d - 1)
    nx, ny, nz = W.grid_shape(dims)
    idx = np.arange(A.shape[0])
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    for r in range(A.shape[0]):
        nb = [c for c in range(A.shape[0]) if c != r and max(abs(i[c] - i[r]), abs(j[c] - j[r]), abs(k[c] - k[r])) == 1]
        assert np.all(A[r, nb] == -1) and np.count_nonzero(A[r]) == len(nb) + 1
    rows = A.sum(axis=1)
    interior = (i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1)
    if d == 3:
        interior &= (k > 0) & (k < nz - 1)
    assert np.all(rows[interior] == 0) and np.all(rows[~interior] > 0)
    x = rng.uniform(7, A.shape[0])
    assert np.allclose(A @ x, W.box_apply(dims, x), rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims", [(8, 6), (5, 4, 3)])
def test_jacobi_box_stencil_spectrum_closed_form(dims):
    """A = 3^d I - (T x ... x T) with T = tridiag(1, 1, 1), whose eigenvalues are
    1 + 2 cos(k pi / (N + 1)); so eig(D^-1 A) = (3^d - prod_i (1 + 2 cos(k_i pi / (N_i + 1)))) / (3^d - 1)."""
    op = O.Operator(*W.box_csr(dims))
    got = np.sort(np.linalg.eigvals(np.diag(op.minv) @ _dense(op)).real)
    d = len(dims)
    grids = np.meshgrid(*[np.arange(1, N + 1) for N in dims], indexing="ij")
    prod = np.ones_like(grids[0], dtype=np.float64)
    for g, N in zip(grids, dims):
        prod = prod * (1.0 + 2.0 * np.cos(g * np.pi / (N + 1)))
    lam = (3.0 ** d - prod) / (3.0 ** d - 1)
    assert np.allclose(got, np.sort(lam.ravel()), atol=1e-12)


def test_box_stencil_lanczos_bounds_and_gershgorin():
    """Gershgorin bounds D^-1 A by 2 while the 27-point spectrum ends near 36/26 (one cosine
    factor near -1, two near 3), so the paper's Lanczos-10 bounds with their 10% margins
    enclose the spectrum far more tightly."""
    dims = (12, 11, 10)
    op = O.Operator(*W.box_csr(dims))
    grids = np.meshgrid(*[np.arange(1, N + 1) for N in dims], indexing="ij")
    prod = np.ones_like(grids[0], dtype=np.float64)
    for g, N in zip(grids, dims):
        prod = prod * (1.0 + 2.0 * np.cos(g * np.pi / (N + 1)))
    lam = (27.0 - prod) / 26.0
    a, b = OS.lanczos(op, W.lanczos_start(op.n), 10)
    ev = OS.tridiag_eigvals(a, b)
    assert lam.min() - 1e-12 <= ev[0] and ev[-1] <= lam.max() + 1e-12
    assert OS.gershgorin_upper(op) == 2.0 and lam.max() < 36.0 / 26.0
    lo, hi = OS.bounds(op, "lanczos10", W.lanczos_start(op.n))
    assert lo == pytest.approx(0.9 * ev[0]) and hi == pytest.approx(1.1 * ev[-1])
    assert lo < lam.min() and hi > lam.max()


def test_diffusion_generator_spd_and_matrix_free_agree():
    dims = (6, 5, 4)
    kappa = W.lognormal_kappa(dims, 1.0, 99)
    op = O.Operator(*W.csr(dims, kappa))
    A = _dense(op)
    assert np.allclose(A, A.T, rtol=0, atol=1e-14)
    assert np.linalg.eigvalsh(A).min() > 0
    x = rng.uniform(3, A.shape[0])
    assert np.allclose(A @ x, W.apply(dims, x, kappa), rtol=1e-13, atol=1e-13)
    # kappa = 1: interior faces weigh 1, each boundary face adds 2 to the diagonal
    A1 = _dense(O.Operator(*W.csr((3, 3), np.ones(9))))
    assert A1[4, 4] == 4 and A1[0, 0] == 2 + 2 * 2


# --- Chebyshev basis (Section 2, Definition) --------------------------------------------

@pytest.mark.parametrize("case", ["poisson_inside", "diffusion_inside", "diffusion_narrow"])
def test_chebyshev_basis_is_T_j_of_mapped_operator(case):
    if case == "poisson_inside":
        op = O.Operator(*W.csr((6, 5)))
    else:
        dims = (3, 3, 4)
        op = O.Operator(*W.csr(dims, W.lognormal_kappa(dims, 1.0, 5)))
    A = _dense(op)
    dh = np.sqrt(op.minv)
    B = dh[:, None] * A * dh[None, :]             # D^-1/2 A D^-1/2, same spectrum as D^-1 A
    lam, V = np.linalg.eigh(B)
    if case == "diffusion_narrow":
        lmin, lmax = lam[0] + 0.3 * (lam[-1] - lam[0]), lam[-1] - 0.2 * (lam[-1] - lam[0])
    else:
        lmin, lmax = 0.95 * lam[0], 1.02 * lam[-1]
    theta, sigma = 2.0 / (lmax - lmin), (lmax + lmin) / 2.0
    r = rng.uniform(21, op.n)
    s = 9
    P = O.chebyshev_basis(op, r, s, lmin, lmax)
    y = V.T @ (r / dh)                            # D^1/2 r in the eigenbasis
    for j in range(s):
        ref = dh * (V @ (_cheb_T(j, theta * (lam - sigma)) * y))
        assert np.linalg.norm(P[:, j] - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref)), j


def test_gram_gives_galerkin_orthogonality():
    """With an exact Gram solve the new residual is orthogonal to span(P): P^T r_(k+1) = 0.

    Exercises G = P^T A P, c = P^T r, the column scaling, alpha = S a and r -= (AP) alpha
    together (Section 2); a transposed or mis-scaled piece leaves P^T r_(k+1) far from 0.
    """
    p = W.make("t", (9, 7), kappa_sigma=1.0, config=9)
    op = O.Operator(*p.csr())
    r = p.b.copy()
    P = O.chebyshev_basis(op, r, 5, 0.05, 2.2)
    G, c, AP = O.gram(op, P, r)
    assert np.array_equal(G, G.T)
    d, Gt, ct = O.column_scaling(G, c)
    assert np.allclose(np.diag(Gt), 1.0, atol=1e-15)
    alpha = d * O.cholesky_solve(Gt, ct)
    r1 = r - AP @ alpha
    assert np.linalg.norm(P.T @ r1) <= 1e-12 * np.linalg.norm(P.T @ r)
    assert np.allclose(AP, _dense(op) @ P, rtol=0, atol=1e-12 * np.abs(AP).max())


# --- Gram solves (Sections 2, 3) ---------------------------------------------------------

def _cheb_gram(s=6, side=10, seed=3):
    dims = (side, side)
    op = O.Operator(*W.csr(dims, W.lognormal_kappa(dims, 0.5, seed)))
    r = rng.uniform(seed + 100, op.n)
    P = O.chebyshev_basis(op, r, s, 0.02, 2.1)
    G, c, AP = O.gram(op, P, r)
    return op, P, r, G, c


def test_fgs_one_sweep_is_exact_for_diagonal_gram():
    c = rng.uniform(8, 7)
    a = O.fgs(np.eye(7), c, 1)
    assert np.array_equal(a, c)


def test_fgs_converges_to_cholesky_and_dense_solve():
    _, _, _, G, c = _cheb_gram(s=6)
    d, Gt, ct = O.column_scaling(G, c)
    # spectral radius of the sweep operator is about 0.99 here: 4000 sweeps reach rounding level
    a_fgs = O.fgs(Gt, ct, 4000)
    a_chol = O.cholesky_solve(Gt, ct)
    a_np = np.linalg.solve(Gt, ct)
    assert np.linalg.norm(a_chol - a_np) <= 1e-12 * np.linalg.norm(a_np)
    assert np.linalg.norm(a_fgs - a_np) <= 1e-10 * np.linalg.norm(a_np)


def test_cholesky_factor_matches_library():
    _, _, _, G, c = _cheb_gram(s=7)
    R = O.cholesky(G)
    assert np.allclose(R, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-12 * np.abs(R).max())


def test_fgs_residual_structure():
    """Section 3, Proposition "FGS Residual Structure" (general D, unscaled G):
    r^(l+1) = P^T r - G a^(l+1) = -L^T a^(l+1) + L^T a^(l), and r^(1) = -L^T a^(1)."""
    _, _, _, G, c = _cheb_gram(s=6)
    Lt = np.triu(G, 1)
    its = O.fgs_iterates(G, c, 6)
    scale = np.linalg.norm(c)
    assert np.linalg.norm((c - G @ its[1]) - (-Lt @ its[1])) <= 1e-13 * scale
    for l in range(1, 6):
        lhs = c - G @ its[l + 1]
        rhs = -Lt @ its[l + 1] + Lt @ its[l]
        assert np.linalg.norm(lhs - rhs) <= 1e-13 * scale, l


def test_one_fgs_sweep_equals_A_norm_mgs():
    """Section 5, Theorem "Algebraic Equivalence": one FGS sweep on G~ a = P~^T A r with
    a^(0) = 0 gives the A-norm MGS coefficients gamma_j of r against the columns of P~."""
    op, P, r, G, c = _cheb_gram(s=6)
    d, Gt, _ = O.column_scaling(G, c)
    Pt = P * d[None, :]
    A = _dense(op)
    a1 = O.fgs(Gt, Pt.T @ (A @ r), 1)
    w = r.copy()
    gam = np.zeros(P.shape[1])
    for j in range(P.shape[1]):
        gam[j] = w @ (A @ Pt[:, j])
        w = w - gam[j] * Pt[:, j]
    assert np.linalg.norm(a1 - gam) <= 1e-13 * np.linalg.norm(gam)


def test_fgs_backward_error_bound_in_exact_arithmetic():
    """Section 3, Theorem "Backward Stability": the computed sweep satisfies
    (D+L) a~ = b - L^T a_old + delta with |delta_j| <= (j-1) eps (|b_j| + sum |L_ji||a~_i|)
    componentwise (b_j = c~_j); delta is evaluated exactly in rational arithmetic."""
    _, _, _, G, c = _cheb_gram(s=8)
    d, Gt, ct = O.column_scaling(G, c)
    its = O.fgs_iterates(Gt, ct, 4)
    u = EPS / 2
    cs_eps = 0.0
    for l in range(4):
        old, new = its[l], its[l + 1]
        s = len(ct)
        for j in range(s):
            # right-hand side of the forward substitution for row j in this sweep
            rhs = Fraction(ct[j]) - sum(Fraction(Gt[j, i]) * Fraction(old[i]) for i in range(j + 1, s))
            lhs = sum(Fraction(Gt[j, i]) * Fraction(new[i]) for i in range(j)) + Fraction(Gt[j, j]) * Fraction(new[j])
            delta = abs(float(lhs - rhs))
            mag = abs(ct[j]) + sum(abs(Gt[j, i] * old[i]) for i in range(j + 1, s)) \
                + sum(abs(Gt[j, i] * new[i]) for i in range(j))
            assert delta <= (s + 1) * u * mag + 1e-300, (l, j)
            if mag > 0:
                cs_eps = max(cs_eps, delta / mag)
    assert cs_eps <= _claims()["backward_stability_Cs_eps"]


def test_multi_sweep_error_propagation_and_bound():
    """Section 3, Lemma "Multi-Sweep Analysis": e^(l+1) = T e^(l) with T = -(D+L)^-1 L^T and
    e = a* - a^(l), hence ||e^(nu)|| <= ||T||_2^nu ||a*||, geometric when ||T||_2 < 1."""
    for s, side, seed in [(4, 12, 4), (3, 8, 2)]:
        _, _, _, G, c = _cheb_gram(s=s, side=side, seed=seed)
        d, Gt, ct = O.column_scaling(G, c)
        T = -np.linalg.solve(np.tril(Gt), np.triu(Gt, 1))
        rho = np.linalg.norm(T, 2)
        a_star = np.linalg.solve(Gt, ct)
        its = O.fgs_iterates(Gt, ct, 30)
        for nu in range(30):
            e0, e1 = a_star - its[nu], a_star - its[nu + 1]
            assert np.linalg.norm(e1 - T @ e0) <= 1e-12 * np.linalg.norm(a_star)
            assert np.linalg.norm(e1) <= rho ** (nu + 1) * np.linalg.norm(a_star) * (1 + 1e-10) + 1e-13
        if rho < 1:
            assert np.linalg.norm(a_star - its[30]) <= rho ** 30 * np.linalg.norm(a_star) + 1e-13


def test_L_frobenius_growth_is_sublinear():
    """Section 4, Theorem "Polynomial Growth": ||L||_F = O(sqrt(s)) for the scaled Chebyshev
    Gram; the log-log slope over s = 4..20 is checked to lie in [0.3, 0.8]."""
    p = W.poisson3d(16)
    op = O.Operator(*p.csr())
    lm = 1 - np.cos(np.pi / 17)
    r = rng.uniform(12, p.n)
    ss = [4, 8, 12, 16, 20]
    Ls = []
    for s in ss:
        P = O.chebyshev_basis(op, r, s, lm, 2 - lm)
        G, c, _ = O.gram(op, P, r)
        _, Gt, _ = O.column_scaling(G, c)
        Ls.append(np.linalg.norm(np.tril(Gt, -1)))
    slope = np.polyfit(np.log(ss), np.log(Ls), 1)[0]
    assert 0.3 <= slope <= 0.8, slope


def test_monomial_versus_chebyshev_conditioning():
    """Section 4, "Monomial comparison" (claims in tests/golden/paper_claims.txt)."""
    cl = _claims()
    kap = cl["mono_kappa_MinvA"]
    lam = np.linspace(1.0, kap, 300)
    op = O.Operator.from_dense(np.diag(lam), precond="none")
    r = rng.uniform(11, 300)
    s = int(cl["mono_kappa_exceeds_inv_eps_at_s"])
    Pm = O.monomial_basis(op, r, s)
    Gm, _, _ = O.gram(op, Pm, r)
    assert np.linalg.cond(Gm) > 1.0 / EPS
    Pc = O.chebyshev_basis(op, r, 10, 1.0, kap)
    Gc, cc, _ = O.gram(op, Pc, r)
    k10 = np.linalg.cond(Gc)
    assert cl["cheb_kappa_order_at_s10"] / 10 <= k10 <= cl["cheb_kappa_order_at_s10"] * 10


def test_monomial_basis_is_the_matrix_powers():
    """Section 4's contrast basis p_j = (M^-1 A)^j r against explicit dense matrix powers, with
    a non-constant Jacobi diagonal (so a dropped M^-1 or a misplaced one shows) and with M = I
    (against the eigendecomposition A^j r = V diag(lambda^j) V^T r)."""
    p = W.make("mono", (9, 8), kappa_sigma=0.7, config=21)
    for precond in ("jacobi", "none"):
        op = O.Operator(*p.csr(), precond=precond)
        A = _dense(op)
        d = np.diag(A)
        assert np.ptp(d) > 0.5   # the diagonal is far from constant
        B = A / d[:, None] if precond == "jacobi" else A
        r = rng.uniform(31, op.n)
        s = 7
        P = O.monomial_basis(op, r, s)
        assert P.shape == (op.n, s)
        for j in range(s):
            ref = np.linalg.matrix_power(B, j) @ r
            assert np.linalg.norm(P[:, j] - ref) <= 1e-12 * np.linalg.norm(ref), (precond, j)
        if precond == "none":
            lam, V = np.linalg.eigh(A)
            for j in range(s):
                ref = V @ (lam ** j * (V.T @ r))
                assert np.linalg.norm(P[:, j] - ref) <= 1e-11 * np.linalg.norm(ref), j


# --- whole solves -----------------------------------------------------------------------

def test_s1_is_steepest_descent():
    p = W.make("t", (10, 8), kappa_sigma=0.7, config=9)
    op = O.Operator(*p.csr())
    res = O.solve(op, p.b, s=1, nu=1, lam_min=0.1, lam_max=2.0, tol=1e-30, max_outer=3, history=3)
    A = _dense(op)
    x = np.zeros(op.n)
    for k in range(3):
        r = p.b - A @ x
        x = x + (r @ r) / (r @ (A @ r)) * r
        assert np.linalg.norm(res.history[k].x - x) <= 1e-13 * np.linalg.norm(x)


def test_minv_r_start_s1_is_preconditioned_steepest_descent():
    """The alternative start p_0 = M^-1 r_k at s = 1: x += a z with z = M^-1 r and
    a = z^T r / z^T A z, the Jacobi-preconditioned steepest descent step (textbook)."""
    p = W.make("t", (10, 8), kappa_sigma=0.7, config=9)
    op = O.Operator(*p.csr())
    res = O.solve(op, p.b, s=1, nu=1, lam_min=0.1, lam_max=2.0, tol=1e-30, max_outer=4, history=4,
                  basis_start="minv_r")
    A = _dense(op)
    minv = 1.0 / np.diag(A)
    x = np.zeros(op.n)
    for k in range(4):
        r = p.b - A @ x
        z = minv * r
        x = x + (z @ r) / (z @ (A @ z)) * z
        assert np.linalg.norm(res.history[k].x - x) <= 1e-13 * np.linalg.norm(x)


@pytest.mark.parametrize("dims", [(9, 7), (6, 5, 4)])
def test_minv_r_start_equals_r_start_for_constant_preconditioner(dims):
    """With a constant M = m I (Jacobi on the Poisson stencil, m = 2d) the start M^-1 r_k
    scales the basis by 1/m; the column scaling takes that factor out of G and c, so alpha
    grows by m and x_k, r_k are those of the p_0 = r_k start of Section 2. With a varying
    diagonal (diffusion) the two starts give different iterates."""
    p = W.make("t", dims, config=9)
    op = O.Operator(*p.csr())
    kw = dict(s=4, nu=20, lam_min=0.05, lam_max=2.0, tol=1e-30, max_outer=5, history=5)
    a = O.solve(op, p.b, **kw)
    b = O.solve(op, p.b, basis_start="minv_r", **kw)
    for ha, hb in zip(a.history, b.history):
        assert np.linalg.norm(ha.x - hb.x) <= 1e-12 * np.linalg.norm(ha.x)
        assert np.linalg.norm(ha.r - hb.r) <= 1e-11 * np.linalg.norm(ha.r)
        assert np.allclose(hb.alpha, 2 * len(dims) * ha.alpha, rtol=1e-10, atol=0)
    q = W.make("t", dims, kappa_sigma=1.0, config=9)
    opq = O.Operator(*q.csr())
    a = O.solve(opq, q.b, **kw)
    b = O.solve(opq, q.b, basis_start="minv_r", **kw)
    assert np.linalg.norm(a.history[0].x - b.history[0].x) > 1e-3 * np.linalg.norm(a.history[0].x)


def test_resuming_from_an_iterate_continues_the_iteration():
    """Section 2's outer iteration is restarted: its state is x alone (r = b - A x). Stopping
    after 3 outer iterations and solving again from x_3 gives the uninterrupted run's x_5, up
    to the rounding of the recomputed residual."""
    p = W.make("p3", (20, 13, 11), config=12)
    op = O.Operator(*p.csr())
    kw = dict(s=8, nu=25, lam_min=0.04, lam_max=2.0, tol=1e-30)
    run = O.solve(op, p.b, max_outer=5, history=5, **kw)
    x3 = O.solve(op, p.b, max_outer=3, **kw).x
    assert np.linalg.norm(x3 - run.history[2].x) == 0.0
    resumed = O.solve(op, p.b, x3, max_outer=2, history=2, **kw)
    assert resumed.outer_iters == 2
    assert np.linalg.norm(resumed.history[-1].x - run.history[-1].x) <= 1e-13 * np.linalg.norm(run.history[-1].x)


def test_tiny_system_one_outer_with_cholesky_is_exact():
    n = 5
    M = rng.uniform(31, n * n).reshape(n, n)
    A = M @ M.T + n * np.eye(n)
    b = rng.uniform(32, n)
    op = O.Operator.from_dense(A)
    lam = np.linalg.eigvals(np.diag(op.minv) @ A).real
    res = O.solve(op, b, s=n, nu=1, lam_min=0.9 * lam.min(), lam_max=1.1 * lam.max(), tol=1e-30,
                  max_outer=1, gram_solver="cholesky")
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - x) <= 1e3 * np.linalg.cond(A) * EPS * np.linalg.norm(x)


def test_full_solve_matches_dense_solution_and_stops_at_tol():
    p = W.make("t", (14, 11), kappa_sigma=1.0, config=9, tol=1e-10)
    op = O.Operator(*p.csr())
    lam = np.linalg.eigvals(np.diag(op.minv) @ _dense(op)).real
    res = O.solve(op, p.b, s=5, nu=30, lam_min=0.9 * lam.min(), lam_max=1.05 * lam.max(), tol=p.tol,
                  history=10 ** 6)
    assert res.converged and res.rel_res_true < p.tol
    kA = np.linalg.cond(_dense(op))
    assert np.linalg.norm(res.x - p.x_star) <= 10 * kA * p.tol * np.linalg.norm(p.x_star)
    # first iterate below tol is where it stopped (Section 8 stopping rule)
    rel = [h.r for h in res.history]
    norms = [np.linalg.norm(v) / res.r0_norm for v in rel]
    assert norms[-1] < p.tol and all(v >= p.tol for v in norms[:-1])


def test_more_sweeps_reduce_gram_inexactness():
    """Section 7: delta_k = ||c~ - G~ a|| / ||c~|| shrinks as nu grows."""
    p = W.make("t", (12, 12), config=9)
    op = O.Operator(*p.csr())
    ds = []
    for nu in (2, 6, 30):
        res = O.solve(op, p.b, s=6, nu=nu, lam_min=0.02, lam_max=2.0, max_outer=3, tol=1e-30, history=3)
        ds.append(np.mean([h.delta for h in res.history]))
    assert ds[0] > ds[1] > ds[2]


# --- spectral bounds (Section 8) --------------------------------------------------------

def test_tridiagonal_bisection_matches_library():
    a = rng.uniform(41, 10, 0.5, 2.0)
    b = rng.uniform(42, 9, 0.1, 0.6)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    assert np.allclose(OS.tridiag_eigvals(a, b), np.linalg.eigvalsh(T), atol=1e-13)


def test_lanczos_ritz_values_inside_closed_form_spectrum():
    p = W.poisson2d_64()
    op = O.Operator(*p.csr())
    a, b = OS.lanczos(op, W.lanczos_start(p.n), 10)
    ev = OS.tridiag_eigvals(a, b)
    lmin = 1 - np.cos(np.pi / 65)
    assert lmin <= ev[0] and ev[-1] <= 2 - lmin
    assert OS.gershgorin_upper(op) == 2.0
    lo, hi = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    assert lo == pytest.approx(0.9 * ev[0]) and hi == 2.0
    lo2, hi2 = OS.bounds(op, "lanczos10", W.lanczos_start(p.n))
    assert hi2 == pytest.approx(1.1 * ev[-1])
    # Lanczos on a dense diagonal matrix finds its extreme eigenvalues once k = n
    op_d = O.Operator.from_dense(np.diag(np.arange(1.0, 9.0)), precond="none")
    a, b = OS.lanczos(op_d, rng.uniform(5, 8), 8)
    assert np.allclose(OS.tridiag_eigvals(a, b), np.arange(1.0, 9.0), atol=1e-8)


# --- block-conjugated s-step CG (Section 1's Chronopoulos-Gear method) ------------------

def _textbook_cg(A, b, iters):
    """Unpreconditioned CG by its two-term recurrences (Hestenes-Stiefel), x_0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    out = []
    for _ in range(iters):
        Ap = A @ p
        a = rr / (p @ Ap)
        x = x + a * p
        r = r - a * Ap
        rn = r @ r
        p = r + (rn / rr) * p
        rr = rn
        out.append(x.copy())
    return out


@pytest.mark.parametrize("dims", [(12, 10), (7, 6, 5)])
@pytest.mark.parametrize("s", [1, 2, 4])
def test_conjugated_sstep_equals_cg_every_s_steps(dims, s):
    """With a constant Jacobi diagonal the basis spans K_s(A, r_k); with exact Gram solves the
    A-conjugate blocks make outer iteration k equal to CG after k s steps (CG's optimality over
    the Krylov space), so every term of the block recurrence is pinned."""
    p = W.make("c", dims, config=41)
    op = O.Operator(*p.csr())
    lam_min = 0.9 * np.linalg.eigvals(np.diag(op.minv) @ _dense(op)).real.min()
    res = O.solve_conjugated(op, p.b, s=s, nu=1, lam_min=lam_min, lam_max=2.0, tol=1e-30, max_outer=6,
                             history=6, gram_solver="cholesky")
    ref = _textbook_cg(op.A, p.b, 6 * s)
    for k, h in enumerate(res.history):
        want = ref[(k + 1) * s - 1]
        assert np.linalg.norm(h.x - want) <= 1e-12 * np.linalg.norm(want), (k, s)


def test_conjugated_s1_with_fgs_equals_cg_on_diffusion():
    """s = 1: p_0 = r_k, the 1x1 Gram systems are solved exactly by one scaled sweep, so the
    method is unpreconditioned CG whatever the coefficients (first nine iterations, before
    finite-precision drift separates the two recurrences)."""
    p = W.make("c", (12, 10), kappa_sigma=1.0, config=42)
    op = O.Operator(*p.csr())
    res = O.solve_conjugated(op, p.b, s=1, nu=1, lam_min=0.01, lam_max=2.0, tol=1e-30, max_outer=9, history=9)
    ref = _textbook_cg(op.A, p.b, 9)
    for k, h in enumerate(res.history):
        assert np.linalg.norm(h.x - ref[k]) <= 1e-11 * np.linalg.norm(ref[k]), k


def test_conjugated_fgs_converges_in_fewer_outer_iterations():
    """With inexact (nu-sweep FGS) Gram solves the conjugated method still reaches tol, in far
    fewer outer iterations than the restarted iteration of Section 2."""
    p = W.poisson2d_64()
    op = O.Operator(*p.csr())
    lam = OS.bounds(op, "gersh_lanczos10", W.lanczos_start(p.n))
    lit = O.solve(op, p.b, s=4, nu=20, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    con = O.solve_conjugated(op, p.b, s=4, nu=20, lam_min=lam[0], lam_max=lam[1], tol=1e-8)
    assert con.converged and con.rel_res_true < 1e-8
    assert np.linalg.norm(p.b - op.matvec(con.x)) / np.linalg.norm(p.b) < 1e-8
    assert con.outer_iters * 3 < lit.outer_iters


def test_scaled_solve_with_many_columns_matches_dense_solve():
    rng_ = np.random.default_rng(3)
    X = rng_.standard_normal((6, 6))
    Wm = X @ X.T + 6 * np.eye(6)
    R = rng_.standard_normal((6, 3))
    assert np.allclose(O.scaled_solve(Wm, R, 200), np.linalg.solve(Wm, R), rtol=1e-12, atol=1e-12)
    assert np.allclose(O.scaled_solve(Wm, R, 1, "cholesky"), np.linalg.solve(Wm, R), rtol=1e-12, atol=1e-12)


# --- AMG coarse-grid FGS (Section 6) ------------------------------------------------------

@pytest.mark.parametrize("dims,block", [((8, 6, 4), (2, 2, 2)), ((12, 8), (4, 4)), ((9, 6, 6), (3, 3, 3))])
def test_coarse_operator_of_box_aggregation_is_scaled_coarse_laplacian(dims, block):
    """Piecewise-constant aggregation of the Dirichlet Laplacian into b x ... x b boxes: the
    aggregate sums give A_c = b^(d-1) times the Laplacian of the coarse grid (diagonal 2d
    b^(d-1) from 2d b^d minus the in-box couplings, -b^(d-1) per face crossing)."""
    from oracle import coarse as OC
    op = O.Operator(*W.csr(dims))
    agg, nc, cdims = OC.box_aggregates(dims, block)
    Ac = OC.coarse_operator(op, agg, nc)
    b = block[0]
    Lc = _dense(O.Operator(*W.csr(cdims[:len(dims)])))
    assert np.array_equal(Ac, b ** (len(dims) - 1) * Lc)


def test_coarse_condition_number_independent_of_fine_size():
    """Proposition "AMG Convergence": at a fixed coarse level kappa(A_c) does not grow with n_f
    (here exactly constant: A_c is a scaled coarse Laplacian)."""
    from oracle import coarse as OC
    kap = []
    for N in (8, 16, 32):
        op = O.Operator(*W.csr((N, N, N)))
        agg, nc, _ = OC.box_aggregates((N, N, N), (N // 4,) * 3)
        ev = np.linalg.eigvalsh(OC.coarse_operator(op, agg, nc))
        kap.append(ev[-1] / ev[0])
    assert np.allclose(kap, kap[0], rtol=1e-10)


@pytest.mark.parametrize("dims,block,sigma", [((13, 11), (3, 3), 1.0), ((7, 6, 5), (2, 3, 2), 0.5), ((10, 10), (1, 1), 0.7)])
def test_streaming_coarse_fgs_equals_fgs_on_formed_operator(dims, block, sigma):
    """Section 6's streaming form (A_c never formed, rows of A_c y from the fine level) gives
    the FGS iterates of the formed A_c; ragged aggregates at the grid edge included; with 1 x 1
    aggregates A_c = A_f."""
    from oracle import coarse as OC
    p = W.make("c", dims, kappa_sigma=sigma, config=51)
    op = O.Operator(*p.csr())
    agg, nc, _ = OC.box_aggregates(dims, block)
    Ac = OC.coarse_operator(op, agg, nc)
    if block == (1, 1):
        assert np.allclose(Ac, _dense(op), rtol=0, atol=1e-14)
    g = rng.normal(52, nc)
    y0 = rng.uniform(53, nc)
    for nu in (1, 3, 8):
        a = OC.coarse_fgs(Ac, g, nu, y0)
        s = OC.coarse_fgs_streaming(op, agg, nc, g, nu, y0)
        assert np.linalg.norm(a - s) <= 1e-13 * np.linalg.norm(a), nu
    ref = np.linalg.solve(Ac, g)
    assert np.linalg.norm(OC.coarse_fgs(Ac, g, 2000) - ref) <= 1e-10 * np.linalg.norm(ref)


# --- adjoint ----------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(6, 5), (4, 3, 3)])
def test_adjoint_gradient_matches_complex_step_dense_reference(dims):
    """dL/dkappa_c = -lambda^T (dA/dkappa_c) x, with (dA/dkappa_c) x taken by complex-step
    differentiation of the assembled operator (exact to rounding), lambda, x by dense solves."""
    kappa = W.lognormal_kappa(dims, 0.5, 17)
    op = O.Operator(*W.csr(dims, kappa))
    A = _dense(op)
    b = rng.uniform(18, op.n)
    xt = rng.uniform(19, op.n)
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A, 2 * (x - xt))
    g = OA.grad_kappa(dims, kappa, x, lam)
    h = 1e-30
    ref = np.empty(op.n)
    for cidx in range(op.n):
        kc = kappa.astype(np.complex128)
        kc[cidx] += 1j * h
        dAx = W.apply(dims, x.astype(np.complex128), kc).imag / h
        ref[cidx] = -lam @ dAx
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)


def test_adjoint_gradient_matches_finite_differences():
    dims = (7, 6)
    kappa = W.lognormal_kappa(dims, 0.5, 23)
    b = rng.uniform(24, 42)
    xt = rng.uniform(25, 42)

    def loss(k):
        A = _dense(O.Operator(*W.csr(dims, k)))
        x = np.linalg.solve(A, b)
        return np.sum((x - xt) ** 2)

    A = _dense(O.Operator(*W.csr(dims, kappa)))
    L, g, lam, x = OA.loss_and_grad(dims, kappa, b, xt, lambda rhs: np.linalg.solve(A, rhs))
    assert L == pytest.approx(loss(kappa))
    for cidx in [0, 5, 17, 41]:
        h = 1e-6 * kappa[cidx]
        kp, km = kappa.copy(), kappa.copy()
        kp[cidx] += h
        km[cidx] -= h
        fd = (loss(kp) - loss(km)) / (2 * h)
        assert fd == pytest.approx(g[cidx], rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_every_oracle_function_cites_its_passage():
    """Every public function of the oracle (and its Gram-solve helper) names the section,
    definition, proposition or cited method it follows, or says that the paper has none."""
    import ast
    import glob
    words = ("Section", "Definition", "Proposition", "Theorem", "Lemma", "paper", "textbook", "Chronopoulos")
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    for f in sorted(glob.glob(os.path.join(here, "*.py"))):
        tree = ast.parse(open(f).read())
        for node in tree.body:
            if isinstance(node, ast.FunctionDef) and (not node.name.startswith("_") or node.name == "_gram_solve_scaled"):
                doc = ast.get_docstring(node) or ""
                assert any(w in doc for w in words), f"{os.path.basename(f)}:{node.name}"


def test_oracle_and_library_share_no_code():
    """The CUDA library's Python side never imports the oracle, the oracle never imports the
    library, and the seeded input generators (`workloads`) import neither."""
    import ast
    import glob
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def imported(path):
        mods = set()
        for node in ast.walk(ast.parse(open(path).read())):
            if isinstance(node, ast.Import):
                mods |= {a.name.split(".")[0] for a in node.names}
            elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
                mods.add(node.module.split(".")[0])
        return mods

    for f in glob.glob(os.path.join(root, "paper_2512_09642_gb300", "*.py")):
        assert "oracle" not in imported(f), f
    for f in glob.glob(os.path.join(root, "oracle", "*.py")):
        assert "paper_2512_09642_gb300" not in imported(f), f
    for f in glob.glob(os.path.join(root, "workloads", "*.py")):
        assert not imported(f) & {"oracle", "paper_2512_09642_gb300"}, f
    for f in glob.glob(os.path.join(root, "paper_2512_09642_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read(), f
