"""Pins of the mapped-cube system and the geometry-aware preconditioner P^G
(oracle/geometry.py; Sec. 4.4, App. A.3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.geometry import MappedProblem, separate
from oracle.fd import FD
from oracle.solve import pcg, direct_solve
from paper_1809_10026_gb300 import synth


@pytest.mark.parametrize("d,p,n_el,a", [(1, 2, 3, [0.6]), (1, 3, 2, [-0.7]), (2, 2, 2, [0.5, -0.3]),
                                         (2, 3, 2, [0.7, 0.4])])
def test_direct_and_kronecker_assembly_agree(d, p, n_el, a):
    """Two independent routes to A^G: quadrature of the form with the chain-rule
    Laplacian of the mapped basis (general J, Hess G), and the weighted 1D
    Kronecker factors (integration by parts in space for the W_t term).  With
    24 Gauss points per element both integrate to rounding."""
    mp = MappedProblem(d, p, n_el, a, nq=24)
    Ad = mp.assemble_direct()
    Ak = mp.assemble_kron().toarray()
    assert np.abs(Ad - Ak).max() <= 1e-13 * np.abs(Ak).max()
    x = synth.uniform(mp.N, 3)
    assert np.abs(mp.apply_kron(x) - Ak @ x).max() <= 1e-14 * np.abs(Ak @ x).max()


def test_mapped_matrix_is_spd():
    mp = MappedProblem(2, 3, 3, [0.6, -0.5])
    A = mp.assemble_kron().toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    np.linalg.cholesky(A)


@pytest.mark.parametrize("d,p,n_el", [(1, 2, 5), (2, 3, 3), (3, 2, 2)])
def test_identity_map_gives_the_cube(d, p, n_el):
    """a = 0: A^G is Eq. A_kron and Pbar^G is Eq. preconditioner (T = 1); the
    separated coefficients are all 1."""
    mp = MappedProblem(d, p, n_el, [0.0] * d)
    A = mp.cube.assemble_A_kron().toarray()
    assert np.abs(mp.assemble_kron().toarray() - A).max() <= 1e-13 * np.abs(A).max()
    mu, om, _, _ = mp.preconditioner_factors()
    for v in mu + om:
        assert np.allclose(v, 1.0, rtol=0, atol=1e-14)
    P = FD(mp.cube).explicit_P().toarray()
    Pg = mp.preconditioner().explicit_Pbar().toarray()
    assert np.abs(Pg - P).max() <= 1e-13 * np.abs(P).max()


def test_separation_recovers_separable_tensors():
    """If every C^(k) is exactly omega^(k) times the mu^(l) of the other
    directions, Algorithm 2 reproduces every entry (ratios 1)."""
    rng = np.random.default_rng(7)
    shape = (4, 3, 5)
    mu_t = [rng.uniform(0.5, 2.0, n) for n in shape]
    om_t = [rng.uniform(0.5, 2.0, n) for n in shape]
    C = []
    for k in range(3):
        f = [mu_t[l] if l != k else om_t[l] for l in range(3)]
        C.append(np.einsum("i,j,k->ijk", *f))
    mu, om = separate(C, maxit=2)
    for k in range(3):
        f = [mu[l] if l != k else om[l] for l in range(3)]
        approx = np.einsum("i,j,k->ijk", *f)
        assert np.abs(np.log(C[k] / approx)).max() <= 1e-13


def test_separation_improves_a_non_separable_fit():
    """On coefficients that are not products (a curved-looking field), the
    worst log-ratio after the algorithm is well below that of the all-ones start."""
    x = np.linspace(0.05, 0.95, 6)
    X, Y, Tt = np.meshgrid(x, x, x[:3], indexing="ij")
    C = [np.exp(X + 2 * Y + 0.3 * X * Y) + Tt, np.exp(-X + Y) * (1 + 0.2 * X * Y), 1 + X + Y + Tt]
    mu, om = separate(C, maxit=2)
    worst0 = max(np.abs(np.log(c)).max() for c in C)
    worst = 0.0
    for k in range(3):
        f = [mu[l] if l != k else om[l] for l in range(3)]
        worst = max(worst, np.abs(np.log(C[k] / np.einsum("i,j,k->ijk", *f))).max())
    assert worst < 0.25 * worst0


@pytest.mark.parametrize("d,p,n_el,a", [(1, 3, 4, [0.5]), (2, 2, 3, [0.6, -0.4]), (3, 2, 2, [0.3, 0.5, -0.4])])
def test_geometry_fd_equals_explicit_inverse(d, p, n_el, a):
    """(P^G)^{-1} r by Algorithm 1 with the scaling equals
    D^{-1/2} Pbar^{-1} D^{-1/2} r with Pbar assembled; P^G is symmetric."""
    mp = MappedProblem(d, p, n_el, a)
    PG = mp.preconditioner()
    Pbar = PG.explicit_Pbar()
    r = synth.uniform(mp.N, 11)
    s = 1 / np.sqrt(PG.D)
    ref = s * direct_solve(Pbar, s * r)
    z = PG.apply(r)
    assert np.abs(z - ref).max() <= 1e-11 * np.abs(ref).max()
    A = mp.assemble_kron()
    assert np.allclose(PG.D, A.diagonal() / Pbar.diagonal(), rtol=1e-14, atol=0)
    y = synth.uniform(mp.N, 12)
    assert abs(y @ PG.apply(r) - r @ PG.apply(y)) <= 1e-12 * np.linalg.norm(y) * np.linalg.norm(PG.apply(r))


@pytest.mark.parametrize("d,n_el,a", [(2, 16, [0.5, 0.5]), (2, 32, [0.7, -0.6])])
def test_geometry_preconditioner_reduces_iterations(d, n_el, a):
    """Sec. 4.4 / Table 2: on a stretched parametrization the cube's P needs
    several times the iterations of P^G (measured: 68 vs 21 for a = 0.5 on 16
    elements, 218 vs 51 for a = (0.7, -0.6) on 32; the terms P^G leaves out
    matter more on coarse meshes: 172 vs 78 on 16 elements)."""
    mp = MappedProblem(d, 3, n_el, a)
    F = synth.uniform(mp.N, 4)
    _, itP, _ = pcg(mp.apply_kron, FD(mp.cube).apply, F, 1e-8, 800)
    _, itG, hist = pcg(mp.apply_kron, mp.preconditioner().apply, F, 1e-8, 800)
    assert hist[-1] <= 1e-8 and itG * 2.5 <= itP, (itP, itG)


def test_mapped_solution_converges_in_physical_space():
    """The mapped discretization solves the heat equation on the physical
    cube: for u = sin(pi x) sin(pi t) (d = 1, p = 3, a = 0.5) the L2 error of
    the least-squares solution falls like h^(p+1) (L2 rate of Sec. 5.1 for
    p >= 3)."""
    pi = np.pi
    u = lambda xs, t: np.sin(pi * xs[:, 0]) * np.sin(pi * t)
    f = lambda xs, t: pi * np.sin(pi * xs[:, 0]) * np.cos(pi * t) + pi ** 2 * np.sin(pi * xs[:, 0]) * np.sin(pi * t)
    errs = []
    for n in (4, 8, 16):
        mp = MappedProblem(1, 3, n, [0.5], nq=12)
        c = direct_solve(mp.assemble_direct(), mp.load_direct(f))
        errs.append(mp.l2_error(c, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= 3.5, (errs, rates)
