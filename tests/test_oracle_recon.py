"""Pins of the oracle's GRPrec reconstruction (Section 3.1) against facts the
paper fixes: the conservation condition, the interpolation conditions, the
least-squares optimality of the degree-1 and degree-3 functionals, exact
reproduction of polynomials of degree <= M, and uniqueness (Section 3.2)."""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(20260221)


def peval(c, x):
    return sum(ck * x ** k for k, ck in enumerate(c))


def pavg(c, a, b):
    return sum(ck * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, ck in enumerate(c)) / (b - a)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_conservation_in_cell_i(M):
    for _ in range(50):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(M, qb, g)
        assert abs(pavg(c, -0.5, 0.5) - qb[1]) < 1e-13


@pytest.mark.parametrize("M", [2, 4])
def test_interpolates_both_interfaces(M):
    for _ in range(50):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(M, qb, g)
        assert abs(peval(c, -0.5) - g[0]) < 1e-13
        assert abs(peval(c, 0.5) - g[1]) < 1e-13


def test_degree4_conserves_neighbour_cells():
    for _ in range(50):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(4, qb, g)
        assert abs(pavg(c, -1.5, -0.5) - qb[0]) < 1e-12
        assert abs(pavg(c, 0.5, 1.5) - qb[2]) < 1e-12


def _objective(M, c, qb, g):
    r = [peval(c, -0.5) - g[0], peval(c, 0.5) - g[1]]
    if M == 3:
        r += [pavg(c, -1.5, -0.5) - qb[0], pavg(c, 0.5, 1.5) - qb[2]]
    return float(np.sum(np.square(r)))


@pytest.mark.parametrize("M", [1, 3])
def test_least_squares_is_optimal_among_conservative_polynomials(M):
    """Any conservative perturbation (zero cell average) raises the functional."""
    for _ in range(20):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(M, qb, g)
        f0 = _objective(M, c, qb, g)
        for _ in range(20):
            dc = RNG.normal(size=M + 1)
            dc[0] -= pavg(dc, -0.5, 0.5)          # make the perturbation mean-free
            for eps in (1e-3, 1e-1):
                assert _objective(M, c + eps * dc, qb, g) >= f0 - 1e-13


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_reproduces_polynomials_of_degree_M(M):
    """Data sampled from any global polynomial of degree <= M give it back."""
    for _ in range(20):
        true = RNG.normal(size=M + 1)
        qb = [pavg(true, -1.5, -0.5), pavg(true, -0.5, 0.5), pavg(true, 0.5, 1.5)]
        g = [peval(true, -0.5), peval(true, 0.5)]
        c = O.recon(M, qb, g)
        assert np.allclose(c, true, atol=1e-12, rtol=0)


def test_degree1_closed_form_slope():
    """Degree 1: the symmetric least-squares problem gives slope g_R - g_L."""
    for _ in range(20):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(1, qb, g)
        assert abs(c[1] - (g[1] - g[0])) < 1e-14
        assert abs(c[0] - qb[1]) < 1e-14


def test_uniqueness_argument_degree2():
    """Section 3.2: a quadratic with one conservation and two interface values is
    unique -- the same data from a different quadratic basis give the same
    polynomial (checked through an independent Vandermonde solve)."""
    for _ in range(20):
        qb, g = RNG.normal(size=3), RNG.normal(size=2)
        c = O.recon(2, qb, g)
        # basis 1, (xi - 1/2), (xi - 1/2)^2 written out by hand
        A = np.array([[1.0, -1.0, 1.0], [1.0, 0.0, 0.0], [1.0, -0.5, 1.0 / 3.0]])
        rhs = np.array([g[0], g[1], qb[1]])
        a = np.linalg.solve(A, rhs)
        x = np.linspace(-0.5, 0.5, 7)
        other = a[0] + a[1] * (x - 0.5) + a[2] * (x - 0.5) ** 2
        assert np.allclose(peval(c, x), other, atol=1e-12)
