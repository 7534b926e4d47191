"""Pins of the oracle's source terms (Section 2: the balance law
d_t Q + d_x F(Q) = S(Q), the numerical source of eq. eq:source in the update
eq. eq_finite_volume, and the GRP with a source, eq. eq:GRP; the
well-balanced property of degree <= 2 reconstructions, Section 3.5).

Two sources, both linear in Q: S(q) = k q for linear advection, and a
constant acceleration -g for the Euler equations, S = (0, -g rho, -g m)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from parity import oracle_run
from test_oracle_riemann import G, RNG, cons, jacobian


def _run(prob, avg, lm, lp, n, t_end=np.inf):
    return oracle_run(prob, avg, lm, lp, n, t_end)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_ck_advection_with_source_is_the_series_of_the_exact_solution(M):
    """q_t + lam q_x = k q: Q(x, t) = exp(k t) p(x - lam t); its bivariate
    Taylor coefficients written out: q_ab = sum_{i+j=b} k^j/j! C(a+i, a)
    (-lam)^i p_{a+i}."""
    lam, k = 0.7, -1.3
    p = RNG.normal(size=M + 1)
    q = O.ck_series_src(O.ADVECTION, lam, G, M, O.SOURCE_LINEAR, k, p)
    for a in range(M + 1):
        for b in range(M + 1 - a):
            exact = sum(k ** (b - i) / math.factorial(b - i) * math.comb(a + i, a) * (-lam) ** i * p[a + i]
                        for i in range(0, min(b, M - a) + 1))
            assert q[a, b, 0] == pytest.approx(exact, rel=1e-13, abs=1e-14), (a, b)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_ck_euler_with_gravity_solves_the_balance_law_to_order_M(M):
    """The residual d_tau Q + A(Q) d_x Q - S(Q) of the truncated series is
    O(eps^M) at distance eps from the expansion point; without the source
    term in the series it is O(1)."""
    g = 0.8
    qa0 = np.zeros((M + 1, 3))
    qa0[0] = cons((1.3, 0.4, 0.9))
    for a in range(1, M + 1):
        qa0[a] = 0.3 * RNG.normal(size=3)

    def residual(q, x, t):
        Q = sum(q[a, b] * x ** a * t ** b for a in range(M + 1) for b in range(M + 1 - a))
        Qt = sum(b * q[a, b] * x ** a * t ** (b - 1) for a in range(M + 1) for b in range(1, M + 1 - a))
        Qx = sum(a * q[a, b] * x ** (a - 1) * t ** b for a in range(1, M + 1) for b in range(M + 1 - a))
        S = np.array([0.0, -g * Q[0], -g * Q[1]])
        return Qt + jacobian(Q) @ Qx - S

    q = O.ck_series_src(O.EULER, 0.0, G, M, O.SOURCE_GRAVITY, g, qa0)
    pts = ((1, 0), (0, 1), (0.7, 0.7))
    r1 = max(np.abs(residual(q, 1e-2 * c, 1e-2 * s)).max() for c, s in pts)
    r2 = max(np.abs(residual(q, 5e-3 * c, 5e-3 * s)).max() for c, s in pts)
    assert math.log2(r1 / r2) > M - 0.3
    q0 = O.ck_series(O.EULER, 0.0, G, M, qa0)                     # no source in the series
    assert np.abs(residual(q0, 1e-3, 0.0)).max() > 0.1


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_uniform_advection_grows_by_the_truncated_exponential(M):
    """Uniform data: the fluxes cancel, one step multiplies the averages by
    the Taylor polynomial of exp(k dt) of degree M + 1 (the interface series
    has degree M in time, and the source term integrates it once more), and
    the interface data by that of degree M."""
    N, k = 16, -2.5
    prob, avg, lm, lp = I.advection_sine_source(N, k, M=M)
    avg = np.full_like(avg, 0.7)
    lm = lp = np.full_like(lm, 0.7)
    S = _run(prob, avg, lm, lp, 1)
    dt = prob["cfl"] * (1.0 / N)
    taylor = lambda deg: sum((k * dt) ** b / math.factorial(b) for b in range(deg + 1))
    assert np.allclose(S.avg, 0.7 * taylor(M + 1), rtol=1e-14, atol=0)
    assert np.allclose(S.iface, 0.7 * taylor(M), rtol=1e-14, atol=0)
    assert S.t[0] == dt


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_with_source_converges_at_order_M_plus_1(M):
    k = -1.0
    e = []
    for N in (32, 64, 128):
        prob, avg, lm, lp = I.advection_sine_source(N, k, M=M)
        S = _run(prob, avg, lm, lp, 10 ** 6, 1.0)
        e.append(np.abs(S.avg - I.advection_sine_source_exact(N, k, 1.0)).sum() / N)
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(orders > M + 1 - 0.3), (M, e, orders)
    # the source matters: the error against the sourceless solution is O(1)
    assert np.abs(S.avg - I.advection_sine_exact(128, 1.0)).max() > 0.1


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_uniform_free_fall_is_exact(M):
    """A uniform gas under the acceleration -g: rho and p stay constant, the
    momentum falls linearly and the energy follows it, exactly in every step
    for every degree (the fluxes cancel; the source's space-time average is
    exact for this state)."""
    g = 0.6
    prob, avg, lm, lp = I.euler_uniform(12, M, g=g)
    n = 7
    S = _run(prob, avg, lm, lp, n)
    t = S.t[0]
    rho, m0, E0 = avg[:, 0]
    m = m0 - g * rho * t
    E = E0 - g * m0 * t + 0.5 * g * g * rho * t * t
    assert np.allclose(S.avg[0], rho, rtol=1e-15)
    assert np.allclose(S.avg[1], m, rtol=1e-13)
    assert np.allclose(S.avg[2], E, rtol=1e-13)
    # pressure unchanged
    p = 0.4 * (S.avg[2] - 0.5 * S.avg[1] ** 2 / S.avg[0])
    assert np.allclose(p, 0.9, rtol=1e-13)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_hydrostatic_polynomial_state_is_preserved(M):
    """Well-balancing (Section 3.5): the polytropic (gamma = 2, p = rho^2)
    hydrostatic state has linear density and quadratic energy; reconstructions
    of degree >= 2 reproduce it, the GRP returns it unchanged in time, and
    the update keeps it to round-off.  The transmissive ends are not
    equilibrium boundaries, so only cells out of their reach after n steps are
    compared (at most one cell plus four repair rounds per step)."""
    N, n = 200, 10
    prob, avg, lm, lp = I.hydrostatic_polytrope(N, M)
    S = _run(prob, avg, lm, lp, n)
    assert S.status[0] == O.OK
    inner = slice(5 * (n + 1), N - 5 * (n + 1))
    scale = np.abs(avg).max()
    assert (np.abs(S.avg[:, inner] - avg[:, inner]) / scale).max() < 1e-13
    assert (np.abs(S.iface[:, inner] - lm[:, inner]) / scale).max() < 1e-13


def test_hydrostatic_state_needs_the_source_and_degree_two():
    """The same state moves without the source term, and with degree 1 (whose
    reconstruction does not reproduce the quadratic energy)."""
    N, n = 200, 10
    inner = slice(5 * (n + 1), N - 5 * (n + 1))
    prob, avg, lm, lp = I.hydrostatic_polytrope(N, 2)
    S = _run(dict(prob, source=O.SOURCE_NONE), avg, lm, lp, n)
    assert np.abs(S.avg[1, inner]).max() > 1e-4
    prob, avg, lm, lp = I.hydrostatic_polytrope(N, 1)
    S = _run(prob, avg, lm, lp, n)
    assert np.abs(S.avg[1, inner]).max() > 1e-9


def test_zero_source_coefficient_is_the_sourceless_scheme():
    prob, avg, lm, lp = I.advection_sine_source(50, 0.0, M=3)
    a = _run(prob, avg, lm, lp, 20).avg
    b = _run(dict(prob, source=O.SOURCE_NONE), avg, lm, lp, 20).avg
    assert np.array_equal(a, b)
    prob, avg, lm, lp = I.sod(80, M=2)
    a = _run(dict(prob, source=O.SOURCE_GRAVITY, source_coef=0.0), avg, lm, lp, 30).avg
    b = _run(prob, avg, lm, lp, 30).avg
    assert np.array_equal(a, b)


def test_source_combinations_the_oracle_rejects():
    prob, avg, lm, lp = I.sod(20, M=2)
    for bad in (dict(source=O.SOURCE_LINEAR, source_coef=1.0), dict(source=O.SOURCE_GRAVITY, source_coef=1.0,
                                                                     solver=O.SOLVER_DET)):
        with pytest.raises(ValueError):
            _run(dict(prob, **bad), avg, lm, lp, 1)
