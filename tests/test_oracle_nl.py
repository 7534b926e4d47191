"""Pins of the oracle's GRPrecNL reconstruction (Sections 3.3-3.4) and of its
characteristic variables: each side polynomial meets its conditions, every
polynomial of degree <= M is reproduced, the weights follow their formula and
pick the smooth side at a jump, the eigenvectors diagonalise the flux
Jacobian, and the scheme keeps order M+1 on smooth data."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I


def _poly_data(P):
    Pi = P.integ()
    avg = lambda a, b: (Pi(b) - Pi(a)) / (b - a)
    return [avg(-1.5, -0.5), avg(-0.5, 0.5), avg(0.5, 1.5), P(-1.5), P(-0.5), P(0.5), P(1.5)]


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_reproduces_polynomials_of_degree_M(M):
    rng = np.random.default_rng(10 + M)
    for _ in range(5):
        c = rng.normal(size=M + 1)
        coef, beta = O.recon_nl(M, _poly_data(np.polynomial.Polynomial(c)), 0.01)
        assert np.abs(coef - c).max() < 1e-12
        assert beta.sum() == pytest.approx(1.0, abs=1e-15)




def test_weights_follow_their_formula_degree1():
    """Degree 1 by hand: p_L through g_{i-1/2}, p_R through g_{i+1/2}, p_C the
    least-squares line (slope g_{i+1/2} - g_{i-1/2}); OI_k = dx * int (p_k')^2
    by Gauss quadrature; omega_k = lambda_k / (1e-14 + OI_k)^4 with lambda =
    (1, 1e9, 1); the oracle's weights and combined polynomial follow."""
    rng = np.random.default_rng(7)
    xs, ws = np.polynomial.legendre.leggauss(4)
    for _ in range(20):
        d7 = rng.normal(size=7) * rng.choice([1e-3, 1.0, 30.0])
        dx = rng.choice([1e-3, 0.05, 1.0])
        q0, gm, gp = d7[1], d7[4], d7[5]
        slopes = [2 * (q0 - gm), gp - gm, 2 * (gp - q0)]
        OI = [dx * np.dot(ws * 0.5, np.full(4, s) ** 2) for s in slopes]
        om = np.array([lam / (1e-14 + oi) ** 4 for lam, oi in zip((1.0, 1e9, 1.0), OI)])
        beta_ref = om / om.sum()
        coef, beta = O.recon_nl(1, d7, dx)
        assert np.allclose(beta, beta_ref, rtol=1e-12, atol=1e-300)
        assert coef[0] == pytest.approx(q0, abs=1e-14 * max(1.0, abs(q0)))
        assert coef[1] == pytest.approx(np.dot(beta_ref, slopes), rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_convex_combination_conserves_and_weights_scale_with_lambda(M):
    rng = np.random.default_rng(20 + M)
    d7 = rng.normal(size=7)
    dx = 0.05
    coef, beta = O.recon_nl(M, d7, dx)
    # a convex combination of polynomials that all conserve cell i conserves it
    avg_i = sum(coef[k] * ((0.5) ** (k + 1) - (-0.5) ** (k + 1)) / (k + 1) for k in range(M + 1))
    assert avg_i == pytest.approx(d7[1], abs=1e-13)
    assert np.all(beta >= 0) and beta.sum() == pytest.approx(1.0, abs=1e-14)
    # linear data: the three polynomials coincide, their indicators too, so
    # the weights are proportional to lambda = (1, 1e9, 1)
    lin = _poly_data(np.polynomial.Polynomial([0.3, 1.7]))
    _, b = O.recon_nl(M, lin, dx)
    assert b[1] / b[0] == pytest.approx(1e9, rel=1e-9) and b[0] == pytest.approx(b[2], rel=1e-12)


def test_degree1_flat_side_takes_the_weight_at_a_jump():
    """Flat data left of a jump at x_{i+1/2}: p_L (through g_{i-1/2}) is
    constant, its indicator is 0, and its weight 1/eps^4 outweighs
    1e9 / OI_C^4: the reconstruction is flat.  (Only degree 1 has a one-sided
    polynomial that avoids the jump: every side polynomial of degrees 2-4 uses
    data on both sides of cell i.)"""
    d7 = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 0.5, 1.0])
    coef, beta = O.recon_nl(1, d7, 0.04)
    assert beta[1] < 1e-30 and beta[2] < 1e-30
    assert abs(coef[1]) < 1e-30


def test_char_basis_diagonalises_the_flux_jacobian():
    g = 1.4
    rng = np.random.default_rng(3)
    for _ in range(10):
        rho, u, p = rng.uniform(0.2, 3), rng.uniform(-2, 2), rng.uniform(0.2, 3)
        Q = np.array([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])
        R, L = O.char_basis(g, Q)
        assert np.abs(L @ R - np.eye(3)).max() < 1e-12
        # Jacobian of F by complex step on the flux definition (Section 4.3)
        def F(q):
            uu = q[1] / q[0]
            pp = (g - 1) * (q[2] - 0.5 * q[1] * uu)
            return np.array([q[1], q[1] * uu + pp, uu * (q[2] + pp)])
        A = np.zeros((3, 3))
        for k in range(3):
            dq = np.zeros(3, dtype=complex)
            dq[k] = 1e-30j
            A[:, k] = F(Q.astype(complex) + dq).imag / 1e-30
        c = math.sqrt(g * p / rho)
        assert np.abs(L @ A @ R - np.diag([u - c, u, u + c])).max() < 1e-11


def _run(prob, avg, lm, lp, t_end, recon):
    st, g = O.init_iface(prob["system"], prob.get("lam", 1.0), prob.get("gamma", 1.4), lm, lp)
    S = O.State(prob, avg, g)
    O.run(dict(prob, recon=recon), S, 10 ** 8, t_end=t_end)
    return S


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_nl_keeps_the_order_on_the_advected_sine(M):
    e = []
    for N in (50, 100):
        prob, avg, lm, lp = I.advection_sine(N, M=M)
        S = _run(prob, avg, lm, lp, 1.0, O.RECON_GRPRECNL)
        e.append(np.abs(S.avg[0] - I.advection_sine_exact(N, 1.0)[0]).sum() / N)
    assert math.log2(e[0] / e[1]) == pytest.approx(M + 1, abs=0.3)


@pytest.mark.parametrize("M", [2, 3])
def test_nl_euler_wave_order_and_conservation(M):
    e = []
    for N in (32, 64):
        prob, avg, lm, lp = I.euler_wave(N, M)
        S = _run(prob, avg, lm, lp, 1.0, O.RECON_GRPRECNL)
        assert S.status[0] == O.OK
        assert np.allclose(S.avg.sum(axis=1), avg.sum(axis=1), rtol=1e-13)
        e.append(np.abs(S.avg[0] - I.euler_wave_exact(N, 1.0)[0]).sum() / N)
    assert math.log2(e[0] / e[1]) == pytest.approx(M + 1, abs=0.4)


def test_nl_square_wave_conserves_and_stays_close_to_linear():
    """Section 4.2 square wave, degrees 1-4: the nonlinear scheme conserves the
    total and its profile stays within the linear scheme's range of
    oscillation (with the printed weights the central polynomial keeps almost
    all of the weight wherever both neighbours vary)."""
    for M in (1, 2, 3, 4):
        prob, avg, lm, lp = I.advection_square(50, M=M)
        lin = _run(prob, avg, lm, lp, 4.0, O.RECON_GRPREC)
        nl = _run(prob, avg, lm, lp, 4.0, O.RECON_GRPRECNL)
        assert nl.avg[0].sum() == pytest.approx(avg[0].sum(), rel=1e-12)
        over = lambda a: max(a.max() - 1.0, -a.min())
        assert over(nl.avg[0]) < 1.1 * over(lin.avg[0]) + 1e-3
