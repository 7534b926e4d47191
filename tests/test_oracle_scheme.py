"""Whole-scheme pins of the oracle: the paper's printed advection errors
(Section 4.2), orders M+1 on smooth data, the unit Courant limit (Section 4.1),
exact translation at Courant number 1, conservation, the reduction of the
smooth Euler density wave to advection, batch independence, the dt_hold rule
and the a-posteriori repair on Sod's problem."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def run_adv(N, M, t_end, maker=I.advection_sine, cfl=0.9):
    prob, avg, lm, lp = maker(N, M=M, cfl=cfl)
    st, g = O.init_iface(O.ADVECTION, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    O.run(prob, S, 10 ** 8, t_end=t_end)
    return prob, S


def norms(err, dx):
    e = np.abs(err)
    return e.max(), e.sum() * dx, math.sqrt((e ** 2).sum() * dx)


def test_paper_table_degree1_errors():
    rows = np.loadtxt(os.path.join(GOLD, "paper_advection_sin4_m1.txt"))
    for N, linf, l1, l2 in rows:
        N = int(N)
        prob, S = run_adv(N, 1, 4.0, maker=I.advection_sin4)
        got = norms(S.avg[0] - I.advection_sin4_exact(N, 4.0)[0], 2.0 / N)
        for g, ref in zip(got, (linf, l1, l2)):
            assert g == pytest.approx(ref, rel=0.012)      # printed with 3 digits


def test_paper_table_orders():
    rows = np.loadtxt(os.path.join(GOLD, "paper_advection_sin4_orders.txt"))
    for M, order, l1_256 in rows:
        M = int(M)
        e = []
        for N in (128, 256):
            prob, S = run_adv(N, M, 4.0, maker=I.advection_sin4)
            e.append(norms(S.avg[0] - I.advection_sin4_exact(N, 4.0)[0], 2.0 / N)[1])
        assert math.log2(e[0] / e[1]) == pytest.approx(order, abs=0.25)
        # The paper's DET runs are reproduced within a factor, not to the digit
        # (its degree >= 2 error constants sit 5-25 % above these).
        assert 0.6 * l1_256 < e[1] < 1.05 * l1_256


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_sine_order(M):
    e = []
    for N in (50, 100, 200):
        prob, S = run_adv(N, M, 1.0)
        e.append(np.abs(S.avg[0] - I.advection_sine_exact(N, 1.0)[0]).sum() / N)
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(orders - (M + 1)) < 0.2)


def one_step_matrix(M, N, nu):
    """The linear one-step map of (averages, interface data) on a periodic grid."""
    prob, _, _, _ = I.advection_sine(N, M=M)
    dx = 1.0 / N
    A = np.zeros((2 * N, 2 * N))
    for k in range(2 * N):
        v = np.zeros(2 * N)
        v[k] = 1.0
        S = O.State(prob, v[:N][None, :], v[N:][None, :])
        O.run(prob, S, 1, dt_fixed=[nu * dx])
        A[:N, k] = S.avg[0]
        A[N:, k] = S.iface[0]
    return A


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_unit_courant_limit(M):
    """Section 4.1: every GRPrec finite volume scheme is stable up to Courant 1."""
    for nu in (0.3, 0.6, 0.9, 1.0):
        rho = np.abs(np.linalg.eigvals(one_step_matrix(M, 24, nu))).max()
        # at nu = 1 unimodular eigenvalues may be defective: eigvals then errs by ~sqrt(eps)
        assert rho <= 1.0 + (1e-10 if nu < 1.0 else 1e-7)
    rho = np.abs(np.linalg.eigvals(one_step_matrix(M, 24, 1.1))).max()
    assert rho > 1.0 + 1e-3


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_courant_one_shifts_the_averages(M):
    N = 20
    prob, avg, lm, lp = I.advection_sine(N, M=M)
    rng = np.random.default_rng(M)
    avg = rng.normal(size=(1, N))
    g = rng.normal(size=(1, N))
    S = O.State(prob, avg, g)
    O.run(prob, S, 1, dt_fixed=[1.0 / N])
    assert np.allclose(S.avg[0], np.roll(avg[0], 1), atol=1e-13)
    if M in (2, 4):        # interpolatory degrees also shift the interface data
        assert np.allclose(S.iface[0], np.roll(g[0], 1), atol=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_wave_order_and_conservation(M):
    e = []
    for N in (32, 64):
        prob, avg, lm, lp = I.euler_wave(N, M)
        st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
        S = O.State(prob, avg, g)
        O.run(prob, S, 10 ** 8, t_end=1.0)
        assert S.status[0] == O.OK
        e.append(np.abs(S.avg[0] - I.euler_wave_exact(N, 1.0)[0]).sum() / N)
        # conservation of every summed average (periodic)
        assert np.allclose(S.avg.sum(axis=1), avg.sum(axis=1), rtol=1e-13)
    assert math.log2(e[0] / e[1]) == pytest.approx(M + 1, abs=0.35)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_density_wave_is_advection_of_rho(M):
    """u = 1 and p = const make every Euler GRP a contact: the scheme equals
    GRPrec advection of rho on the same dt sequence."""
    N = 40
    prob, avg, lm, lp = I.euler_wave(N, M)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    dts = []
    for _ in range(60):
        t0 = S.t[0]
        O.run(prob, S, 1)
        dts.append(S.t[0] - t0)
    pa, _, _, _ = I.advection_sine(N, M=M)
    A = O.State(pa, avg[:1], g[:1])
    O.run(pa, A, 60, dt_fixed=dts)
    assert np.abs(S.avg[0] - A.avg[0]).max() < 1e-12
    assert np.abs(S.avg[1] - S.avg[0]).max() < 1e-12


def test_sod_runs_positive_and_conserves():
    N = 200
    prob, avg, lm, lp = I.sod(N)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    O.run(prob, S, 10 ** 6, t_end=0.2)
    assert S.status[0] == O.OK and S.t[0] == 0.2
    rho, m, E = S.avg
    p = 0.4 * (E - 0.5 * m * m / rho)
    assert rho.min() > 0 and p.min() > 0
    dx = 1.0 / N
    assert rho.sum() * dx == pytest.approx(0.5625, rel=1e-13)
    assert m.sum() * dx == pytest.approx(0.2 * (1.0 - 0.1), rel=1e-12)   # boundary pressures
    assert E.sum() * dx == pytest.approx(0.5 * 2.5 + 0.5 * 0.25, rel=1e-13)
    assert S.stats[0, O.ST_LOW_ORDER] > 0      # the repair was needed and used


def test_batched_domain_is_independent_of_the_batch():
    ids = [3, 17, 40, 41, 99]
    prob, avg, lm, lp = I.batched(domains=ids)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    O.run(prob, S, 30)
    co, io = I.cell_offsets(prob), I.iface_offsets(prob)
    for k, d in enumerate(ids):
        p1, a1, m1, l1 = I.batched(domains=[d])
        s1, g1 = O.init_iface(O.EULER, 1.0, 1.4, m1, l1)
        S1 = O.State(p1, a1, g1)
        O.run(p1, S1, 30)
        assert np.array_equal(S1.avg, S.avg[:, co[k]:co[k + 1]])
        assert np.array_equal(S1.iface, S.iface[:, io[k]:io[k + 1]])


def test_dt_hold_recomputes_every_h_steps():
    prob, avg, lm, lp = I.sod(100)
    prob = dict(prob, dt_hold=3)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    dts = []
    for _ in range(9):
        O.run(prob, S, 1)
        dts.append(S.dt_prev[0])
    assert dts[0] == dts[1] == dts[2] and dts[3] == dts[4] == dts[5]
    assert dts[3] != dts[0]


def test_initial_interface_data_of_smooth_data_are_point_values():
    prob, avg, lm, lp = I.euler_wave(16, 2)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    assert np.allclose(g, lm, rtol=1e-15, atol=1e-15)


def test_step_clips_to_t_end():
    prob, S = run_adv(30, 2, 0.05)
    assert S.t[0] == 0.05


def _exact_sod_averages(N, t, nsub=16):
    """Cell averages of the exact shock-tube solution (x_c = 0.5), by Gauss
    quadrature of the self-similar solution sampled through Galilean shifts."""
    xs, ws = np.polynomial.legendre.leggauss(nsub)
    dx = 1.0 / N
    out = np.zeros(N)
    g = 1.4
    for i in range(N):
        acc = 0.0
        for x, w in zip(xs, ws):
            xi = ((i + 0.5 + 0.5 * x) * dx - 0.5) / t
            WL = np.array([1.0, -xi, 1.0]); WR = np.array([0.125, -xi, 0.1])
            QL = np.array([WL[0], WL[0] * WL[1], WL[2] / (g - 1) + 0.5 * WL[0] * WL[1] ** 2])
            QR = np.array([WR[0], WR[0] * WR[1], WR[2] / (g - 1) + 0.5 * WR[0] * WR[1] ** 2])
            st, Q, _ = O.riemann_state(g, QL, QR)
            acc += 0.5 * w * Q[0]
        out[i] = acc
    return out


def test_sod_converges_to_the_exact_solution():
    """With the a-posteriori repair (admissibility and a relaxed discrete
    maximum principle) the degree-2 scheme converges to the exact shock-tube
    solution: first order in L1, as for any captured discontinuity."""
    e = []
    for N in (100, 200, 400):
        prob, avg, lm, lp = I.sod(N)
        st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
        S = O.State(prob, avg, g)
        O.run(prob, S, 10 ** 6, t_end=0.2)
        assert S.status[0] == O.OK
        e.append(np.abs(S.avg[0] - _exact_sod_averages(N, 0.2)).sum() / N)
    assert e[0] > 1.5 * e[1] > 2.25 * e[2]
    assert e[2] < 5e-3
