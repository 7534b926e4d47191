"""Convergence of the GPU path against exact solutions (no oracle in the
loop): the paper's sin^4 advection table (Section 4.2, degree M = 1..4, t = 4,
mesh 128 -> 256), the sine advection sweep N = 25..400 at M = 2, the smooth
Euler density wave at M = 1..4 (orders M + 1), conservation, and first-order
convergence of the shock tube to the exact Riemann solution."""
import math
import os

import numpy as np
import pytest

from paper_2602_21911_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_advection_sin4_orders.txt")


def _run(prob, avg, lm, lp, t_end):
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.advance_to(t_end)
    a, g, t = s.get_state()
    stats, status = s.get_stats()
    assert (status == 0).all() and np.allclose(t, t_end, rtol=0, atol=0)
    return s, a




def test_paper_sin4_table_orders_and_errors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for M_s, order_s, err_s in rows:
        M = int(M_s)
        e = []
        for N in (128, 256):
            prob, avg, lm, lp = I.advection_sin4(N, M)
            s, a = _run(prob, avg, lm, lp, 4.0)
            l1, l2, linf = s.error_norms(np.ascontiguousarray(I.advection_sin4_exact(N, 4.0)[0]))
            e.append(float(l1[0]))
        order = math.log2(e[0] / e[1])
        assert order == pytest.approx(float(order_s), abs=0.25), (M, order)
        # finest-mesh L1 error: the paper's digits for M = 1 (printed with 3
        # digits); for M >= 2 its solver's error constants sit 5-25 % above
        if M == 1:
            assert e[1] == pytest.approx(float(err_s), rel=0.012)
        else:
            assert 0.6 * float(err_s) < e[1] < 1.05 * float(err_s), (M, e[1])


def test_sine_advection_sweep_m2():
    e = []
    for N in (25, 50, 100, 200, 400):
        prob, avg, lm, lp = I.advection_sine(N, M=2)
        s, a = _run(prob, avg, lm, lp, 1.0)
        l1, _, _ = s.error_norms(np.ascontiguousarray(I.advection_sine_exact(N, 1.0)[0]))
        e.append(float(l1[0]))
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.25), orders


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_wave_orders(M):
    e = []
    Ns = (64, 128, 256)
    for N in Ns:
        prob, avg, lm, lp = I.euler_wave(N, M)
        s, a = _run(prob, avg, lm, lp, 1.0)
        # conservation of every summed average (periodic)
        assert np.allclose(a.sum(axis=1), avg.sum(axis=1), rtol=1e-13)
        l1, _, _ = s.error_norms(np.ascontiguousarray(I.euler_wave_exact(N, 1.0)[0]))
        e.append(float(l1[0]))
    e = np.array(e)
    keep = e > 1e-11                                        # above the rounding floor
    orders = np.log2(e[:-1] / e[1:])[keep[1:]]
    assert len(orders) >= 1
    assert np.all(orders > M + 1 - 0.4), (M, e, orders)


def test_sod_converges_first_order():
    from test_oracle_scheme import _exact_sod_averages
    e = []
    for N in (200, 400, 800):
        prob, avg, lm, lp = I.sod(N)
        s, a = _run(prob, avg, lm, lp, 0.2)
        e.append(np.abs(a[0] - _exact_sod_averages(N, 0.2)).sum() / N)
    assert e[0] > 1.5 * e[1] > 2.25 * e[2]
    assert e[2] < 3e-3
