"""GPU GRPrecNL (Sections 3.3-3.4) against the oracle: smooth and
discontinuous advection, the Euler density wave, the shock tube, the 123
problem, transmissive ghost handling at degree 4, and every launch form on a
batch of domains.

Every case holds the stated tolerance except the degree-1 Euler density wave
run to t = 1, which is listed as out of tolerance (tests/out_of_tolerance.py):
there the oracle itself answers a one-ulp input change with ~1e-9, so its
first 100 steps are held to 1e-11 and the full run is checked for that
ill-conditioning instead."""
import numpy as np
import pytest

from paper_2602_21911_gb300 import inputs as I

from out_of_tolerance import NL_EULER_WAVE_M1_T1, check_exempt
from parity import (DISC_TOL, SMOOTH_TOL, check_parity, gpu_run, oracle_run, oracle_ulp_sensitivity, rel_diff,
                    rel_diff_iface)

pytestmark = pytest.mark.gpu

NL = 1


def _nl(prob):
    return dict(prob, recon=NL)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_sine(M):
    prob, avg, lm, lp = I.advection_sine(80, M=M)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_square_wave(M):
    prob, avg, lm, lp = I.advection_square(50, M=M)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=4.0)


def test_multiwave_many_periods():
    prob, avg, lm, lp = I.advection_multiwave(100, M=2)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=20.0)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_euler_wave(M):
    prob, avg, lm, lp = I.euler_wave(64, M)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


def test_euler_wave_degree1_first_100_steps():
    prob, avg, lm, lp = I.euler_wave(64, 1)
    check_parity(_nl(prob), avg, lm, lp, 100, SMOOTH_TOL)


def test_euler_wave_degree1_to_t1_is_listed_out_of_tolerance():
    """Not held to 1e-11: the oracle's own one-ulp response is ~1e-9 (the
    listed entry); the test asserts that ill-conditioning and reports the
    GPU difference."""
    prob, avg, lm, lp = I.euler_wave(64, 1)
    prob = _nl(prob)
    sens = oracle_ulp_sensitivity(prob, avg, lm, lp, 10 ** 6, 1.0)
    check_exempt(sens, SMOOTH_TOL, "GRPrecNL degree-1 Euler wave to t = 1")
    S = oracle_run(prob, avg, lm, lp, 10 ** 6, 1.0)
    s, a, g, t, stats, status = gpu_run(prob, avg, lm, lp, 10 ** 6, 1.0)
    assert np.array_equal(status, S.status) and t[0] == S.t[0] == 1.0
    d = max(rel_diff(a, S.avg, prob).max(), rel_diff_iface(g, S.iface, prob).max())
    print("GRPrecNL degree-1 Euler wave to t = 1: GPU - oracle %.2e, oracle one-ulp response %.2e "
          "(listed: %s)" % (d, sens, NL_EULER_WAVE_M1_T1))


def test_euler_wave_transmissive_degree4_ghosts():
    prob, avg, lm, lp = I.euler_wave(77, 4, bc=I.TRANSMISSIVE)
    check_parity(_nl(prob), avg, lm, lp, 60, SMOOTH_TOL)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_sod(M):
    prob, avg, lm, lp = I.sod(200, M=M, xc=0.3)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)


def test_123_problem():
    prob, avg, lm, lp = I.euler_123(200, M=2)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.15)


@pytest.mark.parametrize("form", [1, 2, 3])
def test_batched_forms(form):
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 331)[:150])
    s = grprec.Solver(_nl(prob))
    s.set_launch(form, 256, 2048, 4)
    check_parity(_nl(prob), avg, lm, lp, 30, DISC_TOL, solver=s)
