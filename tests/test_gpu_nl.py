"""GPU GRPrecNL (Sections 3.3-3.4) against the oracle: smooth and
discontinuous advection, the Euler density wave, the shock tube, the 123
problem, transmissive ghost handling at degree 4, and every launch form on a
batch of domains.

The nonlinear weights (r = 4, eps = 1e-14) switch steeply where an
indicator of a nearly constant characteristic field crosses eps; a run that
passes such a point answers a one-ulp change of its input with up to ~1e-9
(the Euler density wave at degree 1: 2.6e-9 in the oracle itself).  The
Euler tests therefore take the tolerance max(base, 100 x the oracle's own
one-ulp sensitivity of the same run)."""
import numpy as np
import pytest

from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, SMOOTH_TOL, check_parity

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


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_wave(M):
    prob, avg, lm, lp = I.euler_wave(64, M)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0, conditioned=True)


def test_euler_wave_transmissive_degree4_ghosts():
    prob, avg, lm, lp = I.euler_wave(77, 4, bc=I.TRANSMISSIVE)
    check_parity(_nl(prob), avg, lm, lp, 60, SMOOTH_TOL, conditioned=True)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_sod(M):
    prob, avg, lm, lp = I.sod(200, M=M, xc=0.3)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2, conditioned=True)


def test_123_problem():
    prob, avg, lm, lp = I.euler_123(200, M=2)
    check_parity(_nl(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.15, conditioned=True)


@pytest.mark.parametrize("form", [1, 2, 3])
def test_batched_forms(form):
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 331)[:150])
    s = grprec.Solver(_nl(prob))
    s.set_launch(form, 256, 2048, 4)
    check_parity(_nl(prob), avg, lm, lp, 30, DISC_TOL, solver=s, conditioned=True)
