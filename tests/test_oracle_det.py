"""Pins of the oracle's DET solver (space-time Galerkin predictor + Riemann
problems at the time integration points; the solver of the paper's
computations, Section 4.1): for linear advection it coincides with the
Toro-Titarev solver (both evolve the reconstruction exactly), on the Euler
density wave it is advection of the density, it keeps order M+1, it leaves
constant states unchanged, and it converges on the shock tube."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I


def _run(prob, avg, lm, lp, t_end, steps=10 ** 8, **kw):
    st, g = O.init_iface(prob["system"], prob.get("lam", 1.0), prob.get("gamma", 1.4), lm, lp)
    S = O.State(prob, avg, g)
    O.run(dict(prob, **kw), S, steps, t_end=t_end)
    return S


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("recon", [0, 1])
def test_det_equals_tt_for_linear_advection(M, recon):
    """Both GRP solvers evolve the reconstruction exactly for a linear flux:
    the space-time predictor of degree M is exact for q(x - t), and the
    Riemann problems at the nodes are upwind values of the evolved traces."""
    prob, avg, lm, lp = I.advection_sine(40, M=M)
    a = _run(prob, avg, lm, lp, 1.0, solver=O.SOLVER_TT, recon=recon)
    b = _run(prob, avg, lm, lp, 1.0, solver=O.SOLVER_DET, recon=recon)
    assert np.abs(a.avg - b.avg).max() < 1e-12
    assert np.abs(a.iface - b.iface).max() < 1e-12


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_det_keeps_the_order(M):
    e = []
    for N in (32, 64):
        prob, avg, lm, lp = I.euler_wave(N, M)
        S = _run(prob, avg, lm, lp, 1.0, solver=O.SOLVER_DET)
        assert S.status[0] == O.OK
        assert np.allclose(S.avg.sum(axis=1), avg.sum(axis=1), rtol=1e-13)
        e.append(np.abs(S.avg[0] - I.euler_wave_exact(N, 1.0)[0]).sum() / N)
    assert math.log2(e[0] / e[1]) == pytest.approx(M + 1, abs=0.35)


@pytest.mark.parametrize("M", [2, 4])
def test_det_euler_wave_is_advection_of_rho(M):
    """u = 1 and p constant: every edge Riemann problem is a contact, the
    predictor transports the density; DET on the Euler wave equals DET (= TT)
    on the advected density with the same time steps."""
    N = 40
    prob, avg, lm, lp = I.euler_wave(N, M)
    S = _run(prob, avg, lm, lp, 0.5, solver=O.SOLVER_DET)
    T = _run(prob, avg, lm, lp, 0.5, solver=O.SOLVER_TT)
    assert np.abs(S.avg - T.avg).max() < 1e-11


def test_det_constant_state_is_steady():
    """Steady up to the rounding of the nodal operators (the rows of the
    differentiation matrix sum to zero, T^{-1} maps the end-value vector to
    ones, each only to about an ulp): well below 1e-12 after 20 steps."""
    prob, avg, lm, lp = I.riemann_problem(30, (1.3, 0.4, 2.0), (1.3, 0.4, 2.0), M=3)
    S = _run(prob, avg, lm, lp, np.inf, steps=20, solver=O.SOLVER_DET)
    assert np.abs(S.avg - avg).max() < 1e-12 * np.abs(avg).max()


def test_det_sod_converges_first_order():
    from test_oracle_scheme import _exact_sod_averages
    e = []
    for N in (100, 200, 400):
        prob, avg, lm, lp = I.sod(N)
        S = _run(prob, avg, lm, lp, 0.2, solver=O.SOLVER_DET)
        assert S.status[0] == O.OK
        e.append(np.abs(S.avg[0] - _exact_sod_averages(N, 0.2)).sum() / N)
    assert e[0] > 1.5 * e[1] > 2.25 * e[2]
    assert e[2] < 5e-3
