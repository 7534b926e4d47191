"""Source terms on the GPU (Section 2: d_t Q + d_x F(Q) = S(Q), the GRP with
the source and the numerical source of eq. eq:source) against the oracle,
plus what the mathematics fixes without the oracle: the well-balanced
hydrostatic state of degree 2 (Section 3.5) kept to round-off, and the
convergence order with a linear source."""
import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, SMOOTH_TOL, check_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_with_linear_source_to_t1(M):
    prob, avg, lm, lp = I.advection_sine_source(80, -1.3, M=M)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_uniform_free_fall(M):
    prob, avg, lm, lp = I.euler_uniform(40, M, g=0.6)
    check_parity(prob, avg, lm, lp, 50, SMOOTH_TOL)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_hydrostatic_polytrope(M):
    """gamma = 2 (the generic-gamma kernels), transmissive ends."""
    prob, avg, lm, lp = I.hydrostatic_polytrope(150, M)
    check_parity(prob, avg, lm, lp, 60, SMOOTH_TOL)


@pytest.mark.parametrize("M", [2, 3])
def test_shock_tube_under_gravity(M):
    """Sod's data under the acceleration -1 (gamma = 7/5 kernels, repair
    rounds included)."""
    prob, avg, lm, lp = I.sod(300, M=M)
    prob = dict(prob, source=I.SOURCE_GRAVITY, source_coef=1.0)
    check_parity(prob, avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_gpu_keeps_the_hydrostatic_state(M):
    from paper_2602_21911_gb300 import grprec
    N, n = 200, 10
    prob, avg, lm, lp = I.hydrostatic_polytrope(N, M)
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.step(n)
    a, g, t = s.get_state()
    inner = slice(5 * (n + 1), N - 5 * (n + 1))
    scale = np.abs(avg).max()
    assert (np.abs(a[:, inner] - avg[:, inner]) / scale).max() < 1e-13
    assert (np.abs(g[:, inner] - lm[:, inner]) / scale).max() < 1e-13


def test_linear_source_converges_at_order_M_plus_1_on_the_gpu():
    from paper_2602_21911_gb300 import grprec
    for M in (1, 2, 3, 4):
        e = []
        for N in (32, 64, 128):
            prob, avg, lm, lp = I.advection_sine_source(N, -1.0, M=M)
            s = grprec.Solver(prob)
            s.set_initial(avg, lm, lp)
            s.advance_to(1.0)
            l1, _, _ = s.error_norms(np.ascontiguousarray(I.advection_sine_source_exact(N, -1.0, 1.0)[0]))
            e.append(float(l1[0]))
        orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(orders > M + 1 - 0.3), (M, e, orders)
