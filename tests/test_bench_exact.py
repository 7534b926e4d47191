"""The exact Riemann solutions bench.py measures L1 errors against (a numpy
restatement of the textbook solution) agree with the oracle's exact solver
sampled through Galilean shifts."""
import os
import sys

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

from test_oracle_scheme import _exact_sod_averages  # noqa: E402


def test_sod_averages_match_the_oracle():
    N = 200
    e = np.linspace(0.0, 1.0, N + 1)[None, :]
    mine = bench.exact_riemann_averages((np.ones(1), np.zeros(1), np.ones(1)),
                                        (np.full(1, 0.125), np.zeros(1), np.full(1, 0.1)), 0.5, 0.2, e)[0]
    assert np.abs(mine - _exact_sod_averages(N, 0.2)).max() < 1e-10


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_riemann_rays_match_the_oracle(seed):
    rng = np.random.default_rng(seed)
    g = 1.4
    WL = (np.ones(1), rng.uniform(-2, 2, 1), np.ones(1))
    WR = (np.exp(rng.uniform(-6.9, 6.9, 1)), rng.uniform(-2, 2, 1), np.exp(rng.uniform(-6.9, 6.9, 1)))
    xi = np.linspace(-30.0, 30.0, 241)
    rho, smax = bench.exact_riemann_density(WL, WR, xi[None, :], g)
    for k, x in enumerate(xi):
        # the solution at ray x: the state at x/t = 0 of the data seen by an
        # observer moving with speed x
        ql = np.array([WL[0][0], WL[0][0] * (WL[1][0] - x), WL[2][0] / (g - 1) + 0.5 * WL[0][0] * (WL[1][0] - x) ** 2])
        qr = np.array([WR[0][0], WR[0][0] * (WR[1][0] - x), WR[2][0] / (g - 1) + 0.5 * WR[0][0] * (WR[1][0] - x) ** 2])
        st, Q, _ = O.riemann_state(g, ql, qr)
        assert st == O.OK
        assert rho[0, k] == pytest.approx(Q[0], rel=1e-9), (x, rho[0, k], Q[0])
    assert smax[0] > 0
