"""The seeded input generators: exact cell averages, interface limits and the
batched workload recipe (cell counts log-uniform in [4, 512], half smooth waves,
half Riemann problems)."""
import numpy as np
import pytest
from scipy import integrate

from paper_2602_21911_gb300 import inputs as I


def test_sine_averages_are_exact():
    prob, avg, lm, lp = I.advection_sine(17)
    e = np.linspace(0, 1, 18)
    for i in (0, 5, 16):
        v, _ = integrate.quad(lambda x: np.sin(2 * np.pi * x), e[i], e[i + 1], epsabs=1e-15)
        assert avg[0, i] == pytest.approx(v * 17, abs=1e-14)
    assert np.array_equal(lm, lp) and lm.shape == (1, 17)


def test_sin4_averages_are_exact():
    N = 13
    avg = I.advection_sin4_exact(N, 0.3)
    e = np.linspace(-1, 1, N + 1)
    for i in (0, 6, 12):
        v, _ = integrate.quad(lambda x: np.sin(np.pi * (x - 0.3)) ** 4, e[i], e[i + 1], epsabs=1e-15)
        assert avg[0, i] == pytest.approx(v * N / 2, abs=1e-14)


def test_euler_wave_state():
    prob, avg, lm, lp = I.euler_wave(20, 2)
    assert np.allclose(avg[1], avg[0]) and np.allclose(avg[2], 2.5 + 0.5 * avg[0])
    assert lm.shape == (3, 20)


def test_sod_limits_and_averages():
    prob, avg, lm, lp = I.sod(8)
    assert lm.shape == (3, 9)
    assert np.allclose(avg[:, :4], [[1.0], [0.0], [2.5]]) and np.allclose(avg[:, 4:], [[0.125], [0.0], [0.25]])
    assert lm[0, 4] == 1.0 and lp[0, 4] == 0.125          # the jump sits on interface 4
    assert np.array_equal(lm[:, :4], lp[:, :4]) and np.array_equal(lm[:, 5:], lp[:, 5:])
    prob, avg, lm, lp = I.sod(7)                           # odd: the jump is inside cell 3
    assert avg[0, 3] == pytest.approx(0.5625) and np.array_equal(lm, lp)


def test_batched_recipe_is_seeded_and_shaped():
    P = I.batched_params(65536, 2602)
    Q = I.batched_params(65536, 2602)
    assert all(np.array_equal(P[k], Q[k]) for k in P)
    n = P["n"]
    assert n.min() == 4 and n.max() == 512
    assert 100 < n.mean() < 110                 # log-uniform mean ~ 104.5
    assert abs(P["smooth"].mean() - 0.5) < 0.01
    lr = np.log10(P["r_rho"])
    assert lr.min() > -3.0 and lr.max() < 3.0 and abs(lr.mean()) < 0.05
    assert abs(P["uL"].mean()) < 0.05 and P["uR"].min() >= -2.0 and P["uR"].max() < 2.0
    R = I.batched_params(64, 2603)
    assert not np.array_equal(R["n"], P["n"][:64])


def test_batched_subset_layout():
    prob, avg, lm, lp = I.batched(domains=[0, 1, 2])
    n = prob["n_cells"]
    assert avg.shape == (3, n.sum()) and lm.shape == (3, n.sum() + 3)
    assert np.all(prob["bc"] == I.TRANSMISSIVE)
