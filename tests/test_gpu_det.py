"""GPU DET solver against the oracle: smooth and discontinuous advection,
the Euler density wave (degrees 1-4), the shock tube, GRPrecNL with DET, a
batch of domains, and the graph replay of the DET step."""
import numpy as np
import pytest

from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, SMOOTH_TOL, check_parity

pytestmark = pytest.mark.gpu

DET = 1


def _det(prob, **kw):
    return dict(prob, solver=DET, **kw)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_sine(M):
    prob, avg, lm, lp = I.advection_sine(80, M=M)
    check_parity(_det(prob), avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


def test_square_wave():
    prob, avg, lm, lp = I.advection_square(50, M=3)
    check_parity(_det(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=4.0)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_wave(M):
    prob, avg, lm, lp = I.euler_wave(64, M)
    check_parity(_det(prob), avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


def test_euler_wave_transmissive():
    prob, avg, lm, lp = I.euler_wave(50, 3, bc=I.TRANSMISSIVE)
    check_parity(_det(prob), avg, lm, lp, 50, SMOOTH_TOL)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_sod(M):
    prob, avg, lm, lp = I.sod(200, M=M)
    check_parity(_det(prob), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)


def test_sod_grprecnl():
    prob, avg, lm, lp = I.sod(150, M=2, xc=0.3)
    check_parity(_det(prob, recon=1), avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)


def test_batched_subset():
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 401)[:120])
    check_parity(_det(prob), avg, lm, lp, 25, DISC_TOL)


def test_det_runs_flat_and_graphs_replay_bitwise():
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 257)[:100])
    out = []
    for graph in (0, 16):
        s = grprec.Solver(_det(prob))
        s.set_launch(grprec.GRP_LAUNCH_FUSED, 256, 2048, 4)       # DET keeps the flat form
        assert s.get_launch()["form"] == grprec.GRP_LAUNCH_FLAT
        s.set_graph(graph)
        s.set_initial(avg, lm, lp)
        s.step(32)
        out.append(s.get_state())
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
