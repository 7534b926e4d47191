"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (flat form, CUDA graphs), on outputs the oracle
can compute one by one:

* the batched workload (65,536 domains, 500 steps) at degrees 1-4: domains
  are independent, so 64 sampled domains are run alone through the oracle and
  compared within 1e-9; the domains listed as out of tolerance
  (tests/out_of_tolerance.py) are checked for their ill-conditioning instead;
* the smooth Euler density wave on 8192 cells (the largest grid of its
  convergence sweep), 200 steps at degrees 1-4, within 1e-11;
* Sod's shock tube on 2^22 cells: after k steps only a window around the
  initial jump has moved, and the oracle on that window (transmissive ends,
  same dx) reproduces it, S_max included; the far field stays the initial
  state."""
import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from out_of_tolerance import FULL_BATCH, check_exempt
from parity import DISC_TOL, SMOOTH_TOL, _rel, check_parity, oracle_run

pytestmark = pytest.mark.gpu

_rng = np.random.default_rng(11)
SAMPLE = np.concatenate([[0, 1, 65535], _rng.choice(65536, 21, replace=False), _rng.choice(65536, 40, replace=False)])


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_batched_full_size_sampled_domains(M):
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(65536, seed=2602, M=M)
    s = grprec.Solver(prob)
    s.set_launch(grprec.GRP_LAUNCH_FLAT)
    s.set_graph(5)
    s.set_initial(avg, lm, lp)
    s.step(500)
    a, g, t = s.get_state()
    stats, status = s.get_stats()
    s.close()
    co, io = I.cell_offsets(prob), I.iface_offsets(prob)
    listed = FULL_BATCH[M]
    report = []
    for d in SAMPLE:
        p1, a1, m1, l1 = I.batched(65536, seed=2602, M=M, domains=[d])
        S = oracle_run(p1, a1, m1, l1, 500)
        assert status[d] == S.status[0], d
        if S.status[0] not in (O.OK, O.NONPHYSICAL):
            continue
        assert stats[d, 0] == S.stats[0, 0]
        rd = _rel(a[:, co[d]:co[d + 1]], S.avg).max()
        ri = _rel(g[:, io[d]:io[d + 1]], S.iface).max()
        if int(d) in listed:
            # out of tolerance: the oracle's own response to a one-ulp change
            # of one input value must show the ill-conditioning
            ap = a1.copy()
            ap[0, a1.shape[1] // 2] = np.nextafter(ap[0, a1.shape[1] // 2], 10.0)
            sens = _rel(oracle_run(p1, ap, m1, l1, 500).avg, S.avg).max()
            check_exempt(sens, DISC_TOL, "batch domain %d at degree %d" % (d, M))
            report.append((int(d), max(rd, ri), sens))
            continue
        assert rd <= DISC_TOL and ri <= DISC_TOL, (d, rd, ri)
    print("degree %d, listed out of tolerance (domain, GPU - oracle, oracle one-ulp response):" % M, report)
    # most of the batch runs all 500 steps; a few domains may freeze
    assert (status == 0).mean() > 0.99


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_euler_wave_8192_cells(M):
    prob, avg, lm, lp = I.euler_wave(8192, M)
    check_parity(prob, avg, lm, lp, 200, SMOOTH_TOL)


def test_sod_2pow22_window():
    from paper_2602_21911_gb300 import grprec
    N, k, W = 2 ** 22, 200, 1024
    prob, avg, lm, lp = I.sod(N, M=2)
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.step(k)
    a, g, t = s.get_state()
    dx = 1.0 / N
    c0 = N // 2 - W
    pw, aw, mw, lw = I.riemann_problem(2 * W, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), M=2,
                                       x0=0.5 - W * dx, x1=0.5 + W * dx)
    assert pw["x_right"][0] - pw["x_left"][0] == 2 * W * dx
    S = oracle_run(pw, aw, mw, lw, k)
    assert S.status[0] == O.OK and t[0] == pytest.approx(S.t[0], rel=1e-13)
    ga = a[:, c0:c0 + 2 * W]
    rd = _rel(ga, S.avg).max()
    assert rd <= DISC_TOL, rd
    # the far field still holds the initial states (up to round-off of the
    # conserved/primitive round trip in the interface data)
    far = np.r_[0:c0 - 8, c0 + 2 * W + 8:N]
    assert np.abs(a[:, far] - avg[:, far]).max() < 1e-13
