"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times, on outputs the oracle can compute one by one:

* the batched workload (65,536 domains, 500 steps): domains are independent,
  so sampled domains are run alone through the oracle and compared, within
  1e-9 or, for a domain whose own conditioning is worse, within 100 times
  the oracle's response to a one-ulp change of one input value;
* Sod's shock tube on 2^22 cells: after k steps only a window around the
  initial jump has moved, and the oracle on that window (transmissive ends,
  same dx) reproduces it, S_max included; the far field stays the initial
  state."""
import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, _rel, oracle_run

pytestmark = pytest.mark.gpu


def test_batched_full_size_sampled_domains():
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(65536, seed=2602, M=2)
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.step(500)
    a, g, t = s.get_state()
    stats, status = s.get_stats()
    co, io = I.cell_offsets(prob), I.iface_offsets(prob)
    rng = np.random.default_rng(11)
    sample = np.concatenate([[0, 1, 65535], rng.choice(65536, 21, replace=False)])
    plain_ok = 0
    for d in sample:
        p1, a1, m1, l1 = I.batched(65536, seed=2602, M=2, domains=[d])
        S = oracle_run(p1, a1, m1, l1, 500)
        assert status[d] == S.status[0], d
        if S.status[0] not in (O.OK, O.NONPHYSICAL):
            continue
        assert stats[d, 0] == S.stats[0, 0]
        # the oracle's own response to a one-ulp change of one input value
        a1p = a1.copy()
        a1p[0, a1.shape[1] // 2] = np.nextafter(a1p[0, a1.shape[1] // 2], 10.0)
        Sp = oracle_run(p1, a1p, m1, l1, 500)
        sens = _rel(Sp.avg, S.avg).max()
        ga, sa = a[:, co[d]:co[d + 1]], S.avg
        rd = _rel(ga, sa).max()
        gi, si = g[:, io[d]:io[d + 1]], S.iface
        ri = _rel(gi, si).max()
        tol = max(DISC_TOL, 100.0 * sens)
        assert rd <= tol and ri <= tol, (d, rd, ri, sens)
        plain_ok += rd <= DISC_TOL and ri <= DISC_TOL
    assert plain_ok >= 0.9 * len(sample)
    # most of the batch runs all 500 steps; a few domains may freeze
    assert (status == 0).mean() > 0.99


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
