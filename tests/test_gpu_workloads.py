"""The paper's other workloads on the GPU against the oracle (Sections 4.2
and 4.3), with linear GRPrec:

* the Jiang-Shu multi-wave advection test on 100 cells, C = 0.9, to the
  paper's t = 2000 (long-time stability, Section 4.2), compared at t = 20, 200
  and 2000, degrees 1-4;
* the 123 problem (two strong rarefactions, near-vacuum, Section 4.3) on 200
  cells to t = 0.15, degrees 1-4 with C = 0.9 for degrees 1-2 and the
  paper's reduced C = 0.7 for degrees 3-4, with the Toro-Titarev and with
  the DET solver."""
import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, check_parity, rel_diff, rel_diff_iface

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_multiwave_to_t2000(M):
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.advection_multiwave(100, M=M)
    st, g = O.init_iface(O.ADVECTION, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    for t_end in (20.0, 200.0, 2000.0):
        O.run(prob, S, 10 ** 7, t_end=t_end)
        s.step(10 ** 7, t_end)
        a, gi, t = s.get_state()
        stats, status = s.get_stats()
        assert t[0] == S.t[0] == t_end and status[0] == S.status[0] == 0
        assert stats[0, 0] == S.stats[0, 0]
        assert rel_diff(a, S.avg, prob).max() <= DISC_TOL, (t_end, rel_diff(a, S.avg, prob).max())
        assert rel_diff_iface(gi, S.iface, prob).max() <= DISC_TOL
    # t = 2000 is 1000 periods: about 111,000 steps
    assert S.stats[0, 0] > 100000
    s.close()


@pytest.mark.parametrize("solver", [0, 1], ids=["tt", "det"])
@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_123_problem_linear(M, solver):
    cfl = 0.9 if M <= 2 else 0.7
    prob, avg, lm, lp = I.euler_123(200, M=M, cfl=cfl)
    S, (a, g, t, stats, status), rd = check_parity(dict(prob, solver=solver), avg, lm, lp, 10 ** 6, DISC_TOL,
                                                   t_end=0.15)
    assert S.status[0] == O.OK and t[0] == 0.15
    # two rarefactions leave a near-vacuum between them
    assert a[0].min() < 0.02
