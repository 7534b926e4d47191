"""The op-counting build of the oracle (the bench's roofline numerator) counts
without changing a value, and books the equal-data leading Riemann problems
the way the flux kernel resolves them."""
import numpy as np
import pytest

import oracle as O
from oracle import opcount
from paper_2602_21911_gb300 import inputs as I


@pytest.mark.parametrize("M", [1, 2])
def test_counting_build_changes_no_value(M):
    prob, avg, lm, lp = I.euler_wave(64, M)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    plain = O.State(prob, avg, g)
    O.run(prob, plain, 20)
    # the counting build on the same data: its own state object
    import ctypes
    from oracle import _f64, _ip, _dp
    counted = O.State(prob, avg, g)
    L = ctypes.CDLL(opcount.build())
    L.or_run.argtypes = O.lib().or_run.argtypes
    n = np.ascontiguousarray(prob["n_cells"], dtype=np.int32)
    bc = np.ascontiguousarray(prob["bc"], dtype=np.int32)
    rc = L.or_run(prob["system"], 1.0, 1.4, M, prob["cfl"], len(n), _ip(n), _dp(_f64(prob["x_left"])),
                  _dp(_f64(prob["x_right"])), _ip(bc), 1e-12, 50, 0, 1, _dp(counted.avg), _dp(counted.iface),
                  _dp(counted.t), _ip(counted.nstep), _dp(counted.dt_prev), _ip(counted.status), 20,
                  float("inf"), counted.stats.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), None, 1)
    assert rc == 0
    assert np.array_equal(counted.avg, plain.avg)
    assert np.array_equal(counted.iface, plain.iface)


def test_equal_data_are_booked_for_the_interpolating_degree_only():
    """Degree 2 interpolates the interface data: on the smooth periodic wave
    every leading Riemann problem has equal data (one per cell-update) and
    their Newton work leaves the flux count; with degree 1 the two traces
    differ, and only the rare interface whose traces agree by chance counts."""
    for M, expect_all in ((1, False), (2, True)):
        prob, avg, lm, lp = I.euler_wave(64, M)
        st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
        counts, updates, neq = opcount.count(prob, avg, g, 10)
        if expect_all:
            assert neq == updates
            assert sum(counts["rs_equal"].values()) > 0
        else:
            assert neq < 0.05 * updates
