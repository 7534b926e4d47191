"""Algorithmic FP64 operation counts of the scheme (measurement only).

Builds oracle/opcount.cpp -- the oracle compiled as C++ with a counting
scalar -- and runs it on a sample of a workload.  Every +, -, *, /, sqrt and
pow with at least one operand derived from the state counts one flop;
operations on constants only, negation, fabs and comparisons count none.
The per-cell-update figure is the roofline numerator of the bench.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "opcount.cpp")
LIB = os.path.join(HERE, "libopcount.so")
KINDS = ("add", "mul", "div", "sqrt", "pow")
PHASES = ("cfl", "flux", "update", "rs_equal")
# Algorithmic flops of resolving one leading Riemann problem as equal data
# (the test of the traces: 3 differences, 2 sums, 5 products; admissibility:
# 3 products; the primitive state of the common trace: 1 division, 5 more)
EQUAL_DATA_FLOPS = 19


def build(force=False):
    deps = [SRC, os.path.join(HERE, "grprec_oracle.c"), os.path.join(HERE, "grprec_oracle.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(map(os.path.getmtime, deps)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17",
                           "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


def count(prob, avg, iface, n_steps):
    """Counts (dict) of one single-threaded run of n_steps from (avg, iface),
    the number of cell-updates performed and the number of leading Riemann
    problems with equal data (their operations are in counts["rs_equal"])."""
    import oracle as O
    L = ctypes.CDLL(build())
    L.or_opcount.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    L.or_opcount_reset.argtypes = []
    S = O.State(prob, avg, iface)
    L.or_run.argtypes = O.lib().or_run.argtypes
    L.or_opcount_reset()
    n = np.ascontiguousarray(prob["n_cells"], dtype=np.int32)
    xl = np.ascontiguousarray(prob["x_left"], dtype=np.float64)
    xr = np.ascontiguousarray(prob["x_right"], dtype=np.float64)
    bc = np.ascontiguousarray(prob["bc"], dtype=np.int32)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    rc = L.or_run(prob["system"], prob.get("lam", 1.0), prob.get("gamma", 1.4), prob["M"], prob["cfl"],
                  len(n), n.ctypes.data_as(I), xl.ctypes.data_as(D), xr.ctypes.data_as(D),
                  bc.ctypes.data_as(I), prob.get("newton_rtol", 1e-12), prob.get("newton_max_iter", 50),
                  prob.get("guess", 0), prob.get("dt_hold", 1), S.avg.ctypes.data_as(D),
                  S.iface.ctypes.data_as(D), S.t.ctypes.data_as(D), S.nstep.ctypes.data_as(I),
                  S.dt_prev.ctypes.data_as(D), S.status.ctypes.data_as(I), n_steps, float("inf"),
                  S.stats.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), None, 1)
    assert rc == 0
    out = (ctypes.c_longlong * 21)()
    L.or_opcount(out)
    counts = {ph: dict(zip(KINDS, [int(v) for v in out[5 * i:5 * i + 5]]))
              for i, ph in enumerate(PHASES)}
    updates = int((S.stats[:, 0] * n).sum())
    return counts, updates, int(out[20])


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import oracle as O
    from paper_2602_21911_gb300 import inputs as I
    for name, maker, steps in (
            ("batched M=1 (every 128th domain)", lambda: I.batched(domains=np.arange(0, 65536, 128), M=1), 50),
            ("batched M=2 (every 128th domain)", lambda: I.batched(domains=np.arange(0, 65536, 128)), 50),
            ("batched M=3 (every 128th domain)", lambda: I.batched(domains=np.arange(0, 65536, 128), M=3), 50),
            ("batched M=4 (every 128th domain)", lambda: I.batched(domains=np.arange(0, 65536, 128), M=4), 50),
            ("euler wave N=256 M=1", lambda: I.euler_wave(256, 1), 100),
            ("euler wave N=256 M=2", lambda: I.euler_wave(256, 2), 100),
            ("euler wave N=256 M=3", lambda: I.euler_wave(256, 3), 100),
            ("euler wave N=256 M=4", lambda: I.euler_wave(256, 4), 100),
            ("sod N=1024 M=2", lambda: I.sod(1024, 2), 200),
            ("advection N=256 M=2", lambda: I.advection_sine(256, 2), 100)):
        prob, avg, lm, lp = maker()
        st, g = O.init_iface(prob["system"], 1.0, 1.4, lm, lp)
        c, u, neq = count(prob, avg, g, steps)
        per = {ph: sum(c[ph].values()) / u for ph in PHASES}
        # the flux phase as the product path computes it: equal-data leading
        # Riemann problems resolved by the test instead of Newton
        flux_eq = per["flux"] + neq / u * EQUAL_DATA_FLOPS
        print("%-36s flops/cell-update: total %7.1f  cfl %5.1f  flux %7.1f (equal data resolved: %7.1f, "
              "%.3f per cell-update)  update %6.1f" % (
                  name, sum(per.values()), per["cfl"], per["flux"] + per["rs_equal"], flux_eq,
                  neq / u, per["update"]))
