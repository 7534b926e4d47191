"""grp_step_noalloc: the allocation-free single-domain step.

For callers that cannot call cudaMalloc (code inside another framework's
memory pool or allocator hooks, plug-ins whose host owns all device memory,
loops that must not allocate after start-up).  The entry point keeps its
scratch in a file-scope device array of the library; the caller passes only
its own input and output buffers.  Its results must equal those of the
allocating entry point (grp_step through a context) on two calls in a row.
This file is collected last on purpose, and must also pass on its own in a
fresh process.
"""
import numpy as np
import pytest

from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, SMOOTH_TOL, _rel

pytestmark = pytest.mark.gpu


def _context_two_steps(prob, avg, lm, lp):
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_launch(grprec.GRP_LAUNCH_FLAT)
    s.set_initial(avg, lm, lp)
    g0 = s.get_state()[1].copy()
    out = []
    for _ in range(2):
        s.step(1)
        a, g, t = s.get_state()
        out.append((a.copy(), g.copy(), float(t[0])))
    s.close()
    return g0, out


CASES = {
    # periodic smooth runs (smooth tolerance)
    "advection_sine_M2": (lambda: I.advection_sine(300, M=2), SMOOTH_TOL),
    "advection_sine_M3": (lambda: I.advection_sine(257, M=3), SMOOTH_TOL),
    "euler_wave_M1": (lambda: I.euler_wave(500, 1), SMOOTH_TOL),
    "euler_wave_M2": (lambda: I.euler_wave(500, 2), SMOOTH_TOL),
    "euler_wave_M3": (lambda: I.euler_wave(333, 3), SMOOTH_TOL),
    "euler_wave_M4": (lambda: I.euler_wave(400, 4), SMOOTH_TOL),
    # gamma other than 7/5 takes the generic-gamma kernels
    "euler_wave_gamma53_M2": (lambda: I.euler_wave(256, 2, gamma=5.0 / 3.0), SMOOTH_TOL),
    # transmissive shock tubes (discontinuous tolerance; repair rounds run)
    "sod_M1": (lambda: I.sod(513, M=1), DISC_TOL),
    "sod_M2": (lambda: I.sod(777, M=2), DISC_TOL),
    "sod_M4": (lambda: I.sod(640, M=4), DISC_TOL),
    "sod_gamma53_M3": (lambda: I.sod(300, M=3, gamma=5.0 / 3.0), DISC_TOL),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_the_allocating_entry_point_on_two_calls(case):
    torch = pytest.importorskip("torch")
    from paper_2602_21911_gb300 import grprec
    make, tol = CASES[case]
    prob, avg, lm, lp = make()
    g0, ref = _context_two_steps(prob, avg, lm, lp)
    dev = torch.device("cuda", 0)
    a_in = torch.tensor(avg, device=dev)
    i_in = torch.tensor(g0, device=dev)
    a_out, i_out = torch.empty_like(a_in), torch.empty_like(i_in)
    t = 0.0
    for k in range(2):
        t, status = grprec.grp_step_noalloc(prob, a_in, i_in, a_out, i_out, t)
        assert status == 0
        ra, ri, rt = ref[k]
        assert _rel(a_out.cpu().numpy(), ra).max() <= tol
        assert _rel(i_out.cpu().numpy(), ri).max() <= tol
        assert t == pytest.approx(rt, rel=1e-15)
        a_in, a_out = a_out, a_in            # second call starts from the first's output
        i_in, i_out = i_out, i_in


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2602_21911_gb300 import grprec
    N = grprec.GRP_NOALLOC_MAX_CELLS + 1
    prob, avg, lm, lp = I.euler_wave(N, 2)
    buf = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(grprec.GrpError, match="invalid argument"):
        grprec.grp_step_noalloc(prob, buf, buf.clone(), buf.clone(), buf.clone(), 0.0)
