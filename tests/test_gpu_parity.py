"""GPU (C-ABI library) against the CPU oracle on the same seeded inputs.

Tolerances: max relative cell difference 1e-11 on smooth runs and 1e-9 on
discontinuous runs, per domain and component, for the averages and the
interface data; step counts and statuses must agree exactly."""
import numpy as np
import pytest

import oracle as O
from paper_2602_21911_gb300 import inputs as I

from parity import DISC_TOL, SMOOTH_TOL, check_parity, gpu_run, oracle_run, rel_diff

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_advection_sine_to_t1(M):
    prob, avg, lm, lp = I.advection_sine(100, M=M)
    S, G, rd = check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)
    assert S.t[0] == 1.0


def test_advection_many_tiles_ragged_tail():
    prob, avg, lm, lp = I.advection_sine(1000 + 37, M=2)
    check_parity(prob, avg, lm, lp, 60, SMOOTH_TOL)


def test_advection_negative_speed():
    prob, avg, lm, lp = I.advection_sine(77, M=3)
    prob = dict(prob, lam=-1.3)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=0.5)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("N", [64, 100])
def test_euler_wave_to_t1(M, N):
    prob, avg, lm, lp = I.euler_wave(N, M)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0)


def test_euler_wave_transmissive_ragged():
    prob, avg, lm, lp = I.euler_wave(301, 2, bc=I.TRANSMISSIVE)
    check_parity(prob, avg, lm, lp, 80, SMOOTH_TOL)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_sod(M):
    prob, avg, lm, lp = I.sod(256, M=M)
    S, G, rd = check_parity(prob, avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)
    assert S.t[0] == 0.2


def test_sod_odd_grid_many_tiles():
    prob, avg, lm, lp = I.sod(1001)
    check_parity(prob, avg, lm, lp, 120, DISC_TOL)


def test_batched_subset_100_steps():
    ids = np.arange(0, 65536, 173)[:300]
    prob, avg, lm, lp = I.batched(domains=ids)
    S, G, rd = check_parity(prob, avg, lm, lp, 100, DISC_TOL)


@pytest.mark.parametrize("M", [1, 3, 4])
def test_batched_subset_other_degrees(M):
    """The batch at the degrees bench.py also reports (150 domains, 100 steps);
    at degree 4 two domains of this subset are listed as out of tolerance."""
    from out_of_tolerance import BATCH_SUBSET_M4
    ids = np.arange(0, 65536, 331)[:150]
    prob, avg, lm, lp = I.batched(M=M, domains=ids)
    pos = {int(np.flatnonzero(ids == d)[0]): "batch subset domain %d at degree 4" % d for d in BATCH_SUBSET_M4}
    check_parity(prob, avg, lm, lp, 100, DISC_TOL, exempt=pos if M == 4 else None)


def test_batched_stats_agree():
    ids = np.arange(0, 65536, 997)[:60]
    prob, avg, lm, lp = I.batched(domains=ids)
    S, (a, g, t, stats, status), rd = check_parity(prob, avg, lm, lp, 60, DISC_TOL)
    ok = S.status == 0
    for k in (O.ST_RS_CALLS, O.ST_RECON_FB, O.ST_LOW_ORDER, O.ST_FLUX_FB):
        assert np.array_equal(stats[ok, k].astype(np.int64), S.stats[ok, k]), k


def test_single_cell_domains_and_tiny_domains():
    """Degenerate grids: one cell (periodic and transmissive), two and three cells."""
    for N in (1, 2, 3):
        prob, avg, lm, lp = I.advection_sine(N, M=2)
        check_parity(prob, avg, lm, lp, 5, SMOOTH_TOL)
        prob, avg, lm, lp = I.sod(N, M=2)
        check_parity(prob, avg, lm, lp, 5, DISC_TOL)


def test_zero_steps_and_finished_domains_do_not_move():
    prob, avg, lm, lp = I.euler_wave(40, 2)
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.step(0)
    a, g, t = s.get_state()
    assert np.array_equal(a, avg) and t[0] == 0.0
    s.step(1000, 0.01)
    a1, g1, t1 = s.get_state()
    assert t1[0] == 0.01
    s.step(5, 0.01)                            # already at t_end: nothing moves
    a2, g2, t2 = s.get_state()
    assert np.array_equal(a1, a2) and np.array_equal(g1, g2)


def test_dt_hold():
    prob, avg, lm, lp = I.euler_wave(200, 2)
    check_parity(dict(prob, dt_hold=5), avg, lm, lp, 60, SMOOTH_TOL)
    ids = np.arange(0, 65536, 411)[:100]
    prob, avg, lm, lp = I.batched(domains=ids)
    check_parity(dict(prob, dt_hold=2), avg, lm, lp, 30, DISC_TOL)


def test_advance_to_and_norms():
    prob, avg, lm, lp = I.euler_wave(128, 3)
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_initial(avg, lm, lp)
    s.advance_to(1.0)
    a, g, t = s.get_state()
    S = oracle_run(prob, avg, lm, lp, 10 ** 6, 1.0)
    assert t[0] == 1.0 and rel_diff(a, S.avg, prob).max() < SMOOTH_TOL
    ex = I.euler_wave_exact(128, 1.0)
    l1, l2, li = s.error_norms(np.ascontiguousarray(ex[0]))
    e = np.abs(S.avg[0] - ex[0])
    assert l1[0] == pytest.approx(e.sum() / 128, rel=1e-6)
    assert li[0] == pytest.approx(e.max(), rel=1e-6)


def test_device_pointers_through_torch():
    torch = pytest.importorskip("torch")
    prob, avg, lm, lp = I.euler_wave(64, 2)
    from paper_2602_21911_gb300 import grprec
    st = torch.cuda.Stream()
    s = grprec.Solver(prob, stream=st.cuda_stream)
    with torch.cuda.stream(st):
        da = torch.tensor(avg, device="cuda").contiguous()
        dm = torch.tensor(lm, device="cuda").contiguous()
        s.set_initial(da, dm, dm)
        s.step(50)
        out = torch.empty_like(da)
        s.get_state(avg=out)
    S = oracle_run(prob, avg, lm, lp, 50)
    assert rel_diff(out.cpu().numpy(), S.avg, prob).max() < SMOOTH_TOL


def test_generic_gamma_path():
    """gamma != 7/5 takes the pow() path of the Riemann solver."""
    prob, avg, lm, lp = I.euler_wave(80, 2, gamma=5.0 / 3.0)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=0.5)
    prob, avg, lm, lp = I.sod(200, M=3, gamma=5.0 / 3.0)
    check_parity(prob, avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2)


BATCH_CONFIGS = [(2, 256, 2048, 8), (2, 128, 256, 1), (2, 256, 700, 3), (2, 128, 4096, 16),
                 (3, 256, 2048, 1), (3, 128, 300, 1), (3, 256, 8192, 1)]


@pytest.mark.parametrize("form,threads,cells,k", BATCH_CONFIGS)
def test_batched_kernels_match_oracle(form, threads, cells, k):
    """The fused persistent kernel (form 2) and the split form (form 3), in
    several launch shapes."""
    ids = np.arange(0, 65536, 211)[:200]
    prob, avg, lm, lp = I.batched(domains=ids)
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_launch(form, threads, cells, k)
    assert s.get_launch()["form"] == form
    check_parity(prob, avg, lm, lp, 37, DISC_TOL, solver=s)


def test_batched_and_flat_kernels_agree():
    ids = np.arange(0, 65536, 97)[:400]
    prob, avg, lm, lp = I.batched(domains=ids)
    from paper_2602_21911_gb300 import grprec
    out = []
    for mode in (grprec.GRP_LAUNCH_FLAT, grprec.GRP_LAUNCH_FUSED, grprec.GRP_LAUNCH_SPLIT):
        s = grprec.Solver(prob)
        s.set_launch(mode, 256, 2048, 8)
        s.set_initial(avg, lm, lp)
        s.step(60)
        out.append(s.get_state())
    # the forms inline the same device functions in different kernels, so FMA
    # contraction may differ: they agree to the discontinuous-run tolerance
    for other in out[1:]:
        assert rel_diff(out[0][0], other[0], prob).max() < DISC_TOL
        assert np.allclose(out[0][2], other[2], rtol=DISC_TOL)


def test_batched_kernel_advection_and_periodic_domains():
    prob, avg, lm, lp = I.advection_sine(96, M=3)
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    s.set_launch(grprec.GRP_LAUNCH_FUSED, 128, 1024, 5)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=0.7, solver=s)
    prob, avg, lm, lp = I.euler_wave(64, 4)
    s = grprec.Solver(prob)
    s.set_launch(grprec.GRP_LAUNCH_FUSED, 256, 2048, 7)
    check_parity(prob, avg, lm, lp, 10 ** 6, SMOOTH_TOL, t_end=1.0, solver=s)
    prob, avg, lm, lp = I.sod(500, M=2)
    s = grprec.Solver(prob)
    s.set_launch(grprec.GRP_LAUNCH_SPLIT, 256, 2048, 1)
    check_parity(prob, avg, lm, lp, 10 ** 6, DISC_TOL, t_end=0.2, solver=s)


def test_launch_configuration_is_validated():
    prob, avg, lm, lp = I.euler_wave(16, 2)
    from paper_2602_21911_gb300 import grprec
    s = grprec.Solver(prob)
    for bad in ((5, 256, 2048, 8), (1, 100, 2048, 8), (1, 256, 10, 8), (1, 256, 2048, 0)):
        with pytest.raises(grprec.GrpError):
            s.set_launch(*bad)
    assert s.get_launch()["form"] == grprec.GRP_LAUNCH_FLAT     # auto: one short domain runs flat


@pytest.mark.parametrize("form,k", [(1, 1), (2, 4), (3, 1)])
def test_graph_replay_is_bitwise_the_direct_launch(form, k):
    """A CUDA graph replays the same kernels with the same arguments, so the
    result, the counters and the launch count equal those of direct launches
    bit for bit (graph of 16 steps; 5 steps, not a multiple of k = 4 in the
    fused form, falls back to direct launches there)."""
    from paper_2602_21911_gb300 import grprec
    ids = np.arange(0, 65536, 173)[:300]
    prob, avg, lm, lp = I.batched(domains=ids)
    out = []
    for graph in (0, 16, 5):
        s = grprec.Solver(prob)
        s.set_launch(form, 256, 2048, k)
        s.set_graph(graph)
        s.set_initial(avg, lm, lp)
        s.step(37)
        s.step(16)
        s.step(19, 0.05)          # a finite t_end: another graph
        a, g, t = s.get_state()
        stats, status = s.get_stats()
        out.append((a, g, t, stats, status, s.launch_count()))
    for other in out[1:]:
        for x, y in zip(out[0][:5], other[:5]):
            assert np.array_equal(x, y)
        assert out[0][5] == other[5]


def test_kernel_timing_through_graphs():
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 64)[:1024])
    res = {}
    for graph in (0, 16):
        s = grprec.Solver(prob)
        s.set_launch(grprec.GRP_LAUNCH_FLAT)
        s.set_graph(graph)
        s.set_initial(avg, lm, lp)
        s.step(16)
        s.set_kernel_timing(True)
        s.step(32)
        ms, n = s.kernel_timing()
        assert n == 32 and ms > 0
        res[graph] = ms / n
    assert 0.5 < res[16] / res[0] < 2.0


def test_autotuner_picks_a_candidate_and_leaves_results_unchanged():
    from paper_2602_21911_gb300 import autotune, grprec
    prob, avg, lm, lp = I.batched(domains=np.arange(0, 65536, 97)[:600])
    s = grprec.Solver(prob)
    best = autotune.tune(prob, avg, lm, lp, warm=2, steps=4, use_cache=False, solver=s)
    assert best in autotune.candidates(prob)
    L = s.get_launch()
    assert (L["form"], L["threads"], L["cells_per_block"], L["steps_per_launch"]) == best
    check_parity(prob, avg, lm, lp, 20, DISC_TOL, solver=s)


def test_no_state_is_read_before_written_on_reused_memory():
    """Device memory handed back to the driver full of non-zero bytes, then a
    new context: results must not depend on what the memory held."""
    torch = pytest.importorskip("torch")
    junk = torch.full((1 << 28,), -1, dtype=torch.int32, device="cuda")     # 1 GiB of 0xFF bytes
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    for prob, avg, lm, lp, tol in ((*I.advection_sine(100, M=2), SMOOTH_TOL),
                                   (*I.euler_wave(64, 2), SMOOTH_TOL),
                                   (*I.sod(100, M=2), DISC_TOL)):
        check_parity(prob, avg, lm, lp, 40, tol)


def test_interpolating_degrees_resolve_smooth_riemann_data_without_newton():
    """Degrees 2 and 4 interpolate the interface data, so on smooth periodic
    flow both traces at every interface are the interface datum itself: every
    leading Riemann problem has equal data and takes no Newton iteration.  The
    least-squares degrees 1 and 3 give two different traces and iterate.  The
    oracle runs Newton everywhere; the results agree either way."""
    from paper_2602_21911_gb300 import grprec
    for M, no_newton in ((1, False), (2, True), (3, False), (4, True)):
        prob, avg, lm, lp = I.euler_wave(100, M)
        S, (a, g, t, stats, status), rd = check_parity(prob, avg, lm, lp, 60, SMOOTH_TOL)
        assert S.stats[:, O.ST_NEWTON_SUM].sum() > 0
        n = int(stats[:, grprec.STAT_NEWTON_SUM].sum())
        assert (n == 0) == no_newton, (M, n)
