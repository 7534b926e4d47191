"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

import oracle as O
from paper_2602_21911_gb300 import inputs as I

SMOOTH_TOL = 1e-11        # max relative cell difference on smooth runs
DISC_TOL = 1e-9           # ... on discontinuous runs


def oracle_run(prob, avg, lm, lp, n_steps, t_end=np.inf, threads=1):
    st, g = O.init_iface(prob["system"], prob.get("lam", 1.0), prob.get("gamma", 1.4), lm, lp)
    S = O.State(prob, avg, g)
    O.run(prob, S, n_steps, t_end=t_end, n_threads=threads)
    return S


def gpu_run(prob, avg, lm, lp, n_steps, t_end=np.inf, solver=None, **kw):
    from paper_2602_21911_gb300 import grprec
    s = solver or grprec.Solver(prob, **kw)
    s.set_initial(np.ascontiguousarray(avg), np.ascontiguousarray(lm), np.ascontiguousarray(lp))
    s.step(n_steps, t_end)
    a, g, t = s.get_state()
    stats, status = s.get_stats()
    return s, a, g, t, stats, status


def _rel(sa, sb):
    """max_i |a_i - b_i| / max_i |b_i| per component (normwise).  The
    denominator is floored at 1e-6 of the largest component magnitude of the
    domain, so that a component that is zero up to round-off (the momentum of
    a fluid at rest) is compared on the scale of the state."""
    mag = np.abs(sb).max(axis=1)
    den = np.maximum(mag, max(1e-6 * mag.max(), 1e-300))
    return np.abs(sa - sb).max(axis=1) / den


def rel_diff(a, b, prob):
    """Per domain and component, over the cell averages."""
    co = I.cell_offsets(prob)
    out = np.zeros((len(co) - 1, a.shape[0]))
    for d in range(len(co) - 1):
        out[d] = _rel(a[:, co[d]:co[d + 1]], b[:, co[d]:co[d + 1]])
    return out


def rel_diff_iface(a, b, prob):
    """Per domain and component, over the interface data."""
    io = I.iface_offsets(prob)
    out = np.zeros((len(io) - 1, a.shape[0]))
    for d in range(len(io) - 1):
        out[d] = _rel(a[:, io[d]:io[d + 1]], b[:, io[d]:io[d + 1]])
    return out


def oracle_ulp_sensitivity(prob, avg, lm, lp, n_steps, t_end=np.inf, seed=0):
    """How far the oracle's own result moves when every input average moves
    by one ulp (seeded signs): the conditioning of the run."""
    rng = np.random.default_rng(seed)
    a0 = oracle_run(prob, avg, lm, lp, n_steps, t_end)
    pert = np.where(rng.random(avg.shape) < 0.5, np.nextafter(avg, -np.inf), np.nextafter(avg, np.inf))
    a1 = oracle_run(prob, pert, lm, lp, n_steps, t_end)
    return float(rel_diff(a1.avg, a0.avg, prob).max())


def oracle_one_value_sensitivity(prob, avg, lm, lp, n_steps, t_end=np.inf):
    """The oracle's response to a one-ulp increase of one input value (the
    density of the middle cell of the first domain)."""
    a0 = oracle_run(prob, avg, lm, lp, n_steps, t_end)
    ap = avg.copy()
    k = I.cell_offsets(prob)[1] // 2
    ap[0, k] = np.nextafter(ap[0, k], np.inf)
    a1 = oracle_run(prob, ap, lm, lp, n_steps, t_end)
    return float(rel_diff(a1.avg, a0.avg, prob).max())


def check_parity(prob, avg, lm, lp, n_steps, tol, t_end=np.inf, exempt=None, **kw):
    """GPU vs oracle after n_steps (or at t_end): statuses and step counts
    exactly, times, averages and interface data within tol per domain and
    component.  exempt: {domain position: label} of domains listed as out of
    tolerance (tests/out_of_tolerance.py); each such domain is checked for
    ill-conditioning instead of the bound.  Returns (oracle state, GPU
    results, largest difference over the domains held to the bound)."""
    from out_of_tolerance import check_exempt
    S = oracle_run(prob, avg, lm, lp, n_steps, t_end)
    s, a, g, t, stats, status = gpu_run(prob, avg, lm, lp, n_steps, t_end, **kw)
    assert np.array_equal(status, S.status), (status, S.status)
    # a frozen (NONPHYSICAL) domain keeps the state of its last step on both sides
    ok = (S.status == O.OK) | (S.status == O.NONPHYSICAL)
    assert ok.any()
    assert np.array_equal(stats[ok, 0].astype(np.int64), S.stats[ok, 0]), "step counts differ"
    held = ok.copy()
    for d, label in (exempt or {}).items():
        held[d] = False
        if ok[d]:
            one = I.split_domains(prob, avg, lm, lp, which=[d])[0]
            check_exempt(oracle_one_value_sensitivity(*one, n_steps, t_end), tol, label)
    assert np.allclose(t[held], S.t[held], rtol=tol, atol=0)   # dt follows S_max of the state
    rd = rel_diff(a, S.avg, prob)[held]
    ri = rel_diff_iface(g, S.iface, prob)[held]
    assert rd.max() <= tol, ("averages", rd.max())
    assert ri.max() <= tol, ("interface data", ri.max())
    return S, (a, g, t, stats, status), rd.max()
