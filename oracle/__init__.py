"""ORACLE — test infrastructure only.

A plain FP64 CPU implementation of the FV+GRPrec scheme of arXiv 2602.21911
(GRPrec reconstruction, Section 3.1; exact leading Riemann problem, derivative
Riemann problems, Cauchy-Kovalevskaya series and Gauss flux of the Toro-Titarev
GRP solver, Section 2; the conservative update, Section 2; the CFL rule,
Section 4.1), plus the FP64 reference of the learned Newton guess network in
``oracle.mlp``.  It shares no code with the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ADVECTION, EULER = 0, 1
RECON_GRPREC, RECON_GRPRECNL = 0, 1
SOLVER_TT, SOLVER_DET = 0, 1
SOURCE_NONE, SOURCE_LINEAR, SOURCE_GRAVITY = 0, 1, 2
PERIODIC, TRANSMISSIVE = 0, 1
GUESS_PVRS, GUESS_TRRS, GUESS_GIVEN = 0, 1, 2
OK, NEWTON_NO_CONV, VACUUM, NONPHYSICAL = 0, 1, 2, 3
ST_STEPS, ST_NEWTON_SUM, ST_NEWTON_MAX, ST_RECON_FB, ST_FLUX_FB, ST_RS_CALLS, ST_LOW_ORDER = range(7)
NSTATS = 7

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_longlong)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_recon.argtypes = [ctypes.c_int, _D, _D, _D]
        L.or_star_pressure.argtypes = [ctypes.c_double, _D, _D, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, _D]
        L.or_riemann_state.argtypes = [ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_int, _D, _I]
        L.or_deriv_rp.argtypes = [ctypes.c_double, _D, _D, _D, _D]
        L.or_deriv_rp.restype = None
        L.or_ck_series.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D]
        L.or_ck_series.restype = None
        L.or_grp_interface.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, _D, _D, _I, _I]
        L.or_init_iface.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    _D, _D, _D]
        L.or_run.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.c_double, ctypes.c_int, _I, _D, _D, _I, ctypes.c_double,
                             ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _I, _D, _I,
                             ctypes.c_int, ctypes.c_double, _L, _D, ctypes.c_int]
        L.or_run_ex.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int, _I, _D, _D, _I, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _I, _D, _I,
                                ctypes.c_int, ctypes.c_double, _L, _D, ctypes.c_int]
        L.or_run_solver.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int, _I, _D, _D, _I,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _I,
                                    _D, _I, ctypes.c_int, ctypes.c_double, _L, _D, ctypes.c_int]
        L.or_recon_nl.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D, _D]
        L.or_run_full.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  _I, _D, _D, _I, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  _D, _D, _D, _I, _D, _I, ctypes.c_int, ctypes.c_double, _L, _D, ctypes.c_int]
        L.or_ck_series_src.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, _D, _D]
        L.or_ck_series_src.restype = None
        L.or_char_basis.argtypes = [ctypes.c_double, _D, _D, _D]
        L.or_update_repair.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _D, _D, _D, ctypes.c_char_p, _D, _L]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def recon_nl(M, d7, dx):
    """GRPrecNL monomial coefficients and the weights (beta_L, beta_C, beta_R)
    (Sections 3.3-3.4); d7 = (q_{i-1}, q_i, q_{i+1}, g_{i-3/2}, g_{i-1/2},
    g_{i+1/2}, g_{i+3/2})."""
    d7 = _f64(d7)
    coef, beta = np.zeros(5), np.zeros(3)
    if lib().or_recon_nl(M, _dp(d7), float(dx), _dp(coef), _dp(beta)) != 0:
        raise ValueError("bad degree")
    return coef[:M + 1], beta


def char_basis(gamma, Q):
    """(R, L): right eigenvectors (columns) of the Euler flux Jacobian at Q and L = R^-1."""
    Q = _f64(Q)
    R, L = np.zeros(9), np.zeros(9)
    lib().or_char_basis(float(gamma), _dp(Q), _dp(R), _dp(L))
    return R.reshape(3, 3), L.reshape(3, 3)


def update_repair(gamma, avg, flux, gnew, bc, dx, dt, low=None):
    """The update and a-posteriori repair of one Euler step on given fluxes
    (Section 2, eq. eq_finite_volume; the repair is a reading, not in the
    paper).  avg [3, N]; flux, gnew [nif, 3] high-order fluxes and interface
    data; low [nif] (1 = already first order).  Returns (status, cand [3, N],
    flux, gnew, low, stats) after the repair."""
    avg = _f64(avg)
    N = avg.shape[1]
    nif = N if bc == PERIODIC else N + 1
    f = _f64(flux).reshape(nif, 3).copy()
    g = _f64(gnew).reshape(nif, 3).copy()
    lo = np.zeros(nif, dtype=np.int8) if low is None else np.ascontiguousarray(low, dtype=np.int8).copy()
    cand = np.zeros((3, N))
    stats = np.zeros(NSTATS, dtype=np.int64)
    st = lib().or_update_repair(float(gamma), N, int(bc), float(dx), float(dt), _dp(avg), _dp(f), _dp(g),
                                lo.ctypes.data_as(ctypes.c_char_p), _dp(cand), stats.ctypes.data_as(_L))
    return st, cand, f, g, lo, stats


def recon(M, qbar, g):
    """GRPrec monomial coefficients c_k of p(xi) = sum c_k xi^k (Section 3.1)."""
    qbar, g = _f64(qbar), _f64(g)
    coef = np.zeros(5)
    if lib().or_recon(M, _dp(qbar), _dp(g), _dp(coef)) != 0:
        raise ValueError("reconstruction system is singular")
    return coef[:M + 1]


def star_pressure(gamma, WL, WR, guess_kind=GUESS_PVRS, guess=0.0, rtol=1e-12, max_iter=50):
    """(status, p*, u*, iterations) of the exact ideal-gas Riemann problem."""
    out = np.zeros(3)
    st = lib().or_star_pressure(gamma, _dp(_f64(WL)), _dp(_f64(WR)), guess_kind, guess, rtol,
                                max_iter, _dp(out))
    return st, out[0], out[1], int(out[2])


def riemann_state(gamma, QL, QR, rtol=1e-12, max_iter=50):
    """(status, Q at x/t=0, iterations) for conserved states QL, QR."""
    Q = np.zeros(3)
    it = ctypes.c_int(0)
    st = lib().or_riemann_state(gamma, _dp(_f64(QL)), _dp(_f64(QR)), rtol, max_iter, _dp(Q),
                                ctypes.byref(it))
    return st, Q, it.value


def deriv_rp(gamma, Q0, DL, DR):
    D = np.zeros(3)
    lib().or_deriv_rp(gamma, _dp(_f64(Q0)), _dp(_f64(DL)), _dp(_f64(DR)), _dp(D))
    return D


def ck_series(system, lam, gamma, M, qa0):
    """qa0[a, c] = q_{a,0}; returns q[a, b, c] for a+b <= M (zeros elsewhere)."""
    C = 3 if system == EULER else 1
    qa0 = _f64(np.reshape(qa0, (M + 1, C)))
    out = np.zeros((M + 1, M + 1, C))
    lib().or_ck_series(system, lam, gamma, M, _dp(qa0), _dp(out))
    return out


def ck_series_src(system, lam, gamma, M, source, coef, qa0):
    """ck_series with a source term S(Q) (SOURCE_LINEAR: S = coef q for
    advection; SOURCE_GRAVITY: S = (0, -coef rho, -coef m) for Euler)."""
    C = 3 if system == EULER else 1
    qa0 = _f64(np.reshape(qa0, (M + 1, C)))
    out = np.zeros((M + 1, M + 1, C))
    lib().or_ck_series_src(system, lam, gamma, M, source, float(coef), _dp(qa0), _dp(out))
    return out


def grp_interface(system, lam, gamma, M, dt, trL, trR, rtol=1e-12, max_iter=50,
                  guess_kind=GUESS_PVRS):
    """(status, flux[C], g_new[C], iterations, truncated) for traces tr[k, c]."""
    C = 3 if system == EULER else 1
    trL = _f64(np.reshape(trL, (M + 1, C)))
    trR = _f64(np.reshape(trR, (M + 1, C)))
    flux, gnew = np.zeros(C), np.zeros(C)
    it, tr = ctypes.c_int(0), ctypes.c_int(0)
    st = lib().or_grp_interface(system, lam, gamma, M, dt, _dp(trL), _dp(trR), rtol, max_iter,
                                guess_kind, _dp(flux), _dp(gnew), ctypes.byref(it), ctypes.byref(tr))
    return st, flux, gnew, it.value, tr.value


def init_iface(system, lam, gamma, lim_minus, lim_plus):
    """Initial interface data: leading Riemann state of the one-sided IC limits."""
    lm, lp = _f64(lim_minus), _f64(lim_plus)
    n = lm.shape[-1]
    out = np.zeros_like(lm)
    st = lib().or_init_iface(system, lam, gamma, n, _dp(lm), _dp(lp), _dp(out))
    return st, out


class State:
    """Mutable per-run state of a set of domains (same layout as the library)."""

    def __init__(self, prob, avg, iface):
        D = len(prob["n_cells"])
        self.avg = _f64(avg).copy()
        self.iface = _f64(iface).copy()
        self.t = np.zeros(D)
        self.nstep = np.zeros(D, dtype=np.int32)
        self.dt_prev = np.zeros(D)
        self.status = np.zeros(D, dtype=np.int32)
        self.stats = np.zeros((D, NSTATS), dtype=np.int64)


def run(prob, state, n_steps, t_end=np.inf, dt_fixed=None, n_threads=1):
    """Advance ``state`` in place by n_steps or to t_end (Section 2 update).

    ``prob`` keys: system, lam, gamma, M, cfl, n_cells, x_left, x_right, bc,
    newton_rtol, newton_max_iter, guess, dt_hold, recon, solver, source and
    source_coef (the last four optional).
    """
    n_cells = np.ascontiguousarray(prob["n_cells"], dtype=np.int32)
    xl = _f64(prob["x_left"])
    xr = _f64(prob["x_right"])
    bc = np.ascontiguousarray(prob["bc"], dtype=np.int32)
    dtf = None
    if dt_fixed is not None:
        dtf = _f64(dt_fixed)
        assert len(dtf) >= n_steps
    rc = lib().or_run_full(prob["system"], prob.get("lam", 1.0), prob.get("gamma", 1.4), prob["M"],
                      prob.get("recon", RECON_GRPREC), prob.get("solver", SOLVER_TT),
                      prob.get("source", SOURCE_NONE), float(prob.get("source_coef", 0.0)),
                      prob["cfl"], len(n_cells), _ip(n_cells), _dp(xl), _dp(xr), _ip(bc),
                      prob.get("newton_rtol", 1e-12), prob.get("newton_max_iter", 50),
                      prob.get("guess", GUESS_PVRS), prob.get("dt_hold", 1),
                      _dp(state.avg), _dp(state.iface), _dp(state.t), _ip(state.nstep),
                      _dp(state.dt_prev), _ip(state.status), n_steps, float(t_end),
                      state.stats.ctypes.data_as(_L), _dp(dtf) if dtf is not None else None,
                      n_threads)
    if rc != 0:
        raise ValueError("oracle run rejected its arguments")
    return state


def cpu_threads():
    return len(os.sched_getaffinity(0))
