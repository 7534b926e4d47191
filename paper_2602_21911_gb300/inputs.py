"""Seeded synthetic inputs for the GRPrec scheme.

This module only *builds initial data* (cell averages, the one-sided limits of
the initial condition at each interface, and exact solutions where one is
known in closed form).  It holds none of the scheme's arithmetic, and both the
CUDA path and the CPU oracle take their inputs from it.

Every array is float64, component-major (SoA) and concatenated over domains:
``avg[c, cell]`` and ``lim[c, interface]``.  A domain's interface j sits at the
left edge of its cell j; periodic domains have N interfaces, transmissive ones
N + 1.  Workloads follow the paper's tests: the linear advection sine
(Section 4.2), the smooth Euler density wave (Section 4.3), Sod's shock tube
(Section 4.3, Riemann problems) and a batch of short uneven 1D domains like the
vessel and pipe networks that motivate compact stencils (Section 1).
"""
import math

import numpy as np

ADVECTION, EULER = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
TWO_PI = 2.0 * math.pi


def _edges(x0, x1, n):
    dx = (x1 - x0) / n
    return x0 + dx * np.arange(n + 1, dtype=np.float64), dx


def _sin_avg(xl, xr, k, shift=0.0):
    """Exact cell averages of sin(k (x - shift)) over [xl, xr]."""
    return (np.cos(k * (xl - shift)) - np.cos(k * (xr - shift))) / (k * (xr - xl))


def _cons(rho, u, p, gamma):
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def _problem(system, M, cfl, n_cells, x_left, x_right, bc, lam=1.0, gamma=1.4):
    return dict(system=system, lam=lam, gamma=gamma, M=M, cfl=cfl,
                n_cells=np.asarray(n_cells, dtype=np.int32),
                x_left=np.asarray(x_left, dtype=np.float64),
                x_right=np.asarray(x_right, dtype=np.float64),
                bc=np.asarray(bc, dtype=np.int32),
                newton_rtol=1e-12, newton_max_iter=50, guess=0, dt_hold=1)


# --------------------------------------------------------------------------
# Linear advection q_t + q_x = 0 on periodic [0, 1], q0 = sin(2 pi x).
# --------------------------------------------------------------------------
def advection_sine(N, M=2, cfl=0.9, t=0.0):
    e, dx = _edges(0.0, 1.0, N)
    avg = _sin_avg(e[:-1], e[1:], TWO_PI, t)[None, :]
    lim = np.sin(TWO_PI * (e[:-1] - t))[None, :]
    prob = _problem(ADVECTION, M, cfl, [N], [0.0], [1.0], [PERIODIC])
    return prob, avg, lim, lim.copy()


def advection_sine_exact(N, t):
    e, _ = _edges(0.0, 1.0, N)
    return _sin_avg(e[:-1], e[1:], TWO_PI, t)[None, :]


# The paper's convergence test: q0 = sin^4(pi x) on periodic [-1, 1] (Section 4.2).
# sin^4(a) = 3/8 - cos(2a)/2 + cos(4a)/8
def _sin4_avg(xl, xr, t):
    h = xr - xl
    s2 = (np.sin(TWO_PI * (xr - t)) - np.sin(TWO_PI * (xl - t))) / (TWO_PI * h)
    s4 = (np.sin(2 * TWO_PI * (xr - t)) - np.sin(2 * TWO_PI * (xl - t))) / (2 * TWO_PI * h)
    return 0.375 - 0.5 * s2 + 0.125 * s4


def advection_sin4(N, M, cfl=0.9, t=0.0):
    e, dx = _edges(-1.0, 1.0, N)
    avg = _sin4_avg(e[:-1], e[1:], t)[None, :]
    lim = (np.sin(math.pi * (e[:-1] - t)) ** 4)[None, :]
    prob = _problem(ADVECTION, M, cfl, [N], [-1.0], [1.0], [PERIODIC])
    return prob, avg, lim, lim.copy()


def advection_sin4_exact(N, t):
    e, _ = _edges(-1.0, 1.0, N)
    return _sin4_avg(e[:-1], e[1:], t)[None, :]


# --------------------------------------------------------------------------
# The paper's discontinuous advection tests on periodic [-1, 1] (Section 4.2):
# the square wave (1 on [-0.3, 0.3]) and the Jiang-Shu multi-wave profile.
# Averages by Gauss-Legendre quadrature on the smooth pieces of each cell;
# interface data are the one-sided limits.
# --------------------------------------------------------------------------
def _square(x):
    return np.where((x >= -0.3) & (x <= 0.3), 1.0, 0.0)


def _multiwave(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    m = (x >= -0.8) & (x <= -0.6)
    out[m] = np.exp(-math.log(2.0) * (x[m] + 0.7) ** 2 / 0.0009)
    m = (x >= -0.4) & (x <= -0.2)
    out[m] = 1.0
    m = (x >= 0.0) & (x <= 0.2)
    out[m] = 1.0 - np.abs(10.0 * x[m] - 1.0)
    m = (x >= 0.4) & (x <= 0.6)
    out[m] = np.sqrt(np.maximum(1.0 - 100.0 * (x[m] - 0.5) ** 2, 0.0))
    return out


def _piecewise_avg(f, breaks, xl, xr, n_gauss=16):
    """Cell averages of f, integrating each smooth piece separately."""
    xs, ws = np.polynomial.legendre.leggauss(n_gauss)
    out = np.zeros(len(xl))
    for i, (a, b) in enumerate(zip(xl, xr)):
        pts = [a] + [p for p in breaks if a < p < b] + [b]
        acc = 0.0
        for u, v in zip(pts[:-1], pts[1:]):
            acc += 0.5 * (v - u) * np.dot(ws, f(0.5 * (v - u) * xs + 0.5 * (u + v)))
        out[i] = acc / (b - a)
    return out


def _advection_profile(N, M, f, breaks, cfl):
    e, dx = _edges(-1.0, 1.0, N)
    avg = _piecewise_avg(f, breaks, e[:-1], e[1:])[None, :]
    eps = 1e-13
    minus = f(e[:-1] - eps)[None, :]            # left limits
    plus = f(e[:-1] + eps)[None, :]             # right limits
    prob = _problem(ADVECTION, M, cfl, [N], [-1.0], [1.0], [PERIODIC])
    return prob, avg, minus, plus


def advection_square(N, M=2, cfl=0.9):
    return _advection_profile(N, M, _square, [-0.3, 0.3], cfl)


def advection_multiwave(N, M=2, cfl=0.9):
    return _advection_profile(N, M, _multiwave, [-0.8, -0.6, -0.4, -0.2, 0.0, 0.1, 0.2, 0.4, 0.6], cfl)


def euler_123(N, M=2, cfl=0.9, gamma=1.4):
    """The 123 problem (Section 4.3): (1, -2, 0.4) | (1, 2, 0.4) at x = 0.5."""
    return riemann_problem(N, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4), M=M, cfl=cfl, xc=0.5, gamma=gamma)


# --------------------------------------------------------------------------
# Euler smooth density wave on periodic [0, 1]: rho = 1 + A sin(2 pi (x - t)),
# u = 1, p = p0; exact solution is the translated wave.
# --------------------------------------------------------------------------
def euler_wave(N, M, cfl=0.9, amp=0.2, p0=1.0, gamma=1.4, t=0.0, bc=PERIODIC):
    e, dx = _edges(0.0, 1.0, N)
    rho_avg = 1.0 + amp * _sin_avg(e[:-1], e[1:], TWO_PI, t)
    avg = np.stack([rho_avg, rho_avg, p0 / (gamma - 1.0) + 0.5 * rho_avg])
    xi = e if bc == TRANSMISSIVE else e[:-1]
    rho_i = 1.0 + amp * np.sin(TWO_PI * (xi - t))
    lim = _cons(rho_i, np.ones_like(rho_i), np.full_like(rho_i, p0), gamma)
    prob = _problem(EULER, M, cfl, [N], [0.0], [1.0], [bc], gamma=gamma)
    return prob, avg, lim, lim.copy()


def euler_wave_exact(N, t, amp=0.2, p0=1.0, gamma=1.4):
    e, _ = _edges(0.0, 1.0, N)
    rho = 1.0 + amp * _sin_avg(e[:-1], e[1:], TWO_PI, t)
    return np.stack([rho, rho, p0 / (gamma - 1.0) + 0.5 * rho])


# --------------------------------------------------------------------------
# Riemann problems on transmissive [x0, x1] (Sod: Section 4.3, at x_c = 0.5).
# --------------------------------------------------------------------------
def _riemann_domain(N, WL, WR, xc, gamma, x0=0.0, x1=1.0):
    """Averages and one-sided interface limits of a piecewise-constant IC."""
    e, dx = _edges(x0, x1, N)
    QL = _cons(*[np.float64(v) for v in WL], gamma)
    QR = _cons(*[np.float64(v) for v in WR], gamma)
    frac_left = np.clip((xc - e[:-1]) / dx, 0.0, 1.0)          # share of each cell left of xc
    avg = QL[:, None] * frac_left[None, :] + QR[:, None] * (1.0 - frac_left)[None, :]
    exact_left = frac_left == 1.0
    exact_right = frac_left == 0.0
    avg[:, exact_left] = QL[:, None]
    avg[:, exact_right] = QR[:, None]
    minus = np.where((e <= xc)[None, :], QL[:, None], QR[:, None])   # left limits
    plus = np.where((e < xc)[None, :], QL[:, None], QR[:, None])     # right limits
    return avg, minus, plus


def sod(N, M=2, cfl=0.9, xc=0.5, gamma=1.4):
    avg, minus, plus = _riemann_domain(N, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), xc, gamma)
    prob = _problem(EULER, M, cfl, [N], [0.0], [1.0], [TRANSMISSIVE], gamma=gamma)
    return prob, avg, minus, plus


def riemann_problem(N, WL, WR, M=2, cfl=0.9, xc=0.5, gamma=1.4, x0=0.0, x1=1.0):
    avg, minus, plus = _riemann_domain(N, WL, WR, xc, gamma, x0, x1)
    prob = _problem(EULER, M, cfl, [N], [x0], [x1], [TRANSMISSIVE], gamma=gamma)
    return prob, avg, minus, plus


# --------------------------------------------------------------------------
# Source terms (Section 2, S(Q) of the balance law).
# --------------------------------------------------------------------------
SOURCE_NONE, SOURCE_LINEAR, SOURCE_GRAVITY = 0, 1, 2


def advection_sine_source(N, kappa, M=2, cfl=0.9):
    """q_t + q_x = kappa q on periodic [0, 1], q0 = sin(2 pi x); the exact
    solution is exp(kappa t) sin(2 pi (x - t))."""
    prob, avg, lm, lp = advection_sine(N, M=M, cfl=cfl)
    return dict(prob, source=SOURCE_LINEAR, source_coef=kappa), avg, lm, lp


def advection_sine_source_exact(N, kappa, t):
    return np.exp(kappa * t) * advection_sine_exact(N, t)


def euler_uniform(N, M, rho=1.3, u=0.4, p=0.9, g=0.0, gamma=1.4, cfl=0.9):
    """A uniform state on periodic [0, 1], under the constant acceleration -g
    when g != 0 (exact solution: rho and p constant, u = u0 - g t)."""
    e, dx = _edges(0.0, 1.0, N)
    Q = _cons(np.float64(rho), np.float64(u), np.float64(p), gamma)
    avg = np.repeat(Q[:, None], N, axis=1)
    lim = np.repeat(Q[:, None], N, axis=1)
    prob = _problem(EULER, M, cfl, [N], [0.0], [1.0], [PERIODIC], gamma=gamma)
    if g != 0.0:
        prob = dict(prob, source=SOURCE_GRAVITY, source_coef=g)
    return prob, avg, lim, lim.copy()


def hydrostatic_polytrope(N, M, g=1.0, K=1.0, rho0=2.0, cfl=0.9, bc=TRANSMISSIVE):
    """Gas at rest in equilibrium with the constant acceleration -g on [0, 1]
    for gamma = 2 and p = K rho^2: dp/dx = -g rho gives the linear density
    rho = rho0 - g x / (2 K), and E = p / (gamma - 1) = K rho^2 is quadratic:
    a steady state of polynomial degree 2 (exact averages, point values at
    the interfaces)."""
    gamma = 2.0
    e, dx = _edges(0.0, 1.0, N)
    slope = -g / (2.0 * K)
    xc = 0.5 * (e[:-1] + e[1:])
    rho_avg = rho0 + slope * xc
    E_avg = K * (rho_avg ** 2 + (slope * dx) ** 2 / 12.0)      # average of K rho^2 over a cell
    avg = np.stack([rho_avg, np.zeros(N), E_avg])
    xi = e if bc == TRANSMISSIVE else e[:-1]
    rho_i = rho0 + slope * xi
    lim = np.stack([rho_i, np.zeros_like(rho_i), K * rho_i ** 2])
    prob = dict(_problem(EULER, M, cfl, [N], [0.0], [1.0], [bc], gamma=gamma),
                source=SOURCE_GRAVITY, source_coef=g)
    return prob, avg, lim, lim.copy()


# --------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea, Flood 2014) applied
# to (seed, domain, draw).  Used only to draw workload parameters.
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix_u01(seed, idx, k):
    """Uniform [0, 1) doubles for integer array idx, draw number k."""
    golden = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        x = (np.uint64(seed & _M64) * golden
             + (np.asarray(idx, dtype=np.uint64) * np.uint64(16) + np.uint64(k + 1)) * golden)
        z = x
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def batched_params(n_domains=65536, seed=2602, n_min=4, n_max=512):
    """Per-domain parameters of the batched workload (documented recipe)."""
    d = np.arange(n_domains, dtype=np.uint64)
    u = [splitmix_u01(seed, d, k) for k in range(7)]
    lo, hi = math.log(n_min), math.log(n_max + 1)
    n = np.clip(np.floor(np.exp(lo + u[0] * (hi - lo))), n_min, n_max).astype(np.int32)
    smooth = u[1] < 0.5
    amp = 0.01 + 0.29 * u[2]
    lr = math.log(1e-3), math.log(1e3)
    r_rho = np.exp(lr[0] + u[3] * (lr[1] - lr[0]))
    r_p = np.exp(lr[0] + u[4] * (lr[1] - lr[0]))
    uL = -2.0 + 4.0 * u[5]
    uR = -2.0 + 4.0 * u[6]
    return dict(n=n, smooth=smooth, amp=amp, r_rho=r_rho, r_p=r_p, uL=uL, uR=uR)


def batched(n_domains=65536, seed=2602, M=2, cfl=0.9, gamma=1.4, domains=None):
    """65,536 independent transmissive Euler domains on [0, 1]; half smooth waves
    rho = 1 + A sin(2 pi x), u = p = 1 with A ~ U(0.01, 0.3), half Riemann
    problems at x = 0.5 with rho_L = p_L = 1, (rho_R, p_R) log-uniform in
    [1e-3, 1e3], u_L, u_R ~ U(-2, 2).  ``domains`` selects a subset (ids kept)."""
    P = batched_params(n_domains, seed)
    ids = np.arange(n_domains) if domains is None else np.asarray(domains)
    n = P["n"][ids]
    avgs, minus, plus = [], [], []
    for j, d in enumerate(ids):
        N = int(n[j])
        if P["smooth"][d]:
            e, dx = _edges(0.0, 1.0, N)
            rho = 1.0 + P["amp"][d] * _sin_avg(e[:-1], e[1:], TWO_PI)
            a = np.stack([rho, rho, 1.0 / (gamma - 1.0) + 0.5 * rho])
            rho_i = 1.0 + P["amp"][d] * np.sin(TWO_PI * e)
            lim = _cons(rho_i, np.ones_like(rho_i), np.ones_like(rho_i), gamma)
            avgs.append(a); minus.append(lim); plus.append(lim)
        else:
            a, mi, pl = _riemann_domain(N, (1.0, P["uL"][d], 1.0),
                                        (P["r_rho"][d], P["uR"][d], P["r_p"][d]), 0.5, gamma)
            avgs.append(a); minus.append(mi); plus.append(pl)
    prob = _problem(EULER, M, cfl, n, np.zeros(len(ids)), np.ones(len(ids)),
                    np.full(len(ids), TRANSMISSIVE), gamma=gamma)
    return prob, np.concatenate(avgs, axis=1), np.concatenate(minus, axis=1), np.concatenate(plus, axis=1)


def split_domains(prob, avg, lim_minus, lim_plus, which=None):
    """The domains of a multi-domain problem as single-domain problems
    (prob, avg, lim_minus, lim_plus), for the domain positions ``which``."""
    co, io = cell_offsets(prob), iface_offsets(prob)
    out = []
    for j in (range(len(prob["n_cells"])) if which is None else which):
        pj = dict(prob)
        for k in ("n_cells", "x_left", "x_right", "bc"):
            pj[k] = np.asarray(prob[k])[j:j + 1].copy()
        c = slice(int(co[j]), int(co[j + 1]))
        f = slice(int(io[j]), int(io[j + 1]))
        out.append((pj, np.ascontiguousarray(avg[:, c]), np.ascontiguousarray(lim_minus[:, f]),
                    np.ascontiguousarray(lim_plus[:, f])))
    return out


def n_ifaces(prob):
    return int(np.sum(prob["n_cells"] + (prob["bc"] == TRANSMISSIVE)))


def cell_offsets(prob):
    return np.concatenate([[0], np.cumsum(prob["n_cells"])]).astype(np.int64)


def iface_offsets(prob):
    return np.concatenate([[0], np.cumsum(prob["n_cells"] + (prob["bc"] == TRANSMISSIVE))]).astype(np.int64)
