"""Pins of the oracle's exact Riemann solver, derivative Riemann problem,
Cauchy-Kovalevskaya series and single-interface GRP (Toro-Titarev structure,
Section 2) against facts fixed by the conservation law itself: integral
conservation of the self-similar solution, Rankine-Hugoniot and isentropic
relations, Galilean invariance, closed forms for linear advection and for two
rarefactions, and the PDE residual of the produced series."""
import math

import numpy as np
import pytest

import oracle as O

G = 1.4
RNG = np.random.default_rng(7)


def cons(W, g=G):
    r, u, p = W
    return np.array([r, r * u, p / (g - 1) + 0.5 * r * u * u])


def prim(Q, g=G):
    r, m, E = Q
    u = m / r
    return np.array([r, u, (g - 1) * (E - 0.5 * m * u)])


def flux(Q, g=G):
    """Euler flux written from its definition (Section 4.3); complex-safe."""
    r, m, E = Q
    u = m / r
    p = (g - 1) * (E - 0.5 * m * u)
    return np.array([m, m * u + p, u * (E + p)])


def sample(WL, WR, xi):
    """Exact solution at x/t = xi, by Galilean invariance from the x/t = 0 sampler."""
    sh = np.array([0.0, xi, 0.0])
    st, Q, _ = O.riemann_state(G, cons(np.array(WL) - sh), cons(np.array(WR) - sh))
    assert st in (O.OK, O.VACUUM)
    if Q[0] == 0.0:
        return np.zeros(3)
    return cons(prim(Q) + sh)


CASES = [
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),           # shock tube
    ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),            # two strong rarefactions
    ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),         # strong shock
    ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.0950)),  # colliding shocks
    ((0.3, 0.7, 0.2), (2.0, -0.4, 3.0)),
    ((1.0, 1.2, 1.0), (0.9, 1.3, 0.8)),             # supersonic to the right
]


@pytest.mark.parametrize("WL,WR", CASES)
def test_integral_conservation_of_the_fan(WL, WR):
    """F(Q(0)) = F(Q_L) - int_{-inf}^0 (Q(xi) - Q_L) dxi = F(Q_R) + int_0^inf (Q(xi) - Q_R) dxi."""
    QL, QR = cons(WL), cons(WR)
    Q0 = sample(WL, WR, 0.0)
    F0 = flux(Q0) if Q0[0] > 0 else np.zeros(3)
    smax = 40.0
    xs = np.linspace(-smax, 0.0, 40001)
    left = np.array([sample(WL, WR, x) - QL for x in xs])
    xs2 = np.linspace(0.0, smax, 40001)
    right = np.array([sample(WL, WR, x) - QR for x in xs2])
    il = np.trapezoid(left, xs, axis=0)
    ir = np.trapezoid(right, xs2, axis=0)
    scale = 1.0 + np.abs(flux(QL)) + np.abs(flux(QR)) + np.abs(F0)
    assert np.all(np.abs(F0 - (flux(QL) - il)) / scale < 2e-3)
    assert np.all(np.abs(F0 - (flux(QR) + ir)) / scale < 2e-3)


def test_shock_states_satisfy_rankine_hugoniot():
    """Across the right shock of the shock tube, one speed S solves all three
    jump conditions S [Q] = [F(Q)]."""
    WL, WR = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    st, ps, us, _ = O.star_pressure(G, WL, WR)
    Qs = sample(WL, WR, us + 1e-9)            # right star state, just right of the contact
    QR = cons(WR)
    S = (flux(Qs) - flux(QR)) / (Qs - QR)
    assert abs(S[0] - S[1]) < 1e-9 * abs(S[0]) and abs(S[0] - S[2]) < 1e-9 * abs(S[0])
    assert prim(Qs)[2] == pytest.approx(ps, rel=1e-14)


def test_rarefaction_states_keep_entropy_and_riemann_invariant():
    WL, WR = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    st, ps, us, _ = O.star_pressure(G, WL, WR)
    Ws = prim(sample(WL, WR, us - 1e-9))      # left star state
    cL = math.sqrt(G * WL[2] / WL[0])
    cs = math.sqrt(G * Ws[2] / Ws[0])
    assert Ws[2] / Ws[0] ** G == pytest.approx(WL[2] / WL[0] ** G, rel=1e-13)
    assert Ws[1] + 2 * cs / (G - 1) == pytest.approx(WL[1] + 2 * cL / (G - 1), rel=1e-13)
    # inside the fan the sonic state carries the same invariants and u = c
    Wf = prim(sample(WL, WR, 0.3 * (WL[1] - cL) + 0.7 * (us - cs)))
    cf = math.sqrt(G * Wf[2] / Wf[0])
    assert Wf[2] / Wf[0] ** G == pytest.approx(WL[2] / WL[0] ** G, rel=1e-12)
    assert Wf[1] + 2 * cf / (G - 1) == pytest.approx(WL[1] + 2 * cL / (G - 1), rel=1e-12)


def test_equal_states_give_the_state_exactly():
    for _ in range(20):
        W = (RNG.uniform(0.1, 5), RNG.uniform(-3, 3), RNG.uniform(0.1, 5))
        st, ps, us, it = O.star_pressure(G, W, W)
        assert st == O.OK and ps == W[2] and us == W[1]


def test_two_rarefactions_match_closed_form():
    """When both waves are rarefactions the star pressure has a closed form."""
    z = (G - 1) / (2 * G)
    tested = 0
    for _ in range(50):
        WL = (RNG.uniform(0.2, 3), RNG.uniform(-2, -0.2), RNG.uniform(0.2, 3))
        WR = (RNG.uniform(0.2, 3), RNG.uniform(0.2, 2), RNG.uniform(0.2, 3))
        cL, cR = math.sqrt(G * WL[2] / WL[0]), math.sqrt(G * WR[2] / WR[0])
        du = WR[1] - WL[1]
        if 2 * (cL + cR) / (G - 1) <= du:
            continue
        p_tr = ((cL + cR - 0.5 * (G - 1) * du) / (cL * WL[2] ** -z + cR * WR[2] ** -z)) ** (1 / z)
        if p_tr >= min(WL[2], WR[2]):
            continue
        st, ps, us, it = O.star_pressure(G, WL, WR)
        assert st == O.OK
        assert ps == pytest.approx(p_tr, rel=1e-13)
        tested += 1
    assert tested >= 10


@pytest.mark.parametrize("WL,WR", CASES)
def test_root_is_start_independent(WL, WR):
    st, ps, us, it = O.star_pressure(G, WL, WR)
    for f in (0.3, 0.9, 1.1, 4.0):
        st2, p2, u2, _ = O.star_pressure(G, WL, WR, O.GUESS_GIVEN, f * ps)
        assert st2 == O.OK and p2 == pytest.approx(ps, rel=4e-15, abs=1e-300)
    st3, p3, _, _ = O.star_pressure(G, WL, WR, O.GUESS_TRRS)
    assert p3 == pytest.approx(ps, rel=4e-15)


def test_vacuum_generation_is_reported():
    st, *_ = O.star_pressure(G, (1.0, -10.0, 0.4), (1.0, 10.0, 0.4))
    assert st == O.VACUUM


# --------------------------------------------------------------------------- derivative RP
def jacobian(Q):
    """Complex-step Jacobian of the flux definition: exact to rounding."""
    h = 1e-30
    J = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3, dtype=complex)
        e[j] = 1j * h
        J[:, j] = np.imag(flux(Q.astype(complex) + e)) / h
    return J


def test_derivative_rp_matches_numerical_eigendecomposition():
    for _ in range(50):
        W = (RNG.uniform(0.2, 3), RNG.uniform(-3, 3), RNG.uniform(0.2, 3))
        Q0 = cons(W)
        DL, DR = RNG.normal(size=3), RNG.normal(size=3)
        lam, Rm = np.linalg.eig(jacobian(Q0))
        lam, Rm = lam.real, Rm.real
        wl, wr = np.linalg.solve(Rm, DL), np.linalg.solve(Rm, DR)
        w = np.where(lam > 0, wl, np.where(lam < 0, wr, 0.5 * (wl + wr)))
        ref = Rm @ w
        assert np.allclose(O.deriv_rp(G, Q0, DL, DR), ref, rtol=1e-10, atol=1e-10)


def test_derivative_rp_equal_data():
    Q0 = cons((1.0, 0.3, 2.0))
    D = RNG.normal(size=3)
    assert np.allclose(O.deriv_rp(G, Q0, D, D), D, atol=1e-14)


# --------------------------------------------------------------------------- CK series
@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("lam", [1.0, -0.7])
def test_ck_advection_is_translation(M, lam):
    qa0 = RNG.normal(size=M + 1)
    q = O.ck_series(O.ADVECTION, lam, G, M, qa0)[:, :, 0]
    for a in range(M + 1):
        for b in range(M + 1 - a):
            assert q[a, b] == pytest.approx(math.comb(a + b, b) * (-lam) ** b * qa0[a + b], abs=1e-13)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_ck_euler_series_solves_the_pde_to_order_M(M):
    """The residual d_tau Q + A(Q) d_x Q of the truncated series is O(eps^M)
    at distance eps from the expansion point."""
    W = (1.3, 0.4, 0.9)
    qa0 = np.zeros((M + 1, 3))
    qa0[0] = cons(W)
    for a in range(1, M + 1):
        qa0[a] = 0.3 * RNG.normal(size=3)
    q = O.ck_series(O.EULER, 0.0, G, M, qa0)

    def residual(x, t):
        Q = sum(q[a, b] * x ** a * t ** b for a in range(M + 1) for b in range(M + 1 - a))
        Qt = sum(b * q[a, b] * x ** a * t ** (b - 1) for a in range(M + 1) for b in range(1, M + 1 - a))
        Qx = sum(a * q[a, b] * x ** (a - 1) * t ** b for a in range(1, M + 1) for b in range(M + 1 - a))
        return Qt + jacobian(Q) @ Qx

    r1 = max(np.abs(residual(1e-2 * c, 1e-2 * s)).max() for c, s in ((1, 0), (0, 1), (0.7, 0.7)))
    r2 = max(np.abs(residual(5e-3 * c, 5e-3 * s)).max() for c, s in ((1, 0), (0, 1), (0.7, 0.7)))
    order = math.log2(r1 / r2)
    assert order > M - 0.3


def test_ck_euler_contact_wave_moves_with_u():
    """u = 1, p = const, m = rho: the series is the translated density."""
    M = 4
    qa0 = np.zeros((M + 1, 3))
    d = RNG.normal(size=M + 1)
    d[0] = 1.2
    qa0[:, 0] = d
    qa0[:, 1] = d
    qa0[:, 2] = 0.5 * d
    qa0[0, 2] += 1.0 / (G - 1)
    q = O.ck_series(O.EULER, 0.0, G, M, qa0)
    for b in range(M + 1):
        assert q[0, b, 0] == pytest.approx((-1) ** b * d[b], abs=1e-12)


# --------------------------------------------------------------------------- one GRP
@pytest.mark.parametrize("M", [1, 2, 3, 4])
@pytest.mark.parametrize("lam", [1.0, -1.0])
def test_grp_advection_flux_is_exact_translation(M, lam):
    trL, trR = RNG.normal(size=M + 1), RNG.normal(size=M + 1)
    dt = 0.37
    st, F, g, it, tr = O.grp_interface(O.ADVECTION, lam, G, M, dt, trL, trR)
    up = trL if lam > 0 else trR
    coef = [up[k] / math.factorial(k) for k in range(M + 1)]
    poly = np.polynomial.Polynomial(coef)
    # q(0, tau) = p(-lam tau); flux = lam / dt * int_0^dt p(-lam tau) dtau
    integ = (poly.integ()(0.0) - poly.integ()(-lam * dt)) / lam
    assert F[0] == pytest.approx(lam * integ / dt, rel=1e-13, abs=1e-14)
    assert g[0] == pytest.approx(poly(-lam * dt), rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_grp_euler_constant_state_is_steady(M):
    Q = cons((0.8, -0.3, 1.7))
    tr = np.zeros((M + 1, 3))
    tr[0] = Q
    st, F, g, it, trn = O.grp_interface(O.EULER, 0.0, G, M, 0.1, tr, tr)
    assert st == O.OK
    assert np.allclose(F, flux(Q), rtol=1e-14) and np.allclose(g, Q, rtol=1e-14)


def test_grp_euler_flux_tends_to_godunov_flux():
    M = 2
    trL = np.zeros((M + 1, 3)); trR = np.zeros((M + 1, 3))
    trL[0], trR[0] = cons((1.0, 0.2, 1.0)), cons((0.5, -0.1, 0.6))
    trL[1:], trR[1:] = 0.1 * RNG.normal(size=(M, 3)), 0.1 * RNG.normal(size=(M, 3))
    Q0 = sample((1.0, 0.2, 1.0), (0.5, -0.1, 0.6), 0.0)
    errs = []
    for dt in (1e-3, 5e-4):
        st, F, g, it, tr = O.grp_interface(O.EULER, 0.0, G, M, dt, trL, trR)
        errs.append(np.abs(F - flux(Q0)).max())
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)


# --------------------------------------------------------------------------- tie reading
def test_stationary_contact_is_not_decided_by_rounding():
    """A contact speed within 1e-10 of the sound-speed scale counts as zero:
    the sampled state is the same for u* = 0 and u* = +-1e-14."""
    WL, WR = (1.0, 0.0, 1.0), (0.5, 0.0, 1.0)           # stationary contact
    s0 = sample(WL, WR, 0.0)
    for eps in (1e-14, -1e-14):
        s1 = sample((1.0, eps, 1.0), (0.5, eps, 1.0), 0.0)
        assert np.allclose(s1, s0, rtol=1e-12, atol=1e-12)
    assert s0[0] == pytest.approx(1.0)                 # ties take the left side


def test_derivative_rp_tie_averages_and_is_continuous_there():
    DL, DR = RNG.normal(size=3), RNG.normal(size=3)
    base = O.deriv_rp(G, cons((1.0, 0.0, 1.0)), DL, DR)
    for eps in (1e-13, -1e-13):
        assert np.allclose(O.deriv_rp(G, cons((1.0, eps, 1.0)), DL, DR), base, rtol=1e-10, atol=1e-10)
    # away from the tie the contact component is upwinded
    up = O.deriv_rp(G, cons((1.0, 1e-3, 1.0)), DL, DR)
    assert not np.allclose(up, base, rtol=1e-6)


def test_nearly_equal_data_give_the_left_state_to_the_jump():
    """Riemann data whose conserved states agree to a relative 2^-49 (each
    component on its own scale, the momentum on sqrt(rho E)): the exact
    solution at x/t = 0 lies within the jump of either state.  This is what
    lets the flux kernel resolve such data as the constant state without a
    Newton solve; here the oracle's full Newton solver is the judge."""
    rng = np.random.default_rng(11)
    eps = 2.0 ** -49
    worst = 0.0
    for _ in range(400):
        W = np.array([rng.uniform(0.05, 5.0), rng.uniform(-2.0, 2.0), rng.uniform(0.05, 5.0)])
        QL = cons(W)
        scale = np.array([QL[0], math.sqrt(QL[0] * QL[2]), QL[2]])
        QR = QL + eps * scale * rng.uniform(-1.0, 1.0, 3)
        st, Q, it = O.riemann_state(G, QL, QR)
        assert st == 0 and it >= 1            # the oracle iterates
        worst = max(worst, float(np.max(np.abs(Q - QL) / scale)))
    assert worst <= 4.0 * eps, worst
