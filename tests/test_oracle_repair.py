"""Pins of the oracle's a-posteriori repair (a reading, not in the paper: the
update of Section 2, eq. eq_finite_volume, followed by a MOOD-like check of
each candidate average against a relaxed discrete maximum principle and a
first-order Godunov recomputation of the interfaces of troubled cells).

Every case is built on gas at rest with one pressure, so that the first-order
Godunov flux of any two neighbouring averages is known by hand: the Riemann
problem is a stationary contact, its state at x/t = 0 is the left state, and
its flux carries no mass and no energy.  The high-order fluxes are chosen so
that the candidate averages land where each case wants them, and the
expected results are written out by hand (in the operation order of the
update, so that they compare exactly).  Each case would fail under a
plausible mistake: a wrong neighbour set, a wrong base of the 1 % band, a
missing or extra repair round, a repaired interface recomputed twice, or a
frozen domain that does not report NONPHYSICAL."""
import numpy as np
import pytest

import oracle as O

G = 1.4
E0 = 1.0 / (G - 1.0)                      # energy of unit pressure at rest
P0 = (G - 1.0) * (E0 - 0.5 * 0.0 * 0.0)   # its pressure as the update computes it
# momentum flux of the first-order Godunov state: pressure of the sampled
# left state, which is rebuilt from (rho, 0, P0)
PM = (G - 1.0) * ((P0 / (G - 1.0) + 0.5 * 1.0 * 0.0 * 0.0) - 0.5 * 0.0 * 0.0)
NU = 0.5                                  # dt / dx
DX, DT = 0.1, 0.05


def _state(rho, E=None):
    rho = np.asarray(rho, dtype=np.float64)
    E = np.full_like(rho, E0) if E is None else np.asarray(E, dtype=np.float64)
    return np.stack([rho, np.zeros_like(rho), E])


def _fluxes(mass, energy=None):
    mass = np.asarray(mass, dtype=np.float64)
    energy = np.zeros_like(mass) if energy is None else np.asarray(energy, dtype=np.float64)
    return np.stack([mass, np.full_like(mass, PM), energy], axis=1)


def _cand(avg, F, bc):
    """The update of eq. eq_finite_volume written out: q_i - dt/dx (F_{i+1/2} - F_{i-1/2})."""
    N = avg.shape[1]
    out = np.empty_like(avg)
    for i in range(N):
        jr = (i + 1) % N if bc == O.PERIODIC else i + 1
        out[:, i] = avg[:, i] - DT / DX * (F[jr] - F[i])
    return out


def _run(avg, F, bc, low=None):
    gn = np.zeros_like(F)
    return O.update_repair(G, avg, F, gn, bc, DX, DT, low)


def test_constants():
    assert DT / DX == NU and P0 == PM


def test_density_band_is_one_percent_of_the_larger_bound():
    # cell 2 sees old densities {2.0, 1.5, 1.2}: band [1.2 - 0.02, 2.0 + 0.02]
    rho = [1.0, 2.0, 1.5, 1.2, 1.1]
    avg = _state(rho)
    for target, troubled in ((2.017, False), (2.0195, False), (2.0205, True)):
        s = (target - 1.5) / NU                       # mass flux into cell 2 through interface 2
        F = _fluxes([0, 0, s, 0, 0, 0])
        st, cand, f, g, low, stats = _run(avg, F, O.TRANSMISSIVE)
        assert st == O.OK
        if not troubled:
            # 2.017 lies inside the band only when the band is 1 % of
            # max(|min|, |max|) = 2.0; 1 % of the range (0.8), of the minimum
            # (1.2) or of the cell's own value (1.5) would reject it
            assert np.array_equal(cand, _cand(avg, F, O.TRANSMISSIVE))
            assert not low.any() and stats[O.ST_LOW_ORDER] == 0
        else:
            # both interfaces of cell 2 take the first-order flux (no mass):
            # cells 1, 2, 3 return to their old densities
            assert low.tolist() == [0, 0, 1, 1, 0, 0]
            assert cand[0].tolist() == rho
            assert stats[O.ST_LOW_ORDER] == 2 and stats[O.ST_RS_CALLS] == 2
            # the interface data of a repaired interface: the Godunov state,
            # here the left state of a stationary contact
            assert g[2, 0] == 2.0 and g[3, 0] == 1.5 and g[2, 1] == 0.0 and g[3, 1] == 0.0
            assert np.array_equal(g[[0, 1, 4, 5]], np.zeros((4, 3)))


def test_density_band_lower_bound():
    rho = [1.0, 2.0, 1.5, 1.2, 3.0]
    avg = _state(rho)
    for target, troubled in ((1.1805, False), (1.1795, True)):
        s = (1.5 - target) / NU                       # mass flux out of cell 2 through interface 3
        F = _fluxes([0, 0, 0, s, 0, 0])
        st, cand, f, g, low, stats = _run(avg, F, O.TRANSMISSIVE)
        assert st == O.OK
        if troubled:
            assert low.tolist() == [0, 0, 1, 1, 0, 0] and cand[0].tolist() == rho
        else:
            # cell 3 receives the mass: 1.2 + 0.3195 = 1.5195, inside its band
            # [1.2 - 0.03, 3.0 + 0.03] as well
            assert not low.any()
            assert np.array_equal(cand, _cand(avg, F, O.TRANSMISSIVE))


def test_pressure_band():
    avg = _state([1.0] * 5)
    for dp, troubled in ((0.0099, False), (0.0101, True)):
        # energy flux e through interface 2 moves (g-1) nu e of pressure from
        # cell 1 to cell 2; the band is [1 - 0.01, 1 + 0.01]
        e = dp / ((G - 1.0) * NU)
        F = _fluxes([0] * 6, [0, 0, e, 0, 0, 0])
        st, cand, f, g, low, stats = _run(avg, F, O.TRANSMISSIVE)
        assert st == O.OK
        if troubled:
            # cells 1 and 2 are both troubled; interfaces 1, 2, 3 go first order
            assert low.tolist() == [0, 1, 1, 1, 0, 0]
            assert np.array_equal(cand, avg)
            assert stats[O.ST_LOW_ORDER] == 3
        else:
            assert not low.any()
            assert np.array_equal(cand, _cand(avg, F, O.TRANSMISSIVE))


def test_neighbour_set_at_the_ends_follows_the_boundary_rule():
    rho = [1.0, 1.5, 1.5, 1.5, 3.0]
    avg = _state(rho)
    # raise cell 0 to 2.0 through interface 0
    s = (2.0 - 1.0) / NU
    # periodic: cell 0's neighbours are cells 4 and 1, band [0.97, 3.03]: no repair
    Fp = _fluxes([s, 0, 0, 0, 0])
    st, cand, f, g, low, stats = _run(avg, Fp, O.PERIODIC)
    assert st == O.OK and not low.any()
    assert cand[0].tolist() == [2.0, 1.5, 1.5, 1.5, 2.0]
    # transmissive: the ghost copies cell 0, band [0.985, 1.515]: repaired,
    # and the boundary interface's Godunov state is cell 0 itself
    Ft = _fluxes([s, 0, 0, 0, 0, 0])
    st, cand, f, g, low, stats = _run(avg, Ft, O.TRANSMISSIVE)
    assert st == O.OK
    assert low.tolist() == [1, 1, 0, 0, 0, 0]
    assert cand[0].tolist() == rho
    assert g[0, 0] == 1.0 and g[1, 0] == 1.0


def _cascade(nu_c, N=8):
    """Mass fluxes c on every interface but the first, c + delta there: each
    repair round fixes one cell and uncovers the next."""
    c = nu_c / NU
    delta = 0.05 / NU
    F = _fluxes([c + delta] + [c] * N)
    return _run(_state([1.0] * N), F, O.TRANSMISSIVE)


def test_repair_stops_after_four_rounds():
    st, cand, f, g, low, stats = _cascade(0.05)
    assert st == O.OK
    # rounds 0..3 repair cells 0..3 (interfaces 0..4); the check after round
    # 3 finds cell 4 outside its band, and no fifth round runs
    assert low.tolist() == [1, 1, 1, 1, 1, 0, 0, 0, 0]
    exp = [1.0, 1.0, 1.0, 1.0, 1.0 - NU * (0.05 / NU - 0.0), 1.0, 1.0, 1.0]
    assert cand[0].tolist() == exp
    # an interface repaired in an earlier round is not solved again
    assert stats[O.ST_LOW_ORDER] == 5 and stats[O.ST_RS_CALLS] == 5


def test_a_cell_still_inadmissible_after_the_last_round_freezes_the_domain():
    st, cand, f, g, low, stats = _cascade(1.5)
    assert st == O.NONPHYSICAL
    assert low.tolist() == [1, 1, 1, 1, 1, 0, 0, 0, 0]
    assert cand[0, 4] == 1.0 - NU * (1.5 / NU - 0.0) < 0.0      # kept: the domain freezes on it
    assert (cand[0, :4] == 1.0).all()


def test_a_troubled_cell_next_to_a_first_order_interface_repairs_only_the_other():
    # interface 2 is already first order (as the flux kernel marks a failed
    # GRP); cell 2 is troubled: only interface 3 is recomputed
    rho = [1.0, 2.0, 1.5, 1.2, 3.0]
    avg = _state(rho)
    s = (1.5 - 1.1) / NU                              # cell 2 drops to 1.1, below 1.2 - 0.02
    # (cell 3 receives it: 1.6, inside its band [1.2 - 0.03, 3.0 + 0.03])
    F = _fluxes([0, 0, 0, s, 0, 0])
    st, cand, f, g, low, stats = _run(avg, F, O.TRANSMISSIVE, low=[0, 0, 1, 0, 0, 0])
    assert st == O.OK
    assert low.tolist() == [0, 0, 1, 1, 0, 0]
    assert stats[O.ST_LOW_ORDER] == 1 and stats[O.ST_RS_CALLS] == 1
    assert cand[0].tolist() == rho
