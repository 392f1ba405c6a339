"""Pins of the oracle's conversion step (readings O5-O7 of the rules the paper
cites: precedence of filling over emptying, new interface cells, equal
excess shares) on configurations whose outcome follows from the rules by
counting: a flat interface plane at rest with sigma = 0, where streaming,
the free-boundary condition (Eq. reconstruct gives w_q back at rest) and the
mass exchange leave every cell unchanged, so the only change is the
conversion of the one or two cells given an out-of-range mass.

Geometry (arrays [z][y][x], every axis periodic): liquid at z = 0..2,
interface planes at z = 3 (gas above) and z = 7 (gas below, liquid above
through the wrap), gas at z = 4..6; interface mass 0.5.  A cell of the z = 3
plane has 8 interface neighbours in its plane, 5 liquid neighbours below and
5 gas neighbours above (D3Q19)."""
import numpy as np
import pytest

LIQ, IF, GAS = 1, 2, 4
SHAPE = (8, 6, 6)
ABOVE = [(1, 0, 0), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1)]   # (dz, dy, dx) with c_z = +1
BELOW = [(-1, 0, 0), (-1, 1, 0), (-1, -1, 0), (-1, 0, 1), (-1, 0, -1)]
PLANE = [(0, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0) and abs(dy) + abs(dx) <= 2]


def _plane_state(orc):
    phi = np.zeros(SHAPE)
    phi[0:3] = 1.0
    phi[3] = 0.5
    phi[7] = 0.5
    P = orc.params(SHAPE, sigma=0.0, tau=0.8)
    st = orc.init_state(P, phi)
    assert np.all(st.flags[0:3] == LIQ) and np.all(st.flags[3] == IF) and np.all(st.flags[4:7] == GAS)
    w = np.array([orc.feq(q, 1.0, np.zeros(3)) for q in range(19)])
    fluid = (st.flags & 3) > 0
    assert np.array_equal(st.f[:, fluid], np.repeat(w[:, None], fluid.sum(), 1))
    return P, st


def _at(c, d):
    return tuple((np.array(c) + np.array(d)) % np.array(SHAPE))


def _set_mass(st, c, m):
    st.mass[c] = m
    st.phi[c] = m


def test_plane_at_rest_is_stationary(orc):
    P, st = _plane_state(orc)
    nxt, counts, _, _ = orc.step(P, st)
    assert counts[3:7].sum() == 0
    assert np.array_equal(nxt.flags, st.flags)
    assert np.max(np.abs(nxt.f - st.f)) < 1e-15 and np.max(np.abs(nxt.mass - st.mass)) < 1e-15


def test_filling_cell_shares_its_excess_with_thirteen_receivers(orc):
    """m = 1.01 > (1 + eps) rho: the cell becomes liquid with m = rho = 1; its 5
    gas neighbours become interface with f = feq(1, 0) and m = 0; the excess
    0.01 goes in equal shares to the 13 neighbours that are interface after
    that (8 in the plane, 5 new), none to the liquid below."""
    P, st = _plane_state(orc)
    c = (3, 2, 2)
    _set_mass(st, c, 1.01)
    M0 = orc.mass(P, st)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [1, 0, 5, 0] and counts[8] == 0
    share = 0.01 / 13
    assert nxt.flags[c] == LIQ and abs(nxt.mass[c] - 1.0) < 1e-15
    w = np.array([orc.feq(q, 1.0, np.zeros(3)) for q in range(19)])
    for d in ABOVE:
        a = _at(c, d)
        assert nxt.flags[a] == IF
        assert abs(nxt.mass[a] - share) < 1e-15 and abs(nxt.phi[a] - share) < 1e-15
        assert np.max(np.abs(nxt.f[(slice(None),) + a] - w)) < 1e-16
    for d in PLANE:
        a = _at(c, d)
        assert nxt.flags[a] == IF and abs(nxt.mass[a] - (0.5 + share)) < 1e-15
    for d in BELOW:
        assert nxt.flags[_at(c, d)] == LIQ
    changed = np.argwhere(np.abs(nxt.mass - st.mass) > 1e-12)  # beyond rounding: the cell and its 13 receivers
    assert len(changed) == 1 + 5 + 8
    assert abs(orc.mass(P, nxt) + nxt.lost - M0) < 1e-12 * M0


def test_emptying_cell_turns_liquid_below_into_interface(orc):
    """m = -0.01 < -eps rho: the cell becomes gas (m = 0, phi = 0); its 5 liquid
    neighbours below become interface with m = rho = 1; the excess -0.01 goes
    in equal shares to the 8 plane neighbours and the 5 new cells."""
    P, st = _plane_state(orc)
    c = (3, 3, 1)
    _set_mass(st, c, -0.01)
    M0 = orc.mass(P, st)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [0, 1, 0, 5] and counts[8] == 0
    share = -0.01 / 13
    assert nxt.flags[c] == GAS and nxt.mass[c] == 0.0 and nxt.phi[c] == 0.0
    for d in BELOW:
        a = _at(c, d)
        assert nxt.flags[a] == IF
        assert abs(nxt.mass[a] - (1.0 + share)) < 1e-15 and abs(nxt.phi[a] - (1.0 + share)) < 1e-15
    for d in PLANE:
        assert abs(nxt.mass[_at(c, d)] - (0.5 + share)) < 1e-15
    for d in ABOVE:
        assert nxt.flags[_at(c, d)] == GAS
    assert abs(orc.mass(P, nxt) + nxt.lost - M0) < 1e-12 * M0


def test_filling_beats_an_emptying_neighbour(orc):
    """An emptying cell next to a filling one stays interface (readings O5-O7): only
    the filling cell converts, and the emptying neighbour is one of its 13
    receivers, keeping its own negative mass plus one share."""
    P, st = _plane_state(orc)
    cf, ce = (3, 2, 2), (3, 2, 3)
    _set_mass(st, cf, 1.01)
    _set_mass(st, ce, -0.01)
    M0 = orc.mass(P, st)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [1, 0, 5, 0] and counts[8] == 0
    share = 0.01 / 13
    assert nxt.flags[cf] == LIQ and nxt.flags[ce] == IF
    assert abs(nxt.mass[ce] - (-0.01 + share)) < 1e-15
    for d in BELOW:  # the emptying cell did not convert: nothing below it became interface
        assert nxt.flags[_at(ce, d)] == LIQ
    assert abs(orc.mass(P, nxt) + nxt.lost - M0) < 1e-12 * M0


@pytest.mark.parametrize("m", [1.0009, -0.0009])
def test_masses_inside_the_eps_band_do_not_convert(orc, m):
    """The conversion thresholds are m > (1 + eps) rho and m < -eps rho with
    eps = 1e-3 (readings O5-O7): masses just inside the band leave every type."""
    P, st = _plane_state(orc)
    _set_mass(st, (3, 1, 4), m)
    nxt, counts, _, _ = orc.step(P, st)
    assert counts[3:7].sum() == 0 and np.array_equal(nxt.flags, st.flags)


def test_new_cells_take_the_equilibrium_of_their_fluid_neighbours(orc):
    """With a uniform flow u parallel to the plane the state is still stationary
    (the gas links reconstruct feq(1, u), the exchange terms cancel in pairs);
    a cell made interface from gas starts from feq(rho, u) of its fluid
    neighbours, here feq(1, u), not from rest."""
    P, st = _plane_state(orc)
    u = np.array([0.05, 0.02, 0.0])
    fe = np.array([orc.feq(q, 1.0, u) for q in range(19)])
    fluid = (st.flags & 3) > 0
    st.f[:, fluid] = fe[:, None]
    nxt, counts, _, _ = orc.step(P, st)
    assert counts[3:7].sum() == 0
    assert np.max(np.abs(nxt.f[:, fluid] - fe[:, None])) < 1e-15
    assert np.max(np.abs(nxt.mass - st.mass)) < 1e-15
    c = (3, 4, 1)
    _set_mass(st, c, 1.01)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [1, 0, 5, 0]
    for d in ABOVE:
        a = _at(c, d)
        assert nxt.flags[a] == IF
        assert np.max(np.abs(nxt.f[(slice(None),) + a] - fe)) < 1e-15


def test_normal_weighted_excess_of_a_filling_cell(orc):
    """Reading K1 (Koerner's normal-weighted shares): the plane's normal points
    down into the liquid, n = (0, 0, -1); a filled cell gives with weights
    max(0, -n.c) = max(0, c_z): the 5 new cells above (c_z = 1) get 1/5 of the
    excess each, the 8 in-plane receivers (c_z = 0) nothing."""
    P, st = _plane_state(orc)
    P.excess_rule = 1
    c = (3, 2, 2)
    _set_mass(st, c, 1.01)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [1, 0, 5, 0]
    for d in ABOVE:
        assert abs(nxt.mass[_at(c, d)] - 0.01 / 5) < 1e-15
    for d in PLANE:
        assert abs(nxt.mass[_at(c, d)] - 0.5) < 1e-15
    assert abs(orc.mass(P, nxt) + nxt.lost - orc.mass(P, st)) < 1e-13


def test_normal_weighted_excess_of_an_emptying_cell(orc):
    """An emptied cell (m = -0.01) gives with weights max(0, n.c) = max(0, -c_z):
    its negative excess goes in fifths to the 5 liquid cells below, which
    become interface with m = rho = 1; the in-plane cells keep 0.5."""
    P, st = _plane_state(orc)
    P.excess_rule = 1
    c = (3, 2, 2)
    _set_mass(st, c, -0.01)
    nxt, counts, _, _ = orc.step(P, st)
    assert list(counts[3:7]) == [0, 1, 0, 5]
    for d in BELOW:
        a = _at(c, d)
        assert nxt.flags[a] == IF and abs(nxt.mass[a] - (1.0 - 0.01 / 5)) < 1e-15
    for d in PLANE:
        assert abs(nxt.mass[_at(c, d)] - 0.5) < 1e-15


def test_normal_weighted_rule_falls_back_to_equal_shares(orc):
    """A filled cell whose gas-side neighbours are not interface after the
    conversion would give zero weight to every receiver: equal shares then.
    Here the neighbours above are obstacle cells (no new interface cells), so
    the 8 in-plane cells take 1/8 each."""
    P, st = _plane_state(orc)
    P.excess_rule = 1
    st.flags[4] = 8  # obstacle layer above the plane
    st.phi[4] = 0.0
    c = (3, 2, 2)
    _set_mass(st, c, 1.01)
    nxt, counts, _, _ = orc.step(P, st)
    assert counts[3] == 1 and counts[5] == 0
    for d in PLANE:
        assert abs(nxt.mass[_at(c, d)] - (0.5 + 0.01 / 8)) < 1e-14
