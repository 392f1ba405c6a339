"""Pins of the oracle's bubble model (Sec. III.A: the gas pressure follows the
gas volume; reading B1: isothermal ideal gas, p_g = p0 V0 / V):

* the gas volume of a sub-sampled spherical bubble is 4/3 pi R^3 (the fill
  levels are exact sub-sample counts, so within 1e-3 relative);
* at V = V0 the model gives p_g = p0 exactly;
* Boyle's law with mass conservation: a bubble in a closed liquid box whose
  liquid starts at density 1.02 shrinks until its pressure p0 V0 / V equals
  the liquid's c_s^2 rho_l, rho_l = M / (N - V) with the liquid mass M
  conserved; at sigma = 0 that fixes V_eq = 3 p0 V0 N / (M + 3 p0 V0)."""
import math

import numpy as np
import pytest


def _bubble_state(orc, L=20, R=5.0, rho_l=1.0, sigma=0.0):
    phi = orc.fill(orc.geom("sphere", c=(L / 2 - 0.3, L / 2 + 0.2, L / 2 + 0.1), R=R, sub=16, invert=1), (L, L, L))
    P = orc.params((L, L, L), sigma=sigma, tau=0.8, curv_model=2)
    st = orc.init_state(P, phi)
    if rho_l != 1.0:
        fe = np.array([orc.feq(q, rho_l, np.zeros(3)) for q in range(19)])
        liq = (st.flags & 3) > 0
        st.f[:, liq] = fe[:, None]
        st.mass[st.flags == 1] = rho_l
        st.mass[st.flags == 2] = st.phi[st.flags == 2] * rho_l
    return P, st


def test_gas_volume_of_a_bubble(orc):
    R = 6.0
    P, st = _bubble_state(orc, L=24, R=R)
    assert orc.gas_volume(st) == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=1e-3)


def test_pressure_equals_p0_at_the_initial_volume(orc):
    P, st = _bubble_state(orc)
    V0 = orc.gas_volume(st)
    _, pg = orc.bubble_step(P, st, 1.0 / 3.0, V0)
    assert pg == 1.0 / 3.0


@pytest.mark.slow
def test_boyle_law_with_liquid_mass_conservation(orc):
    P, st = _bubble_state(orc, rho_l=1.02)
    p0 = 1.0 / 3.0
    V0 = orc.gas_volume(st)
    N = st.flags.size
    M = orc.mass(P, st)
    V_eq = 3 * p0 * V0 * N / (M + 3 * p0 * V0)
    assert V_eq < 0.99 * V0  # the bubble must shrink by more than the tolerance below
    vols, pgs, pls = [], [], []
    for k in range(300):
        (st, counts, _, _), pg = orc.bubble_step(P, st, p0, V0)
        if k >= 150:
            vols.append(orc.gas_volume(st))
            pgs.append(pg)
            pls.append(st.f.sum(0)[st.flags == 1].mean() / 3.0)
    assert np.mean(vols) == pytest.approx(V_eq, rel=3e-3)
    assert np.mean(pgs) == pytest.approx(np.mean(pls), rel=2e-3)
    assert abs(orc.mass(P, st) + st.lost - M) < 1e-10 * M
