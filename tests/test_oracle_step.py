"""Pins of the oracle's time step (stream, free-boundary condition, mass
exchange, collision, conversion).

Each check compares the oracle with what physics or the paper fixes: a fluid
at rest stays at rest, uniform flow is stationary, a shear wave decays at
nu k^2 with nu = (tau - 1/2)/3 (Sec. II), total mass is conserved exactly,
no liquid cell touches a gas cell (Sec. II), the Laplace pressure of a
droplet is 2 sigma/R (Sec. II), and the translation test of Tab. advection
(Sec. III.A) reaches the printed error magnitude."""
import os

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _advection_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "advection_table.txt")) if l.strip() and l[0] != "#"]
    return {int(r[0]): dict(u0=float(r[3]), L1=float(r[4]) / 100, L2=float(r[5]) / 100) for r in rows}


def _liquid_box(orc, shape, collision=0, tau=0.8):
    P = orc.params(shape, collision=collision, tau=tau)
    st = orc.init_state(P, np.ones(shape))
    return P, st


@pytest.mark.parametrize("collision", [0, 1])
def test_rest_state_is_stationary(orc, collision):
    P, st = _liquid_box(orc, (5, 6, 7), collision)
    f0 = st.f.copy()
    for _ in range(3):
        st, counts, _, _ = orc.step(P, st)
    assert np.max(np.abs(st.f - f0)) < 1e-16
    assert counts[0] == 5 * 6 * 7


@pytest.mark.parametrize("collision", [0, 1])
def test_uniform_flow_is_stationary(orc, collision):
    P, st = _liquid_box(orc, (4, 5, 6), collision)
    u0 = np.array([0.04, -0.03, 0.02])
    fe = np.array([orc.feq(q, 1.02, u0) for q in range(19)])
    st.f[:] = fe[:, None, None, None]
    for _ in range(3):
        st, _, _, _ = orc.step(P, st)
    assert np.max(np.abs(st.f - fe[:, None, None, None])) < 1e-15


def test_droplet_without_surface_tension_stays_at_rest(orc):
    """With sigma = 0 and f = feq(1, 0), Eq. (reconstruct) returns w_q on every gas
    link and the mass fluxes of Eq. (advection1) cancel: nothing moves."""
    shape = (20, 20, 20)
    phi = orc.fill(orc.geom("sphere", c=(9.7, 10.2, 10.1), R=5.5, sub=8), shape)
    P = orc.params(shape, sigma=0.0, tau=0.9)
    st = orc.init_state(P, phi)
    f0, phi0, fl0 = st.f.copy(), st.phi.copy(), st.flags.copy()
    for _ in range(2):
        st, counts, _, _ = orc.step(P, st)
    fluid = (fl0 & 3) > 0
    assert np.max(np.abs(st.f[:, fluid] - f0[:, fluid])) < 1e-16
    assert np.max(np.abs(st.phi - phi0)) < 1e-15
    assert np.all(st.flags == fl0)


@pytest.mark.parametrize("collision,tau", [(0, 0.8), (1, 0.8), (0, 1.3)])
def test_shear_wave_decay_rate(orc, collision, tau):
    """u_x(z) = U sin(k z) decays as exp(-nu k^2 t), nu = c_s^2 (tau - 1/2) (Sec. II)."""
    L = 32
    shape = (L, 1, 1)
    P, st = _liquid_box(orc, shape, collision, tau)
    k = 2 * np.pi / L
    z = np.arange(L)
    U = 1e-3
    for iz in range(L):
        u = np.array([U * np.sin(k * iz), 0, 0])
        st.f[:, iz, 0, 0] = [orc.feq(q, 1.0, u) for q in range(19)]
    c, _, _ = orc.lattice()

    def amp(s):
        ux = (c[:, 0].astype(float) @ s.f[:, :, 0, 0]) / s.f[:, :, 0, 0].sum(0)
        return 2 * np.mean(ux * np.sin(k * z))

    a0 = amp(st)
    T = 150
    for _ in range(T):
        st, _, _, _ = orc.step(P, st)
    nu = (tau - 0.5) / 3.0
    rate = -np.log(amp(st) / a0) / T
    assert rate == pytest.approx(nu * k * k, rel=0.02)


def _moving_droplet(orc, shape=(24, 24, 24), u=(0.04, 0.02, -0.01), sigma=5e-4):
    phi = orc.fill(orc.geom("sphere", c=(11.6, 12.3, 11.9), R=6.3, sub=8), shape)
    P = orc.params(shape, sigma=sigma, tau=0.7)
    st = orc.init_state(P, phi)
    u = np.array(u)
    fe = np.array([orc.feq(q, 1.0, u) for q in range(19)])
    fluid = (st.flags & 3) > 0
    st.f[:, fluid] = fe[:, None]
    return P, st


@pytest.mark.parametrize("model", [0, 1])
def test_mass_conservation_and_invariants_through_conversions(orc, model):
    """Sum of interface m plus liquid rho plus the lost-mass counter is exactly
    conserved (the mass exchange is antisymmetric and conversion only moves
    mass); no liquid cell touches gas after any step (Sec. II)."""
    P, st = _moving_droplet(orc)
    P.curv_model = model
    M0 = orc.mass(P, st)
    conversions = 0
    for _ in range(25):
        st, counts, _, _ = orc.step(P, st)
        conversions += counts[3] + counts[4]
        assert counts[8] == 0
        assert abs(orc.mass(P, st) + st.lost - M0) < 1e-12 * M0
    assert conversions > 20


@pytest.mark.slow
@pytest.mark.parametrize("model", [0, 1])
def test_laplace_pressure_of_droplet(orc, model):
    """The 32^3 droplet (R = 8, sigma = 1e-4, BGK tau = 1): the pressure jump
    c_s^2 (rho_in - 1) oscillates acoustically around 2 sigma / R; its mean over
    steps 100..199 is within 15% of it (Sec. II, p_s = 2 sigma kappa)."""
    w = S.workload("droplet32")
    g = w["geometry"]
    shape = w["shape"]
    phi = orc.fill(orc.geom("sphere", c=g["c"], R=g["R"], sub=16), shape)
    P = orc.params(shape, sigma=w["sigma"], tau=w["tau"], curv_model=model)
    st = orc.init_state(P, phi)
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    r = np.sqrt((xx - g["c"][0]) ** 2 + (yy - g["c"][1]) ** 2 + (zz - g["c"][2]) ** 2)
    dps = []
    for it in range(200):
        st, counts, _, _ = orc.step(P, st)
        if it >= 100:
            inner = (st.flags == 1) & (r < g["R"] - 2)
            dps.append((st.f.sum(0)[inner].mean() - 1.0) / 3.0)
    assert np.mean(dps) == pytest.approx(2 * w["sigma"] / g["R"], rel=0.15)


@pytest.mark.slow
def test_translation_of_bubble_matches_printed_magnitude(orc):
    """Tab. advection, d = 10, u0 = 0.05: the bubble is carried by a constant
    f = feq(1, u0) for T = d/u0 = 200 steps and compared with the initial field
    shifted by d.  The paper prints L1 = 3.00 %, L2 = 9.38 %; the domain is not
    stated, so the norms are taken of the bubble indicator 1 - phi, which does
    not depend on it.  The conversion rules are readings, so the check is on
    magnitude: L2 within 25 %, L1 within a factor 2.5."""
    ref = _advection_table()[10]
    d, u0 = 10, ref["u0"]
    T = int(round(d / u0))
    L = 20
    shape = (L, L, L)
    phi0 = orc.fill(orc.geom("sphere", c=(L / 2, L / 2, L / 2), R=d / 2, sub=16, invert=1), shape)
    P = orc.params(shape, sigma=0.0, tau=1.0, curv_model=2)
    st = orc.init_state(P, phi0)
    fe = np.array([orc.feq(q, 1.0, np.array([u0, 0, 0])) for q in range(19)])
    g0 = 1 - st.phi.copy()
    for _ in range(T):
        st.f[:] = fe[:, None, None, None]
        st, _, _, _ = orc.step(P, st)
    g1 = 1 - np.roll(st.phi, -d, axis=2)
    L1 = np.abs(g1 - g0).sum() / g0.sum()
    L2 = np.sqrt(((g1 - g0) ** 2).sum() / (g0 ** 2).sum())
    assert L2 == pytest.approx(ref["L2"], rel=0.25)
    assert ref["L1"] / 2.5 < L1 < ref["L1"] * 2.5


@pytest.mark.slow
def test_sessile_cap_height_follows_contact_angle(orc):
    """A spherical cap built for theta_eq = 60 deg on a wall (Sec. III.B):
    with theta_eq = 60 its height stays at the cap height of its volume,
    h = (V / (pi (1/(1 - cos theta) - 1/3)))^(1/3), within 1 %; run with
    theta_eq = 120 it beads up and with 30 it spreads.  This fixes the
    direction of the whole wetting path (LSQR contact rows, corner rule)."""
    R, L, H = 8.0, 32, 16
    t = np.radians(60.0)
    c = (L / 2 + 0.25, L / 2 - 0.125, 0.5 - R * np.cos(t))
    phi = orc.fill(orc.geom("cap", c=c, R=R, zw=0.5, sub=8), (H, L, L))
    obs = np.zeros((H, L, L), np.uint8)
    obs[0] = obs[H - 1] = 1
    ratio = {}
    for th in (60.0, 120.0, 30.0):
        P = orc.params((H, L, L), collision=1, tau=0.8, sigma=1e-3, theta=np.radians(th))
        st = orc.init_state(P, phi, obs)
        V = st.phi[(st.flags & 3) > 0].sum()
        h = (V / (np.pi * (1 / (1 - np.cos(t)) - 1 / 3))) ** (1 / 3)
        for _ in range(200):
            st, counts, _, _ = orc.step(P, st)
        z = np.nonzero(st.flags == 2)[0]
        hstar = (z + st.phi[st.flags == 2] - 0.5).max() - 0.5  # wall plane at z = 1/2
        ratio[th] = hstar / h
    assert abs(ratio[60.0] - 1) < 0.01
    assert ratio[120.0] > 1.04
    assert ratio[30.0] < 0.98
