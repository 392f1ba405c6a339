"""Pins of the oracle's step with frozen cell types (the forward map of the
adjoint windows) and of the finite-difference reference gradient built on it.

What fixes them: where the plain step converts nothing, the frozen step is
the plain step (bit for bit); with types frozen the mass exchange is still
antisymmetric, so total mass (liquid rho + interface m) is conserved exactly
while no cell changes type; and the window map is smooth in sigma and theta,
so central differences at h and h/2 agree to O(h^2) (which is what makes a
central difference of the FP64 oracle a reference gradient)."""
import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S


def _moving_droplet(orc, frozen, shape=(24, 24, 24), u=(0.04, 0.02, -0.01), sigma=5e-4):
    phi = orc.fill(orc.geom("sphere", c=(11.6, 12.3, 11.9), R=6.3, sub=8), shape)
    P = orc.params(shape, sigma=sigma, tau=0.7, frozen=frozen)
    st = orc.init_state(P, phi)
    fe = np.array([orc.feq(q, 1.0, np.array(u)) for q in range(19)])
    st.f[:, (st.flags & 3) > 0] = fe[:, None]
    return P, st


def test_frozen_step_equals_plain_step_where_nothing_converts(orc):
    shape = (20, 20, 20)
    phi = orc.fill(orc.geom("sphere", c=(9.7, 10.2, 10.1), R=5.5, sub=8), shape)
    P = orc.params(shape, sigma=1e-4, tau=0.9)
    st = orc.init_state(P, phi)
    s1, c1, _, _ = orc.step(P, st)
    assert c1[3:7].sum() == 0  # the plain step converts nothing here
    Pf = orc.params(shape, sigma=1e-4, tau=0.9, frozen=1)
    s2, c2, _, _ = orc.step(Pf, st)
    for a, b in ((s1.f, s2.f), (s1.mass, s2.mass), (s1.phi, s2.phi), (s1.flags, s2.flags)):
        assert np.array_equal(a, b)


def test_frozen_steps_keep_types_and_conserve_mass(orc):
    P, st = _moving_droplet(orc, frozen=0)
    _, counts, _, _ = orc.step(P, st)
    assert counts[3] + counts[4] > 0  # the plain step converts from this state
    P, st = _moving_droplet(orc, frozen=1)
    fl0, M0 = st.flags.copy(), orc.mass(P, st)
    for _ in range(15):
        st, counts, _, _ = orc.step(P, st)
        assert counts[3:7].sum() == 0
        assert np.array_equal(st.flags, fl0)
        assert abs(orc.mass(P, st) - M0) < 1e-12 * M0
    assert st.lost == 0.0
    p = st.phi[st.flags == 2]
    assert p.max() > 1.001 or p.min() < -0.001  # held where the plain step would convert


def _sessile_small(orc, theta, sigma, frozen=1):
    H, L, R = 12, 20, 6.0
    phi = orc.fill(orc.geom("cap", c=(L / 2 + 0.3, L / 2 - 0.2, 0.5), R=R, zw=0.5, sub=8), (H, L, L))
    obs = S.obstacle_mask((H, L, L), (0, H - 1))
    P = orc.params((H, L, L), collision=1, tau=0.8, sigma=sigma, theta=theta, frozen=frozen)
    return P, orc.init_state(P, phi, obs)


def _window_phi(orc, theta, sigma, steps=8):
    P, st = _sessile_small(orc, theta, sigma)
    for _ in range(steps):
        st, _, _, _ = orc.step(P, st)
    return st.phi, st.flags


def test_window_map_is_smooth_in_sigma_and_theta(orc):
    target, fl = _window_phi(orc, np.radians(70.0), 3e-4)
    iface = fl == 2
    assert np.any(fl == 8)

    def loss(theta, sigma):
        phi, fl2 = _window_phi(orc, theta, sigma)
        assert np.array_equal(fl2, fl)
        return float(np.sum((phi[iface] - target[iface]) ** 2))

    th0, s0 = np.radians(90.0), 2e-4
    for k, scale in ((0, 1e-3), (1, 1e-3 * s0)):
        def Lk(h):
            d = np.zeros(2)
            d[k] = h
            return loss(th0 + d[0], s0 + d[1])
        D1 = (Lk(scale) - Lk(-scale)) / (2 * scale)
        D2 = (Lk(scale / 2) - Lk(-scale / 2)) / scale
        assert D1 != 0.0
        assert abs(D1 - D2) <= 1e-5 * abs(D2), (k, D1, D2)
