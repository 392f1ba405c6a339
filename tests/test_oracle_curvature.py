"""Pins of the oracle's curvature models (LSQR, Sec. II.C; FD, Sec. II.A).

Each check compares the oracle with something other than itself: exact
quadric point sets, the mean curvature of a graph computed from its first
and second fundamental forms, planes (kappa = 0), spheres (kappa = 1/R),
cube symmetries and spherical caps at a wall with a given contact angle."""
import itertools

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S


def _rows(u, v):
    return np.stack([u * u, v * v, u * v, u, v], 1)


def _coef(seed):
    r = S.uniform(seed, 5) - 0.5
    return np.array([0.3 * r[0], 0.3 * r[1], 0.3 * r[2], 0.8 * r[3], 0.8 * r[4]])


@pytest.mark.parametrize("seed", range(6))
def test_ls_fit_recovers_exact_quadric(orc, seed):
    coef = _coef(seed)
    uv = (S.uniform(100 + seed, 40).reshape(20, 2) - 0.5) * 3.0
    rows = _rows(uv[:, 0], uv[:, 1])
    fit, mode = orc.ls_fit(rows, rows @ coef)
    assert mode == 0
    assert np.allclose(fit, coef, atol=1e-12)


def test_ls_fit_with_centre_constraint(orc):
    """A constraint that the true surface satisfies leaves the exact fit unchanged;
    a constraint it violates is met exactly by the fit (Eq. contactConstraint)."""
    coef = _coef(11)
    uv = (S.uniform(12, 24).reshape(12, 2) - 0.5) * 3.0
    rows = _rows(uv[:, 0], uv[:, 1])
    uc, vc = 0.3, -0.7
    C = np.array([[2 * uc, 0, vc, 1, 0], [0, 2 * vc, uc, 0, 1]])
    fit, mode = orc.ls_fit(rows, rows @ coef, C, C @ coef)
    assert mode == 0 and np.allclose(fit, coef, atol=1e-12)
    g = C @ coef + np.array([0.1, -0.05])
    fit, mode = orc.ls_fit(rows, rows @ coef, C, g)
    assert mode == 0
    assert np.allclose(C @ fit, g, atol=1e-12)
    # and the fit is the constrained minimiser: perturbing inside the null space of C raises the error
    _, _, vt = np.linalg.svd(C)
    e0 = np.sum((rows @ fit - rows @ coef) ** 2)
    for k in range(2, 5):
        for s in (1e-3, -1e-3):
            assert np.sum((rows @ (fit + s * vt[k]) - rows @ coef) ** 2) > e0


def test_ls_fit_fallbacks(orc):
    uv = np.array([[0.5, 0.2], [-0.4, 0.9], [1.0, -1.0], [0.1, 0.3]])
    rows = _rows(uv[:, 0], uv[:, 1])
    iso = np.array([0.05, 0.05, 0.0, 0.2, -0.1])
    fit, mode = orc.ls_fit(rows, rows @ iso)  # 4 rows < 5 unknowns: isotropic model
    assert mode == 1 and np.allclose(fit, iso, atol=1e-12)
    fit, mode = orc.ls_fit(rows[:2], rows[:2] @ iso)
    assert mode == 2 and np.all(fit == 0)
    # collinear points (v = 0): rank deficient in both models
    u = np.linspace(-1, 1, 9)
    rows = _rows(u, 0 * u)
    fit, mode = orc.ls_fit(rows, 0.1 * u * u)
    assert mode == 2


def _mean_curvature_fundamental_forms(c):
    """Mean curvature of z = f(u,v) at the origin from the shape operator
    S = I^-1 II (first and second fundamental forms), H = tr(S)/2."""
    A, B, C, H, I = c
    fu, fv, fuu, fvv, fuv = H, I, 2 * A, 2 * B, C
    first = np.array([[1 + fu * fu, fu * fv], [fu * fv, 1 + fv * fv]])
    second = np.array([[fuu, fuv], [fuv, fvv]]) / np.sqrt(1 + fu * fu + fv * fv)
    return 0.5 * np.trace(np.linalg.solve(first, second))


@pytest.mark.parametrize("seed", range(8))
def test_kappa_formula_is_mean_curvature(orc, seed):
    c = _coef(200 + seed)
    assert orc.kappa_from_coef(c) == pytest.approx(_mean_curvature_fundamental_forms(c), abs=1e-14)


def test_ls_fit_of_sphere_points(orc):
    """Points on a sphere of radius R around the pole: the paraboloid fit gives
    kappa = 1/R up to the quartic term of the sphere's height function, an O(1/R^2)
    relative bias for points within 1.5 cells."""
    for R in (4.0, 10.0, 30.0):
        uv = (S.uniform(int(R), 60).reshape(30, 2) - 0.5) * 3.0
        f = R - np.sqrt(R * R - (uv ** 2).sum(1))
        fit, mode = orc.ls_fit(_rows(uv[:, 0], uv[:, 1]), f)
        assert abs(orc.kappa_from_coef(fit) * R - 1) < 1.5 / R ** 2


# ------------------------------------------------------------ fields

def _state(orc, phi, obstacle=None, **kw):
    P = orc.params(phi.shape, **kw)
    st = orc.init_state(P, phi, obstacle)
    return P, st


def _exact_plane_phi(orc, shape, n, d):
    """Fill levels of the half-space {x : x.n >= d} computed from the exact cut volume."""
    nz, ny, nx = shape
    phi = np.zeros(shape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                phi[z, y, x] = orc.plic_volume(n, d - (n[0] * x + n[1] * y + n[2] * z))
    phi[phi > 1 - 1e-12] = 1.0  # rounding of full cells
    phi[phi < 1e-12] = 0.0
    return phi


@pytest.mark.parametrize("n", [(0.0, 0.0, 1.0), (1.0, 0.0, 1.0), (0.0, 1.0, 1.0), (1.0, 1.0, 0.0)])
def test_lsqr_plane_has_zero_curvature(orc, n):
    n = np.array(n) / np.linalg.norm(n)
    shape = (16, 16, 16)
    phi = _exact_plane_phi(orc, shape, n, 0.37 + 7.5 * n.sum())
    # cells near the periodic seam see the jump of the wrapped field: only inner cells are checked
    P, st = _state(orc, phi)
    kappa, n4, stats = orc.curvature(P, st.flags, st.phi)
    z, y, x = np.nonzero(st.flags == 2)
    inner = (x > 2) & (x < 13) & (y > 2) & (y < 13) & (z > 2) & (z < 13)
    assert inner.sum() > 10
    assert np.max(np.abs(kappa[z[inner], y[inner], x[inner]])) < 1e-9
    assert np.allclose(n4[z[inner], y[inner], x[inner], :3], n, atol=1e-12)


def test_fd_linear_field_has_zero_curvature(orc):
    shape = (12, 12, 32)
    x = np.arange(32)
    phi = np.broadcast_to(0.5 + 0.012 * (x - 15.5), shape).copy()
    P = orc.params(shape, curv_model=1)
    flags = np.full(shape, 2, np.uint8)
    kappa, _, _ = orc.curvature(P, flags, phi)
    assert np.max(np.abs(kappa[:, :, 4:28])) < 1e-13


def _sphere_phi(orc, R, seed=5):
    L = int(2 * R + 12)
    L += L % 2
    c = L / 2 + S.centre_offset(seed)
    G = orc.geom("sphere", c=tuple(c), R=R, sub=16)
    return orc.fill(G, (L, L, L))


@pytest.mark.parametrize("R,tol_lsqr,tol_fd", [(6.0, 0.03, 0.03), (12.0, 0.012, 0.03)])
def test_sphere_mean_curvature(orc, R, tol_lsqr, tol_fd):
    """kappa = 1/R on the interface of a sub-sampled sphere (Sec. III.A); the
    LSQR mean converges with R; FD is first order and biased low."""
    phi = _sphere_phi(orc, R)
    P, st = _state(orc, phi)
    kappa, _, stats = orc.curvature(P, st.flags, st.phi)
    m = (st.flags == 2) & (st.phi > 0.02) & (st.phi < 0.98)
    assert abs(np.mean(kappa[m]) * R - 1) < tol_lsqr
    assert stats[1] == 0 and stats[2] == 0
    P.curv_model = 1
    kfd, _, _ = orc.curvature(P, st.flags, st.phi)
    assert abs(np.mean(kfd[m]) * R - 1) < tol_fd


def _transforms():
    """a few of the 48 cube symmetries as (axes permutation, flips) of the (z,y,x) array"""
    return [((0, 1, 2), (False, False, True)), ((0, 2, 1), (False, False, False)),
            ((2, 1, 0), (True, False, False)), ((1, 2, 0), (False, True, True))]


@pytest.mark.parametrize("model", [0, 1])
def test_curvature_cube_symmetry(orc, model):
    phi = _sphere_phi(orc, 6.0, seed=9)
    # break the sphere's own symmetry with a second blob so that index mistakes show
    G = orc.geom("sphere", c=(7.3, 8.1, 15.6), R=3.2, sub=8)
    phi = np.maximum(phi, orc.fill(G, phi.shape))
    P, st = _state(orc, phi, curv_model=model)
    k0, _, _ = orc.curvature(P, st.flags, st.phi)
    for perm, flips in _transforms():
        def T(a):
            a = np.transpose(a, perm)
            for ax, fl in enumerate(flips):
                if fl:
                    a = np.flip(a, ax)
            return np.ascontiguousarray(a)
        k1, _, _ = orc.curvature(P, T(st.flags), T(st.phi))
        assert np.max(np.abs(k1 - T(k0))) < 1e-9


def _cap(orc, theta_deg, R=12.0, L=40, H=24):
    t = np.radians(theta_deg)
    c = (L / 2 + 0.25, L / 2 - 0.125, 0.5 - R * np.cos(t))
    G = orc.geom("cap", c=c, R=R, zw=0.5, sub=16)
    phi = orc.fill(G, (H, L, L))
    obs = np.zeros((H, L, L), np.uint8)
    obs[0] = obs[H - 1] = 1
    return phi, obs


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_lsqr_wetting_spherical_cap(orc, theta):
    """A spherical cap meeting the wall at theta_eq has kappa = 1/R at the
    contact line when the wetting rows use theta_eq (Sec. II.C, Eq.
    contactNormal); using 180 - theta_eq instead breaks it.  This fixes the
    sign convention of the wall normal (into the wall) and of m."""
    R = 12.0
    phi, obs = _cap(orc, theta, R)
    P, st = _state(orc, phi, obs, theta=np.radians(theta))
    kappa, _, stats = orc.curvature(P, st.flags, st.phi)
    cl = (st.flags == 2) & (np.roll(st.flags, 1, 0) == 8)
    assert cl.sum() > 50 and stats[3] == cl.sum()
    assert abs(np.mean(kappa[cl]) * R - 1) < 0.1
    if theta != 90.0:
        P.theta = np.radians(180.0 - theta)
        kw, _, _ = orc.curvature(P, st.flags, st.phi)
        assert abs(np.mean(kw[cl]) * R - 1) > 1.0
