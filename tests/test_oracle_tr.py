"""Pins of the oracle's TR curvature (Sec. II.B: a triangle fan of PLIC
points after Pohl, curvature after Taubin), each against something other
than the oracle:

* exact point sets: PLIC points placed exactly on a sphere (normals along
  the radius) give kappa = 1/R for every fan, because each directional
  curvature 2 h / |p|^2 is that of a great circle; a bubble gives -1/R; points
  on a plane give 0;
* rings of points on the quadric h = A u^2 + B v^2 + C uv: equally spaced
  rings give the mean curvature A + B (the average of the normal curvature
  over all directions); an uneven ring needs the triangle-area weights to
  stay near it (the plain mean of the directional curvatures is 30 % off);
* degenerate fans: fewer than two points, all gaps of at least pi;
* sub-sampled spheres: the mean of kappa R over the interface is 1 within
  1.5 % (R = 6 ... 24 cells);
* the curvature field commutes with cube symmetries, and a fan does not
  depend on where the angle is measured from."""
import math

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S


def _block(orc, centre_fn):
    """A 5x5x5 periodic grid whose middle 3x3x3 block is interface; normal4
    from centre_fn(o) -> (n_hat, a) for each block cell at offset o."""
    shape = (5, 5, 5)
    flags = np.full(shape, orc.GAS, np.uint8)
    flags[1:4, 1:4, 1:4] = orc.INTERFACE
    n4 = np.zeros(shape + (4,))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                n, a = centre_fn(np.array([dx, dy, dz], float))
                n4[2 + dz, 2 + dy, 2 + dx, :3] = n
                n4[2 + dz, 2 + dy, 2 + dx, 3] = a
    P = orc.params(shape, curv_model=4)
    return P, flags, n4, 2 + 5 * (2 + 5 * 2)


def _sphere_normals(c, R, bubble):
    def fn(o):
        d = c - o
        r = np.linalg.norm(d)
        if bubble:  # liquid outside: the normal points away from the centre
            return -d / r, R - r
        return d / r, r - R
    return fn


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("bubble", [False, True])
def test_exact_sphere_points(orc, seed, bubble):
    u = S.uniform(900 + seed, 6)
    R = [2.5, 4.0, 10.0, 40.0][seed % 4]
    zc, ph = 2 * u[0] - 1, 2 * math.pi * u[1]
    direction = np.array([math.sqrt(1 - zc * zc) * math.cos(ph), math.sqrt(1 - zc * zc) * math.sin(ph), zc])
    # sphere surface passing near the middle cell's centre (offset < 0.3 along the normal)
    c = direction * (R + 0.6 * (u[2] - 0.5))
    P, flags, n4, i = _block(orc, _sphere_normals(c, R, bubble))
    k = orc.tr_cell(P, flags, n4, i)
    assert k == pytest.approx(-1.0 / R if bubble else 1.0 / R, rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_exact_plane_points(orc, seed):
    u = S.uniform(950 + seed, 4)
    n = np.array([u[0] - 0.5, u[1] - 0.5, u[2] - 0.5])
    n /= np.linalg.norm(n)
    q = n * (u[3] - 0.5) * 0.8
    P, flags, n4, i = _block(orc, lambda o: (n, float(np.dot(n, q - o))))
    assert abs(orc.tr_cell(P, flags, n4, i)) < 1e-13


def _quadric_ring(angles, d, A, B, C):
    u = d * np.cos(angles)
    v = d * np.sin(angles)
    return u, v, A * u * u + B * v * v + C * u * v


@pytest.mark.parametrize("nring", [6, 8, 12])
def test_symmetric_ring_gives_mean_curvature(orc, nring):
    """kappa_j -> 2 (A cos^2 + B sin^2 + C cos sin) as d -> 0; over equally
    spaced angles cos^2 and sin^2 average to 1/2 and cos sin to 0."""
    A, B, C = 0.31, -0.07, 0.23
    off = 0.37  # the ring need not start at angle 0
    ang = off + 2 * math.pi * np.arange(nring) / nring
    u, v, h = _quadric_ring(ang, 1e-3, A, B, C)
    assert orc.tr_fan(u, v, h) == pytest.approx(A + B, abs=1e-5)


def test_uneven_ring_needs_area_weights(orc):
    """On h = A u^2 with points at 0,10,20,30,40,90,180,270 degrees the
    Taubin weights (areas of the triangles at each edge, about sin of the
    neighbouring gaps) keep the estimate within 5 % of the mean curvature A;
    the unweighted mean of the directional curvatures would be 1.3 A."""
    A = 0.2
    ang = np.radians([0, 10, 20, 30, 40, 90, 180, 270])
    u, v, h = _quadric_ring(ang, 1e-3, A, 0.0, 0.0)
    k = orc.tr_fan(u, v, h)
    assert abs(k / A - 1) < 0.05
    plain = np.mean(2 * h / (u * u + v * v + h * h))
    assert abs(plain / A - 1) > 0.25


def test_weights_are_surface_areas(orc):
    """Worked example with large heights: four points at 90 degree steps, unit
    projected radius, heights 0.9, 0.1, 0.5, 0.2.  The weight of an edge is
    the summed surface area of its two fan triangles (Heron's formula on the
    3D side lengths here); projected areas would all be 1/2 and give the
    plain mean 0.5943, the surface areas give 0.5989"""
    h = np.array([0.9, 0.1, 0.5, 0.2])
    ang = np.radians([0.0, 90.0, 180.0, 270.0])
    u, v = np.cos(ang), np.sin(ang)
    pts = np.stack([u, v, h], 1)
    kap = 2 * h / (1 + h * h)

    def heron(a, b):
        la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(a - b)
        s2 = (la + lb + lc) / 2
        return math.sqrt(s2 * (s2 - la) * (s2 - lb) * (s2 - lc))

    areas = [heron(pts[k], pts[(k + 1) % 4]) for k in range(4)]
    want = sum(areas[k] * (kap[k] + kap[(k + 1) % 4]) for k in range(4)) / (2 * sum(areas))
    assert orc.tr_fan(u, v, h) == pytest.approx(want, rel=1e-12)
    assert abs(want - np.mean(kap)) > 0.004


def test_degenerate_fans(orc):
    # one point: no triangle
    assert orc.tr_fan([0.5], [0.2], [0.1]) == 0.0
    # two points opposite each other: both gaps are pi, the fan is open everywhere
    assert orc.tr_fan([0.5, -0.5], [0.0, 0.0], [0.1, 0.1]) == 0.0
    # a point on the normal axis is dropped (no direction)
    k3 = orc.tr_fan([0.0, 0.4, -0.2, -0.2], [0.0, 0.0, 0.35, -0.35], [0.3, 0.02, 0.02, 0.02])
    k2 = orc.tr_fan([0.4, -0.2, -0.2], [0.0, 0.35, -0.35], [0.02, 0.02, 0.02])
    assert k3 == k2 and k2 > 0


def test_open_fan_on_a_sphere(orc):
    """Points on a sphere covering only part of the circle (a gap >= pi stays
    open): still 1/R, every directional curvature being 1/R."""
    R = 5.0
    ang = np.radians([10, 50, 95, 140])
    pts = []
    for a in ang:
        t = 0.8  # arc angle along the great circle in direction a
        s = R * math.sin(t / R * 2)
        hh = R * (1 - math.cos(t / R * 2))
        pts.append((s * math.cos(a), s * math.sin(a), hh))
    u, v, h = np.array(pts).T
    assert orc.tr_fan(u, v, h) == pytest.approx(1.0 / R, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_fan_independent_of_angle_origin(orc, seed):
    """Rotating the tangent frame about the normal changes every angle by the
    same amount: the cyclic order, the triangles and kappa stay."""
    r = S.uniform(970 + seed, 40)
    u = (r[:10] - 0.5) * 2.4
    v = (r[10:20] - 0.5) * 2.4
    h = (r[20:30] - 0.5) * 0.3
    k0 = orc.tr_fan(u, v, h)
    for rot in (0.3, 1.7, -2.9):
        c, s = math.cos(rot), math.sin(rot)
        assert orc.tr_fan(c * u - s * v, s * u + c * v, h) == pytest.approx(k0, rel=1e-12, abs=1e-15)


def _sphere_state(orc, R, seed=3):
    L = int(2 * R + 10)
    off = S.centre_offset(seed)
    c = tuple(np.array([L / 2] * 3) - 0.4 + off)
    phi = orc.fill(orc.geom("sphere", c=c, R=R, sub=16), (L, L, L))
    P = orc.params((L, L, L), curv_model=4)
    return P, orc.init_state(P, phi)


@pytest.mark.parametrize("R", [6.0, 12.0, 24.0])
def test_subsampled_sphere_mean(orc, R):
    P, st = _sphere_state(orc, R)
    k, _, _ = orc.curvature(P, st.flags, st.phi)
    sel = st.flags == orc.INTERFACE
    assert sel.sum() > 100
    assert abs(np.mean(k[sel]) * R - 1) < 0.015


def test_tr_cube_symmetry(orc):
    phi = orc.fill(orc.geom("sphere", c=(11.3, 10.6, 12.2), R=6.0, sub=8), (24, 24, 24))
    G = orc.geom("sphere", c=(7.3, 8.1, 15.6), R=3.2, sub=8)
    phi = np.maximum(phi, orc.fill(G, phi.shape))
    P = orc.params(phi.shape, curv_model=4)
    st = orc.init_state(P, phi)
    k0, _, _ = orc.curvature(P, st.flags, st.phi)
    for perm, flips in [((0, 1, 2), (False, False, True)), ((0, 2, 1), (False, False, False)),
                        ((2, 1, 0), (True, False, False)), ((1, 2, 0), (False, True, True))]:
        def T(a):
            a = np.transpose(a, perm)
            for ax, fl in enumerate(flips):
                if fl:
                    a = np.flip(a, ax)
            return np.ascontiguousarray(a)
        k1, _, _ = orc.curvature(P, T(st.flags), T(st.phi))
        assert np.max(np.abs(k1 - T(k0))) < 1e-9
