"""Pins of the oracle's wall treatment, each against values fixed by the paper
and worked out by hand (no call of the oracle's own helpers for the expected
side):

* the reflection of fill levels into obstacle cells (Sec. II.A, the formula
  with aperture alpha = sqrt(2)/2): which neighbours enter and with which
  weights, on an axis wall, a 45-degree staircase wall and next to a concave
  edge;
* the FD wetting normal (Sec. II.A, Eq. contactNormal with the constant
  extrapolation of reading O16): a vertical interface plane on a floor has
  kappa_FD = -cos(theta_eq)/4 at its contact-line cells, and spherical caps
  meet kappa R ~ 1 only with the right contact angle;
* the corner rule at contact-line cells (Sec. II, Fig. inhomo): the obstacle
  links whose outgoing direction points against the interface normal
  projected into the wall take Eq. (reconstruct), the others bounce back,
  checked link by link on a hand-built cell;
* invariance of both curvature models under the cube symmetries that map a
  walled box onto itself (no tie-break by lattice order)."""
import itertools
import math

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S

ALPHA = math.sqrt(2.0) / 2.0
# D3Q19 velocities written out here (the order of the C ABI)
C = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
              (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])


def _at(a, x, y, z):
    """a[z, y, x] with periodic wrap (arrays are (nz, ny, nx))."""
    nz, ny, nx = a.shape
    return a[z % nz, y % ny, x % nx]


def _paper_reflection(phi, obs, x, y, z, nw):
    """The paper's reflection formula at obstacle cell (x, y, z) for a given
    unit wall normal nw pointing out of the wall, evaluated literally:
    neighbours x_o + c_q inside Omega with |nw . c_q/|c_q|| > alpha (with a
    margin for exact ties), weights |nw . c_q/|c_q||."""
    num = den = 0.0
    for c in C[1:]:
        if _at(obs, x + c[0], y + c[1], z + c[2]):
            continue
        w = abs(float(np.dot(nw, c))) / math.sqrt(float(np.dot(c, c)))
        if w > ALPHA + 1e-9:
            num += w * _at(phi, x + c[0], y + c[1], z + c[2])
            den += w
    return num / den if den > 0 else 0.0


def _random_phi(shape, seed):
    return S.uniform(seed, int(np.prod(shape))).reshape(shape)


def test_reflection_axis_walls_take_the_face_neighbour(orc):
    """A flat wall normal to an axis: the face neighbour has |nw.c| = 1, the
    four edge neighbours sit exactly at the aperture (not > alpha), so the
    reflected value is the fill level of the face neighbour, on all six faces.
    Cells two layers deep have no fluid neighbour and get 0."""
    shape = (12, 11, 10)
    phi = _random_phi(shape, 31)
    obs = np.zeros(shape, np.uint8)
    obs[:2] = obs[-2:] = 1
    obs[:, :2] = obs[:, -2:] = 1
    obs[:, :, :2] = obs[:, :, -2:] = 1
    P = orc.params(shape)
    flags = np.where(obs > 0, orc.OBSTACLE, orc.LIQUID).astype(np.uint8)
    ext = orc.reflect_phi(P, flags, phi)
    nz, ny, nx = shape
    checked = 0
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if not obs[z, y, x]:
            assert ext[z, y, x] == phi[z, y, x]
            continue
        inner = [(x, 1, nx - 2), (y, 1, ny - 2), (z, 1, nz - 2)]
        on = [k for k, (v, lo, hi) in enumerate(inner) if v == lo or v == hi]
        deep = any(v < lo or v > hi for v, lo, hi in inner)
        # face cells of the first layer: exactly one axis on the boundary layer
        if len(on) == 1 and not deep:
            k = on[0]
            v, lo, hi = inner[k]
            # away from the edges, where every D3Q19 neighbour on the fluid
            # side exists (next to an edge the lattice-sum normal tilts)
            if not all(inner[j][1] + 1 < inner[j][0] < inner[j][2] - 1 for j in range(3) if j != k):
                continue
            step = [0, 0, 0]
            step[k] = 1 if v == lo else -1
            expect = phi[z + step[2], y + step[1], x + step[0]]
            nw = np.array(step, float)
            assert _paper_reflection(phi, obs, x, y, z, nw) == pytest.approx(expect, abs=0)
            assert ext[z, y, x] == expect
            checked += 1
        elif x in (0, nx - 1) or y in (0, ny - 1) or z in (0, nz - 1):
            assert ext[z, y, x] == 0.0
    assert checked == 2 * ((nx - 6) * (ny - 6) + (ny - 6) * (nz - 6) + (nx - 6) * (nz - 6))


def test_reflection_diagonal_wall(orc):
    """A 45-degree staircase wall (obstacle where x + z <= k): with the
    geometric wall normal (1,0,1)/sqrt2 only the diagonal neighbour (1,0,1)
    passes the aperture (|nw.c| = 1; face and other edge neighbours give
    sqrt2/2 or 1/2), so both obstacle layers reflect phi(x_o + (1,0,1)).  The
    oracle's wall normal (sum of lattice vectors to the non-obstacle
    neighbours) must agree with the geometric one here."""
    shape = (16, 6, 16)
    phi = _random_phi(shape, 32)
    zz, _, xx = np.meshgrid(np.arange(16), np.arange(6), np.arange(16), indexing="ij")
    s = xx + zz
    obs = ((s <= 10) | (s >= 26)).astype(np.uint8)  # two parallel staircases closing the periodic box
    P = orc.params(shape)
    flags = np.where(obs > 0, orc.OBSTACLE, orc.LIQUID).astype(np.uint8)
    ext = orc.reflect_phi(P, flags, phi)
    nw = np.array([1.0, 0.0, 1.0]) / math.sqrt(2.0)
    n = 0
    inner = (xx >= 1) & (xx <= 14) & (zz >= 1) & (zz <= 14)  # neighbourhood does not wrap
    for z, y, x in zip(*np.nonzero(((s == 10) | (s == 9)) & inner)):
        expect = _at(phi, x + 1, y, z + 1)
        assert _paper_reflection(phi, obs, x, y, z, nw) == pytest.approx(expect, abs=1e-15)
        assert ext[z, y, x] == pytest.approx(expect, abs=1e-15)
        n += 1
    assert n > 80


def test_reflection_weights_next_to_a_concave_edge(orc):
    """Obstacle cell (0, y, 1) of a side wall x = 0 right above a floor z = 0.
    Its non-obstacle neighbours are (1,0,0), (1,+-1,0) and (1,0,1), so the wall
    normal of reading O15 is (4,0,1)/sqrt17.  |nw.c| is 4/sqrt17 = 0.970 for
    (1,0,0), 5/sqrt34 = 0.857 for (1,0,1) and 4/sqrt34 = 0.686 < alpha for
    (1,+-1,0): phi_o is the weighted mean of two cells with those weights."""
    shape = (8, 6, 8)
    phi = _random_phi(shape, 33)
    obs = np.zeros(shape, np.uint8)
    obs[0] = obs[-1] = 1
    obs[:, :, 0] = obs[:, :, -1] = 1
    P = orc.params(shape)
    flags = np.where(obs > 0, orc.OBSTACLE, orc.LIQUID).astype(np.uint8)
    ext = orc.reflect_phi(P, flags, phi)
    wa, wb = 4.0 / math.sqrt(17.0), 5.0 / math.sqrt(34.0)
    for y in range(6):
        a, b = phi[1, y, 1], phi[2, y, 1]
        expect = (wa * a + wb * b) / (wa + wb)
        assert ext[1, y, 0] == pytest.approx(expect, rel=1e-14)
        assert _paper_reflection(phi, obs, 0, y, 1, np.array([4.0, 0.0, 1.0]) / math.sqrt(17.0)) == \
            pytest.approx(expect, rel=1e-14)
        # the edge cell (0, y, 0) itself sees only (1,0,1)
        assert ext[0, y, 0] == phi[1, y, 1]


def _vertical_plane(orc, theta_eq_deg, H=12, L=20):
    """Liquid for x < 9.37 between a floor (z = 0) and a lid (z = H-1): the
    interface is the vertical plane x = 9.37 (a 90-degree contact line); a gas
    block at x >= 16 keeps the periodic x wrap from making a second
    interface near it."""
    G = orc.geom("plane", n=(1.0, 0.0, 0.0), d=9.37, sub=16)
    phi = orc.fill(G, (H, L, L))
    obs = np.zeros((H, L, L), np.uint8)
    obs[0] = obs[H - 1] = 1
    P = orc.params((H, L, L), curv_model=1, theta=math.radians(theta_eq_deg))
    st = orc.init_state(P, phi, obs)
    return P, st


@pytest.mark.parametrize("theta_eq", [30.0, 60.0, 80.0, 90.0, 100.0, 135.0])
def test_fd_wetting_vertical_plane_closed_form(orc, theta_eq):
    """For the vertical plane the smoothed fill level depends on x only, so
    every fluid normal near the interface is (-1,0,0) (towards the liquid) and
    n_z = 0; at the floor's obstacle cells Eq. (contactNormal) with n_w =
    (0,0,-1) into the wall gives n_z = -cos(theta_eq) whatever the tangent.
    kappa = -1/2 div n with central differences then leaves only the z term
    at the contact-line cells: kappa = -1/2 * (0 - (-cos theta_eq))/2 =
    -cos(theta_eq)/4.  Under the lid (n_w = (0,0,1), n_z = +cos(theta_eq) at
    its obstacle cells) the z term is cos(theta_eq) - 0 and kappa is the same,
    as the mirror symmetry z -> -z of a scalar requires."""
    P, st = _vertical_plane(orc, theta_eq)
    kappa, _, _ = orc.curvature(P, st.flags, st.phi)
    H = st.flags.shape[0]
    iface = st.flags == orc.INTERFACE
    iface[:, :, 15:] = False
    floor = iface.copy()
    floor[2:] = False
    lid = iface.copy()
    lid[: H - 2] = False
    mid = iface.copy()
    mid[:3] = False
    mid[H - 3:] = False
    assert floor.sum() >= 20 and lid.sum() >= 20
    c = math.cos(math.radians(theta_eq))
    assert np.max(np.abs(kappa[floor] + c / 4)) < 1e-12
    assert np.max(np.abs(kappa[lid] + c / 4)) < 1e-12
    assert np.max(np.abs(kappa[mid])) < 1e-12


def _cap(orc, theta_deg, R=12.0, L=40, H=24):
    t = np.radians(theta_deg)
    c = (L / 2 + 0.25, L / 2 - 0.125, 0.5 - R * np.cos(t))
    G = orc.geom("cap", c=c, R=R, zw=0.5, sub=16)
    phi = orc.fill(G, (H, L, L))
    obs = np.zeros((H, L, L), np.uint8)
    obs[0] = obs[H - 1] = 1
    return phi, obs


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_fd_wetting_spherical_cap(orc, theta):
    """FD on a spherical cap meeting the floor at theta_eq: kappa R ~ 1 at the
    contact-line cells (first order: within 0.2) with the right angle, far
    from it (> 1 away) with 180 - theta_eq."""
    R = 12.0
    phi, obs = _cap(orc, theta, R)
    P = orc.params(phi.shape, curv_model=1, theta=np.radians(theta))
    st = orc.init_state(P, phi, obs)
    kappa, _, _ = orc.curvature(P, st.flags, st.phi)
    cl = (st.flags == orc.INTERFACE) & (np.roll(st.flags, 1, 0) == orc.OBSTACLE)
    assert cl.sum() > 50
    assert abs(np.mean(kappa[cl]) * R - 1) < 0.2
    P.theta = np.radians(180.0 - theta)
    kw, _, _ = orc.curvature(P, st.flags, st.phi)
    assert abs(np.mean(kw[cl]) * R - 1) > 1.0


def _corner_cell_state(orc, n_hat):
    """An 8x6x6 periodic box, obstacle floor z = 0 and lid z = 5.  Row z = 1:
    interface for x <= 4 (the test cell is (4, 2, 1)), gas for x >= 5; gas for
    z >= 2.  Fluid PDFs are w_q plus distinct seeded offsets."""
    shape = (6, 6, 8)
    flags = np.full(shape, orc.GAS, np.uint8)
    flags[0] = flags[5] = orc.OBSTACLE
    flags[1, :, :5] = orc.INTERFACE
    _, w, _ = orc.lattice()
    f = np.zeros((19,) + shape)
    noise = (S.uniform(77, 19 * int(np.prod(shape))).reshape((19,) + shape) - 0.5) * 4e-3
    f[:] = w[:, None, None, None] + noise
    mass = np.where(flags == orc.INTERFACE, 0.5, 0.0)
    phi = mass.copy()
    normal4 = np.zeros(shape + (4,))
    normal4[1, :, :5, :3] = n_hat
    kappa = np.full(shape, 0.05)
    return orc.State(f, flags, mass, phi), normal4, kappa


@pytest.mark.parametrize("n_hat", [(-0.6, 0.48, 0.64), (0.28, -0.96, 0.0), (0.0, 0.0, 1.0)])
def test_corner_rule_link_by_link(orc, n_hat):
    """Fig. inhomo: at a contact-line cell (gas and obstacle neighbours) an
    obstacle link takes Eq. (reconstruct) when its outgoing direction c (from
    the cell into the wall) has c . n_t < 0, n_t the interface normal with its
    wall-normal part removed; otherwise it bounces back.  The floor's five
    outgoing directions are (0,0,-1), (+-1,0,-1), (0,+-1,-1) and n_t =
    (n_x, n_y, 0), so the reconstructed set is written out by hand for each
    normal.  With tau = 10^6 the collision barely changes the streamed
    values, and each link is compared with both candidates."""
    n_hat = np.array(n_hat) / np.linalg.norm(n_hat)
    st, normal4, kappa = _corner_cell_state(orc, n_hat)
    p_gas, sigma = 0.5, 0.01
    P = orc.params(st.flags.shape, tau=1e6, sigma=sigma, p_gas=p_gas)
    out, _, _, _ = orc.step(P, st, kappa=kappa, normal4=normal4)
    x, y, z = 4, 2, 1
    f0 = st.f[:, z, y, x]
    rho0 = f0.sum()
    u0 = (C.T @ f0) / rho0
    rho_b = 3 * p_gas + 6 * sigma * 0.05
    # outgoing direction -> reconstructed?  (c . n_t < 0 strictly)
    nt = np.array([n_hat[0], n_hat[1], 0.0])
    hand = {(0, 0, -1): False,
            (1, 0, -1): 1 * nt[0] < 0, (-1, 0, -1): -1 * nt[0] < 0,
            (0, 1, -1): 1 * nt[1] < 0, (0, -1, -1): -1 * nt[1] < 0}
    opp = [int(np.nonzero((C == -c).all(1))[0][0]) for c in C]
    fs = np.zeros(19)
    fs[0] = f0[0]
    recon_links = 0
    for q in range(1, 19):
        qb = opp[q]
        sx, sy, sz = x - C[q][0], y - C[q][1], z - C[q][2]
        t = _at(st.flags, sx, sy, sz)
        recon = orc.feq(q, rho_b, u0) + orc.feq(qb, rho_b, u0) - f0[qb]
        bounce = f0[qb]
        if t == orc.INTERFACE:
            fs[q] = st.f[q, sz % 6, sy % 6, sx % 8]
        elif t == orc.GAS:
            fs[q] = recon
        else:
            r = hand[tuple(int(v) for v in C[qb])]
            fs[q] = recon if r else bounce
            other = bounce if r else recon
            recon_links += r
            # the oracle's value sits on the chosen candidate, far from the other
            assert abs(out.f[q, z, y, x] - fs[q]) < 1e-6
            assert abs(out.f[q, z, y, x] - other) > 1e-2
    expect = orc.collide(P, fs)
    assert np.max(np.abs(out.f[:, z, y, x] - expect)) < 1e-13
    assert recon_links == sum(hand.values())


def _transforms():
    """cube symmetries that keep z (the walled axis) as an axis: permutations of
    (y, x), flips of any axis (arrays are (z, y, x))"""
    out = []
    for perm in ((0, 1, 2), (0, 2, 1)):
        for flips in itertools.product((False, True), repeat=3):
            out.append((perm, flips))
    return out


@pytest.mark.slow
@pytest.mark.parametrize("model", [0, 1])
def test_curvature_symmetry_with_walls(orc, model):
    """A cap on the floor of a box with side walls and a second blob sitting
    in the edge between the floor and a side wall (where the wall normal of
    an obstacle cell is diagonal, so the tangent taken from the fluid cell
    x_b enters kappa): both curvature models commute with the 16 symmetries
    of the walled box (no choice depends on the lattice order of the
    neighbours)."""
    H, L = 16, 24
    G = orc.geom("cap", c=(11.3, 12.6, -2.0), R=8.0, zw=0.5, sub=8)
    phi = orc.fill(G, (H, L, L))
    G2 = orc.geom("sphere", c=(2.4, 8.2, 2.1), R=3.6, sub=8)
    phi = np.maximum(phi, orc.fill(G2, (H, L, L)))
    obs = np.zeros((H, L, L), np.uint8)
    obs[0] = obs[-1] = 1
    obs[:, 0] = obs[:, -1] = 1
    obs[:, :, 0] = obs[:, :, -1] = 1
    P = orc.params((H, L, L), curv_model=model, theta=np.radians(70.0))
    st = orc.init_state(P, phi, obs)
    k0, _, _ = orc.curvature(P, st.flags, st.phi)
    assert np.count_nonzero(k0) > 100
    for perm, flips in _transforms():
        def T(a):
            a = np.transpose(a, perm)
            for ax, fl in enumerate(flips):
                if fl:
                    a = np.flip(a, ax)
            return np.ascontiguousarray(a)
        k1, _, _ = orc.curvature(P, T(st.flags), T(st.phi))
        assert np.max(np.abs(k1 - T(k0))) < 1e-9, (perm, flips)
