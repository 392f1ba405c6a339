"""GPU parity of the TR curvature (Sec. II.B, triangle fan of PLIC points with
Taubin's mean curvature) against the FP64 oracle, through the C ABI.

Tolerance: |d| <= 1e-4 max(|ref|, 1/L), as for the other curvature models.
The fan is an integer decision taken from floating point (the angular order
of the points and whether a gap reaches pi): cells where two angles of the
oracle's points lie within 1e-4 rad of each other, or a gap lies within 1e-4
of pi, may be triangulated differently in FP32; those cells (a small share,
asserted) must still hold a finite value within the range of their
directional curvatures."""
import math

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL_K = 1e-4


@pytest.fixture(scope="module")
def fsl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1509_07691_gb300 import build
    build.build()
    from paper_1509_07691_gb300 import fsl as F
    return F


def _fan_data(st_flags, n4, z, y, x):
    """angles and directional curvatures of the oracle's fan at one cell (the
    construction of the oracle's TR, repeated here only to find near-ties)"""
    nz, ny, nx = st_flags.shape
    c = n4[z, y, x]
    n = c[:3]
    k = int(np.argmin(np.abs(n)))  # first minimum: lowest index on ties
    e = np.zeros(3)
    e[k] = 1
    tu = np.cross(e, n)
    tu /= np.linalg.norm(tu)
    tv = np.cross(n, tu)
    p = c[3] * n
    ang, kap = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                j = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
                if st_flags[j] != 2 or not np.any(n4[j][:3]):
                    continue
                d = np.array([dx, dy, dz]) + n4[j][3] * n4[j][:3] - p
                u, v, h = d @ tu, d @ tv, d @ n
                if u * u + v * v < 1e-12:
                    continue
                ang.append(math.atan2(v, u))
                kap.append(2 * h / (u * u + v * v + h * h))
    return np.array(ang), np.array(kap)


def _near_tie(ang, eps=1e-4):
    if len(ang) < 2:
        return False
    a = np.sort(ang)
    gaps = np.diff(np.concatenate([a, [a[0] + 2 * math.pi]]))
    return bool(np.any(gaps < eps) or np.any(np.abs(gaps - math.pi) < eps))


def _check_field(orc, st, n4, k_gpu, k_ref, L):
    idx = np.argwhere(st.flags == 2)
    ties = 0
    for z, y, x in idx:
        err = abs(k_gpu[z, y, x] - k_ref[z, y, x])
        if err <= TOL_K * max(abs(k_ref[z, y, x]), 1.0 / L):
            continue
        ang, kap = _fan_data(st.flags, n4, z, y, x)
        assert _near_tie(ang), (z, y, x, k_gpu[z, y, x], k_ref[z, y, x])
        assert np.isfinite(k_gpu[z, y, x]) and kap.min() - 1e-4 <= k_gpu[z, y, x] <= kap.max() + 1e-4
        ties += 1
    assert ties <= max(2, 0.01 * len(idx)), ties
    return len(idx)


@pytest.mark.parametrize("name", ["droplet32", "sessile64", "oscillating128"])
def test_tr_curvature_parity(orc, fsl, name):
    w = S.workload(name)
    g = w["geometry"]
    kw = dict(c=g["c"], R=g.get("R_s", g.get("R")), eps2=g.get("eps2", 0.0), zw=g.get("zw", 0.0), sub=16)
    og = orc.geom(g["kind"], **kw)
    phi = orc.fill(og, w["shape"])
    obs = S.obstacle_mask(w["shape"], w["walls"])
    P = orc.params(w["shape"], curv_model=4, tau=w["tau"], sigma=w["sigma"], theta=w["theta"])
    st = orc.init_state(P, phi, obs)
    k_ref, n4, _ = orc.curvature(P, st.flags, st.phi)
    Fp = fsl.make_params(w["shape"], curv_model=fsl.CURV_TR, tau=w["tau"], sigma=w["sigma"], theta=w["theta"])
    sim = fsl.Sim(Fp, phi0=phi.astype(np.float32), obstacle=obs)
    sim.curvature(fsl.CURV_TR)
    k_gpu = sim.host_state()["kappa"]
    n = _check_field(orc, st, n4, k_gpu, k_ref, max(w["shape"]))
    assert n > 500
    # the model tracks the sphere: mean kappa R within 1.5 % away from walls
    if name != "sessile64":
        R = g.get("R_s", g.get("R"))
        sel = st.flags == 2
        assert abs(np.mean(k_gpu[sel]) * R - 1) < (0.015 if name == "droplet32" else 0.05)
    sim.close()


def test_tr_inside_the_step(orc, fsl):
    """FSL_CURV_TR as the step's model: one step of a moving droplet against
    the oracle's step with TR (types bit-exact, f and phi within 1e-5)."""
    shape = (24, 24, 24)
    off = S.centre_offset(6)
    c = tuple(np.array(shape[::-1]) / 2 - 0.4 + off)
    phi = orc.fill(orc.geom("sphere", c=c, R=6.3, sub=8), shape)
    P = orc.params(shape, sigma=5e-4, tau=0.7, curv_model=4)
    st = orc.init_state(P, phi)
    fe = np.array([orc.feq(q, 1.0, np.array([0.04, 0.02, -0.01])) for q in range(19)])
    fluid = (st.flags & 3) > 0
    st.f[:, fluid] = fe[:, None] + S.pdf_noise(6, shape, 2e-4)[:, fluid]
    for _ in range(3):
        st, _, _, _ = orc.step(P, st)
    st.f = st.f.astype(np.float32).astype(np.float64)
    st.mass = st.mass.astype(np.float32).astype(np.float64)
    st.phi = st.phi.astype(np.float32).astype(np.float64)
    import copy
    Pn = copy.copy(P)
    Pn.eps = 1e9
    s2, _, _, rho = orc.step(Pn, st)  # no cell may sit within 1e-5 rho of a conversion threshold
    near = (np.abs(s2.mass - (1 + P.eps) * rho) < 1e-5 * rho) | (np.abs(s2.mass + P.eps * rho) < 1e-5 * rho)
    assert not np.any(near & (st.flags == 2))
    ref, counts, kref, _ = orc.step(P, st)
    sim = fsl.Sim(fsl.make_params(shape, sigma=5e-4, tau=0.7, curv_model=fsl.CURV_TR), phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    fl = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fl] - ref.f[:, fl])) <= 1e-5
    assert np.max(np.abs(h["phi"][fl] - ref.phi[fl])) <= 1e-5
    assert sim.status() == 0
    sim.close()
