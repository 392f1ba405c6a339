"""The advection test of Sec. III.A (Tab. advection) on the GPU path, against
the FP64 oracle: a gas bubble carried by a prescribed constant flow, the
lattice Boltzmann data held at f = feq(1, u0) before every step
(fsl_prescribe_flow), so that only the mass exchange of Eqs. (advection1/2)
and the conversions move the fill level.

* one step from identical inputs: cell types bit-exact, phi and m within
  1e-5 (the file's float tolerance, as in test_gpu_parity.py);
* the whole translation over d = 10 cells (T = 200 steps at u0 = 0.05): the
  L1 and L2 norms of the bubble indicator 1 - phi against its shifted
  initial field agree with the oracle's within 2 % relative, and with the
  printed 3.00 % / 9.38 % in magnitude (as the oracle's own pin)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1509_07691_gb300 import build
    build.build()
    from paper_1509_07691_gb300 import fsl as F
    return F


def _bubble(orc, d, L, c_off=(0.0, 0.0, 0.0)):
    shape = (L, L, L)
    c = tuple(L / 2 + o for o in c_off)
    return orc.fill(orc.geom("sphere", c=c, R=d / 2, sub=16, invert=1), shape)


def _norms(phi0, phiT, d):
    g0 = 1 - phi0
    g1 = 1 - np.roll(phiT, -d, axis=2)
    return np.abs(g1 - g0).sum() / g0.sum(), np.sqrt(((g1 - g0) ** 2).sum() / (g0 ** 2).sum())


def test_single_step_with_prescribed_flow(orc, fsl):
    L, d, u0 = 20, 10, 0.05
    phi0 = _bubble(orc, d, L, (0.137, -0.213, 0.071))
    P = orc.params(phi0.shape, sigma=0.0, tau=1.0, curv_model=2)
    st = orc.init_state(P, phi0)
    fe = np.array([orc.feq(q, 1.0, np.array([u0, 0, 0])) for q in range(19)])
    for _ in range(7):  # develop a few steps so that conversions are in flight
        st.f[:] = fe[:, None, None, None]
        st, _, _, _ = orc.step(P, st)
    st.mass = st.mass.astype(np.float32).astype(np.float64)
    st.phi = st.phi.astype(np.float32).astype(np.float64)
    st.f[:] = fe[:, None, None, None]
    ref, counts, _, _ = orc.step(P, st)
    sim = fsl.Sim(fsl.make_params(phi0.shape, sigma=0.0, tau=1.0, curv_model=fsl.CURV_NONE),
                  phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    sim.f_current().fill_(0.0)  # whatever the buffer held, the prescribed flow replaces it at fluid cells
    sim.prescribe_flow(1.0, (u0, 0.0, 0.0))
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    fl = (ref.flags & 3) > 0
    assert np.max(np.abs(h["phi"][fl] - ref.phi[fl])) <= 1e-5
    iface = ref.flags == 2
    assert np.max(np.abs(h["mass"][iface] - ref.mass[iface])) <= 1e-5
    sim.close()


@pytest.mark.slow
def test_translation_d10_against_the_oracle(orc, fsl):
    L, d, u0 = 20, 10, 0.05
    T = int(round(d / u0))
    phi0 = _bubble(orc, d, L)
    P = orc.params(phi0.shape, sigma=0.0, tau=1.0, curv_model=2)
    st = orc.init_state(P, phi0)
    fe = np.array([orc.feq(q, 1.0, np.array([u0, 0, 0])) for q in range(19)])
    for _ in range(T):
        st.f[:] = fe[:, None, None, None]
        st, _, _, _ = orc.step(P, st)
    l1_ref, l2_ref = _norms(orc.init_state(P, phi0).phi, st.phi, d)
    sim = fsl.Sim(fsl.make_params(phi0.shape, sigma=0.0, tau=1.0, curv_model=fsl.CURV_NONE),
                  phi0=phi0.astype(np.float32))
    start = sim.host_state()["phi"]
    for _ in range(T):
        sim.prescribe_flow(1.0, (u0, 0.0, 0.0))
        sim.step(1)
    l1, l2 = _norms(start, sim.host_state()["phi"], d)
    assert l1 == pytest.approx(l1_ref, rel=0.02)
    assert l2 == pytest.approx(l2_ref, rel=0.02)
    # the printed d = 10 row: L1 = 3.00 %, L2 = 9.38 % (magnitude, conversion rules are readings)
    assert 0.03 / 2.5 < l1 < 0.03 * 2.5
    assert l2 == pytest.approx(0.0938, rel=0.25)
    assert sim.status() == 0
    sim.close()
