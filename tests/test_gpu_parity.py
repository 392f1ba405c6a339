"""GPU parity of the CUDA path (libfsl via its C ABI) against the FP64 oracle.

Tolerances (the float ones follow the stated targets and are written here):
  flags, conversion results, cell counts   bit-exact (type bits)
  fill levels of spheres and caps          exact (k / sub^3 in both)
  single-step f, m, phi                    |d| <= 1e-5 max(|ref|, 1)
  curvature                                |d| <= 1e-4 max(|ref|, 1/L)
  PLIC normals and offsets                 |d| <= 2e-5
Parity of a step is checked from identical inputs (the oracle runs on the
FP32 state cast to FP64).  Threshold decisions (conversion) are checked for
guard-band cells first: none may lie within 1e-5 rho of a threshold.
"""
import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL_F = 1e-5
TOL_K = 1e-4


@pytest.fixture(scope="module")
def fsl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1509_07691_gb300 import build
    build.build()
    from paper_1509_07691_gb300 import fsl as F
    return F


def _geom_pair(orc, F, g, sub=16):
    kw = dict(c=g.get("c", (0, 0, 0)), R=g.get("R", 0.0), eps2=g.get("eps2", 0.0), c2=g.get("c2", (0, 0, 0)),
              R2=g.get("R2", 0.0), zw=g.get("zw", 0.0), h0=g.get("h0", 0.0), amp=g.get("amp", 0.0),
              wavelength=g.get("wavelength", 1.0), invert=g.get("invert", 0), sub=sub)
    if g["kind"] == "mode2":
        kw["R"] = g["R_s"]
    return orc.geom(g["kind"], **kw), F.make_geometry(g["kind"], **kw)


def _gpu_fill(F, shape, geom):
    import torch
    phi = torch.zeros(shape, dtype=torch.float32, device="cuda")
    F.fill_geometry(F.make_params(shape), geom, phi)
    torch.cuda.synchronize()
    return phi.double().cpu().numpy()


@pytest.mark.parametrize("name", ["droplet32", "sessile64"])
def test_fill_levels_exact(orc, fsl, name):
    w = S.workload(name)
    og, fg = _geom_pair(orc, fsl, w["geometry"])
    ref = orc.fill(og, w["shape"])
    got = _gpu_fill(fsl, w["shape"], fg)
    assert np.array_equal(got, ref)


def test_fill_levels_perturbed_sphere_sampled(orc, fsl):
    """256^3 P2-perturbed droplet (the benchmark geometry): sampled cells near
    the surface and all cells' totals."""
    w = S.workload("oscillating256")
    og, fg = _geom_pair(orc, fsl, w["geometry"])
    got = _gpu_fill(fsl, w["shape"], fg)
    band = np.nonzero((got.ravel() > 0) & (got.ravel() < 1))[0]
    pick = band[(S.uniform(77, 400) * band.size).astype(np.int64)]
    ref = orc.fill_cells(og, w["shape"], pick)
    assert np.max(np.abs(got.ravel()[pick] - ref)) <= 1.0 / 4096
    R = w["geometry"]["R"]
    assert got.sum() == pytest.approx(4.0 / 3.0 * np.pi * R ** 3, rel=2e-3)


def _init_both(orc, F, w, **kw):
    og, fg = _geom_pair(orc, F, w["geometry"])
    phi = orc.fill(og, w["shape"])
    obs = S.obstacle_mask(w["shape"], w["walls"])
    coll = F.TRT if w["collision"] == "trt" else F.BGK
    P = orc.params(w["shape"], collision=coll, tau=w["tau"], sigma=w["sigma"], theta=w["theta"], **kw)
    st = orc.init_state(P, phi, obs)
    Fp = F.make_params(w["shape"], collision=coll, tau=w["tau"], sigma=w["sigma"], theta=w["theta"],
                       curv_model=kw.get("curv_model", 0))
    sim = F.Sim(Fp, phi0=phi.astype(np.float32), obstacle=obs)
    return P, st, sim


@pytest.mark.parametrize("name", ["droplet32", "sessile64"])
def test_initial_state(orc, fsl, name):
    w = S.workload(name)
    P, st, sim = _init_both(orc, fsl, w)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, st.flags)
    fluid = (st.flags & 3) > 0
    assert np.max(np.abs(h["phi"][fluid] - st.phi[fluid])) <= 1e-7
    assert np.max(np.abs(h["mass"][fluid] - st.mass[fluid])) <= 1e-7
    assert np.max(np.abs(h["f"][:, fluid] - st.f[:, fluid])) <= 1e-7
    # near-obstacle bit: set exactly where a D3Q19 neighbour is an obstacle
    obs = st.flags == 8
    c, _, _ = orc.lattice()
    near = np.zeros_like(obs)
    for q in range(1, 19):
        near |= np.roll(obs, shift=(-c[q, 2], -c[q, 1], -c[q, 0]), axis=(0, 1, 2))
    assert np.array_equal((h["flags"] & fsl.NEAR_OBSTACLE) > 0, near)
    sim.close()


def _kappa_tol(ref, L):
    return TOL_K * np.maximum(np.abs(ref), 1.0 / L)


@pytest.mark.parametrize("name,model", [("droplet32", 0), ("droplet32", 1), ("sessile64", 0), ("sessile64", 1)])
def test_curvature_parity(orc, fsl, name, model):
    w = S.workload(name)
    if name == "sessile64":
        w["theta"] = np.radians(60.0)
    P, st, sim = _init_both(orc, fsl, w, curv_model=model)
    P.curv_model = model
    kref, nref, stats = orc.curvature(P, st.flags, st.phi)
    sim.curvature(model)
    h = sim.host_state()
    m = st.flags == 2
    L = max(w["shape"])
    n_gpu = None
    import torch
    ws = sim.workspace[: sim.N * 16].view(torch.float32).view(sim.N, 4).cpu().numpy().reshape(w["shape"] + (4,))
    assert np.max(np.abs(ws[m] - nref[m])) <= 2e-5
    err = np.abs(h["kappa"][m] - kref[m])
    assert np.all(err <= _kappa_tol(kref[m], L)), (err.max(), np.argmax(err))
    sim.close()


def _developed_state(orc, seed, shape=(24, 24, 24), u=(0.04, 0.02, -0.01), sigma=5e-4, steps=4, obstacle=None,
                     theta=np.pi / 2, collision=0, tau=0.7):
    """A droplet in motion (oracle-developed, then cast to FP32) with conversions in flight."""
    off = S.centre_offset(seed)
    c = tuple(np.array(shape[::-1]) / 2 - 0.4 + off)
    if obstacle is None:
        phi = orc.fill(orc.geom("sphere", c=c, R=6.3, sub=8), shape)
    else:
        phi = orc.fill(orc.geom("cap", c=(c[0], c[1], 0.5), R=7.3, zw=0.5, sub=8), shape)
    P = orc.params(shape, sigma=sigma, tau=tau, theta=theta, collision=collision)
    st = orc.init_state(P, phi, obstacle)
    u = np.array(u)
    fe = np.array([orc.feq(q, 1.0, u) for q in range(19)])
    fluid = (st.flags & 3) > 0
    st.f[:, fluid] = fe[:, None] + S.pdf_noise(seed, shape, 2e-4)[:, fluid]
    for _ in range(steps):
        st, _, _, _ = orc.step(P, st)
    st.f = st.f.astype(np.float32).astype(np.float64)
    st.mass = st.mass.astype(np.float32).astype(np.float64)
    st.phi = st.phi.astype(np.float32).astype(np.float64)
    return P, st


def _guard_band(orc, P, st):
    """cells whose pre-conversion mass lies within 1e-5 rho of a threshold"""
    import copy
    Pn = copy.copy(P)
    Pn.eps = 1e9
    s2, _, _, rho = orc.step(Pn, st)
    m = s2.mass
    was_if = st.flags == 2
    near = (np.abs(m - (1 + P.eps) * rho) < 1e-5 * rho) | (np.abs(m + P.eps * rho) < 1e-5 * rho)
    return np.count_nonzero(near & was_if)


def _gpu_from_state(F, P, st, model, obstacle=False):
    Fp = F.make_params(st.phi.shape, collision=P.collision, tau=P.tau, sigma=P.sigma, theta=P.theta,
                       curv_model=model)
    sim = F.Sim(Fp, phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    return sim


@pytest.mark.parametrize("seed,model", [(1, 0), (2, 0), (3, 1), (4, 2)])
def test_single_step_parity(orc, fsl, seed, model):
    P, st = _developed_state(orc, seed)
    P.curv_model = model
    assert _guard_band(orc, P, st) == 0
    ref, counts, kref, _ = orc.step(P, st)
    assert counts[3] + counts[4] + counts[5] + counts[6] > 0, "the seed must exercise conversions"
    sim = _gpu_from_state(fsl, P, st, model)
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    fluid = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fluid] - ref.f[:, fluid])) <= TOL_F
    iface = ref.flags == 2
    assert np.max(np.abs(h["mass"][iface] - ref.mass[iface])) <= TOL_F
    assert np.max(np.abs(h["phi"][fluid] - ref.phi[fluid])) <= TOL_F
    # curvature used inside the step
    was_if = st.flags == 2
    err = np.abs(h["kappa"][was_if] - kref[was_if])
    assert np.all(err <= _kappa_tol(kref[was_if], 24))
    m_gpu, lost_gpu = sim.mass_total()
    assert m_gpu == pytest.approx(orc.mass(P, ref), rel=1e-6)
    assert lost_gpu == pytest.approx(ref.lost - st.lost, abs=1e-6)
    sim.close()


@pytest.mark.parametrize("theta,model", [(60.0, 0), (120.0, 0), (60.0, 1)])
def test_single_step_parity_with_wall(orc, fsl, theta, model):
    """contact-line corner rule, wall reflection and wetting rows/normals"""
    shape = (16, 28, 28)
    obs = np.zeros(shape, np.uint8)
    obs[0] = obs[-1] = 1
    P, st = _developed_state(orc, 11, shape=shape, u=(0.03, -0.02, 0.0), obstacle=obs, theta=np.radians(theta),
                             collision=1, tau=0.8, sigma=1e-3)
    P.curv_model = model
    assert _guard_band(orc, P, st) == 0
    ref, counts, kref, _ = orc.step(P, st)
    sim = _gpu_from_state(fsl, P, st, model)
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    fluid = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fluid] - ref.f[:, fluid])) <= TOL_F
    assert np.max(np.abs(h["phi"][fluid] - ref.phi[fluid])) <= TOL_F
    was_if = st.flags == 2
    err = np.abs(h["kappa"][was_if] - kref[was_if])
    assert np.all(err <= _kappa_tol(kref[was_if], 28))
    sim.close()


def test_ragged_grid_and_stats(orc, fsl):
    """x extent not a multiple of the block size, ny != nz; stats and mass agree."""
    shape = (13, 11, 37)
    phi = orc.fill(orc.geom("sphere", c=(18.3, 5.2, 6.1), R=4.4, sub=8), shape)
    P = orc.params(shape, sigma=2e-4, tau=0.9)
    st = orc.init_state(P, phi)
    sim = fsl.Sim(fsl.make_params(shape, sigma=2e-4, tau=0.9), phi0=phi.astype(np.float32))
    ref = st
    for _ in range(3):
        ref, counts, _, _ = orc.step(P, ref)
    sim.step(3)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    s = sim.stats()
    assert s[0] == counts[0] and s[1] == counts[1] and s[2] == counts[2]
    assert s[4] == counts[7] and s[5] == counts[8] == 0
    assert s[7] == counts[1]
    fluid = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fluid] - ref.f[:, fluid])) <= 3 * TOL_F
    sim.close()


def test_mass_conservation_on_gpu(orc, fsl):
    """Total mass plus lost mass is conserved by the GPU step to FP32 rounding."""
    P, st = _developed_state(orc, 5, steps=1)
    sim = _gpu_from_state(fsl, P, st, 0)
    m0, l0 = sim.mass_total()
    for _ in range(10):
        sim.step(5)
        m, l = sim.mass_total()
        assert abs((m + l) - (m0 + l0)) < 2e-5 * m0
    assert sim.status() == 0
    sim.close()


@pytest.mark.parametrize("storage,tol_f", [(1, 1e-5), (2, 6e-5)])
def test_single_step_parity_reduced_precision(orc, fsl, storage, tol_f):
    """PDFs stored as 16-bit offsets f - w_q scaled by 2^8 (FP16 or BF16), collide
    in FP32.  The oracle steps from the decoded stored state; the tolerance is
    the rounding of the stored output: a half unit in the last place of an
    offset of up to about 0.01 times 2^8 (2^-11 for FP16, 2^-8 for BF16,
    divided by 2^8) plus the FP32 arithmetic."""
    import copy
    P, st = _developed_state(orc, 2)
    Fp = fsl.make_params(st.phi.shape, collision=P.collision, tau=P.tau, sigma=P.sigma, theta=P.theta,
                         storage=storage)
    sim = fsl.Sim(Fp, phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    st_in = copy.copy(st)
    st_in.f = sim.host_state()["f"]  # what the GPU holds after encoding
    assert _guard_band(orc, P, st_in) == 0
    ref, counts, _, _ = orc.step(P, st_in)
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    fluid = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fluid] - ref.f[:, fluid])) <= tol_f
    assert np.max(np.abs(h["phi"][fluid] - ref.phi[fluid])) <= TOL_F
    iface = ref.flags == 2
    # a cell converted from liquid gets m = rho summed over its 19 stored (rounded) PDFs
    assert np.max(np.abs(h["mass"][iface] - ref.mass[iface])) <= max(TOL_F, 10 * tol_f)
    sim.close()


@pytest.mark.parametrize("storage,tol_f", [(1, 1e-5), (2, 6e-5)])
@pytest.mark.parametrize("nx", [70, 71, 128])
def test_reduced_precision_pool_spans_and_x_wrap(orc, fsl, storage, tol_f, nx):
    """16-bit storage on a wavy pool between two walls that fills the whole x
    range: liquid cells at x = 0 and x = nx - 1 pull across the periodic x
    boundary, and the x rows end in a partial 32-cell segment (6 or 7 cells),
    or (nx = 128) in whole segments.  One step against the oracle from the
    decoded stored state, tolerances as above."""
    import copy
    shape = (16, 12, nx)
    phi = orc.fill(orc.geom("pool", h0=8.3, amp=1.2, wavelength=nx / 2.0, sub=8), shape)
    obs = S.obstacle_mask(shape, (0, 15))
    P = orc.params(shape, sigma=5e-4, tau=0.7)
    st = orc.init_state(P, phi, obs)
    fluid = (st.flags & 3) > 0
    assert fluid.reshape(16, -1, nx)[:, :, 0].any() and fluid.reshape(16, -1, nx)[:, :, nx - 1].any()
    fe = np.array([orc.feq(q, 1.0, np.array([0.03, -0.02, 0.01])) for q in range(19)])
    # noise seed: one whose stored (rounded) state has no cell in the guard band
    st.f[:, fluid] = fe[:, None] + S.pdf_noise(8 if nx == 128 else 7, shape, 2e-4)[:, fluid]
    st.f = st.f.astype(np.float32).astype(np.float64)
    Fp = fsl.make_params(shape, collision=P.collision, tau=P.tau, sigma=P.sigma, theta=P.theta, storage=storage)
    sim = fsl.Sim(Fp, phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    st_in = copy.copy(st)
    st_in.f = sim.host_state()["f"]
    assert _guard_band(orc, P, st_in) == 0
    ref, _, _, _ = orc.step(P, st_in)
    sim.step(1)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, ref.flags)
    liquid = ref.flags == 1
    assert np.max(np.abs(h["f"][:, liquid] - ref.f[:, liquid])) <= tol_f
    fl = (ref.flags & 3) > 0
    assert np.max(np.abs(h["f"][:, fl] - ref.f[:, fl])) <= tol_f
    assert sim.status() == 0
    sim.close()


@pytest.mark.parametrize("storage", [1, 2])
def test_reduced_precision_mass_drift_is_small(orc, fsl, storage):
    """Rounding of the stored offsets makes the total mass drift; over 50 steps of
    a moving droplet it stays within the storage resolution times the fluid cells."""
    P, st = _developed_state(orc, 5, steps=1)
    Fp = fsl.make_params(st.phi.shape, collision=P.collision, tau=P.tau, sigma=P.sigma, theta=P.theta,
                         storage=storage)
    sim = fsl.Sim(Fp, phi0=st.phi.astype(np.float32))
    sim.set_state(st.f, st.flags, st.mass, st.phi)
    m0, l0 = sim.mass_total()
    sim.step(50)
    m1, l1 = sim.mass_total()
    nfluid = int(np.count_nonzero(st.flags & 3))
    ulp = 2.0 ** -11 if storage == 1 else 2.0 ** -8
    assert abs((m1 + l1) - (m0 + l0)) < 50 * nfluid * ulp * 0.01 * 19
    assert sim.status() == 0
    sim.close()


def test_checkpoint_round_trip(orc, fsl, tmp_path):
    """fsl_save / fsl_load: the loaded state is the saved one bit for bit (PDFs
    of every cell, types, mass, fill level, total and lost mass), stepping on
    from it repeats the steps taken after the save, a truncated file and a
    context of another size are refused, and a refused load changes nothing."""
    import torch
    P, st = _developed_state(orc, 3)
    sim = _gpu_from_state(fsl, P, st, 0)
    sim.step(3)
    snap0 = sim.snapshot()
    h0 = sim.host_state()
    m0, l0 = sim.mass_total()
    path = str(tmp_path / "state.fslckpt")
    sim.save(path)
    sim.step(4)
    h4 = sim.host_state()
    sim.load(path)
    snap = sim.snapshot()
    for k in ("f", "mass", "phi"):
        assert torch.equal(snap[k].view(torch.uint8), snap0[k].view(torch.uint8)), k
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, h0["flags"] & fsl.TYPE_MASK)
    assert sim.mass_total() == (m0, l0)
    sim.step(4)
    h = sim.host_state()
    assert np.array_equal(h["flags"] & fsl.TYPE_MASK, h4["flags"] & fsl.TYPE_MASK)
    fl = (h4["flags"] & 3) > 0
    assert np.max(np.abs(h["f"][:, fl] - h4["f"][:, fl])) <= 1e-6
    for k in ("mass", "phi"):
        assert np.max(np.abs(h[k] - h4[k])) <= 1e-6, k
    # a truncated checkpoint is refused before any buffer is written
    with open(path, "rb") as fp:
        raw = fp.read()
    short = str(tmp_path / "short.fslckpt")
    with open(short, "wb") as fp:
        fp.write(raw[: len(raw) - 64])
    before = sim.snapshot()
    with pytest.raises(fsl.FslError):
        sim.load(short)
    after = sim.snapshot()
    for k in ("f", "flags", "mass", "phi"):
        assert torch.equal(after[k].view(torch.uint8), before[k].view(torch.uint8)), k
    assert sim.status() == 0
    sim.close()
    other = _gpu_from_state(fsl, *_developed_state(orc, 3, shape=(20, 20, 20)), 0)
    with pytest.raises(fsl.FslError):
        other.load(path)
    other.close()
