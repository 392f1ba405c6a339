"""GPU adjoint windows (frozen cell types) against the FP64 oracle.

  frozen window          f', m, phi after a 12-step window: |d| <= 1e-5 max(|ref|, 1)
                         (the single-step bar; FP32 rounding does not grow
                         past it in 12 steps); types bit-exact
  curvature Jacobian     kappa of the dual pass within the curvature bar
                         (1e-4 relative); dkappa_x/dphi_y and dkappa_x/dtheta
                         against central differences (h = 1e-6) of the oracle's
                         FP64 LSQR curvature, |d| <= 2e-3 max|row| (FP32 dual
                         arithmetic through a least-squares solve)
  dot products           <v, J^T w> (adjoint) = <J v, w> (central differences
                         of the oracle window, FP64) for random v on
                         (phi, m, f') and w on phi: relative 1e-3, from a
                         moving state whose interface fill levels lie in
                         [0.02, 0.98] (phi = 0 or 1 is the PLIC clamp, a kink)
  dL/dsigma, dL/dtheta   sessile droplet 64^3, R 16, 50-step window with a
                         checkpoint every 10 steps, fill-level L2 loss to the
                         oracle's window at theta 70 deg, sigma 3e-4, evaluated
                         at theta 90 deg, sigma 2e-4: within 1e-2 of the FP64
                         reference (central differences of the oracle window,
                         h = 1e-4 relative) and within 3e-2 of central
                         differences of the GPU's own FP32 window (steps
                         5e-2 sigma and 1e-2 rad: at h = 1e-4 the FP32
                         rounding of L, ~1e-6 relative, exceeds the difference)
  fit                    gradient-based descent from (90 deg, 2e-4) recovers
                         theta within 1 deg
"""
import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1509_07691_gb300 import build
    build.build()
    from paper_1509_07691_gb300 import fsl
    return fsl


def _sessile_inputs(orc, shape, R, sub=8):
    H, L = shape[0], shape[1]
    phi = orc.fill(orc.geom("cap", c=(L / 2 + 0.3, L / 2 - 0.2, 0.5), R=R, zw=0.5, sub=sub), shape)
    obs = S.obstacle_mask(shape, (0, H - 1))
    return phi, obs


def _pair(orc, F, shape, R, theta, sigma, tau=0.8):
    phi, obs = _sessile_inputs(orc, shape, R)
    P = orc.params(shape, collision=1, tau=tau, sigma=sigma, theta=theta, frozen=1)
    st = orc.init_state(P, phi, obs)
    Fp = F.make_params(shape, collision=F.TRT, tau=tau, sigma=sigma, theta=theta)
    sim = F.Sim(Fp, phi0=phi.astype(np.float32), obstacle=obs)
    return P, st, sim


def _gpu_state_as_oracle(orc, sim):
    h = sim.host_state()
    st = orc.State(h["f"].copy(), (h["flags"] & 15).astype(np.uint8), h["mass"].copy(), h["phi"].copy())
    return st


def _orc_window(orc, P, st, steps):
    for _ in range(steps):
        st, counts, _, _ = orc.step(P, st)
        assert counts[3:7].sum() == 0
    return st


def test_frozen_window_matches_oracle(orc, F):
    P, st, sim = _pair(orc, F, (20, 24, 24), 7.0, np.radians(60.0), 3e-4)
    st = _gpu_state_as_oracle(orc, sim)
    sim.window_forward(12, 4)
    h = sim.host_state()
    ref = _orc_window(orc, P, st, 12)
    assert np.array_equal(h["flags"] & 15, ref.flags)
    fl = (ref.flags & 3) > 0
    ifc = ref.flags == 2
    assert np.max(np.abs(h["f"][:, fl] - ref.f[:, fl])) <= 1e-5
    assert np.max(np.abs(h["phi"][ifc] - ref.phi[ifc])) <= 1e-5
    assert np.max(np.abs(h["mass"][ifc] - ref.mass[ifc])) <= 1e-5
    # the context continues with plain steps from the window's end state
    P.frozen = 0
    ref2, counts, _, _ = orc.step(P, _gpu_state_as_oracle(orc, sim))
    sim.step(1)
    h2 = sim.host_state()
    assert np.array_equal(h2["flags"] & 15, ref2.flags)
    fl2 = (ref2.flags & 3) > 0
    assert np.max(np.abs(h2["f"][:, fl2] - ref2.f[:, fl2])) <= 1e-5
    sim.close()


def _slots(i, cells_shape):
    nz, ny, nx = cells_shape
    z, rem = divmod(int(i), nx * ny)
    y, x = divmod(rem, nx)
    return x, y, z


def test_kappa_jacobian_matches_oracle_differences(orc, F):
    shape = (14, 20, 20)
    P, st, sim = _pair(orc, F, shape, 6.0, np.radians(60.0), 5e-4)
    sim.window_forward(3, 3)  # a developed, generic fill level
    jac, cells, kval = sim.kappa_jacobian()
    kap = sim.curvature(F.CURV_LSQR).clone()
    h = sim.host_state()
    jac, cells, kval = jac.cpu().numpy().astype(np.float64), cells.cpu().numpy(), kval.cpu().numpy()
    kf = kap.cpu().numpy().ravel()[cells]
    assert np.all(np.abs(kval - kf) <= 1e-4 * np.maximum(np.abs(kf), 1.0 / max(shape)))
    flags = (h["flags"] & 15).astype(np.uint8)
    phi = h["phi"].copy()
    P.curv_model = 0
    near = (h["flags"] & 16) > 0
    nz, ny, nx = shape
    order = np.argsort(-(near.ravel()[cells]).astype(int), kind="stable")
    pick = list(order[:8]) + list(order[8 :: max(1, (len(order) - 8) // 16)][:16])
    hstep = 1e-6
    worst = 0.0
    for k in pick:
        x, y, z = _slots(cells[k], shape)
        row = np.zeros(344)
        for s in range(343):
            dx, dy, dz = s % 7 - 3, (s // 7) % 7 - 3, s // 49 - 3
            j = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
            if flags[j] != 2:
                continue
            pp, pm = phi.copy(), phi.copy()
            pp[j] += hstep
            pm[j] -= hstep
            kp = orc.curvature(P, flags, pp)[0][z, y, x]
            km = orc.curvature(P, flags, pm)[0][z, y, x]
            row[s] = (kp - km) / (2 * hstep)
        P.theta += hstep
        kp = orc.curvature(P, flags, phi)[0][z, y, x]
        P.theta -= 2 * hstep
        km = orc.curvature(P, flags, phi)[0][z, y, x]
        P.theta += hstep
        row[343] = (kp - km) / (2 * hstep)
        used = np.array([flags[((z + s // 49 - 3) % nz, (y + (s // 7) % 7 - 3) % ny, (x + s % 7 - 3) % nx)] == 2
                         for s in range(343)] + [True])
        scale = max(np.max(np.abs(row)), 1e-3)
        err = np.max(np.abs(jac[k][used] - row[used])) / scale
        worst = max(worst, err)
        assert err <= 2e-3, (k, near.ravel()[cells[k]], err)
    print(f"curvature Jacobian: worst row error {worst:.2e} of max|row|")
    sim.close()


def _rand(seed, shape, mask):
    return np.where(mask, S.normal(seed, int(np.prod(shape))).reshape(shape), 0.0)


def test_adjoint_dot_products_against_oracle_differences(orc, F):
    import torch
    shape = (12, 18, 18)
    P, st, sim = _pair(orc, F, shape, 5.5, np.radians(60.0), 5e-4)
    # a moving state (common to both sides, FP32 values)
    fluid = (st.flags & 3) > 0
    u = np.array([0.02, -0.015, 0.01])
    fe = np.array([orc.feq(q, 1.0, u) for q in range(19)])
    f0 = st.f.copy()
    f0[:, fluid] = fe[:, None] + 1e-3 * _rand(3, (19,) + shape, np.broadcast_to(fluid, (19,) + shape))[:, fluid]
    # interface fill levels inside (0, 1): at phi = 0 or 1 the PLIC offset is
    # clamped, a kink with a cube-root branch on the inner side, where the map
    # has no derivative to test
    ifc0 = st.flags == 2
    phi0 = np.where(ifc0, np.clip(st.phi, 0.02, 0.98), st.phi)
    m0 = np.where(ifc0, phi0 * f0.sum(axis=0), st.mass)
    sim.set_state(f0.astype(np.float32), st.flags, m0.astype(np.float32), phi0.astype(np.float32))
    s0 = _gpu_state_as_oracle(orc, sim)
    ifc = s0.flags == 2
    W, K = 5, 2
    w = _rand(11, shape, ifc)
    sim.window_forward(W, K)
    ds, dt, dphi0, dm0, df0 = sim.window_adjoint(torch.from_numpy(w.astype(np.float32)).cuda(), inputs=True)
    dphi0, dm0, df0 = (t.double().cpu().numpy() for t in (dphi0, dm0, df0))
    vp, vm = _rand(12, shape, ifc), _rand(13, shape, ifc)
    vf = _rand(14, (19,) + shape, np.broadcast_to((s0.flags & 3) > 0, (19,) + shape))
    adj = float(np.sum(vp * dphi0) + np.sum(vm * dm0) + np.sum(vf * df0))

    def window_dot(st0, Pw):
        return float(np.sum(w * _orc_window(orc, Pw, st0, W).phi))

    hh = 1e-6

    def shifted(sgn):
        s = s0.copy()
        s.phi = s.phi + sgn * hh * vp
        s.mass = s.mass + sgn * hh * vm
        s.f = s.f + sgn * hh * vf
        return s

    fd = (window_dot(shifted(1), P) - window_dot(shifted(-1), P)) / (2 * hh)
    print(f"dot product: adjoint {adj:.9e}, oracle differences {fd:.9e}")
    assert abs(adj - fd) <= 1e-3 * abs(fd)
    def P_at(sigma, theta):
        return orc.params(shape, collision=1, tau=0.8, sigma=sigma, theta=theta, frozen=1)

    for name, got in (("sigma", ds), ("theta", dt)):
        if name == "sigma":
            step = 1e-4 * P.sigma
            Pp, Pm = P_at(P.sigma + step, P.theta), P_at(P.sigma - step, P.theta)
        else:
            step = 1e-4
            Pp, Pm = P_at(P.sigma, P.theta + step), P_at(P.sigma, P.theta - step)
        ref = (window_dot(s0.copy(), Pp) - window_dot(s0.copy(), Pm)) / (2 * step)
        print(f"d<w,phi>/d{name}: adjoint {got:.9e}, oracle differences {ref:.9e}")
        assert abs(got - ref) <= 1e-3 * abs(ref) + 1e-9
    sim.close()


# ---- sessile droplet 64^3: gradients and the fit ----------------------------------
TARGET = (np.radians(70.0), 3e-4)
START = (np.radians(90.0), 2e-4)
WINDOW, CKPT = 50, 10


@pytest.fixture(scope="module")
def sessile(orc):
    w = S.workload("sessile64")
    g = w["geometry"]
    phi = orc.fill(orc.geom("cap", c=g["c"], R=g["R"], zw=g["zw"], sub=8), w["shape"])
    obs = S.obstacle_mask(w["shape"], w["walls"])

    def window(theta, sigma):
        P = orc.params(w["shape"], collision=1, tau=w["tau"], sigma=sigma, theta=theta, frozen=1)
        return _orc_window(orc, P, orc.init_state(P, phi, obs), WINDOW)

    tgt = window(*TARGET)
    ifc = tgt.flags == 2

    def loss(theta, sigma):
        return float(np.sum((window(theta, sigma).phi[ifc] - tgt.phi[ifc]) ** 2))

    th, sg = START
    ht, hs = 1e-4, 1e-4 * sg
    ref = ((loss(th, sg + hs) - loss(th, sg - hs)) / (2 * hs), (loss(th + ht, sg) - loss(th - ht, sg)) / (2 * ht))
    return dict(w=w, phi=phi, obs=obs, target=tgt.phi, ifc=ifc, ref=ref)


def _sessile_sim(F, case):
    w = case["w"]
    Fp = F.make_params(w["shape"], collision=F.TRT, tau=w["tau"], sigma=START[1], theta=START[0])
    return F.Sim(Fp, phi0=case["phi"].astype(np.float32), obstacle=case["obs"])


def test_window_gradient_against_fp64_reference_and_differences(F, sessile):
    import torch
    sim = _sessile_sim(F, sessile)
    start = sim.snapshot()
    tgt = torch.from_numpy(sessile["target"].astype(np.float32)).cuda()
    ifc = torch.from_numpy(sessile["ifc"]).cuda()

    def run(theta, sigma, grad=False):
        sim.restore(start)
        sim.set_surface(sigma, theta)
        sim.window_forward(WINDOW, CKPT)
        d = torch.where(ifc, sim.phi - tgt, torch.zeros_like(tgt))
        L = float(torch.sum(d.double() ** 2))
        if not grad:
            return L
        ds, dt = sim.window_adjoint(2.0 * d)
        return L, ds, dt

    th, sg = START
    L, ds, dt = run(th, sg, grad=True)
    ref_s, ref_t = sessile["ref"]
    # FP32 differences: L carries rounding of ~1e-6 relative, so the steps are
    # as large as the O(h^2) error allows (5e-2 sigma, 1e-2 rad)
    hs, ht = 5e-2 * sg, 1e-2
    fd_s = (run(th, sg + hs) - run(th, sg - hs)) / (2 * hs)
    fd_t = (run(th + ht, sg) - run(th - ht, sg)) / (2 * ht)
    print(f"L = {L:.6e}; dL/dsigma adjoint {ds:.6e}, FP64 ref {ref_s:.6e}, FP32 differences {fd_s:.6e}")
    print(f"dL/dtheta adjoint {dt:.6e}, FP64 ref {ref_t:.6e}, FP32 differences {fd_t:.6e}")
    assert abs(ds - ref_s) <= 1e-2 * abs(ref_s)
    assert abs(dt - ref_t) <= 1e-2 * abs(ref_t)
    assert abs(ds - fd_s) <= 3e-2 * abs(ref_s)
    assert abs(dt - fd_t) <= 3e-2 * abs(ref_t)
    # the adjoint is bit-reproducible
    L2, ds2, dt2 = run(th, sg, grad=True)
    assert (L2, ds2, dt2) == (L, ds, dt)
    sim.close()


def test_fit_recovers_contact_angle(F, sessile):
    import torch
    from scipy.optimize import minimize
    sim = _sessile_sim(F, sessile)
    start = sim.snapshot()
    tgt = torch.from_numpy(sessile["target"].astype(np.float32)).cuda()
    ifc = torch.from_numpy(sessile["ifc"]).cuda()
    # scaled unknowns: sigma / 1e-4 and theta in units of 10 degrees
    scale = np.array([1e-4, np.radians(10.0)])

    def fun(xs):
        surface = torch.tensor(xs * scale, dtype=torch.float64, requires_grad=True)
        sim.restore(start)
        phi = F.FslStepWindow.apply(surface, sim, WINDOW, CKPT)
        loss = torch.sum(torch.where(ifc, phi - tgt, torch.zeros_like(tgt)).double() ** 2)
        loss.backward()
        return float(loss.detach()), surface.grad.numpy() * scale

    x0 = np.array([START[1], START[0]]) / scale
    res = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=[(0.5, 6.0), (3.0, 15.0)],
                   options=dict(maxiter=60, ftol=1e-14, gtol=1e-12))
    sigma, theta = res.x * scale
    print(f"fit: theta {np.degrees(theta):.3f} deg, sigma {sigma:.4e} after {res.nfev} evaluations ({res.message})")
    assert abs(np.degrees(theta) - 70.0) < 1.0
    assert abs(sigma / 3e-4 - 1.0) < 0.05
    sim.close()
