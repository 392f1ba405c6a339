"""FP64 CPU oracle of the FSLBM step (arXiv 1509.07691) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1509_07691_gb300``) and never imports it.

The numerical work is in ``fsl_oracle.c`` (plain C, FP64, compiled with gcc
without contraction or fast-math); this module marshals numpy arrays to it.

Parity status of the oracle functions
  plic_volume / plic_offset   pinned: brute-force sub-sampling, axis-aligned
                              closed forms, round trip
  ls_fit / kappa_from_coef    pinned: exact quadric point sets, closed-form
                              mean curvature of tilted quadrics
  tr_fan / tr_cell (TR)       pinned: exact sphere points give 1/R and plane
                              points 0 whatever the fan, symmetric rings on
                              quadrics give the mean curvature A + B, uneven
                              rings need the area weights, sub-sampled spheres
                              (magnitude of the paper's TR errors), cube
                              symmetry
  curvature (LSQR, FD)        pinned: planes (kappa = 0), spheres (kappa R -> 1,
                              second order for LSQR), cube symmetries (also of
                              a walled box with an interface in a concave
                              edge), spherical caps at the wall (contact-angle
                              sign, both models), the FD closed form
                              kappa = -cos(theta_eq)/4 of a vertical plane on
                              a wall
  reflect_phi                 pinned: the paper's reflection formula evaluated
                              by hand on axis walls, a 45-degree staircase and
                              next to a concave edge (neighbour set, aperture
                              ties, weights)
  step                        pinned: rest state, uniform flow, shear-wave decay
                              rate, exact mass conservation, type invariants,
                              Laplace pressure of a droplet; corner rule link by
                              link on a hand-built contact-line cell
  gas_volume / bubble_step    pinned: the volume of a sub-sampled bubble against
                              4/3 pi R^3, p_g = p0 at V = V0, and Boyle's law
                              for a bubble compressed by a liquid at higher
                              pressure (the bubble shrinks until p_g matches it)
  conversion readings         pinned on flat-interface scenarios whose outcome
                              (equal shares, and the normal-weighted shares of
                              reading K1: 1/5 to the new cells on the gas side
                              of a filled cell, 1/5 to the cells from liquid on
                              the liquid side of an emptied one)
                              follows from the readings by counting (thresholds,
                              filling beats emptying, new cells from gas and
                              from liquid, 13 equal excess shares, new cells at
                              the fluid neighbours' equilibrium), plus mass
                              conservation and the type invariants (the paper
                              cites, but does not state, the conversion rules)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsl_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
LIQUID, INTERFACE, GAS, OBSTACLE = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile fsl_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("collision", ctypes.c_int), ("curv_model", ctypes.c_int), ("literal_phi", ctypes.c_int),
                ("tau", ctypes.c_double), ("magic", ctypes.c_double), ("sigma", ctypes.c_double),
                ("p_gas", ctypes.c_double), ("theta", ctypes.c_double), ("eps", ctypes.c_double),
                ("frozen", ctypes.c_int), ("excess_rule", ctypes.c_int)]


class Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("invert", ctypes.c_int), ("sub", ctypes.c_int), ("pad_", ctypes.c_int),
                ("c", ctypes.c_double * 3), ("R", ctypes.c_double), ("eps2", ctypes.c_double),
                ("c2", ctypes.c_double * 3), ("R2", ctypes.c_double), ("zw", ctypes.c_double),
                ("n", ctypes.c_double * 3), ("d", ctypes.c_double),
                ("h0", ctypes.c_double), ("amp", ctypes.c_double), ("wavelength", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_L = ctypes.POINTER(ctypes.c_long)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            G = ctypes.POINTER(Geom)
            sig = {
                "orc_lattice": (None, [_I, _I, _I, _D, _I]),
                "orc_collide": (None, [P, _D, _D]),
                "orc_feq": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, _D]),
                "orc_plic_volume": (ctypes.c_double, [_D, ctypes.c_double]),
                "orc_plic_offset": (ctypes.c_double, [_D, ctypes.c_double, ctypes.c_int]),
                "orc_reflect_phi": (None, [P, _U8, _D, _D]),
                "orc_normals": (None, [P, _U8, _D, _D, ctypes.c_int]),
                "orc_ls_fit": (ctypes.c_int, [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D, _I]),
                "orc_kappa_from_coef": (ctypes.c_double, [_D]),
                "orc_curvature": (None, [P, _U8, _D, _D, _D, ctypes.c_int, _L]),
                "orc_tr_fan": (ctypes.c_double, [ctypes.c_int, _D, _D, _D, _I]),
                "orc_tr_cell": (ctypes.c_double, [P, _U8, _D, ctypes.c_long]),
                "orc_step": (None, [P, _D, _D, _U8, _D, _D, _D, _D, _D, _D, _L]),
                "orc_fill_cell": (ctypes.c_double, [G, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_fill": (None, [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]),
                "orc_fill_list": (None, [G, ctypes.c_int, ctypes.c_int, ctypes.c_long, _L, _D]),
                "orc_init_state": (None, [P, _U8, _D, _U8, _D, _D]),
                "orc_mass": (ctypes.c_double, [P, _U8, _D, _D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(l, name)
                fn.restype = res
                fn.argtypes = args
            _lib = l
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _u8(a):
    return a.ctypes.data_as(_U8)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    """(c[19,3] int, w[19], opp[19]) as the oracle defines them."""
    cx, cy, cz, opp = (np.zeros(Q, np.int32) for _ in range(4))
    w = np.zeros(Q)
    I = lambda a: a.ctypes.data_as(_I)
    lib().orc_lattice(I(cx), I(cy), I(cz), _d(w), I(opp))
    return np.stack([cx, cy, cz], 1), w, opp


def params(shape, collision=0, curv_model=0, tau=1.0, magic=3.0 / 16.0, sigma=0.0, p_gas=1.0 / 3.0,
           theta=np.pi / 2, eps=1e-3, literal_phi=0, frozen=0, excess_rule=0) -> Params:
    """shape = (nz, ny, nx) of the numpy arrays (x fastest).  frozen = 1: cell
    types frozen (no conversion test), as in the adjoint windows.
    excess_rule = 1: excess mass shared by normal-weighted shares (reading K1)."""
    nz, ny, nx = shape
    return Params(nx, ny, nz, collision, curv_model, literal_phi, tau, magic, sigma, p_gas, theta, eps, frozen,
                  excess_rule)


def feq(q, rho, u):
    return lib().orc_feq(int(q), float(rho), _d(_f64(u)))


def collide(P: Params, f):
    f = _f64(f)
    out = np.zeros(Q)
    lib().orc_collide(ctypes.byref(P), _d(f), _d(out))
    return out


def plic_volume(n, a):
    return lib().orc_plic_volume(_d(_f64(n)), float(a))


def plic_offset(n, phi, iters=60):
    return lib().orc_plic_offset(_d(_f64(n)), float(phi), int(iters))


def ls_fit(rows, rhs, crow=None, crhs=None):
    """Least-squares fit of (A,B,C,H,I); returns (coef[5], mode)."""
    rows = _f64(np.asarray(rows).reshape(-1, 5))
    rhs = _f64(rhs)
    m = rows.shape[0]
    nc = 0 if crow is None else 2
    crow = _f64(np.zeros((2, 5)) if crow is None else crow)
    crhs = _f64(np.zeros(2) if crhs is None else crhs)
    coef = np.zeros(5)
    mode = ctypes.c_int(0)
    lib().orc_ls_fit(m, _d(rows if m else np.zeros(5)), _d(rhs if m else np.zeros(1)), nc, _d(crow), _d(crhs),
                     _d(coef), ctypes.byref(mode))
    return coef, mode.value


def kappa_from_coef(c):
    return lib().orc_kappa_from_coef(_d(_f64(c)))


def geom(kind, c=(0, 0, 0), R=0.0, eps2=0.0, c2=(0, 0, 0), R2=0.0, zw=0.0, n=(0, 0, 1), d=0.0,
         h0=0.0, amp=0.0, wavelength=1.0, invert=0, sub=16) -> Geom:
    kinds = {"sphere": 0, "mode2": 1, "cap": 2, "two_spheres": 3, "pool": 4, "plane": 5}
    k = kinds[kind] if isinstance(kind, str) else int(kind)
    D3 = ctypes.c_double * 3
    return Geom(k, int(invert), int(sub), 0, D3(*c), R, eps2, D3(*c2), R2, zw, D3(*n), d, h0, amp, wavelength)


def fill(G: Geom, shape):
    nz, ny, nx = shape
    phi = np.zeros(shape)
    lib().orc_fill(ctypes.byref(G), nx, ny, nz, _d(phi))
    return phi


def fill_cells(G: Geom, shape, idx):
    nz, ny, nx = shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.shape[0])
    lib().orc_fill_list(ctypes.byref(G), nx, ny, idx.shape[0], idx.ctypes.data_as(_L), _d(out))
    return out


class State:
    """FP64 state: f[19,nz,ny,nx] (post-collision), flags, mass, phi (x fastest)."""

    def __init__(self, f, flags, mass, phi):
        self.f, self.flags, self.mass, self.phi = f, flags, mass, phi
        self.lost = 0.0

    def copy(self):
        s = State(self.f.copy(), self.flags.copy(), self.mass.copy(), self.phi.copy())
        s.lost = self.lost
        return s


def init_state(P: Params, phi0, obstacle=None) -> State:
    shape = phi0.shape
    phi = _f64(phi0).copy()
    obstacle = np.zeros(shape, np.uint8) if obstacle is None else np.ascontiguousarray(obstacle, np.uint8)
    flags = np.zeros(shape, np.uint8)
    f = np.zeros((Q,) + shape)
    mass = np.zeros(shape)
    lib().orc_init_state(ctypes.byref(P), _u8(obstacle), _d(phi), _u8(flags), _d(f), _d(mass))
    return State(f, flags, mass, phi)


def normals(P: Params, flags, phi, iters=60):
    flags = np.ascontiguousarray(flags, np.uint8)
    phi = _f64(phi)
    out = np.zeros(phi.shape + (4,))
    lib().orc_normals(ctypes.byref(P), _u8(flags), _d(phi), _d(out), int(iters))
    return out


def reflect_phi(P: Params, flags, phi):
    flags = np.ascontiguousarray(flags, np.uint8)
    phi = _f64(phi)
    out = np.zeros_like(phi)
    lib().orc_reflect_phi(ctypes.byref(P), _u8(flags), _d(phi), _d(out))
    return out


def tr_fan(u, v, h, key=None):
    """TR mean curvature of a fan of points (u, v, h) in the centre's tangent frame."""
    u, v, h = (_f64(np.asarray(a).ravel()) for a in (u, v, h))
    key = np.arange(u.size, dtype=np.int32) if key is None else np.ascontiguousarray(key, dtype=np.int32)
    return lib().orc_tr_fan(int(u.size), _d(u), _d(v), _d(h), key.ctypes.data_as(_I))


def tr_cell(P: Params, flags, normal4, i):
    """TR curvature of cell index i from given normals and PLIC offsets (normal4[..., 4])."""
    flags = np.ascontiguousarray(flags, np.uint8)
    n4 = _f64(normal4)
    return lib().orc_tr_cell(ctypes.byref(P), _u8(flags), _d(n4), int(i))


def curvature(P: Params, flags, phi, iters=60):
    """Returns (kappa, normal4, stats[full, isotropic, zero, centre-constrained])."""
    flags = np.ascontiguousarray(flags, np.uint8)
    phi = _f64(phi)
    kappa = np.zeros(phi.shape)
    n4 = np.zeros(phi.shape + (4,))
    stats = np.zeros(4, np.int64)
    lib().orc_curvature(ctypes.byref(P), _u8(flags), _d(phi), _d(kappa), _d(n4), int(iters),
                        stats.ctypes.data_as(_L))
    return kappa, n4, stats


def step(P: Params, S: State, kappa=None, normal4=None, iters=60):
    """One time step; returns (new State, counts[9], kappa used, rho(t+1))."""
    if kappa is None or normal4 is None:
        k2, n2, _ = curvature(P, S.flags, S.phi, iters)
        kappa = k2 if kappa is None else kappa
        normal4 = n2 if normal4 is None else normal4
    out = S.copy()
    fout = S.f.copy()
    rho = np.zeros(S.phi.shape)
    lost = ctypes.c_double(S.lost)
    counts = np.zeros(9, np.int64)
    lib().orc_step(ctypes.byref(P), _d(_f64(S.f)), _d(fout), _u8(out.flags), _d(out.mass), _d(out.phi),
                   _d(_f64(kappa)), _d(_f64(normal4)), _d(rho), ctypes.byref(lost), counts.ctypes.data_as(_L))
    out.f = fout
    out.lost = lost.value
    return out, counts, kappa, rho


def gas_volume(S: State):
    """Gas volume of a state (the bubble model of Sec. III.A): gas cells count
    1, interface cells 1 - phi; liquid and obstacle cells 0."""
    t = S.flags & 15
    return float(np.count_nonzero(t == GAS) + np.sum(1.0 - S.phi[t == INTERFACE]))


def bubble_step(P: Params, S: State, p0: float, V0: float, iters=60):
    """One step with the bubble model (Sec. III.A): the gas pressure follows
    the gas volume as an isothermal ideal gas, p_g = p0 V0 / V(t) (reading
    B1), set from the state at t before the step; returns step()'s tuple and
    the p_g used."""
    import copy
    Pb = copy.copy(P)
    Pb.p_gas = p0 * V0 / gas_volume(S)
    return step(Pb, S, iters=iters), Pb.p_gas


def mass(P: Params, S: State):
    return lib().orc_mass(ctypes.byref(P), _u8(S.flags), _d(_f64(S.f)), _d(_f64(S.mass)))
