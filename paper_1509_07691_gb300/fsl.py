"""Thin Python binding of libfsl (include/fsl.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch only
provides the device buffers (caller-owned, as the C ABI requires) and the
CUDA stream.  If libfsl.so is missing the import of this module fails: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfsl.so")

OK, EINVAL, ECUDA, ECAPACITY, ETIMEOUT, ENAN, EUNSUPPORTED, EIO = 0, -1, -2, -3, -4, -5, -6, -7
LIQUID, INTERFACE, GAS, OBSTACLE, TYPE_MASK, NEAR_OBSTACLE = 1, 2, 4, 8, 15, 16
BGK, TRT = 0, 1
CURV_LSQR, CURV_FD, CURV_NONE, CURV_MLP, CURV_TR = 0, 1, 2, 3, 4
F32, F16_OFS, BF16_OFS = 0, 1, 2
WHERE_NONE, WHERE_HOST, WHERE_DEVICE = 0, 1, 2
JAC_STRIDE = 344  # curvature Jacobian row: 7x7x7 window slots, then theta
GEOMETRY_KINDS = {"sphere": 0, "mode2": 1, "cap": 2, "two_spheres": 3, "pool": 4, "plane": 5}
Q = 19


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("curv_model", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("storage_shift", ctypes.c_int32), ("plic_iters", ctypes.c_int32),
                ("tau", ctypes.c_double), ("magic", ctypes.c_double), ("sigma", ctypes.c_double),
                ("p_gas", ctypes.c_double), ("theta", ctypes.c_double), ("eps_convert", ctypes.c_double),
                ("lsqr_fp64_cond", ctypes.c_double), ("excess_rule", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class Fields(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * 2), ("flags", ctypes.c_void_p * 2), ("mass", ctypes.c_void_p),
                ("phi", ctypes.c_void_p), ("kappa", ctypes.c_void_p), ("workspace", ctypes.c_void_p)]


class Geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("invert", ctypes.c_int32), ("sub", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("c", ctypes.c_double * 3), ("R", ctypes.c_double),
                ("eps2", ctypes.c_double), ("c2", ctypes.c_double * 3), ("R2", ctypes.c_double),
                ("zw", ctypes.c_double), ("n", ctypes.c_double * 3), ("d", ctypes.c_double),
                ("h0", ctypes.c_double), ("amp", ctypes.c_double), ("wavelength", ctypes.c_double)]


_lib = None
_SIGNATURES = {
    "fsl_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Params)]),
    "fsl_fill_geometry": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(Geometry), ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "fsl_init": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(Fields), ctypes.c_void_p, ctypes.c_int,
                                ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "fsl_refresh": (ctypes.c_int, [ctypes.c_void_p]),
    "fsl_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fsl_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fsl_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fsl_curvature": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "fsl_mass": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "fsl_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "fsl_step_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "fsl_prescribe_flow": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_double] * 4),
    "fsl_set_bubble": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    "fsl_bubble": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "fsl_conversions": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p,
                                       ctypes.c_int64]),
    "fsl_mass_static": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "fsl_mlp_param_bytes": (ctypes.c_size_t, []),
    "fsl_mlp_master_count": (ctypes.c_int, []),
    "fsl_mlp_stencils": (ctypes.c_int, [ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_int, ctypes.c_float,
                                                                                   ctypes.c_uint64] + [ctypes.c_void_p] * 3),
    "fsl_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4),
    "fsl_mlp_status": (ctypes.c_int, [ctypes.c_int]),
    "fsl_mlp_train_workspace": (ctypes.c_size_t, [ctypes.c_int]),
    "fsl_mlp_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] +
                          [ctypes.c_void_p] * 4),
    "fsl_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_int, ctypes.c_float, ctypes.c_int] +
                           [ctypes.c_void_p] * 3),
    "fsl_mlp_epoch_workspace": (ctypes.c_size_t, [ctypes.c_int]),
    "fsl_mlp_train_epoch": (ctypes.c_int, [ctypes.c_void_p] * 7 + [ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                                                    ctypes.c_int] + [ctypes.c_void_p] * 3),
    "fsl_mlp_pack": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "fsl_mlp_attach": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "fsl_adjoint_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int]),
    "fsl_set_surface": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    "fsl_window_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_size_t]),
    "fsl_window_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)] + [ctypes.c_void_p] * 3),
    "fsl_kappa_jacobian": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int] +
                           [ctypes.c_void_p] * 3 + [ctypes.POINTER(ctypes.c_int)]),
    "fsl_parity": (ctypes.c_int, [ctypes.c_void_p]),
    "fsl_status": (ctypes.c_int, [ctypes.c_void_p]),
    "fsl_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fsl_destroy": (None, [ctypes.c_void_p]),
}
EXPORTED = tuple(_SIGNATURES)


def lib():
    """Load libfsl.so (raises if it has not been built: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfsl.so not built ({LIB_PATH}); run paper_1509_07691_gb300.build.build()")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(l, name)
            fn.restype = res
            fn.argtypes = args
        _lib = l
    return _lib


class FslError(RuntimeError):
    pass


def check(rc: int, what: str = ""):
    if rc != OK:
        msg = lib().fsl_strerror(rc).decode()
        raise FslError(f"{what}: {msg} ({rc})")


def make_params(shape, collision=BGK, curv_model=CURV_LSQR, storage=F32, storage_shift=8, plic_iters=4, tau=1.0,
                magic=3.0 / 16.0, sigma=0.0, p_gas=1.0 / 3.0, theta=math.pi / 2, eps_convert=1e-3,
                lsqr_fp64_cond=1e6, excess_rule=0) -> Params:
    """shape = (nz, ny, nx) of the numpy/torch arrays (x fastest)."""
    nz, ny, nx = shape
    return Params(nx, ny, nz, collision, curv_model, storage, storage_shift, plic_iters, tau, magic, sigma, p_gas,
                  theta, eps_convert, lsqr_fp64_cond, excess_rule, 0)


def make_geometry(kind, c=(0, 0, 0), R=0.0, eps2=0.0, c2=(0, 0, 0), R2=0.0, zw=0.0, n=(0, 0, 1), d=0.0, h0=0.0,
                  amp=0.0, wavelength=1.0, invert=0, sub=16) -> Geometry:
    k = GEOMETRY_KINDS[kind] if isinstance(kind, str) else int(kind)
    D3 = ctypes.c_double * 3
    return Geometry(k, int(invert), int(sub), 0, D3(*c), R, eps2, D3(*c2), R2, zw, D3(*n), d, h0, amp, wavelength)


def _stream_handle(stream) -> int:
    return 0 if stream is None else int(stream.cuda_stream)


def fill_geometry(params: Params, geom: Geometry, phi: torch.Tensor, stream=None):
    check(lib().fsl_fill_geometry(ctypes.byref(params), ctypes.byref(geom), ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.c_void_p(_stream_handle(stream))), "fsl_fill_geometry")


_STORAGE_DTYPE = {F32: torch.float32, F16_OFS: torch.float16, BF16_OFS: torch.bfloat16}


class Sim:
    """One FSLBM context with its caller-owned device buffers (torch tensors)."""

    def __init__(self, params: Params, phi0=None, obstacle=None, device="cuda", stream=None, phi_on_device=False):
        self.p = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self.device = torch.device(device)
        self.stream = stream
        dt = _STORAGE_DTYPE[params.storage]
        Np = (self.N + 3) // 4 * 4
        self.f = [torch.empty((Q,) + self.shape, dtype=dt, device=self.device) for _ in range(2)]
        self.flags = [torch.zeros(Np, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.mass = torch.zeros(self.shape, dtype=torch.float32, device=self.device)
        self.phi = torch.zeros(self.shape, dtype=torch.float32, device=self.device)
        self.kappa = torch.zeros(self.shape, dtype=torch.float32, device=self.device)
        ws = lib().fsl_workspace_size(ctypes.byref(params))
        if ws == 0:
            raise FslError("fsl_workspace_size: invalid parameters")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.fields = Fields()
        self.fields.f[0], self.fields.f[1] = self.f[0].data_ptr(), self.f[1].data_ptr()
        self.fields.flags[0], self.fields.flags[1] = self.flags[0].data_ptr(), self.flags[1].data_ptr()
        self.fields.mass, self.fields.phi = self.mass.data_ptr(), self.phi.data_ptr()
        self.fields.kappa, self.fields.workspace = self.kappa.data_ptr(), self.workspace.data_ptr()
        self._keep = []
        phi_ptr, phi_where = None, WHERE_NONE
        if phi0 is not None:
            if isinstance(phi0, torch.Tensor) and phi0.is_cuda:
                t = phi0.to(torch.float32).contiguous()
                phi_ptr, phi_where = t.data_ptr(), WHERE_DEVICE
            else:
                t = torch.from_numpy(np.ascontiguousarray(phi0, dtype=np.float32)).pin_memory()
                phi_ptr, phi_where = t.data_ptr(), WHERE_HOST
            self._keep.append(t)
        obs_ptr, obs_where = None, WHERE_NONE
        if obstacle is not None:
            if isinstance(obstacle, torch.Tensor) and obstacle.is_cuda:
                t = obstacle.to(torch.uint8).contiguous()
                obs_ptr, obs_where = t.data_ptr(), WHERE_DEVICE
            else:
                t = torch.from_numpy(np.ascontiguousarray(obstacle, dtype=np.uint8)).pin_memory()
                obs_ptr, obs_where = t.data_ptr(), WHERE_HOST
            self._keep.append(t)
        ctx = ctypes.c_void_p()
        check(lib().fsl_init(ctypes.byref(params), ctypes.byref(self.fields), phi_ptr, phi_where, obs_ptr, obs_where,
                             ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(ctx)), "fsl_init")
        self.ctx = ctx

    # -- calls -----------------------------------------------------------------
    def step(self, n: int = 1):
        check(lib().fsl_step(self.ctx, int(n)), "fsl_step")

    def step_profile(self) -> np.ndarray:
        """One step launched kernel by kernel; device ms of normals, curvature,
        liquid stream-collide, interface stream-collide, conversion, finalize."""
        out = (ctypes.c_float * 6)()
        check(lib().fsl_step_profile(self.ctx, out), "fsl_step_profile")
        return np.array(list(out), dtype=np.float64)

    def curvature(self, model: int, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.kappa if out is None else out
        check(lib().fsl_curvature(self.ctx, int(model), ctypes.c_void_p(out.data_ptr())), "fsl_curvature")
        return out

    def mass_total(self):
        m, lost = ctypes.c_double(), ctypes.c_double()
        check(lib().fsl_mass(self.ctx, ctypes.byref(m), ctypes.byref(lost)), "fsl_mass")
        return m.value, lost.value

    def stats(self) -> np.ndarray:
        out = (ctypes.c_int64 * 10)()
        check(lib().fsl_stats(self.ctx, out), "fsl_stats")
        return np.array(list(out), dtype=np.int64)

    def prescribe_flow(self, rho: float, u):
        """f' = feq(rho, u) at every liquid and interface cell (fsl_prescribe_flow)."""
        check(lib().fsl_prescribe_flow(self.ctx, float(rho), float(u[0]), float(u[1]), float(u[2])),
              "fsl_prescribe_flow")

    def set_bubble(self, p0: float, V0: float = 0.0):
        """Bubble model on (p0 > 0; V0 <= 0: the current gas volume) or off (p0 = 0)."""
        check(lib().fsl_set_bubble(self.ctx, float(p0), float(V0)), "fsl_set_bubble")

    def bubble(self):
        """(gas volume, gas pressure of the next step) of the bubble model."""
        v, p = ctypes.c_double(), ctypes.c_double()
        check(lib().fsl_bubble(self.ctx, ctypes.byref(v), ctypes.byref(p)), "fsl_bubble")
        return v.value, p.value

    def conversions(self):
        """Sorted cell indices filled, emptied, new interface from gas and new
        interface from liquid in the last step (fsl_conversions)."""
        cnt = (ctypes.c_int64 * 4)()
        check(lib().fsl_conversions(self.ctx, cnt, None, 0), "fsl_conversions")
        total = int(sum(cnt))
        cells = np.zeros(max(total, 1), dtype=np.int32)
        check(lib().fsl_conversions(self.ctx, cnt, ctypes.c_void_p(cells.ctypes.data), total), "fsl_conversions")
        out, o = [], 0
        for k in range(4):
            out.append(cells[o: o + cnt[k]].copy())
            o += cnt[k]
        return out

    def mass_static(self, out: torch.Tensor) -> int:
        """fsl_mass_static on the current state into `out` (one float64 on the
        device); no workspace is used.  Returns the status code."""
        return lib().fsl_mass_static(ctypes.byref(self.p), ctypes.c_void_p(self.f_current().data_ptr()),
                                     ctypes.c_void_p(self.flags[0].data_ptr()), ctypes.c_void_p(self.mass.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_handle(self.stream)))

    def attach_mlp(self, net: "Mlp", fallback_rel: float = 0.05):
        self._mlp = net
        check(lib().fsl_mlp_attach(self.ctx, ctypes.c_void_p(net.params.data_ptr()), float(fallback_rel)),
              "fsl_mlp_attach")

    def status(self) -> int:
        return lib().fsl_status(self.ctx)

    @property
    def parity(self) -> int:
        return lib().fsl_parity(self.ctx)

    def refresh(self):
        check(lib().fsl_refresh(self.ctx), "fsl_refresh")

    # -- state access (host copies, for checks) ------------------------------------
    def f_current(self) -> torch.Tensor:
        return self.f[self.parity]

    def flags_current(self) -> torch.Tensor:
        return self.flags[0][: self.N].view(self.shape)

    def pdfs_float(self) -> torch.Tensor:
        """Current PDFs decoded to float32 (16-bit offsets: f = w_q + v 2^-shift)."""
        f = self.f_current()
        if self.p.storage == F32:
            return f
        w = torch.tensor([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, device=f.device).view(Q, 1, 1, 1)
        return f.float() * (2.0 ** -self.p.storage_shift) + w

    def set_state(self, f, flags, mass, phi):
        """Write a state (host arrays) into the current buffers and refresh."""
        p = self.parity
        dt = _STORAGE_DTYPE[self.p.storage]
        fx = torch.as_tensor(np.ascontiguousarray(f, dtype=np.float32))
        if self.p.storage != F32:
            w = torch.tensor([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).view(Q, 1, 1, 1)
            fx = (fx - w) * (2.0 ** self.p.storage_shift)
        self.f[p].copy_(fx.to(dt))
        fl = torch.as_tensor(np.ascontiguousarray(flags, dtype=np.uint8)).reshape(-1)
        self.flags[0][: self.N].copy_(fl)
        self.mass.copy_(torch.as_tensor(np.ascontiguousarray(mass, dtype=np.float32)))
        self.phi.copy_(torch.as_tensor(np.ascontiguousarray(phi, dtype=np.float32)))
        torch.cuda.synchronize(self.device)
        self.refresh()

    def host_state(self) -> dict:
        torch.cuda.synchronize(self.device)
        return dict(f=self.pdfs_float().double().cpu().numpy(), flags=self.flags_current().cpu().numpy(),
                    mass=self.mass.double().cpu().numpy(), phi=self.phi.double().cpu().numpy(),
                    kappa=self.kappa.double().cpu().numpy())

    # -- adjoint windows (frozen cell types) ----------------------------------------
    def set_surface(self, sigma: float, theta: float):
        """New surface tension and contact angle (radians) for the next steps."""
        check(lib().fsl_set_surface(self.ctx, float(sigma), float(theta)), "fsl_set_surface")
        self.p.sigma, self.p.theta = float(sigma), float(theta)

    def interface_count(self) -> int:
        return int(self.stats()[1])

    def _adj_workspace(self, window, ckpt_every, max_interface, slot="_adj_ws"):
        nbytes = lib().fsl_adjoint_workspace_size(ctypes.byref(self.p), int(window), int(ckpt_every),
                                                  int(max_interface))
        if nbytes == 0:
            raise FslError("fsl_adjoint_workspace_size: invalid arguments")
        ws = getattr(self, slot, None)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            setattr(self, slot, ws)
        return ws, nbytes

    def window_forward(self, window: int, ckpt_every: int = 10, max_interface: int | None = None):
        """`window` steps with frozen cell types, checkpoints every `ckpt_every`."""
        if max_interface is None:
            max_interface = 2 * self.interface_count() + 1024
        ws, nbytes = self._adj_workspace(window, ckpt_every, max_interface)
        check(lib().fsl_window_forward(self.ctx, int(window), int(ckpt_every), int(max_interface),
                                       ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())),
              "fsl_window_forward")
        self._adj_window = (int(window), int(ckpt_every), int(max_interface))

    def window_adjoint(self, dL_dphi: torch.Tensor, inputs: bool = False):
        """dL/dsigma, dL/dtheta of the last window from dL/dphi at its end; with
        inputs=True also dL/dphi, dL/dm and dL/df' at its start."""
        g = dL_dphi.to(device=self.device, dtype=torch.float32).contiguous()
        assert g.numel() == self.N
        outs = [None, None, None]
        if inputs:
            outs = [torch.zeros(self.shape, dtype=torch.float32, device=self.device),
                    torch.zeros(self.shape, dtype=torch.float32, device=self.device),
                    torch.zeros((Q,) + self.shape, dtype=torch.float32, device=self.device)]
        ds, dt = ctypes.c_double(), ctypes.c_double()
        torch.cuda.current_stream(self.device).synchronize()
        check(lib().fsl_window_adjoint(self.ctx, ctypes.c_void_p(g.data_ptr()), ctypes.byref(ds), ctypes.byref(dt),
                                       *[_ptr(t) for t in outs]), "fsl_window_adjoint")
        if inputs:
            return ds.value, dt.value, outs[0], outs[1], outs[2]
        return ds.value, dt.value

    def kappa_jacobian(self, max_interface: int | None = None):
        """(jac [n, JAC_STRIDE], cells [n], kappa [n]) of the current state."""
        if max_interface is None:
            max_interface = self.interface_count() + 64
        ws, nbytes = self._adj_workspace(1, 1, max_interface, slot="_jac_ws")
        jac = torch.zeros((max_interface, JAC_STRIDE), dtype=torch.float32, device=self.device)
        cells = torch.zeros(max_interface, dtype=torch.int32, device=self.device)
        kap = torch.zeros(max_interface, dtype=torch.float32, device=self.device)
        n = ctypes.c_int()
        check(lib().fsl_kappa_jacobian(self.ctx, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                                       int(max_interface), _ptr(jac), _ptr(cells), _ptr(kap), ctypes.byref(n)),
              "fsl_kappa_jacobian")
        return jac[: n.value], cells[: n.value], kap[: n.value]

    def save(self, path: str):
        """Checkpoint of the current state (PDFs, types, mass, fill level, lost
        mass) to a file; synchronising."""
        check(lib().fsl_save(self.ctx, os.fsencode(path)), "fsl_save")

    def load(self, path: str):
        """Resume from a checkpoint written by save() on a grid of the same size
        and storage; the lists are rebuilt.  Synchronising."""
        check(lib().fsl_load(self.ctx, os.fsencode(path)), "fsl_load")

    def snapshot(self) -> dict:
        """Device copy of the current state (PDFs, types, mass, fill level)."""
        torch.cuda.synchronize(self.device)
        return dict(f=self.f_current().clone(), flags=self.flags[0].clone(), mass=self.mass.clone(),
                    phi=self.phi.clone())

    def restore(self, snap: dict):
        """Put a snapshot back as the current state (lists rebuilt by refresh)."""
        torch.cuda.synchronize(self.device)
        self.f_current().copy_(snap["f"])
        self.flags[0].copy_(snap["flags"])
        self.mass.copy_(snap["mass"])
        self.phi.copy_(snap["phi"])
        torch.cuda.synchronize(self.device)
        self.refresh()

    def close(self):
        if getattr(self, "ctx", None):
            lib().fsl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Mlp:
    """Learned curvature network: packed BF16 parameters and FP32 master weights
    with Adam moments, all torch device tensors."""

    def __init__(self, init: dict, device="cuda", stream=None):
        self.device = torch.device(device)
        self.stream = stream
        cnt = lib().fsl_mlp_master_count()
        master = np.concatenate([np.asarray(init[k], np.float32).ravel() for k in ("W1", "W2", "w3", "b1", "b2", "b3")])
        assert master.size == cnt
        self.master = torch.from_numpy(master).to(self.device)
        self.m = torch.zeros(cnt, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(cnt, dtype=torch.float32, device=self.device)
        self.params = torch.zeros(lib().fsl_mlp_param_bytes(), dtype=torch.uint8, device=self.device)
        self.step = 0
        self._ws = None
        check(lib().fsl_mlp_pack(_ptr(self.master), _ptr(self.params), _stream_handle(stream)), "fsl_mlp_pack")

    def _workspace(self, n):
        need = lib().fsl_mlp_train_workspace(int(n))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._ws

    def forward(self, X, keep=False):
        n = X.shape[0]
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        z1 = torch.empty((n, 128), dtype=torch.float32, device=self.device) if keep else None
        z2 = torch.empty((n, 128), dtype=torch.float32, device=self.device) if keep else None
        check(lib().fsl_mlp_forward(_ptr(self.params), _ptr(X), n, _ptr(y), _ptr(z1), _ptr(z2),
                                    _stream_handle(self.stream)), "fsl_mlp_forward")
        return (y, z1, z2) if keep else y

    @staticmethod
    def status(reset: bool = False) -> int:
        """Sticky status of the tensor-core MLP kernels (0, or FSL_ETIMEOUT)."""
        return lib().fsl_mlp_status(1 if reset else 0)

    def gradients(self, X, target):
        n = X.shape[0]
        g = torch.empty(self.master.numel(), dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        check(lib().fsl_mlp_gradients(_ptr(self.params), _ptr(X), _ptr(target), n, _ptr(g), _ptr(loss),
                                      _ptr(self._workspace(n)), _stream_handle(self.stream)), "fsl_mlp_gradients")
        return g, loss

    def train_step(self, X, target, lr, loss_out=None):
        self.step += 1
        n = X.shape[0]
        check(lib().fsl_mlp_train_step(_ptr(self.params), _ptr(self.master), _ptr(self.m), _ptr(self.v), _ptr(X),
                                       _ptr(target), n, float(lr), self.step, _ptr(loss_out),
                                       _ptr(self._workspace(n)), _stream_handle(self.stream)), "fsl_mlp_train_step")

    def train_epoch(self, X, target, perm, batch, lr, losses=None):
        """One pass over (X, target) in the order perm, `batch` rows per Adam
        step, the batch loop inside the library; a ragged tail is left out.
        losses: None or a device tensor of n // batch floats for the batch
        losses.  Returns the number of steps taken."""
        n = X.shape[0]
        assert perm.dtype == torch.int64 and perm.is_contiguous() and perm.numel() == n
        need = lib().fsl_mlp_epoch_workspace(int(batch))
        if getattr(self, "_ews", None) is None or self._ews.numel() < need:
            self._ews = torch.empty(need, dtype=torch.uint8, device=self.device)
        check(lib().fsl_mlp_train_epoch(_ptr(self.params), _ptr(self.master), _ptr(self.m), _ptr(self.v), _ptr(X),
                                        _ptr(target), _ptr(perm), n, int(batch), float(lr), self.step, _ptr(losses),
                                        _ptr(self._ews), _stream_handle(self.stream)), "fsl_mlp_train_epoch")
        nb = n // batch
        self.step += nb
        return nb

    def master_dict(self):
        a = self.master.cpu().numpy()
        o = [0, 16384, 32768, 32896, 33024, 33152, 33153]
        shp = [(128, 128), (128, 128), (128,), (128,), (128,), (1,)]
        return {k: a[o[i]:o[i + 1]].reshape(shp[i]) for i, k in enumerate(("W1", "W2", "w3", "b1", "b2", "b3"))}


def mlp_stencils(params: dict, sub=8, noise=1e-3, noise_seed=0, device="cuda", stream=None):
    """Training stencils on the GPU from synthetic.mlp_sample_params(...)."""
    n = int(params["axes"].shape[0])
    dev = torch.device(device)
    t = {k: torch.from_numpy(np.ascontiguousarray(params[k], np.float32)).to(dev) for k in ("axes", "quat", "dir", "delta")}
    inv = torch.from_numpy(np.ascontiguousarray(params["invert"], np.int32)).to(dev)
    X = torch.empty((n, 128), dtype=torch.bfloat16, device=dev)
    target = torch.empty(n, dtype=torch.float32, device=dev)
    check(lib().fsl_mlp_stencils(n, _ptr(t["axes"]), _ptr(t["quat"]), _ptr(t["dir"]), _ptr(t["delta"]), _ptr(inv),
                                 int(sub), float(noise), int(noise_seed), _ptr(X), _ptr(target),
                                 _stream_handle(stream)), "fsl_mlp_stencils")
    return X, target


class FslStepWindow(torch.autograd.Function):
    """phi after `window` steps with frozen cell types, as a function of
    surface = tensor([sigma, theta]) (float64, theta in radians).  The forward
    pass runs fsl_window_forward from the simulation's current state (the
    caller puts the start state in place, e.g. Sim.restore); the backward pass
    is fsl_window_adjoint (checkpointed recomputation, hand-written reverse
    kernels)."""

    @staticmethod
    def forward(ctx, surface, sim, window, ckpt_every=10):
        s = surface.detach().cpu().double()
        sim.set_surface(float(s[0]), float(s[1]))
        sim.window_forward(int(window), int(ckpt_every))
        ctx.sim = sim
        torch.cuda.synchronize(sim.device)
        return sim.phi.clone()

    @staticmethod
    def backward(ctx, grad_phi):
        ds, dt = ctx.sim.window_adjoint(grad_phi)
        return torch.tensor([ds, dt], dtype=torch.float64), None, None, None
