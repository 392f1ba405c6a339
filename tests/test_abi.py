"""CPU checks of the C ABI: libfsl.so builds for sm_103a, loads, and exports
every function include/fsl.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fsl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(fsl_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1509_07691_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fsl_init", "fsl_step", "fsl_curvature", "fsl_mass", "fsl_workspace_size", "fsl_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fsl_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_1509_07691_gb300 import fsl
    assert sorted(fsl.EXPORTED) == _declared()
    lib = ctypes.CDLL(libpath)
    for n in fsl.EXPORTED:
        assert hasattr(lib, n)


def test_workspace_size_and_validation_without_gpu(libpath):
    from paper_1509_07691_gb300 import fsl
    p = fsl.make_params((8, 8, 8), tau=0.8)
    ws = fsl.lib().fsl_workspace_size(ctypes.byref(p))
    N = 512
    assert ws >= N * (16 + 4 + 4 + 5 * 4)
    bad = fsl.make_params((8, 8, 8), tau=0.4)  # tau <= 1/2 is not a valid relaxation time
    assert fsl.lib().fsl_workspace_size(ctypes.byref(bad)) == 0
    bad = fsl.make_params((2, 8, 8))
    assert fsl.lib().fsl_workspace_size(ctypes.byref(bad)) == 0
    assert fsl.lib().fsl_strerror(fsl.EINVAL).decode().startswith("invalid")
    # fsl_init rejects a null fields pointer before touching the device
    ctx = ctypes.c_void_p()
    assert fsl.lib().fsl_init(ctypes.byref(p), None, None, 0, None, 0, None, ctypes.byref(ctx)) == fsl.EINVAL
    # the training epoch: workspace = gathered batch (256 B rows + targets) + the step's workspace;
    # bad arguments are rejected before any device work (the pointers below are never dereferenced)
    L = fsl.lib()
    assert L.fsl_mlp_epoch_workspace(0) == 0
    assert L.fsl_mlp_epoch_workspace(4096) >= L.fsl_mlp_train_workspace(4096) > 0
    fake = [ctypes.c_void_p(1 << 20)] * 7
    def epoch(n, batch, lr=1e-3, step0=0, ptrs=fake, ws=ctypes.c_void_p(1 << 20)):
        return L.fsl_mlp_train_epoch(*ptrs, n, batch, lr, step0, None, ws, None)
    assert epoch(100, 4096) == fsl.EINVAL                       # fewer rows than one batch
    assert epoch(8192, 0) == fsl.EINVAL
    assert epoch(8192, 4096, lr=0.0) == fsl.EINVAL
    assert epoch(8192, 4096, step0=-1) == fsl.EINVAL
    assert epoch(8192, 4096, ptrs=[None] + fake[1:]) == fsl.EINVAL
    assert epoch(8192, 4096, ptrs=fake[:4] + [ctypes.c_void_p((1 << 20) + 8)] + fake[5:]) == fsl.EINVAL  # X misaligned
    assert epoch(8192, 4096, ws=ctypes.c_void_p((1 << 20) + 64)) == fsl.EINVAL  # workspace misaligned
    # checkpoints: a NULL context or path is rejected before any file or device access
    assert L.fsl_save(None, b"x.fslckpt") == fsl.EINVAL
    assert L.fsl_load(None, b"x.fslckpt") == fsl.EINVAL
    assert L.fsl_strerror(fsl.EIO).decode().startswith("checkpoint")
