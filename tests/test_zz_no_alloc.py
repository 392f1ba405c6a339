"""The allocation-free mass entry point (fsl_mass_static) against fsl_mass.

fsl_mass_static serves callers that may not allocate device memory (a host
application that owns all of it, or a time-critical monitoring loop): it
keeps its block partial sums in a fixed array inside the library instead of
the caller's workspace.  Two calls in a row must each agree with fsl_mass,
which shows that the shared array is fully rewritten by every call.  This
file is collected last so that a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1509_07691_gb300 import build
    build.build()
    from paper_1509_07691_gb300 import fsl
    return fsl


def _droplet(F, storage):
    import torch
    shape = (40, 48, 56)
    P = F.make_params(shape, sigma=5e-4, tau=0.7, storage=storage)
    phi = torch.zeros(shape, dtype=torch.float32, device="cuda")
    F.fill_geometry(P, F.make_geometry("sphere", c=(27.3, 23.6, 19.8), R=11.0, sub=8), phi)
    sim = F.Sim(P, phi0=phi)
    sim.step(12)
    return sim


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_mass_static_matches_fsl_mass_on_two_calls(F, storage):
    import torch
    sim = _droplet(F, storage)
    m_ref, _ = sim.mass_total()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        assert sim.mass_static(out) == F.OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(m_ref, rel=1e-12)
    # a different state right after: the array holds the previous call's
    # partials, which the next call must overwrite
    sim.step(7)
    m2, _ = sim.mass_total()
    assert sim.mass_static(out) == F.OK
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(m2, rel=1e-12)
    sim.close()


def test_mass_static_rejects_grids_beyond_its_array(F):
    import torch
    big = F.make_params((1024, 1024, 512))  # 2^29 cells > FSL_MASS_STATIC_MAX_CELLS
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(4, dtype=torch.uint8, device="cuda")
    rc = F.lib().fsl_mass_static(ctypes.byref(big), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert rc == F.EINVAL
