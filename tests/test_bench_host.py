"""Host-side logic of bench.py (no GPU): the algorithmic bytes behind the
roofline figures, the roofline arithmetic, and the period estimator of the
configuration reports."""
import math

import numpy as np

import bench


def test_algorithmic_bytes_per_cell():
    nb = bench.algorithmic_bytes(n_fluid=1000, n_if=100, n_seg_cells=1000)
    assert nb["sc_liquid"] == 152.0 * 900 + 1000       # 19 PDFs in + 19 out, 4 B each, + flags
    assert nb["sc_interface"] == 248.0 * 100            # own + pulled + written PDFs, m, phi, kappa, rho, flag
    nb16 = bench.algorithmic_bytes(n_fluid=1000, n_if=100, n_seg_cells=1000, pdf_bytes=2)
    assert nb16["sc_liquid"] == 76.0 * 900 + 1000
    assert nb16["sc_interface"] == 134.0 * 100
    # the LSQR fit fused with the interface stream-collide
    fused = bench.algorithmic_bytes(n_fluid=1000, n_if=100, n_seg_cells=1000, fused=True)
    assert fused["sc_interface"] == 0.0
    assert fused["lsqr_curvature"] == nb["lsqr_curvature"] + nb["sc_interface"]
    assert fused["lsqr_curvature"] == (21.0 + 248.0) * 100


def test_roofline_fraction_is_bytes_over_time_over_peak():
    ph = np.array([0.01, 0.02, 0.1, 0.0, 0.01, 0.01])   # ms per phase, sc_liquid the largest
    nb = bench.algorithmic_bytes(n_fluid=10 ** 6, n_if=10 ** 4, n_seg_cells=10 ** 6)
    r = bench.roofline_of(ph, nb, {"hbm_gbs": 6000.0})
    assert r["kernel"] == "sc_liquid" and r["bound"] == "hbm"
    assert math.isclose(r["achieved"], nb["sc_liquid"] / 1e-4 / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / 6000.0)


def test_zero_crossings_give_the_period_of_a_damped_cosine():
    every, period = 200, 18600.0
    t = np.arange(0, 24001, every)
    a = 3.0 * np.exp(-1e-4 * t) * np.cos(2 * math.pi * t / period)
    zc = bench.zero_crossings(a, every)
    assert len(zc) == 3
    assert abs(2 * np.mean(np.diff(zc)) - period) < 1e-3 * period
    assert abs(zc[0] - period / 4) < 0.01 * period


def test_launches_per_step_follow_the_domain():
    # LSQR: the general-path kernel is launched only where some cell has an
    # obstacle neighbour (contact lines); the other models always take 7
    walls = np.zeros((4, 4, 4), dtype=np.uint8)
    assert bench.launches_per_step("lsqr", None) == 6
    assert bench.launches_per_step("lsqr", walls) == 6
    walls[0] = 1
    assert bench.launches_per_step("lsqr", walls) == 7
    assert bench.launches_per_step("fd", None) == 7
    assert bench.launches_per_step("none", walls) == 7
