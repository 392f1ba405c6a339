"""Seeded synthetic inputs for the FSLBM workloads.

This module holds no arithmetic of the method.  It only draws the seeded
numbers a run needs (centre offsets, perturbation noise) with a
counter-based splitmix64 generator, and states the workload parameters
(grid sizes, radii, sigma, tau, contact angles) as plain numbers.  Both the
CUDA path and the CPU oracle are fed from here; neither derives anything
from the other.

Workloads (geometry shapes follow the paper's test cases, Sec. III):
  droplet32     32^3 periodic, sphere R = 8, BGK tau = 1, sigma = 1e-4
  sessile128    128x128x64, wall layers at z = 0 and z = 63, hemisphere
                R = 30 on the wall, TRT (Lambda = 3/16), tau = 0.8,
                sigma = 5e-4, theta in {30, 60, 90, 120} degrees
  oscillating256  256^3 periodic, P2-perturbed sphere (amplitude 0.1 R,
                volume of R = 40), sigma = 1e-3, tau = 0.6
  oscillating128  the same at half the size (128^3, R = 20): the small case
                for detailed kernel profiles
  sessile64     64^3, wall layers at z = 0 and z = 63, hemisphere R = 16,
                TRT tau = 0.8
  coalescence384  384^3, spheres R = 48 and R = 32 with a 4-cell gap,
                sigma = 1e-3, tau = 0.7
  pool256       256^3, wall layers at z = 0 and z = 255, liquid below
                z = 160 + 2 sin(2 pi x/64) sin(2 pi y/64), sigma = 1e-3, tau = 0.6
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1509
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of splitmix64 started at state `seed` (Steele, Lea, Flood 2014)."""
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed & MASK64)
        inc = np.uint64(0x9E3779B97F4A7C15)
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = s + idx * inc
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        out[:] = z
    return out


def uniform_at(seed: int, index) -> np.ndarray:
    """splitmix64 uniform in [0, 1) at counter positions `index` (the k-th
    output of the stream started at `seed` is uniform_at(seed, k))."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal draws (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, n)
    u2 = uniform(seed ^ 0x5DEECE66D, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def centre_offset(seed: int) -> np.ndarray:
    """Sub-cell offset in [-1/2, 1/2)^3, quantised to 1/1024 so that sample
    coordinates minus the centre are exact in binary floating point."""
    u = uniform(seed, 3) - 0.5
    return np.floor(u * 1024.0) / 1024.0


def p2_volume_radius(R: float, eps2: float) -> float:
    """Base radius R_s such that r(theta) = R_s (1 + eps2 P2(cos theta)) encloses
    the volume of a sphere of radius R: V = (2 pi/3) R_s^3 (2 + 6 eps2^2/5 + 4 eps2^3/35)."""
    return R * (2.0 / (2.0 + 1.2 * eps2 ** 2 + (4.0 / 35.0) * eps2 ** 3)) ** (1.0 / 3.0)


WORKLOADS = {
    "droplet32": dict(shape=(32, 32, 32), collision="bgk", tau=1.0, sigma=1e-4, theta_deg=90.0, steps=200,
                      geometry=dict(kind="sphere", R=8.0, base=(16.0, 16.0, 16.0)), walls=()),
    "sessile128": dict(shape=(64, 128, 128), collision="trt", tau=0.8, sigma=5e-4, theta_deg=90.0, steps=5000,
                       geometry=dict(kind="cap", R=30.0, base=(64.0, 64.0, 0.5), zw=0.5), walls=(0, 63)),
    "oscillating256": dict(shape=(256, 256, 256), collision="bgk", tau=0.6, sigma=1e-3, theta_deg=90.0,
                           steps=1000, geometry=dict(kind="mode2", R=40.0, eps2=0.1, base=(128.0, 128.0, 128.0)),
                           walls=()),
    "oscillating128": dict(shape=(128, 128, 128), collision="bgk", tau=0.6, sigma=1e-3, theta_deg=90.0,
                           steps=1000, geometry=dict(kind="mode2", R=20.0, eps2=0.1, base=(64.0, 64.0, 64.0)),
                           walls=()),
    "sessile64": dict(shape=(64, 64, 64), collision="trt", tau=0.8, sigma=2e-4, theta_deg=90.0, steps=50,
                      geometry=dict(kind="cap", R=16.0, base=(32.0, 32.0, 0.5), zw=0.5), walls=(0, 63)),
    "coalescence384": dict(shape=(384, 384, 384), collision="bgk", tau=0.7, sigma=1e-3, theta_deg=90.0,
                           steps=1000, geometry=dict(kind="two_spheres", R=48.0, R2=32.0, base=(142.0, 192.0, 192.0),
                                                     base2=(226.0, 192.0, 192.0)), walls=()),
    "pool256": dict(shape=(256, 256, 256), collision="bgk", tau=0.6, sigma=1e-3, theta_deg=90.0, steps=1000,
                    geometry=dict(kind="pool", h0=160.0, amp=2.0, wavelength=64.0), walls=(0, 255)),
}


def workload(name: str, seed: int = SEED, **override) -> dict:
    """Parameters of a named workload with its seeded centre offset applied.

    Returns a dict with shape (nz, ny, nx), collision, tau, sigma, theta (rad),
    geometry (plain numbers: kind, centre c, radii, ...) and walls (z indices
    of obstacle layers)."""
    w = {k: (dict(v) if isinstance(v, dict) else v) for k, v in WORKLOADS[name].items()}
    w.update(override)
    g = dict(w["geometry"])
    off = centre_offset(seed)
    if g["kind"] in ("sphere", "mode2", "two_spheres"):
        g["c"] = tuple(float(b + o) for b, o in zip(g.pop("base"), off))
    elif g["kind"] == "cap":
        b = g.pop("base")
        g["c"] = (float(b[0] + off[0]), float(b[1] + off[1]), float(b[2]))
    if g["kind"] == "two_spheres":
        g["c2"] = tuple(float(b + o) for b, o in zip(g.pop("base2"), off))
    if g["kind"] == "mode2":
        g["R_s"] = p2_volume_radius(g["R"], g["eps2"])
    w["geometry"] = g
    w["theta"] = math.radians(w["theta_deg"])
    w["seed"] = seed
    return w


def obstacle_mask(shape, walls) -> np.ndarray:
    """uint8 mask with the listed z layers set (obstacle cells).  All axes wrap,
    so a box closed in z needs a wall layer at each end."""
    m = np.zeros(shape, np.uint8)
    for z in walls:
        m[z] = 1
    return m


def pdf_noise(seed: int, shape, amp: float) -> np.ndarray:
    """Zero-mean uniform noise of half-width `amp` for a (19,)+shape PDF field."""
    n = 19 * int(np.prod(shape))
    return ((uniform(seed, n) - 0.5) * (2.0 * amp)).reshape((19,) + tuple(shape))


def field_noise(seed: int, shape, amp: float) -> np.ndarray:
    """Zero-mean uniform noise of half-width `amp` for a scalar field."""
    return ((uniform(seed, int(np.prod(shape))) - 0.5) * (2.0 * amp)).reshape(shape)


def gaussian_field(seed: int, shape, sd: float) -> np.ndarray:
    return (normal(seed, int(np.prod(shape))) * sd).reshape(shape)


def mlp_sample_params(seed: int, n: int) -> dict:
    """Shape parameters of n training stencils for the learned curvature
    (spheres and ellipsoids, radii log-uniform in [2, 60], uniformly random
    orientation, surface direction and sub-cell offset; 30 % bubbles).

    axes (n,3) semi-axes in cells, quat (n,4) unit quaternion (w,x,y,z),
    dir (n,3) unit direction in the body frame of the surface point that
    passes through the middle cell, delta (n,3) that point's offset from the
    middle cell's centre, invert (n,) 1 if the liquid is outside."""
    u = uniform(seed, 13 * n).reshape(n, 13)
    R = np.exp(np.log(2.0) + u[:, 0] * (np.log(60.0) - np.log(2.0)))
    ell = u[:, 1] >= 0.5
    axes = np.stack([R, R * np.where(ell, 0.6 + 0.4 * u[:, 2], 1.0), R * np.where(ell, 0.6 + 0.4 * u[:, 3], 1.0)], 1)
    axes = np.maximum(axes, 2.0)
    invert = (u[:, 4] < 0.3).astype(np.int32)
    a, b, c = u[:, 5], 2 * np.pi * u[:, 6], 2 * np.pi * u[:, 7]
    quat = np.stack([np.sqrt(a) * np.cos(c), np.sqrt(1 - a) * np.sin(b), np.sqrt(1 - a) * np.cos(b),
                     np.sqrt(a) * np.sin(c)], 1)
    zc = 2 * u[:, 8] - 1
    ph = 2 * np.pi * u[:, 9]
    rxy = np.sqrt(np.maximum(0.0, 1 - zc * zc))
    d = np.stack([rxy * np.cos(ph), rxy * np.sin(ph), zc], 1)
    delta = u[:, 10:13] - 0.5
    return dict(axes=axes, quat=quat, dir=d, delta=delta, invert=invert)


def mlp_init_weights(seed: int) -> dict:
    """Initial MLP parameters: weights N(0, 1/fan_in), biases 0 (FP32)."""
    W1 = normal(seed, 128 * 128).reshape(128, 128) / np.sqrt(125.0)
    W1[:, 125:] = 0.0
    W2 = normal(seed + 1, 128 * 128).reshape(128, 128) / np.sqrt(128.0)
    w3 = normal(seed + 2, 128) / np.sqrt(128.0)
    return dict(W1=W1.astype(np.float32), b1=np.zeros(128, np.float32), W2=W2.astype(np.float32),
                b2=np.zeros(128, np.float32), w3=w3.astype(np.float32), b3=np.zeros(1, np.float32))
