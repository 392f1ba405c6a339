"""FP64 CPU oracle of the learned-curvature extension -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use
it.  Shares no code with the CUDA path.

What it computes (the GPU path must compute the same):
  stencils   5x5x5 fill levels around a cell crossed by the surface of a
             sphere or ellipsoid (sub-sampled like Sec. III.A), Gaussian noise
             on the partially filled cells (clipped to [0,1]), and the target
             kappa = mean curvature at the surface point nearest the centre of
             the middle cell (negative when the liquid is outside)
  canonical  axes flipped so the Parker-Youngs normal of the middle cell has
             non-negative components, then ordered by decreasing |n_k|
  network    x = 2 phi - 1 (BF16), z1 = W1 x + b1, h1 = bf16(gelu(z1)),
             z2 = W2 h1 + b2, h2 = gelu(z2), y = w3 . h2 + b3; W1, W2, w3 BF16,
             biases FP32, gelu(x) = x Phi(x) (erf form)
  loss       mean over the batch of w (y - t)^2 with w = 1 / (t^2 + 7e-5)
  Adam       beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, FP32 master
             weights and BF16 copies

Parity status: gradients pinned by central finite differences; gelu pinned
by its erf definition; ellipsoid curvature pinned by the closed forms at the
axis points and the sphere; the fill levels reuse the pinned sub-sampling of
the main oracle (oracle.fill_cells).
"""
from __future__ import annotations

import math

import numpy as np

NIN, NPAD, NH = 125, 128, 128
LOSS_EPS = 7e-5
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


# ------------------------------------------------------------------ numerics
def bf16(a):
    """Round to bfloat16 (round to nearest even) and return as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


# ------------------------------------------------------------------ network
def forward(params, X, round_bf16=True):
    """X: (n, 125) fill levels.  Returns y (n,) and the activations."""
    rb = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.zeros((X.shape[0], NPAD))
    x[:, :NIN] = rb(2.0 * np.asarray(X, dtype=np.float64) - 1.0)
    W1, b1, W2, b2, w3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    z1 = x @ rb(W1).T + b1
    h1 = rb(gelu(z1))
    z2 = h1 @ rb(W2).T + b2
    h2 = gelu(z2)
    y = h2 @ rb(w3) + b3
    return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_weights(t):
    return 1.0 / (np.asarray(t) ** 2 + LOSS_EPS)


def loss(params, X, t, round_bf16=True):
    y, _ = forward(params, X, round_bf16)
    return float(np.mean(loss_weights(t) * (y - t) ** 2))


def backward(params, X, t, round_bf16=True):
    """Gradients of `loss` with respect to the master parameters (the BF16
    rounding of weights is treated as the identity, straight through)."""
    rb = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, a = forward(params, X, round_bf16)
    n = X.shape[0]
    d3 = 2.0 * loss_weights(t) * (y - t) / n
    w3 = rb(params["w3"])
    W2 = rb(params["W2"])
    d2 = (d3[:, None] * w3[None, :]) * gelu_grad(a["z2"])
    d1 = (d2 @ W2) * gelu_grad(a["z1"])
    return dict(W1=d1.T @ a["x"], b1=d1.sum(0), W2=d2.T @ a["h1"], b2=d2.sum(0), w3=a["h2"].T @ d3, b3=d3.sum())


def adam(params, grads, m, v, step, lr):
    """One Adam step on the master parameters (in place); step counts from 1."""
    for k in params:
        g = grads[k]
        m[k] = BETA1 * m[k] + (1 - BETA1) * g
        v[k] = BETA2 * v[k] + (1 - BETA2) * g * g
        mh = m[k] / (1 - BETA1 ** step)
        vh = v[k] / (1 - BETA2 ** step)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + ADAM_EPS)


# ------------------------------------------------------------------ stencils
def quat_matrix(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def shape_centre(axes, q, d_body, delta):
    """Centre C (world) such that the surface point in body direction d lies at delta."""
    a = np.asarray(axes, dtype=np.float64)
    s_b = d_body / math.sqrt(float(np.sum((d_body / a) ** 2)))
    return np.asarray(delta) - quat_matrix(q) @ s_b


def stencil_fill(axes, q, C, invert, sub):
    """5x5x5 fill levels, index [i+2, j+2, k+2] for cell offsets (x=i, y=j, z=k):
    the fraction of the sub^3 points (i,j,k) + (s + 1/2)/sub - 1/2 of each cell
    that lie inside the (rotated) ellipsoid sum (y_k/a_k)^2 <= 1."""
    Rm = quat_matrix(q)
    s = (np.arange(sub) + 0.5) / sub - 0.5
    cells = np.arange(5) - 2
    gx, gy, gz, sx, sy, sz = np.meshgrid(cells, cells, cells, s, s, s, indexing="ij")
    p = np.stack([gx + sx, gy + sy, gz + sz], -1) - np.asarray(C)
    y = p @ Rm  # rows: R^T (p - C)
    ins = np.sum((y / np.asarray(axes, dtype=np.float64)) ** 2, -1) <= 1.0
    if invert:
        ins = ~ins
    return ins.reshape(5, 5, 5, -1).mean(-1)


def ellipsoid_mean_curvature_nearest(axes, q, C, invert, iters=200):
    """Mean curvature of the surface at the point nearest the origin."""
    a = np.asarray(axes, dtype=np.float64)
    o = quat_matrix(q).T @ (-np.asarray(C))  # origin in the body frame
    # x_k = a_k^2 o_k / (a_k^2 + t); sum (x_k / a_k)^2 = 1; g decreasing in t > -min a^2
    g = lambda t: float(np.sum(a * a * o * o / (a * a + t) ** 2)) - 1.0
    lo = -np.min(a * a) * (1 - 1e-15)
    hi = max(1.0, float(np.max(np.abs(o)) * np.max(a)))
    while g(hi) > 0:
        hi *= 2
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    t = 0.5 * (lo + hi)
    x = a * a * o / (a * a + t)
    grad = 2 * x / (a * a)
    hess = 2 / (a * a)
    gn = float(np.linalg.norm(grad))
    H = (gn * gn * float(np.sum(hess)) - float(np.sum(grad * grad * hess))) / (2 * gn ** 3)
    return -H if invert else H


def parker_youngs_centre(s):
    """Parker-Youngs gradient (weights 4/2/1) of the middle cell of a 5^3 stencil."""
    n = np.zeros(3)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                v = s[2 + dx, 2 + dy, 2 + dz]
                if dx:
                    n[0] += dx * (2 if dy == 0 else 1) * (2 if dz == 0 else 1) * v
                if dy:
                    n[1] += dy * (2 if dx == 0 else 1) * (2 if dz == 0 else 1) * v
                if dz:
                    n[2] += dz * (2 if dx == 0 else 1) * (2 if dy == 0 else 1) * v
    return n


def canonical(s):
    """Flip axes with negative normal component, then order the axes by
    decreasing |n| (stable for ties).  Returns the flattened 125 values with
    index a*25 + b*5 + c along the ordered axes."""
    n = parker_youngs_centre(s)
    t = np.array(s)
    for k in range(3):
        if n[k] < 0:
            t = np.flip(t, axis=k)
    mag = np.abs(n)
    order = sorted(range(3), key=lambda k: (-mag[k], k))
    return np.transpose(t, order).reshape(-1).copy()


def noise_normal(seed, index):
    """Standard normal from two splitmix64 uniforms (Box-Muller), counter based."""
    from paper_1509_07691_gb300 import synthetic as S  # seeded generator module (no method arithmetic)
    u1 = S.uniform_at(seed, 2 * index)
    u2 = S.uniform_at(seed, 2 * index + 1)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def sample(p, k, sub=8, noise=1e-3, noise_seed=0):
    """Stencil k of the parameter set p (arrays from synthetic.mlp_sample_params)."""
    axes, q, d, delta, inv = p["axes"][k], p["quat"][k], p["dir"][k], p["delta"][k], int(p["invert"][k])
    C = shape_centre(axes, q, d, delta)
    s = stencil_fill(axes, q, C, inv, sub)
    if noise > 0:
        idx = k * 125 + np.arange(125)
        nz = noise_normal(noise_seed, idx).reshape(5, 5, 5) * noise
        part = (s > 0) & (s < 1)
        s = np.where(part, np.clip(s + nz, 0.0, 1.0), s)
    return canonical(s), ellipsoid_mean_curvature_nearest(axes, q, C, inv)
