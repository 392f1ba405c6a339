"""Pins of the learned-curvature oracle (oracle/mlp.py) against closed forms,
finite differences and the main oracle's pinned sampler."""
import math

import numpy as np
import pytest

from paper_1509_07691_gb300 import synthetic as S


@pytest.fixture(scope="module")
def M():
    import oracle.mlp as m
    return m


def test_gelu_is_x_times_normal_cdf(M):
    for x in (-2.0, -1.0, -0.3, 0.0, 0.7, 1.0, 3.0):
        Phi = 0.5 * math.erfc(-x / math.sqrt(2.0))
        assert float(M.gelu(np.array(x))) == pytest.approx(x * Phi, abs=1e-15)
        h = 1e-6
        fd = (float(M.gelu(np.array(x + h))) - float(M.gelu(np.array(x - h)))) / (2 * h)
        assert float(M.gelu_grad(np.array(x))) == pytest.approx(fd, abs=1e-8)


def test_bf16_rounding(M):
    # 7 explicit mantissa bits: spacing 2^-7 at 1, ties to even
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1.0 + 2 ** -8) == 1.0  # tie -> even
    assert M.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (upper)
    assert M.bf16(1.0 + 1.5 * 2 ** -8) == 1.0 + 2 ** -7
    assert M.bf16(-0.3) == -0.30078125


def _params(seed, scale=0.4):
    p = {k: v.astype(np.float64) for k, v in S.mlp_init_weights(seed).items()}
    p["b1"] = S.uniform(seed + 7, 128) * 0.2 - 0.1
    p["b2"] = S.uniform(seed + 8, 128) * 0.2 - 0.1
    p["b3"] = np.array([0.05])
    return p


def test_gradients_match_finite_differences(M):
    p = _params(3)
    X = S.uniform(11, 6 * 125).reshape(6, 125)
    t = S.uniform(12, 6) * 0.4 - 0.2
    g = M.backward(p, X, t, round_bf16=False)
    h = 1e-6
    picks = [("W1", (5, 17)), ("W1", (100, 124)), ("b1", (3,)), ("W2", (7, 90)), ("b2", (64,)), ("w3", (12,)),
             ("b3", (0,))]
    for name, idx in picks:
        q = {k: v.copy() for k, v in p.items()}
        q[name][idx] += h
        lp = M.loss(q, X, t, round_bf16=False)
        q[name][idx] -= 2 * h
        lm = M.loss(q, X, t, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        gv = g[name][idx] if name != "b3" else g["b3"]
        assert gv == pytest.approx(fd, rel=1e-5, abs=1e-9), name


def test_adam_first_step_closed_form(M):
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    M.adam(p, g, m, v, 1, 1e-2)
    # first step: m_hat = g, v_hat = g^2 -> update -lr g / (|g| + eps)
    expect = np.array([1.0, -2.0, 0.5]) - 1e-2 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(p["a"], expect, atol=1e-15)


def test_ellipsoid_curvature_closed_forms(M):
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    a = (3.0, 4.0, 5.0)
    # surface point (a, 0, 0) placed at the origin: principal curvatures a/b^2, a/c^2
    C = M.shape_centre(a, ident, np.array([1.0, 0.0, 0.0]), np.zeros(3))
    H = M.ellipsoid_mean_curvature_nearest(a, ident, C, 0)
    assert H == pytest.approx(0.5 * (3 / 16 + 3 / 25), rel=1e-10)
    C = M.shape_centre(a, ident, np.array([0.0, 0.0, 1.0]), np.zeros(3))
    assert M.ellipsoid_mean_curvature_nearest(a, ident, C, 1) == pytest.approx(-0.5 * (5 / 9 + 5 / 16), rel=1e-10)
    # sphere: 1/R from any offset, rotated
    q = S.mlp_sample_params(4, 1)["quat"][0]
    C = M.shape_centre((7.0, 7.0, 7.0), q, np.array([0.0, 0.6, 0.8]), np.array([0.2, -0.3, 0.1]))
    assert M.ellipsoid_mean_curvature_nearest((7.0, 7.0, 7.0), q, C, 0) == pytest.approx(1 / 7, rel=1e-10)


def test_stencil_fill_matches_main_sampler(M, orc):
    """A sphere stencil from oracle.mlp against oracle.fill_cells (independent code)."""
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    R = 5.3
    C = M.shape_centre((R, R, R), ident, np.array([0.48, 0.6, 0.64]) / np.linalg.norm([0.48, 0.6, 0.64]),
                       np.array([0.1, -0.2, 0.05]))
    s = M.stencil_fill((R, R, R), ident, C, 0, 8)
    # main oracle: grid 5^3 with the stencil's cell (i,j,k) at index (i+2, j+2, k+2), centre shifted by 2
    G = orc.geom("sphere", c=tuple(C + 2.0), R=R, sub=8)
    ref = orc.fill(G, (5, 5, 5))  # [z, y, x]
    assert np.max(np.abs(np.transpose(ref, (2, 1, 0)) - s)) <= 1.0 / 512


def test_canonical_form_is_symmetry_invariant(M):
    s = S.uniform(21, 125).reshape(5, 5, 5)
    s[:, :, :2] *= 0.3  # give the centre a generic gradient
    base = M.canonical(s)
    for flips in [(0,), (1,), (2,), (0, 2), (0, 1, 2)]:
        t = s
        for a in flips:
            t = np.flip(t, a)
        for perm in [(0, 1, 2), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
            assert np.allclose(M.canonical(np.transpose(t, perm)), base, atol=0)
