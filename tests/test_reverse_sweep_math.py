"""The reverse sweep of the LSQR fit that k_kappa_rev (csrc/k_adj.cu) runs for
the curvature Jacobian of the adjoint window, written out in numpy and
checked against central differences of the same fit (Sec. II.C: paraboloid
f = A u^2 + B v^2 + C uv + H u + I v through the PLIC points of the 3x3x3
block in the frame of the centre normal, kappa by Eq. anacurv).  The sweep:
  xbar = dkappa/d(A, B, C, H, I), lambda = G^-1 xbar,
  rowbar_j = e_j lambda - (row_j . lambda) x,  fbar_j = row_j . lambda,
then through u, v, f = d . (t_u, t_v, n), d = o_j + a_j n_j - a n, and the
centre frame t_u = w/|w|, t_v = n x t_u.  CPU only; the GPU kernel itself is
checked against FP64 oracle differences in test_gpu_adjoint.py."""
import numpy as np
import pytest


def _frame(n):
    k = 0
    if abs(n[1]) < abs(n[0]):
        k = 1
    if abs(n[2]) < abs(n[k]):
        k = 2
    w = [np.array([0.0, -n[2], n[1]]), np.array([n[2], 0.0, -n[0]]), np.array([-n[1], n[0], 0.0])][k]
    tu = w / np.linalg.norm(w)
    return k, w, tu, np.cross(n, tu)


def _offset(t):
    return np.array([t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1], float)


def _fit(nn, aa, rows):
    n, a = nn[13], aa[13]
    k, w, tu, tv = _frame(n)
    p = a * n
    M, f, dvs = [], [], []
    for t in rows:
        dv = _offset(t) + aa[t] * nn[t] - p
        u, v = dv @ tu, dv @ tv
        M.append([u * u, v * v, u * v, u, v])
        f.append(dv @ n)
        dvs.append(dv)
    M, f = np.array(M), np.array(f)
    G = M.T @ M
    x = np.linalg.solve(G, M.T @ f)
    return k, w, tu, tv, p, M, f, dvs, G, x


def kappa(nn, aa, rows):
    x = _fit(nn, aa, rows)[-1]
    A, B, C, H, I = x
    g = 1 + H * H + I * I
    return (A * (1 + I * I) + B * (1 + H * H) - C * H * I) / g ** 1.5


def reverse(nn, aa, rows, drop_residual=False):
    n, a = nn[13], aa[13]
    k, w, tu, tv, p, M, f, dvs, G, x = _fit(nn, aa, rows)
    A, B, C, H, I = x
    g = 1 + H * H + I * I
    D = g ** 1.5
    Nn = A * (1 + I * I) + B * (1 + H * H) - C * H * I
    xb = np.array([(1 + I * I) / D, (1 + H * H) / D, -H * I / D,
                   (2 * B * H - C * I - 3 * Nn * H / g) / D, (2 * A * I - C * H - 3 * Nn * I / g) / D])
    lam = np.linalg.solve(G, xb)
    gn, ga = np.zeros((27, 3)), np.zeros(27)
    tub, tvb, nb, pb = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    for row, dv, fj, t in zip(M, dvs, f, rows):
        u, v = dv @ tu, dv @ tv
        e, rl = fj - row @ x, row @ lam
        rb = (0.0 if drop_residual else e) * lam - rl * x
        ub = 2 * u * rb[0] + v * rb[2] + rb[3]
        vb = 2 * v * rb[1] + u * rb[2] + rb[4]
        db = ub * tu + vb * tv + rl * n
        gn[t], ga[t] = aa[t] * db, nn[t] @ db
        tub += ub * dv
        tvb += vb * dv
        nb += rl * dv
        pb -= db
    nb += np.cross(tu, tvb)
    tub += np.cross(tvb, n)
    wb = (tub - tu * (tu @ tub)) / np.linalg.norm(w)
    if k == 0:
        nb[2] -= wb[1]; nb[1] += wb[2]
    elif k == 1:
        nb[2] += wb[0]; nb[0] -= wb[2]
    else:
        nb[1] -= wb[0]; nb[0] += wb[1]
    ga[13] = pb @ n
    gn[13] = nb + a * pb
    return gn, ga


@pytest.mark.parametrize("seed", range(6))
def test_reverse_sweep_matches_central_differences(seed):
    nn, aa, rows = _case(seed)
    assert _worst(nn, aa, rows) < 1e-7


def _case(seed):
    rng = np.random.default_rng(100 + seed)
    R = 4.0 + 4.0 * seed
    c = rng.normal(size=3)
    c *= (R + 0.3 * rng.normal()) / np.linalg.norm(c)
    nn, aa = np.zeros((27, 3)), np.zeros(27)
    for t in range(27):
        d = c - _offset(t)
        r = np.linalg.norm(d)
        nn[t] = d / r + 0.05 * rng.normal(size=3)
        aa[t] = r - R + 0.05 * rng.normal()
    rows = [t for t in range(27) if t != 13 and rng.random() < 0.8]
    return nn, aa, rows


def _worst(nn, aa, rows, **kw):
    gn, ga = reverse(nn, aa, rows, **kw)
    h, worst = 1e-6, 0.0
    for t in rows + [13]:
        for comp in range(4):
            pn, pa, mn, ma = nn.copy(), aa.copy(), nn.copy(), aa.copy()
            if comp < 3:
                pn[t, comp] += h
                mn[t, comp] -= h
            else:
                pa[t] += h
                ma[t] -= h
            fd = (kappa(pn, pa, rows) - kappa(mn, ma, rows)) / (2 * h)
            worst = max(worst, abs((gn[t, comp] if comp < 3 else ga[t]) - fd))
    return worst


def test_a_dropped_term_is_caught():
    """The same check fails when the residual term of rowbar is left out
    (a plausible slip in the derivation): the noisy normals put the PLIC
    points off any paraboloid."""
    nn, aa, rows = _case(1)
    assert _worst(nn, aa, rows) < 1e-7
    assert _worst(nn, aa, rows, drop_residual=True) > 1e-4
