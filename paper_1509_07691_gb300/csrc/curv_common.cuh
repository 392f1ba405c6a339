// curv_common.cuh -- the per-cell curvature arithmetic of Sec. II.A-C, written
// once for plain (float, double) and dual numbers: obstacle reflection of the
// fill level, Parker-Youngs gradient, PLIC volume and offset, streaming
// Givens least squares, contact point and contact normal, and the LSQR
// paraboloid fit.  The forward kernels (k_curv.cu) instantiate it with float
// and double; the curvature Jacobian of the adjoint (k_adj.cu) with
// Dual<float> and Dual<double>, one seed per lane.
//
// Cell access goes through an accessor `acc` relative to the centre cell:
//   acc.flag(dx, dy, dz)              flags of the cell at that offset
//   acc.normal(dx, dy, dz, n[3], a)   unit PLIC normal and offset of an
//                                     interface cell (false for a zero normal)
//   acc.theta(ct, st)                 cos and sin of the contact angle
#pragma once

#include "dual.cuh"
#include "fsl_internal.cuh"

namespace fslk {

// ---- fill level at obstacle cells (Sec. II.A reflection, aperture sqrt(2)/2) --
// n_w is the (integer) sum of the lattice vectors from the obstacle cell to
// its non-obstacle neighbours; the aperture test 2 (N.c)^2 > |N|^2 |c|^2 is
// exact.  flag_at / value_at take offsets from the obstacle cell.
template <typename T, typename FL, typename V>
__device__ T reflect_value(FL flag_at, V value_at) {
    int nx = 0, ny = 0, nz = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (flag_at(cx(q), cy(q), cz(q)) & T_OBS) continue;
        nx += cx(q);
        ny += cy(q);
        nz += cz(q);
    }
    const int n2 = nx * nx + ny * ny + nz * nz;
    if (n2 == 0) return T(0);
    T num = T(0);
    float den = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int dx = cx(q), dy = cy(q), dz = cz(q);
        if (flag_at(dx, dy, dz) & T_OBS) continue;
        const int dot = nx * dx + ny * dy + nz * dz;
        const int c2 = dx * dx + dy * dy + dz * dz;
        if (2 * dot * dot > n2 * c2) {
            const float w = fabsf((float)dot) * rsqrtf((float)(n2 * c2));
            num += w * value_at(dx, dy, dz);
            den += w;
        }
    }
    return den > 0.f ? num / den : T(0);
}

// Parker-Youngs gradient: central difference with transverse weights 4/2/1;
// g(dx, dy, dz) is the fill level at that offset from the cell.
template <typename T, typename G>
__device__ __forceinline__ void parker_youngs(G g, T n[3]) {
    n[0] = n[1] = n[2] = T(0);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const T v = g(dx, dy, dz);
                if (dx) n[0] += (float)(dx * (dy == 0 ? 2 : 1) * (dz == 0 ? 2 : 1)) * v;
                if (dy) n[1] += (float)(dy * (dx == 0 ? 2 : 1) * (dz == 0 ? 2 : 1)) * v;
                if (dz) n[2] += (float)(dz * (dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1)) * v;
            }
}

// ---- PLIC ------------------------------------------------------------------
// Volume of {z in [0,1]^3 : m.z <= al} for m >= 0 sorted m1 <= m2 <= m3 with
// m1 + m2 + m3 = 1, al in [0, 1/2].  Inclusion-exclusion of the corner
// simplex, with the divided differences in m1 taken analytically so that no
// branch divides by a component that can vanish there.
template <typename T>
__device__ __forceinline__ T plic_vol_half(T m1, T m2, T m3, T al) {
    if (al < m1) return al * al * al / (6.0f * m1 * m2 * m3);
    const T base = 3.0f * al * al - 3.0f * al * m1 + m1 * m1;  // ((al)^3 - (al-m1)^3)/m1
    if (al < m2) return base / (6.0f * m2 * m3);
    if (al >= m1 + m2) return (2.0f * al - m1 - m2) / (2.0f * m3);
    const T e2 = al - m2;
    if (al < m3) return (base - e2 * e2 * (e2 / m1)) / (6.0f * m2 * m3);
    const T e3 = al - m3;
    return (base - e2 * e2 * (e2 / m1) - e3 * e3 * (e3 / m1)) / (6.0f * m2 * m3);
}

template <typename T>
__device__ __forceinline__ T plic_vol(T m1, T m2, T m3, T al) {
    return al <= 0.5f ? plic_vol_half(m1, m2, m3, al) : 1.0f - plic_vol_half(m1, m2, m3, 1.0f - al);
}

// dV/dal of plic_vol_half, branch by branch
template <typename S>
__device__ __forceinline__ S plic_dvol_half(S m1, S m2, S m3, S al) {
    if (al < m1) return al * al / (2.0f * m1 * m2 * m3);
    if (al < m2) return (2.0f * al - m1) / (2.0f * m2 * m3);
    if (al >= m1 + m2) return S(1) / m3;
    const S e2 = al - m2;
    S t = 6.0f * al - 3.0f * m1 - 3.0f * e2 * (e2 / m1);
    if (al >= m3) {
        const S e3 = al - m3;
        t -= 3.0f * e3 * (e3 / m1);
    }
    return t / (6.0f * m2 * m3);
}

// Inverse of plic_vol: al with V(al) = phi.  By symmetry only V <= 1/2 is
// solved.  The branch is found from V at the break points m1, m2 and
// min(m3, m1 + m2); the corner tetrahedron (cube root), the two-plane wedge
// (quadratic) and the four-edge slab (linear) are solved in closed form, the
// remaining cubic by Newton from the secant between its break points.
template <typename S>
__device__ S plic_alpha(S m1, S m2, S m3, S phi, int iters) {
    const bool mirror = phi > 0.5f;
    const S v = mirror ? S(1) - phi : phi;
    const S V1 = m1 > S(0) ? m1 * m1 / (6.0f * m2 * m3) : S(0);
    const S V2 = m2 > S(0) ? (3.0f * m2 * m2 - 3.0f * m2 * m1 + m1 * m1) / (6.0f * m2 * m3) : S(0);
    const S a3 = fmin(m3, m1 + m2);
    const S V3 = plic_vol_half(m1, m2, m3, a3);
    S al;
    if (v < V1) {
        al = cbrt(6.0f * m1 * m2 * m3 * v);
    } else if (v < V2) {
        al = 0.5f * m1 + sqrt(fmax(72.0f * m2 * m3 * v - 3.0f * m1 * m1, S(0))) * (S(1) / S(6));
    } else if (v >= V3 && m3 >= m1 + m2) {
        al = m3 * v + 0.5f * (m1 + m2);
    } else {
        S lo, hi, vlo, vhi;
        if (v < V3) { lo = m2; hi = a3; vlo = V2; vhi = V3; }
        else { lo = a3; hi = S(0.5); vlo = V3; vhi = S(0.5); }
        al = vhi > vlo ? lo + (hi - lo) * (v - vlo) / (vhi - vlo) : lo;
        for (int it = 0; it < iters; ++it) {
            const S g = plic_vol_half(m1, m2, m3, al) - v;
            al = fmin(fmax(al - g / plic_dvol_half(m1, m2, m3, al), lo), hi);
        }
    }
    return mirror ? S(1) - al : al;
}

// Offset a of the plane {y.n = a} through the cell [-1/2,1/2]^3 whose liquid
// side {y.n >= a} holds volume phi.  With m = |n| / sum|n| and
// al = 1/2 - a / sum|n| the liquid part is {z : m.z <= al} of the unit cube.
template <typename S>
__device__ S plic_offset(S nx, S ny, S nz, S phi, int iters) {
    S a1 = fabs(nx), a2 = fabs(ny), a3 = fabs(nz);
    const S M = a1 + a2 + a3;
    if (phi <= S(0)) return 0.5f * M;
    if (phi >= S(1)) return -0.5f * M;
    S t;
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    const S m1 = a1 / M, m2 = a2 / M, m3 = S(1) - m1 - m2;
    return M * (0.5f - plic_alpha(m1, m2, m3, phi, iters));
}

// The same offset for dual inputs: the value by plic_offset's arithmetic, the
// derivative by the implicit function theorem on V(al; m) = phi,
// dal = (dphi - dV/dm . dm) / (dV/dal), exact at the computed al.
template <typename S>
__device__ Dual<S> plic_offset(Dual<S> nx, Dual<S> ny, Dual<S> nz, Dual<S> phi, int iters) {
    using T = Dual<S>;
    T a1 = fabs(nx), a2 = fabs(ny), a3 = fabs(nz);
    const T M = a1 + a2 + a3;
    if (phi.v <= S(0)) return 0.5f * M;
    if (phi.v >= S(1)) return -0.5f * M;
    T t;
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    const T m1 = a1 / M, m2 = a2 / M, m3 = T(1) - m1 - m2;
    const S al = plic_alpha(m1.v, m2.v, m3.v, phi.v, iters);
    const T V = plic_vol(m1, m2, m3, T(al));  // V.d = dV/dm . dm at fixed al
    const S dV = al <= S(0.5) ? plic_dvol_half(m1.v, m2.v, m3.v, al) : plic_dvol_half(m1.v, m2.v, m3.v, S(1) - al);
    const T alpha(al, dV > S(0) ? (phi.d - V.d) / dV : S(0), 0);
    return M * (0.5f - alpha);
}

// unit normal of the Parker-Youngs gradient and its PLIC offset; false (and
// a zero normal) where the gradient vanishes
template <typename T>
__device__ __forceinline__ bool unit_normal_offset(T nv[3], T phi, int iters, T &a) {
    const T l2 = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
    if (!(value_of(l2) >= 1e-24f)) {
        nv[0] = nv[1] = nv[2] = T(0);
        a = T(0);
        return false;
    }
    const T inv = rsqrt_of(l2);
    nv[0] = nv[0] * inv;
    nv[1] = nv[1] * inv;
    nv[2] = nv[2] * inv;
    a = plic_offset(nv[0], nv[1], nv[2], phi, iters);
    return true;
}

// ---- LSQR --------------------------------------------------------------------
// Streaming Givens QR of a K-column least-squares problem (upper triangle R
// and Q^T b kept in registers; rows are rotated in as they come).
template <typename T, int K>
struct Givens {
    T R[K * (K + 1) / 2];
    T qb[K];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int j = 0; j < K * (K + 1) / 2; ++j) R[j] = T(0);
#pragma unroll
        for (int j = 0; j < K; ++j) qb[j] = T(0);
    }
    __device__ __forceinline__ static int at(int r, int c) { return r * K - r * (r - 1) / 2 + (c - r); }
    __device__ __forceinline__ void add(T a[K], T b, int k) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (j >= k) break;
            const T rjj = R[at(j, j)];
            const T h = sqrt(rjj * rjj + a[j] * a[j]);
            if (h == T(0)) continue;
            const T c = rjj / h, s = a[j] / h;
            R[at(j, j)] = h;
#pragma unroll
            for (int l = j + 1; l < K; ++l) {
                if (l >= k) break;
                const T r = R[at(j, l)];
                R[at(j, l)] = c * r + s * a[l];
                a[l] = c * a[l] - s * r;
            }
            const T z = qb[j];
            qb[j] = c * z + s * b;
            b = c * b - s * z;
        }
    }
    // back substitution; returns false if some |R_jj| <= 1e-6 max|R_ii|; cond = max/min |R_jj|
    __device__ __forceinline__ bool solve(T xo[K], int k, T &cond) {
        T rmax = T(0), rmin = T(3.0e38);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (j >= k) break;
            const T r = fabs(R[at(j, j)]);
            rmax = r > rmax ? r : rmax;
            rmin = r < rmin ? r : rmin;
        }
        cond = rmin > T(0) ? rmax / rmin : T(3.0e38);
        if (!(rmax > T(0)) || !(rmin > T(1e-6) * rmax)) return false;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            if (j >= k) continue;
            T s = qb[j];
#pragma unroll
            for (int l = j + 1; l < K; ++l)
                if (l < k) s -= R[at(j, l)] * xo[l];
            xo[j] = s / R[at(j, j)];
        }
        return true;
    }
};

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Contact point and contact normal of contact-line cell j at offset o from
// the centre (Sec. II.C, Fig. contactPoint, Eq. contactNormal): wall normal
// n_w = unit sum of the vectors to j's obstacle neighbours (into the wall);
// wall plane half way, (y - o).n_w = 1/2; p_c = p_j + s d with d the unit
// projection of n_w onto the PLIC plane (none if |d| < 1e-6);
// m = n_w cos(theta) + n_t sin(theta), n_t the unit projection of n_j onto the wall.
template <typename T, typename Acc>
__device__ bool contact(const Acc &acc, int ox, int oy, int oz, const T o[3], const T nj[3], T aj, T pc[3],
                        T mh[3]) {
    T w[3] = {T(0), T(0), T(0)};
    int cnt = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (acc.flag(ox + cx(q), oy + cy(q), oz + cz(q)) & T_OBS) {
            w[0] += T((double)cx(q));
            w[1] += T((double)cy(q));
            w[2] += T((double)cz(q));
            ++cnt;
        }
    }
    if (!cnt) return false;
    const T wl = sqrt(dot3(w, w));
    if (wl < T(1e-12)) return false;
    w[0] /= wl;
    w[1] /= wl;
    w[2] /= wl;
    const T wn = dot3(w, nj);
    T dv[3] = {w[0] - wn * nj[0], w[1] - wn * nj[1], w[2] - wn * nj[2]};
    const T dl = sqrt(dot3(dv, dv));
    if (dl < T(1e-6)) return false;
    dv[0] /= dl;
    dv[1] /= dl;
    dv[2] /= dl;
    const T rel[3] = {aj * nj[0], aj * nj[1], aj * nj[2]};
    const T s = (T(0.5) - dot3(rel, w)) / dot3(dv, w);
    T nt[3] = {nj[0] - wn * w[0], nj[1] - wn * w[1], nj[2] - wn * w[2]};
    const T ntl = sqrt(dot3(nt, nt));
    if (ntl < T(1e-12)) return false;
    T ct, sn;
    acc.theta(ct, sn);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pc[k] = o[k] + rel[k] + s * dv[k];
        mh[k] = w[k] * ct + (nt[k] / ntl) * sn;
    }
    return true;
}

// LSQR curvature of the centre interface cell (Sec. II.C), with flags fi.
// The model is f(u,v) = A u^2 + B v^2 + C uv + H u + I v (J = 0) in the frame
// (t_u, t_v, n) of the centre normal, through the PLIC points of the
// interface cells of the 3x3x3 neighbourhood, plus two gradient rows per
// contact point of a contact-line neighbour.  A centre constraint
// grad f(u_c, v_c) = g (the centre is a contact-line cell) is eliminated
// exactly (H = g_u - 2 u_c A - v_c C, I = g_v - 2 v_c B - u_c C).  Fallbacks:
// isotropic model B = A, C = 0, then kappa = 0.  kappa by Eq. (anacurv) with
// the mixed term -C H I.  cond_out = max/min |R_jj| of the solve taken.
template <typename T, typename Acc>
__device__ T lsqr_core(const Acc &acc, uint8_t fi, T &cond_out) {
    cond_out = T(1);
    T n[3], a;
    if (!acc.normal(0, 0, 0, n, a)) return T(0);
    int k = 0;
    if (fabs(n[1]) < fabs(n[0])) k = 1;
    if (fabs(n[2]) < fabs(n[k])) k = 2;
    T tu[3];
    if (k == 0) { tu[0] = T(0); tu[1] = -n[2]; tu[2] = n[1]; }
    else if (k == 1) { tu[0] = n[2]; tu[1] = T(0); tu[2] = -n[0]; }
    else { tu[0] = -n[1]; tu[1] = n[0]; tu[2] = T(0); }
    const T tl = sqrt(dot3(tu, tu));
    tu[0] /= tl;
    tu[1] /= tl;
    tu[2] /= tl;
    const T tv[3] = {n[1] * tu[2] - n[2] * tu[1], n[2] * tu[0] - n[0] * tu[2], n[0] * tu[1] - n[1] * tu[0]};
    const T p[3] = {a * n[0], a * n[1], a * n[2]};

    bool cons = false;
    T uc = T(0), vc = T(0), gu = T(0), gv = T(0);
    if (fi & B_NEAR) {
        const T o[3] = {T(0), T(0), T(0)};
        T pc[3], mh[3];
        if (contact<T>(acc, 0, 0, 0, o, n, a, pc, mh)) {
            const T mn = dot3(mh, n);
            if (fabs(mn) >= T(1e-6)) {
                const T dc[3] = {pc[0] - p[0], pc[1] - p[1], pc[2] - p[2]};
                uc = dot3(dc, tu);
                vc = dot3(dc, tv);
                gu = -dot3(mh, tu) / mn;
                gv = -dot3(mh, tv) / mn;
                cons = true;
            }
        }
    }
    Givens<T, 5> full;
    Givens<T, 3> red;
    full.init();
    red.init();
    const int kf = cons ? 3 : 5, kr = cons ? 1 : 3;
    int m = 0;
#pragma unroll 1
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int dx = t % 3 - 1, dy = t / 3 - 1;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const uint8_t fj = acc.flag(dx, dy, dz);
            if (!(fj & T_IF)) continue;
            T nj[3], aj;
            if (!acc.normal(dx, dy, dz, nj, aj)) continue;
            const T o[3] = {T((double)dx), T((double)dy), T((double)dz)};
            const T dv[3] = {o[0] + aj * nj[0] - p[0], o[1] + aj * nj[1] - p[1], o[2] + aj * nj[2] - p[2]};
            const T u = dot3(dv, tu), v = dot3(dv, tv), f = dot3(dv, n);
            if (!cons) {
                T rf[5] = {u * u, v * v, u * v, u, v};
                T rr[3] = {u * u + v * v, u, v};
                full.add(rf, f, kf);
                red.add(rr, f, kr);
            } else {
                const T rhs = f - gu * u - gv * v;
                T rf[5] = {u * u - T(2) * uc * u, v * v - T(2) * vc * v, u * v - vc * u - uc * v, T(0), T(0)};
                T rr[3] = {u * u + v * v - T(2) * uc * u - T(2) * vc * v, T(0), T(0)};
                full.add(rf, rhs, kf);
                red.add(rr, rhs, kr);
            }
            ++m;
            if (fj & B_NEAR) {
                T pc[3], mh[3];
                if (!contact<T>(acc, dx, dy, dz, o, nj, aj, pc, mh)) continue;
                const T mn = dot3(mh, n);
                if (fabs(mn) < T(1e-6)) continue;
                const T dc[3] = {pc[0] - p[0], pc[1] - p[1], pc[2] - p[2]};
                const T uj = dot3(dc, tu), vj = dot3(dc, tv);
                const T g1 = -dot3(mh, tu) / mn, g2 = -dot3(mh, tv) / mn;
                if (!cons) {
                    T r1[5] = {T(2) * uj, T(0), vj, T(1), T(0)};
                    T r2[5] = {T(0), T(2) * vj, uj, T(0), T(1)};
                    T s1[3] = {T(2) * uj, T(1), T(0)};
                    T s2[3] = {T(2) * vj, T(0), T(1)};
                    full.add(r1, g1, kf);
                    full.add(r2, g2, kf);
                    red.add(s1, g1, kr);
                    red.add(s2, g2, kr);
                } else {
                    T r1[5] = {T(2) * (uj - uc), T(0), vj - vc, T(0), T(0)};
                    T r2[5] = {T(0), T(2) * (vj - vc), uj - uc, T(0), T(0)};
                    T s1[3] = {T(2) * (uj - uc), T(0), T(0)};
                    T s2[3] = {T(2) * (vj - vc), T(0), T(0)};
                    full.add(r1, g1 - gu, kf);
                    full.add(r2, g2 - gv, kf);
                    red.add(s1, g1 - gu, kr);
                    red.add(s2, g2 - gv, kr);
                }
                m += 2;
            }
        }
    }
    T A = T(0), B = T(0), C = T(0), H = T(0), I = T(0);
    T cond = T(1);
    T sol[5] = {T(0), T(0), T(0), T(0), T(0)};
    bool done = false;
    if (m >= kf && full.solve(sol, kf, cond)) {
        A = sol[0];
        B = sol[1];
        C = sol[2];
        if (cons) {
            H = gu - T(2) * uc * A - vc * C;
            I = gv - T(2) * vc * B - uc * C;
        } else {
            H = sol[3];
            I = sol[4];
        }
        done = true;
    } else {
        T xr[3] = {T(0), T(0), T(0)};
        T c2;
        if (m >= kr && red.solve(xr, kr, c2)) {
            cond = c2;
            A = B = xr[0];
            if (cons) {
                H = gu - T(2) * uc * A;
                I = gv - T(2) * vc * A;
            } else {
                H = xr[1];
                I = xr[2];
            }
            done = true;
        }
    }
    cond_out = cond;
    if (!done) return T(0);
    const T g = T(1) + H * H + I * I;
    return (A * (T(1) + I * I) + B * (T(1) + H * H) - C * H * I) / (g * sqrt(g));
}

// Accessor of the forward kernels: flags and stored PLIC normals (float4
// n, a) of the grid around cell (x, y, z); periodic wrap.
struct GridAcc {
    const Dev &d;
    int x, y, z;
    __device__ __forceinline__ uint8_t flag(int dx, int dy, int dz) const {
        return d.flags[nbr_index(d, x, y, z, dx, dy, dz)];
    }
    template <typename T>
    __device__ __forceinline__ bool normal(int dx, int dy, int dz, T n[3], T &a) const {
        const float4 q4 = d.normal[nbr_index(d, x, y, z, dx, dy, dz)];
        if (q4.x == 0.f && q4.y == 0.f && q4.z == 0.f) return false;
        n[0] = T(q4.x);
        n[1] = T(q4.y);
        n[2] = T(q4.z);
        a = T(q4.w);
        return true;
    }
    template <typename T>
    __device__ __forceinline__ void theta(T &ct, T &st) const {
        ct = T(d.cos_theta_d);
        st = T(d.sin_theta_d);
    }
};

// Accessor of the general-path kernels: the same values staged in shared
// memory by one warp per cell (stage_block): the flags of the 5x5x5 block
// (contact points look one cell past the 3x3x3 block) and the stored normals
// of the 3x3x3 block.
struct StagedAcc {
    const Dev &d;
    const uint8_t *fl;  // slot ((dz+2)*5 + dy+2)*5 + dx+2
    const float4 *nm;   // slot (dz+1)*9 + (dy+1)*3 + dx+1
    __device__ __forceinline__ uint8_t flag(int dx, int dy, int dz) const {
        return fl[((dz + 2) * 5 + (dy + 2)) * 5 + (dx + 2)];
    }
    template <typename T>
    __device__ __forceinline__ bool normal(int dx, int dy, int dz, T n[3], T &a) const {
        const float4 q4 = nm[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (q4.x == 0.f && q4.y == 0.f && q4.z == 0.f) return false;
        n[0] = T(q4.x);
        n[1] = T(q4.y);
        n[2] = T(q4.z);
        a = T(q4.w);
        return true;
    }
    template <typename T>
    __device__ __forceinline__ void theta(T &ct, T &st) const {
        ct = T(d.cos_theta_d);
        st = T(d.sin_theta_d);
    }
};

// the lanes of a warp stage the block of cell (x, y, z) for StagedAcc
__device__ __forceinline__ void stage_block(const Dev &d, int x, int y, int z, int lane, uint8_t *fl, float4 *nm) {
    for (int e = lane; e < 125; e += 32) fl[e] = d.flags[nbr_index(d, x, y, z, e % 5 - 2, (e / 5) % 5 - 2, e / 25 - 2)];
    if (lane < 27) nm[lane] = d.normal[nbr_index(d, x, y, z, lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1)];
}

// Fast path: FP32 normal equations of the full model for an interface cell
// with no contact-line cell in its neighbourhood.  The 5x5 Gram matrix
// A^T A and A^T f are accumulated row by row (independent FMAs), then solved
// by Cholesky in registers.  The fit is rejected (cell left to the general
// path) when a contact-line cell is present, when there are fewer than five
// rows, or when the Cholesky pivots estimate cond(A^T A) above fp64_cond.
// In three parts so that the rows can be split over several lanes:
// fill level at any cell (periodic wrap); an obstacle cell takes the
// reflected fill level of Sec. II.A (kept out of line: callers unroll over
// their stencils and obstacle cells are rare)
static __device__ __noinline__ float phi_reflected(const Dev &d, int x, int y, int z) {
    return reflect_value<float>([&](int a, int b, int c) { return d.flags[nbr_index(d, x, y, z, a, b, c)]; },
                                [&](int a, int b, int c) { return d.phi[nbr_index(d, x, y, z, a, b, c)]; });
}

static __device__ __forceinline__ float phi_ext(const Dev &d, int x, int y, int z) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    const int i = cell_index(d, x, y, z);
    if (!(d.flags[i] & T_OBS)) return d.phi[i];
    return phi_reflected(d, x, y, z);
}

// lsqr_fast_frame, lsqr_fast_row (for each neighbour slot t of the 3x3x3
// block, t = (dz+1)*9 + (dy+1)*3 + (dx+1), centre 13), lsqr_fast_solve.
struct FastFrame {
    float n[3], tu[3], tv[3], p[3];
};

__device__ __forceinline__ void lsqr_fast_frame(const float4 c4, FastFrame &F) {
    F.n[0] = c4.x;
    F.n[1] = c4.y;
    F.n[2] = c4.z;
    int k = 0;
    if (fabsf(F.n[1]) < fabsf(F.n[0])) k = 1;
    if (fabsf(F.n[2]) < fabsf(F.n[k])) k = 2;
    if (k == 0) { F.tu[0] = 0.f; F.tu[1] = -F.n[2]; F.tu[2] = F.n[1]; }
    else if (k == 1) { F.tu[0] = F.n[2]; F.tu[1] = 0.f; F.tu[2] = -F.n[0]; }
    else { F.tu[0] = -F.n[1]; F.tu[1] = F.n[0]; F.tu[2] = 0.f; }
    const float tl = rsqrtf(dot3(F.tu, F.tu));
    F.tu[0] *= tl;
    F.tu[1] *= tl;
    F.tu[2] *= tl;
    F.tv[0] = F.n[1] * F.tu[2] - F.n[2] * F.tu[1];
    F.tv[1] = F.n[2] * F.tu[0] - F.n[0] * F.tu[2];
    F.tv[2] = F.n[0] * F.tu[1] - F.n[1] * F.tu[0];
    F.p[0] = c4.w * F.n[0];
    F.p[1] = c4.w * F.n[1];
    F.p[2] = c4.w * F.n[2];
}

__device__ __forceinline__ void lsqr_fast_row(int t, uint8_t fj, const float4 q4, const FastFrame &F, float G[15],
                                              float r[5], int &m, bool &contact) {
    const bool use = (fj & T_IF) && t != 13 && !(q4.x == 0.f && q4.y == 0.f && q4.z == 0.f);
    contact |= (fj & T_IF) && (fj & B_NEAR);
    const float w = use ? 1.f : 0.f;
    const float dv[3] = {(float)(t % 3 - 1) + q4.w * q4.x - F.p[0], (float)((t / 3) % 3 - 1) + q4.w * q4.y - F.p[1],
                         (float)(t / 9 - 1) + q4.w * q4.z - F.p[2]};
    const float u = dot3(dv, F.tu), v = dot3(dv, F.tv), f = w * dot3(dv, F.n);
    const float a[5] = {w * u * u, w * v * v, w * u * v, w * u, w * v};
    int c = 0;
#pragma unroll
    for (int a0 = 0; a0 < 5; ++a0) {
#pragma unroll
        for (int a1 = a0; a1 < 5; ++a1) G[c++] += a[a0] * a[a1];
        r[a0] += a[a0] * f;
    }
    m += use ? 1 : 0;
}

__device__ __forceinline__ bool lsqr_fast_solve(const float G[15], const float r[5], int m, bool contact,
                                                float fp64_cond, float &kap) {
    // Cholesky G = R^T R (R upper, packed like G)
    float R[15];
    float dmax = 0.f, dmin = 3.0e38f;
    bool pd = true;
    {
        int c = 0;
#pragma unroll
        for (int a0 = 0; a0 < 5; ++a0) {
#pragma unroll
            for (int a1 = a0; a1 < 5; ++a1, ++c) {
                float sum = G[c];
#pragma unroll
                for (int kk = 0; kk < a0; ++kk) {
                    const int i0 = kk * 5 - kk * (kk - 1) / 2 + (a0 - kk), i1 = kk * 5 - kk * (kk - 1) / 2 + (a1 - kk);
                    sum -= R[i0] * R[i1];
                }
                if (a1 == a0) {
                    pd = pd && sum > 0.f;
                    const float dd = sqrtf(fmaxf(sum, 1e-30f));
                    R[c] = dd;
                    dmax = fmaxf(dmax, dd);
                    dmin = fminf(dmin, dd);
                } else {
                    R[c] = sum / R[a0 * 5 - a0 * (a0 - 1) / 2];
                }
            }
        }
    }
    const float cond = (dmax / dmin) * (dmax / dmin);
    const bool ok = !contact && m >= 5 && pd && !(cond > fp64_cond);
    // R^T y = r, R x = y
    float yv[5], sol[5];
#pragma unroll
    for (int a0 = 0; a0 < 5; ++a0) {
        float sum = r[a0];
#pragma unroll
        for (int kk = 0; kk < a0; ++kk) sum -= R[kk * 5 - kk * (kk - 1) / 2 + (a0 - kk)] * yv[kk];
        yv[a0] = sum / R[a0 * 5 - a0 * (a0 - 1) / 2];
    }
#pragma unroll
    for (int a0 = 4; a0 >= 0; --a0) {
        float sum = yv[a0];
#pragma unroll
        for (int kk = a0 + 1; kk < 5; ++kk) sum -= R[a0 * 5 - a0 * (a0 - 1) / 2 + (kk - a0)] * sol[kk];
        sol[a0] = sum / R[a0 * 5 - a0 * (a0 - 1) / 2];
    }
    const float A = sol[0], B = sol[1], C = sol[2], H = sol[3], I = sol[4];
    const float g = 1.0f + H * H + I * I;
    kap = (A * (1.0f + I * I) + B * (1.0f + H * H) - C * H * I) / (g * sqrtf(g));
    return ok;
}

// one thread per cell: the flags and stored normals of the whole 3x3x3
// block are loaded before any is used (one round of independent loads)
__device__ __forceinline__ bool lsqr_fast(const Dev &d, int i, int x, int y, int z, float &kap) {
    const int xs[3] = {x == 0 ? d.nx - 1 : x - 1, x, x == d.nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? d.ny - 1 : y - 1, y, y == d.ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? d.nz - 1 : z - 1, z, z == d.nz - 1 ? 0 : z + 1};
    uint8_t fjs[27];
    float4 q4s[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int jj = cell_index(d, xs[t % 3], ys[(t / 3) % 3], zs[t / 9]);
        fjs[t] = d.flags[jj];
        q4s[t] = d.normal[jj];
    }
    const float4 c4 = q4s[13];
    kap = 0.f;
    if (c4.x == 0.f && c4.y == 0.f && c4.z == 0.f) return true;
    FastFrame F;
    lsqr_fast_frame(c4, F);
    float G[15], r[5];
#pragma unroll
    for (int t = 0; t < 15; ++t) G[t] = 0.f;
#pragma unroll
    for (int t = 0; t < 5; ++t) r[t] = 0.f;
    int m = 0;
    bool contact = (fjs[13] & B_NEAR) != 0;
#pragma unroll
    for (int t = 0; t < 27; ++t) lsqr_fast_row(t, fjs[t], q4s[t], F, G, r, m, contact);
    return lsqr_fast_solve(G, r, m, contact, d.fp64_cond, kap);
}

}  // namespace fslk
