// k_curv.cu -- interface normals, PLIC points and curvature (Sec. II.A-C).
//   k_normals  Parker-Youngs normal of phi (obstacle cells by the aperture
//              reflection of Sec. II.A) and the PLIC offset a with
//              vol(cell cap {y.n >= a}) = phi (Sec. II.B), per interface cell.
//   k_lsqr     least-squares paraboloid through the PLIC points of the 3x3x3
//              neighbourhood with contact-point rows and centre constraints
//              (Sec. II.C), solved by streaming Givens QR in registers; cells
//              whose R is ill conditioned are re-solved in FP64.
//   k_fd       finite-difference curvature -1/2 div(n) of the K8-smoothed fill
//              level with wetting normals at obstacle cells (Sec. II.A).
#include "fsl_internal.cuh"

namespace fslk {

constexpr int LIST_THREADS = 128;

// ---- fill level at obstacle cells (Sec. II.A reflection, aperture sqrt(2)/2) --
// n_w is the (integer) sum of the lattice vectors to the non-obstacle
// neighbours; the aperture test 2 (N.c)^2 > |N|^2 |c|^2 is exact.
template <typename F>
__device__ float reflect(const Dev &d, int x, int y, int z, F value) {
    int nx = 0, ny = 0, nz = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & T_OBS) continue;
        nx += cx(q);
        ny += cy(q);
        nz += cz(q);
    }
    const int n2 = nx * nx + ny * ny + nz * nz;
    if (n2 == 0) return 0.f;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int dx = cx(q), dy = cy(q), dz = cz(q);
        if (d.flags[nbr_index(d, x, y, z, dx, dy, dz)] & T_OBS) continue;
        const int dot = nx * dx + ny * dy + nz * dz;
        const int c2 = dx * dx + dy * dy + dz * dz;
        if (2 * dot * dot > n2 * c2) {
            const float w = fabsf((float)dot) * rsqrtf((float)(n2 * c2));
            num += w * value(x + dx, y + dy, z + dz);
            den += w;
        }
    }
    return den > 0.f ? num / den : 0.f;
}

__device__ __forceinline__ float phi_ext(const Dev &d, int x, int y, int z) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    const int i = cell_index(d, x, y, z);
    if (!(d.flags[i] & T_OBS)) return d.phi[i];
    return reflect(d, x, y, z, [&](int a, int b, int c) { return d.phi[nbr_index(d, a, b, c, 0, 0, 0)]; });
}

// Parker-Youngs gradient: central difference with transverse weights 4/2/1.
template <typename G>
__device__ __forceinline__ void parker_youngs(int x, int y, int z, G g, float n[3]) {
    n[0] = n[1] = n[2] = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const float v = g(x + dx, y + dy, z + dz);
                if (dx) n[0] += dx * (dy == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dy) n[1] += dy * (dx == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dz) n[2] += dz * (dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1) * v;
            }
}

// ---- PLIC ------------------------------------------------------------------
// Volume of {z in [0,1]^3 : m.z <= al} for m >= 0 sorted m1 <= m2 <= m3 with
// m1 + m2 + m3 = 1, al in [0, 1/2].  Inclusion-exclusion of the corner
// simplex, with the divided differences in m1 taken analytically so that no
// branch divides by a component that can vanish there.
__device__ __forceinline__ float plic_vol_half(float m1, float m2, float m3, float al) {
    if (al < m1) return al * al * al / (6.0f * m1 * m2 * m3);
    const float base = 3.0f * al * al - 3.0f * al * m1 + m1 * m1;  // ((al)^3 - (al-m1)^3)/m1
    if (al < m2) return base / (6.0f * m2 * m3);
    if (al >= m1 + m2) return (2.0f * al - m1 - m2) / (2.0f * m3);
    const float e2 = al - m2;
    if (al < m3) return (base - e2 * e2 * (e2 / m1)) / (6.0f * m2 * m3);
    const float e3 = al - m3;
    return (base - e2 * e2 * (e2 / m1) - e3 * e3 * (e3 / m1)) / (6.0f * m2 * m3);
}

__device__ __forceinline__ float plic_vol(float m1, float m2, float m3, float al) {
    return al <= 0.5f ? plic_vol_half(m1, m2, m3, al) : 1.0f - plic_vol_half(m1, m2, m3, 1.0f - al);
}

// dV/dal of plic_vol_half, branch by branch
__device__ __forceinline__ float plic_dvol_half(float m1, float m2, float m3, float al) {
    if (al < m1) return al * al / (2.0f * m1 * m2 * m3);
    if (al < m2) return (2.0f * al - m1) / (2.0f * m2 * m3);
    if (al >= m1 + m2) return 1.0f / m3;
    const float e2 = al - m2;
    float t = 6.0f * al - 3.0f * m1 - 3.0f * e2 * (e2 / m1);
    if (al >= m3) {
        const float e3 = al - m3;
        t -= 3.0f * e3 * (e3 / m1);
    }
    return t / (6.0f * m2 * m3);
}

// Inverse of plic_vol: al with V(al) = phi.  By symmetry only V <= 1/2 is
// solved.  The branch is found from V at the break points m1, m2 and
// min(m3, m1 + m2); the corner tetrahedron (cube root), the two-plane wedge
// (quadratic) and the four-edge slab (linear) are solved in closed form, the
// remaining cubic by Newton from the secant between its break points.
__device__ float plic_alpha(float m1, float m2, float m3, float phi, int iters) {
    const bool mirror = phi > 0.5f;
    const float v = mirror ? 1.0f - phi : phi;
    const float V1 = m1 > 0.f ? m1 * m1 / (6.0f * m2 * m3) : 0.f;
    const float V2 = m2 > 0.f ? (3.0f * m2 * m2 - 3.0f * m2 * m1 + m1 * m1) / (6.0f * m2 * m3) : 0.f;
    const float a3 = fminf(m3, m1 + m2);
    const float V3 = plic_vol_half(m1, m2, m3, a3);
    float al;
    if (v < V1) {
        al = cbrtf(6.0f * m1 * m2 * m3 * v);
    } else if (v < V2) {
        al = 0.5f * m1 + sqrtf(fmaxf(72.0f * m2 * m3 * v - 3.0f * m1 * m1, 0.f)) * (1.0f / 6.0f);
    } else if (v >= V3 && m3 >= m1 + m2) {
        al = m3 * v + 0.5f * (m1 + m2);
    } else {
        float lo, hi, vlo, vhi;
        if (v < V3) { lo = m2; hi = a3; vlo = V2; vhi = V3; }
        else { lo = a3; hi = 0.5f; vlo = V3; vhi = 0.5f; }
        al = vhi > vlo ? lo + (hi - lo) * (v - vlo) / (vhi - vlo) : lo;
        for (int it = 0; it < iters; ++it) {
            const float g = plic_vol_half(m1, m2, m3, al) - v;
            al = fminf(fmaxf(al - g / plic_dvol_half(m1, m2, m3, al), lo), hi);
        }
    }
    return mirror ? 1.0f - al : al;
}

// Offset a of the plane {y.n = a} through the cell [-1/2,1/2]^3 whose liquid
// side {y.n >= a} holds volume phi.  With m = |n| / sum|n| and
// al = 1/2 - a / sum|n| the liquid part is {z : m.z <= al} of the unit cube.
__device__ float plic_offset(float nx, float ny, float nz, float phi, int iters) {
    float a1 = fabsf(nx), a2 = fabsf(ny), a3 = fabsf(nz);
    const float M = a1 + a2 + a3;
    if (phi <= 0.f) return 0.5f * M;
    if (phi >= 1.f) return -0.5f * M;
    float t;
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    const float m1 = a1 / M, m2 = a2 / M, m3 = 1.0f - m1 - m2;
    return M * (0.5f - plic_alpha(m1, m2, m3, phi, iters));
}

// The first kernel of a step also zeroes that step's counters (conversion
// lists, general-path LSQR list, FP64 re-solves, next interface list); every
// later kernel of the step is ordered after it on the stream.
__global__ void __launch_bounds__(LIST_THREADS) k_normals(Dev d) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    if (blockIdx.x == 0 && threadIdx.x == 8) d.counts[d.cif_next] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const int zero[8] = {C_FILL, C_EMPTY, C_NEWGAS, C_LIQ2IF, C_SLOW, C_FP64, C_MLP, C_MLPKEEP};
        d.counts[zero[threadIdx.x]] = 0;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.iflist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        float nv[3];
        if (d.flags[i] & B_NEAR) parker_youngs(x, y, z, [&](int a, int b, int c) { return phi_ext(d, a, b, c); }, nv);
        else parker_youngs(x, y, z, [&](int a, int b, int c) { return d.phi[nbr_index(d, a, b, c, 0, 0, 0)]; }, nv);
        const float l2 = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
        if (!(l2 >= 1e-24f)) {
            d.normal[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float inv = rsqrtf(l2);
        const float n0 = nv[0] * inv, n1 = nv[1] * inv, n2 = nv[2] * inv;
        d.normal[i] = make_float4(n0, n1, n2, plic_offset(n0, n1, n2, d.phi[i], d.plic_iters));
    }
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
template <typename T>
__device__ bool contact(const Dev &d, int xj, int yj, int zj, const T o[3], const T nj[3], T aj, T pc[3], T mh[3]) {
    T w[3] = {T(0), T(0), T(0)};
    int cnt = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (d.flags[nbr_index(d, xj, yj, zj, cx(q), cy(q), cz(q))] & T_OBS) {
            w[0] += cx(q);
            w[1] += cy(q);
            w[2] += cz(q);
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
    const T ct = T(d.cos_theta_d), sn = T(d.sin_theta_d);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pc[k] = o[k] + rel[k] + s * dv[k];
        mh[k] = w[k] * ct + (nt[k] / ntl) * sn;
    }
    return true;
}

// LSQR curvature of interface cell i (Sec. II.C).  The model is
// f(u,v) = A u^2 + B v^2 + C uv + H u + I v (J = 0).  A centre constraint
// grad f(u_c, v_c) = g is eliminated exactly (H = g_u - 2 u_c A - v_c C,
// I = g_v - 2 v_c B - u_c C).  Fallbacks: isotropic model B = A, C = 0, then
// kappa = 0.  kappa by Eq. (anacurv) with the mixed term -C H I.
template <typename T>
__device__ float lsqr_cell(const Dev &d, int i, int x, int y, int z, float &cond_out) {
    const float4 c4 = d.normal[i];
    cond_out = 1.f;
    if (c4.x == 0.f && c4.y == 0.f && c4.z == 0.f) return 0.f;
    const T n[3] = {T(c4.x), T(c4.y), T(c4.z)};
    const T a = T(c4.w);
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
    const uint8_t fi = d.flags[i];

    bool cons = false;
    T uc = T(0), vc = T(0), gu = T(0), gv = T(0);
    if (fi & B_NEAR) {
        const T o[3] = {T(0), T(0), T(0)};
        T pc[3], mh[3];
        if (contact<T>(d, x, y, z, o, n, a, pc, mh)) {
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
    const int xs[3] = {x == 0 ? d.nx - 1 : x - 1, x, x == d.nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? d.ny - 1 : y - 1, y, y == d.ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? d.nz - 1 : z - 1, z, z == d.nz - 1 ? 0 : z + 1};
    for (int dz = -1; dz <= 1; ++dz) {
        // one z-plane of the neighbourhood: all nine flags and normals are
        // loaded before any of them is used (independent loads in flight)
        int jj[9];
        uint8_t fjs[9];
        float4 q4s[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) jj[t] = cell_index(d, xs[t % 3], ys[t / 3], zs[dz + 1]);
#pragma unroll
        for (int t = 0; t < 9; ++t) fjs[t] = d.flags[jj[t]];
#pragma unroll
        for (int t = 0; t < 9; ++t) q4s[t] = d.normal[jj[t]];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int dx = t % 3 - 1, dy = t / 3 - 1;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const uint8_t fj = fjs[t];
            if (!(fj & T_IF)) continue;
            const float4 q4 = q4s[t];
            if (q4.x == 0.f && q4.y == 0.f && q4.z == 0.f) continue;
            const T nj[3] = {T(q4.x), T(q4.y), T(q4.z)};
            const T aj = T(q4.w);
            const T o[3] = {T(dx), T(dy), T(dz)};
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
                if (!contact<T>(d, xs[dx + 1], ys[dy + 1], zs[dz + 1], o, nj, aj, pc, mh)) continue;
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
    cond_out = (float)cond;
    if (!done) return 0.f;
    const T g = T(1) + H * H + I * I;
    return (float)((A * (T(1) + I * I) + B * (T(1) + H * H) - C * H * I) / (g * sqrt(g)));
}

// Fast path: FP32 normal equations of the full model for an interface cell
// with no contact-line cell in its neighbourhood.  The 5x5 Gram matrix
// A^T A and A^T f are accumulated row by row (independent FMAs), then solved
// by Cholesky in registers.  Returns false (cell left to the general path)
// when a contact-line cell is present, when there are fewer than five rows,
// or when the Cholesky pivots estimate cond(A^T A) above d.fp64_cond.
__device__ bool lsqr_fast(const Dev &d, int i, int x, int y, int z, float &kap) {
    const float4 c4 = d.normal[i];
    kap = 0.f;
    if (c4.x == 0.f && c4.y == 0.f && c4.z == 0.f) return true;
    const float n[3] = {c4.x, c4.y, c4.z};
    int k = 0;
    if (fabsf(n[1]) < fabsf(n[0])) k = 1;
    if (fabsf(n[2]) < fabsf(n[k])) k = 2;
    float tu[3];
    if (k == 0) { tu[0] = 0.f; tu[1] = -n[2]; tu[2] = n[1]; }
    else if (k == 1) { tu[0] = n[2]; tu[1] = 0.f; tu[2] = -n[0]; }
    else { tu[0] = -n[1]; tu[1] = n[0]; tu[2] = 0.f; }
    const float tl = rsqrtf(dot3(tu, tu));
    tu[0] *= tl;
    tu[1] *= tl;
    tu[2] *= tl;
    const float tv[3] = {n[1] * tu[2] - n[2] * tu[1], n[2] * tu[0] - n[0] * tu[2], n[0] * tu[1] - n[1] * tu[0]};
    const float p[3] = {c4.w * n[0], c4.w * n[1], c4.w * n[2]};
    float G[15], r[5];
#pragma unroll
    for (int t = 0; t < 15; ++t) G[t] = 0.f;
#pragma unroll
    for (int t = 0; t < 5; ++t) r[t] = 0.f;
    int m = 0;
    bool contact = (d.flags[i] & B_NEAR) != 0;
    const int xs[3] = {x == 0 ? d.nx - 1 : x - 1, x, x == d.nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? d.ny - 1 : y - 1, y, y == d.ny - 1 ? 0 : y + 1};
#pragma unroll 1
    for (int pz = 0; pz < 3; ++pz) {
        const int zz = z + pz - 1 < 0 ? d.nz - 1 : (z + pz - 1 >= d.nz ? 0 : z + pz - 1);
        int jj[9];
        uint8_t fjs[9];
        float4 q4s[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) jj[t] = cell_index(d, xs[t % 3], ys[t / 3], zz);
#pragma unroll
        for (int t = 0; t < 9; ++t) fjs[t] = d.flags[jj[t]];
#pragma unroll
        for (int t = 0; t < 9; ++t) q4s[t] = d.normal[jj[t]];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float4 q4 = q4s[t];
            const bool use = (fjs[t] & T_IF) && !(pz == 1 && t == 4) && !(q4.x == 0.f && q4.y == 0.f && q4.z == 0.f);
            contact |= (fjs[t] & T_IF) && (fjs[t] & B_NEAR);
            const float w = use ? 1.f : 0.f;
            const float dv[3] = {(float)(t % 3 - 1) + q4.w * q4.x - p[0], (float)(t / 3 - 1) + q4.w * q4.y - p[1],
                                 (float)(pz - 1) + q4.w * q4.z - p[2]};
            const float u = dot3(dv, tu), v = dot3(dv, tv), f = w * dot3(dv, n);
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
    }
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
    const bool ok = !contact && m >= 5 && pd && !(cond > d.fp64_cond);
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

__global__ void __launch_bounds__(LIST_THREADS) k_lsqr_fast(Dev d, float *kappa_out) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    warp_uniform_loop(n, [&](int k, bool valid) {
        bool defer = false;
        int i = 0;
        if (valid) {
            i = d.iflist[k];
            int x, y, z;
            cell_coords(d, i, x, y, z);
            float kap;
            if (lsqr_fast(d, i, x, y, z, kap)) kappa_out[i] = kap;
            else defer = true;
        }
        warp_append(d.slow, d.counts + C_SLOW, defer, i);
    });
}

// General path: contact rows and centre constraint, isotropic fallback, FP64
// re-solve when the FP32 R is ill conditioned
__global__ void __launch_bounds__(LIST_THREADS) k_lsqr_slow(Dev d, float *kappa_out) {
    int cnt[1];
    block_counts<1>(d.counts, {C_SLOW}, cnt);
    const int n = cnt[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.slow[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        float cond;
        float kap = lsqr_cell<float>(d, i, x, y, z, cond);
        if (cond * cond > d.fp64_cond) {
            kap = lsqr_cell<double>(d, i, x, y, z, cond);
            atomicAdd(d.counts + C_FP64, 1);
        }
        kappa_out[i] = kap;
    }
}

// ---- FD ----------------------------------------------------------------------
__device__ __forceinline__ float k8w(int dx, int dy, int dz) {
    const int r2 = dx * dx + dy * dy + dz * dz;
    return r2 == 0 ? 1.0f : (r2 == 1 ? 0.31640625f : (r2 == 2 ? 0.0625f : 0.00390625f));
}

// K8-smoothed fill level (eps = 2 on the 3x3x3 stencil, normalised by the
// discrete weight sum 3.6796875) at a non-obstacle cell
__device__ float smooth_at(const Dev &d, int x, int y, int z) {
    float s = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) s += k8w(dx, dy, dz) * phi_ext(d, x + dx, y + dy, z + dz);
    return s * (1.0f / 3.6796875f);
}

// smoothed field at any cell; obstacle cells reflect the smoothed field
__device__ float smooth_ext(const Dev &d, int x, int y, int z) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    if (!(d.flags[cell_index(d, x, y, z)] & T_OBS)) return smooth_at(d, x, y, z);
    return reflect(d, x, y, z, [&](int a, int b, int c) { return smooth_at(d, a, b, c); });
}

__device__ void unit_or_zero(float n[3]) {
    const float l2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    if (!(l2 >= 1e-24f)) {
        n[0] = n[1] = n[2] = 0.f;
        return;
    }
    const float inv = rsqrtf(l2);
    n[0] *= inv;
    n[1] *= inv;
    n[2] *= inv;
}

// unit normal of the smoothed field; at obstacle cells the wetting normal of
// Eq. (contactNormal) from the neighbour x_b most aligned with the outward wall normal
__device__ void fd_normal(const Dev &d, int x, int y, int z, float n[3]) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    if (!(d.flags[cell_index(d, x, y, z)] & T_OBS)) {
        parker_youngs(x, y, z, [&](int a, int b, int c) { return smooth_ext(d, a, b, c); }, n);
        unit_or_zero(n);
        return;
    }
    int nx = 0, ny = 0, nz = 0;
    for (int q = 1; q < Q; ++q) {
        if (d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & T_OBS) continue;
        nx += cx(q);
        ny += cy(q);
        nz += cz(q);
    }
    n[0] = n[1] = n[2] = 0.f;
    if (nx == 0 && ny == 0 && nz == 0) return;
    int best = -1;
    float bestv = -3.0e38f;
    for (int q = 1; q < Q; ++q) {
        if (d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & T_OBS) continue;
        const int c2 = cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q);
        const float v = (float)(nx * cx(q) + ny * cy(q) + nz * cz(q)) / sqrtf((float)c2);
        if (v > bestv) {
            bestv = v;
            best = q;
        }
    }
    float w[3] = {-(float)nx, -(float)ny, -(float)nz};
    unit_or_zero(w);
    float nb[3];
    const int xb = wrap(x + cx(best), d.nx), yb = wrap(y + cy(best), d.ny), zb = wrap(z + cz(best), d.nz);
    parker_youngs(xb, yb, zb, [&](int a, int b, int c) { return smooth_ext(d, a, b, c); }, nb);
    unit_or_zero(nb);
    const float wn = nb[0] * w[0] + nb[1] * w[1] + nb[2] * w[2];
    float nt[3] = {nb[0] - wn * w[0], nb[1] - wn * w[1], nb[2] - wn * w[2]};
    unit_or_zero(nt);
    for (int k = 0; k < 3; ++k) n[k] = w[k] * d.cos_theta + nt[k] * d.sin_theta;
}

__global__ void __launch_bounds__(LIST_THREADS) k_fd(Dev d, float *kappa_out) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.iflist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        float np[3], nm[3], div = 0.f;
        fd_normal(d, x + 1, y, z, np);
        fd_normal(d, x - 1, y, z, nm);
        div += np[0] - nm[0];
        fd_normal(d, x, y + 1, z, np);
        fd_normal(d, x, y - 1, z, nm);
        div += np[1] - nm[1];
        fd_normal(d, x, y, z + 1, np);
        fd_normal(d, x, y, z - 1, nm);
        div += np[2] - nm[2];
        kappa_out[i] = -0.25f * div;
    }
}

__global__ void k_zero_kappa(Dev d, float *kappa_out) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) kappa_out[d.iflist[k]] = 0.f;
}

void launch_normals(const Dev &d, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_normals, LIST_THREADS, 4);
    k_normals<<<g, LIST_THREADS, 0, s>>>(d);
}
void launch_lsqr(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int gf = list_blocks((const void *)k_lsqr_fast, LIST_THREADS, 4);
    static const int gs = list_blocks((const void *)k_lsqr_slow, LIST_THREADS, 1);
    k_lsqr_fast<<<gf, LIST_THREADS, 0, s>>>(d, kappa_out);
    k_lsqr_slow<<<gs, LIST_THREADS, 0, s>>>(d, kappa_out);
}
void launch_fd(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_fd, LIST_THREADS, 4);
    k_fd<<<g, LIST_THREADS, 0, s>>>(d, kappa_out);
}
void launch_zero_kappa(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_zero_kappa, LIST_THREADS, 4);
    k_zero_kappa<<<g, LIST_THREADS, 0, s>>>(d, kappa_out);
}

}  // namespace fslk
