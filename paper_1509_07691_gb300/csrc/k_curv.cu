// k_curv.cu -- interface normals, PLIC points and curvature (Sec. II.A-C).
//   k_normals  Parker-Youngs normal of phi (obstacle cells by the aperture
//              reflection of Sec. II.A) and the PLIC offset a with
//              vol(cell cap {y.n >= a}) = phi (Sec. II.B), per interface cell.
//   k_lsqr     least-squares paraboloid through the PLIC points of the 3x3x3
//              neighbourhood with contact-point rows and centre constraints
//              (Sec. II.C): FP32 normal equations where that is safe, else
//              streaming Givens QR in registers, re-solved in FP64 when R is
//              ill conditioned.
//   k_fd_warp  finite-difference curvature -1/2 div(n) of the K8-smoothed fill
//              level with wetting normals at obstacle cells (Sec. II.A).
//   k_tr       triangle-fan curvature of the PLIC points (Sec. II.B).
// The per-cell arithmetic is in curv_common.cuh.
#include "curv_common.cuh"

namespace fslk {

constexpr int LIST_THREADS = 128;

// Parker-Youngs normal of a cell next to an obstacle (reflected fill levels at
// the obstacle cells); out of line, so that the loop of k_normals stays short
__device__ __noinline__ void normal_near_wall(const Dev &d, int x, int y, int z, float nv[3]) {
    parker_youngs<float>([&](int dx, int dy, int dz) { return phi_ext(d, x + dx, y + dy, z + dz); }, nv);
}

// The first kernel of a step also runs the step prologue (counters, bubble
// pressure); every later kernel of the step is ordered after it on the stream.
__global__ void __launch_bounds__(LIST_THREADS) k_normals(Dev d) {
    pdl_enter();
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) step_prologue(d);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.iflist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        // the 27 fill levels are loaded with the cell's type (one round); a cell
        // next to a wall takes the reflected ones instead, out of line
        float ph[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) ph[t] = d.phi[nbr_index(d, x, y, z, t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1)];
        const uint8_t fl = d.flags[i];
        float nv[3], a;
        if (fl & B_NEAR)
            normal_near_wall(d, x, y, z, nv);
        else
            parker_youngs<float>([&](int dx, int dy, int dz) { return ph[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; }, nv);
        const bool ok = unit_normal_offset<float>(nv, ph[13], d.plic_iters, a);
        d.normal[i] = ok ? make_float4(nv[0], nv[1], nv[2], a) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
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
    __shared__ uint8_t sfl[LIST_THREADS / 32][128];
    __shared__ float4 snm[LIST_THREADS / 32][27];
    int cnt[1];
    block_counts<1>(d.counts, {C_SLOW}, cnt);
    const int n = cnt[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < n; k += nw) {  // warp per cell: the block staged, one lane fits
        const int i = d.slow[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        stage_block(d, x, y, z, lane, sfl[w], snm[w]);
        __syncwarp();
        if (lane == 0) {
            const StagedAcc acc{d, sfl[w], snm[w]};
            const uint8_t fi = d.flags[i];
            float cond;
            float kap = lsqr_core<float>(acc, fi, cond);
            if (cond * cond > d.fp64_cond) {
                double c2;
                kap = (float)lsqr_core<double>(acc, fi, c2);
                atomicAdd(d.counts + C_FP64, 1);
            }
            kappa_out[i] = kap;
        }
        __syncwarp();
    }
}

// ---- TR (Sec. II.B) -------------------------------------------------------------
// Triangle-fan curvature of the PLIC points (Pohl's fan, Taubin's mean
// curvature).  One warp per interface cell; lane t (0..26) holds block cell
// t = (dz+1)*9 + (dy+1)*3 + (dx+1).  In the tangent frame of the centre
// point (the LSQR frame), lane t takes the PLIC point of its cell if that
// cell is interface with a nonzero normal (centre excluded) and its
// projection is not within 1e-6 of the centre: (u, v, h), the angle
// atan2(v, u) and the directional curvature 2h / |p|^2.  The fan orders the
// points by (angle, t); each lane finds its successor in that cyclic order by
// a scan over the warp, and if the angular gap is below pi the triangle
// (centre, own point, successor) adds its surface area times the two
// directional curvatures to the numerator and twice the area to the
// denominator: kappa = sum / sum, the mean of the directional curvatures
// weighted by the areas of the triangles at each edge.  No triangle: 0.
constexpr float TR_TWO_PI = 6.28318530717958647692f;
constexpr float TR_PI = 3.14159265358979323846f;

__global__ void __launch_bounds__(LIST_THREADS) k_tr(Dev d, float *kappa_out) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int t = lane < 27 ? lane : 13;
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    for (int k = gw; k < n; k += nw) {  // warp-uniform
        const int i = d.iflist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        const float4 c4 = d.normal[i];
        const bool none = c4.x == 0.f && c4.y == 0.f && c4.z == 0.f;  // warp-uniform
        const int j = nbr_index(d, x, y, z, dx, dy, dz);
        const uint8_t fj = d.flags[j];
        const float4 q4 = d.normal[j];
        FastFrame F;
        lsqr_fast_frame(none ? make_float4(0.f, 0.f, 1.f, 0.f) : c4, F);
        const float ex = dx + q4.w * q4.x - F.p[0], ey = dy + q4.w * q4.y - F.p[1], ez = dz + q4.w * q4.z - F.p[2];
        const float u = ex * F.tu[0] + ey * F.tu[1] + ez * F.tu[2];
        const float v = ex * F.tv[0] + ey * F.tv[1] + ez * F.tv[2];
        const float h = ex * F.n[0] + ey * F.n[1] + ez * F.n[2];
        const float r2 = u * u + v * v;
        const bool valid = !none && lane < 27 && t != 13 && (fj & T_IF) &&
                           !(q4.x == 0.f && q4.y == 0.f && q4.z == 0.f) && r2 >= 1e-12f;
        const float ang = atan2f(v, u);
        const float kap = 2.0f * h / (r2 + h * h);
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        // successor in the cyclic (angle, t) order: smallest gap, then smallest t
        float best = 3.0e38f;
        int succ = -1;
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const float as = __shfl_sync(0xffffffffu, ang, s);
            float g = as - ang;
            if (g < 0.f || (g == 0.f && s < lane)) g += TR_TWO_PI;
            if (valid && ((vmask >> s) & 1u) && s != lane && g < best) {
                best = g;
                succ = s;
            }
        }
        const int src = succ < 0 ? lane : succ;
        const float us = __shfl_sync(0xffffffffu, u, src), vs = __shfl_sync(0xffffffffu, v, src);
        const float hs = __shfl_sync(0xffffffffu, h, src), ks = __shfl_sync(0xffffffffu, kap, src);
        float num = 0.f, den = 0.f;
        if (valid && succ >= 0 && best < TR_PI) {
            const float cx_ = v * hs - h * vs, cy_ = h * us - u * hs, cz_ = u * vs - v * us;
            const float area = 0.5f * sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
            num = area * (kap + ks);
            den = 2.0f * area;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (lane == 0) kappa_out[i] = den > 0.f ? num / den : 0.f;
    }
}

// ---- FD ----------------------------------------------------------------------
__device__ __forceinline__ float k8w(int dx, int dy, int dz) {
    const int r2 = dx * dx + dy * dy + dz * dz;
    return r2 == 0 ? 1.0f : (r2 == 1 ? 0.31640625f : (r2 == 2 ? 0.0625f : 0.00390625f));
}

// K8-smoothed fill level (eps = 2 on the 3x3x3 stencil, normalised by the
// discrete weight sum 3.6796875) at a non-obstacle cell
__device__ __noinline__ float smooth_at(const Dev &d, int x, int y, int z) {
    float s = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) s += k8w(dx, dy, dz) * phi_ext(d, x + dx, y + dy, z + dz);
    return s * (1.0f / 3.6796875f);
}

// smoothed field at any cell; obstacle cells reflect the smoothed field
__device__ __noinline__ float smooth_ext(const Dev &d, int x, int y, int z) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    if (!(d.flags[cell_index(d, x, y, z)] & T_OBS)) return smooth_at(d, x, y, z);
    return reflect_value<float>([&](int a, int b, int c) { return d.flags[nbr_index(d, x, y, z, a, b, c)]; },
                                [&](int a, int b, int c) { return smooth_at(d, x + a, y + b, z + c); });
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
__device__ __noinline__ void fd_normal(const Dev &d, int x, int y, int z, float n[3]) {
    x = wrap(x, d.nx);
    y = wrap(y, d.ny);
    z = wrap(z, d.nz);
    if (!(d.flags[cell_index(d, x, y, z)] & T_OBS)) {
        parker_youngs<float>([&](int a, int b, int c) { return smooth_ext(d, x + a, y + b, z + c); }, n);
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
    parker_youngs<float>([&](int a, int b, int c) { return smooth_ext(d, xb + a, yb + b, zb + c); }, nb);
    unit_or_zero(nb);
    const float wn = nb[0] * w[0] + nb[1] * w[1] + nb[2] * w[2];
    float nt[3] = {nb[0] - wn * w[0], nb[1] - wn * w[1], nb[2] - wn * w[2]};
    unit_or_zero(nt);
    for (int k = 0; k < 3; ++k) n[k] = w[k] * d.cos_theta + nt[k] * d.sin_theta;
}

// FD curvature, one warp per interface cell: the fill levels of the 7^3
// block around the cell are staged in shared memory once, the lanes share the
// 5^3 K8-smoothed values, six lanes take the face neighbours' normals and
// lane 0 the central differences.  The sums run in the order of smooth_at,
// parker_youngs and fd_cell, so the values are those of the per-cell path; a
// cell with an obstacle in its 7^3 block (reflected fill levels and wetting
// normals) takes that path (fd_normal) on lane 0.
constexpr int FD_WARPS = 4;

// the per-cell path (walls in reach), out of line so that its registers do not
// weigh on the staged path; its helpers (smooth_at, smooth_ext, fd_normal) are
// out of line too, one copy each instead of an inlined tree of stencils
__device__ __noinline__ float fd_cell(const Dev &d, int x, int y, int z) {
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
    return -0.25f * div;
}

__global__ void __launch_bounds__(32 * FD_WARPS) k_fd_warp(Dev d, float *kappa_out) {
    __shared__ float s_phi[FD_WARPS][343];
    __shared__ float s_sm[FD_WARPS][125];
    __shared__ float s_n[FD_WARPS][6][3];
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    float *ph = s_phi[w], *sm = s_sm[w];
    for (int k = gw; k < n; k += nw) {  // warp-uniform
        const int i = d.iflist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        bool obs = false;
        for (int e = lane; e < 343; e += 32) {
            const int j = nbr_index(d, x, y, z, e % 7 - 3, (e / 7) % 7 - 3, e / 49 - 3);
            obs |= (d.flags[j] & T_OBS) != 0;
            ph[e] = d.phi[j];
        }
        if (__any_sync(0xffffffffu, obs)) {  // walls in reach: the per-cell path
            if (lane == 0) kappa_out[i] = fd_cell(d, x, y, z);
            __syncwarp();
            continue;
        }
        __syncwarp();
        // smoothed fill level of the 5^3 block (offsets -2..2), as smooth_at
        for (int e = lane; e < 125; e += 32) {
            const int ex = e % 5 + 1, ey = (e / 5) % 5 + 1, ez = e / 25 + 1;  // in the 7^3 block
            float acc = 0.f;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        acc += k8w(dx, dy, dz) * ph[(ez + dz) * 49 + (ey + dy) * 7 + ex + dx];
            sm[e] = acc * (1.0f / 3.6796875f);
        }
        __syncwarp();
        // normals at the face neighbours x+e_x, x-e_x, x+e_y, x-e_y, x+e_z, x-e_z
        if (lane < 6) {
            const int ax = lane >> 1, sg = (lane & 1) ? -1 : 1;
            const int cxn = 2 + (ax == 0 ? sg : 0), cyn = 2 + (ax == 1 ? sg : 0), czn = 2 + (ax == 2 ? sg : 0);
            float nv[3];
            parker_youngs<float>(
                [&](int dx, int dy, int dz) { return sm[(czn + dz) * 25 + (cyn + dy) * 5 + cxn + dx]; }, nv);
            unit_or_zero(nv);
            s_n[w][lane][0] = nv[0];
            s_n[w][lane][1] = nv[1];
            s_n[w][lane][2] = nv[2];
        }
        __syncwarp();
        if (lane == 0) {
            float div = 0.f;
            div += s_n[w][0][0] - s_n[w][1][0];
            div += s_n[w][2][1] - s_n[w][3][1];
            div += s_n[w][4][2] - s_n[w][5][2];
            kappa_out[i] = -0.25f * div;
        }
        __syncwarp();
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
    static const int gs = list_blocks((const void *)k_lsqr_slow, LIST_THREADS, 4);
    k_lsqr_fast<<<gf, LIST_THREADS, 0, s>>>(d, kappa_out);
    k_lsqr_slow<<<gs, LIST_THREADS, 0, s>>>(d, kappa_out);
}
void launch_fd(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_fd_warp, 32 * FD_WARPS, 16);
    k_fd_warp<<<g, 32 * FD_WARPS, 0, s>>>(d, kappa_out);
}
void launch_tr(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_tr, LIST_THREADS, 8);
    k_tr<<<g, LIST_THREADS, 0, s>>>(d, kappa_out);
}
void launch_zero_kappa(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_zero_kappa, LIST_THREADS, 4);
    k_zero_kappa<<<g, LIST_THREADS, 0, s>>>(d, kappa_out);
}

}  // namespace fslk
