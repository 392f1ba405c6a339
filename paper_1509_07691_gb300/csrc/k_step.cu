// k_step.cu -- the FSLBM time step (Sec. II): fused pull stream-collide with the
// free-boundary condition and mass exchange, conversion of interface cells
// with excess-mass redistribution, and the update of the cell types, of the
// interface list and of the active segments for the next step.
//
// Work decomposition: liquid cells are processed by k_sc_bulk over the active
// x-row segments (coalesced SoA loads, one thread per cell); interface cells
// by k_curv_iface_fast (LSQR model, fit and stream-collide fused) or
// k_sc_iface (other models) over the interface list; everything after the
// collision only touches list entries, so no pass sweeps the whole grid.
#include "collide.cuh"
#include "curv_common.cuh"

namespace fslk {

constexpr int LIST_BLOCK = 128;

// index of the source cell x - c_q of every direction
__device__ __forceinline__ void sources(const Dev &d, int x, int y, int z, int src[Q]) {
    const int xs[3] = {x == d.nx - 1 ? 0 : x + 1, x, x == 0 ? d.nx - 1 : x - 1};  // x - c for c = -1, 0, 1
    const int ys[3] = {y == d.ny - 1 ? 0 : y + 1, y, y == 0 ? d.ny - 1 : y - 1};
    const int zs[3] = {z == d.nz - 1 ? 0 : z + 1, z, z == 0 ? d.nz - 1 : z - 1};
#pragma unroll
    for (int q = 0; q < Q; ++q) src[q] = cell_index(d, xs[cx(q) + 1], ys[cy(q) + 1], zs[cz(q) + 1]);
}

// Liquid cells of the active segments: pull stream (Eq. lbe1) and collide.
// One warp per 32-cell x-row segment, one thread per cell (coalesced SoA
// loads and stores).  A liquid cell next to a wall takes bounce-back
// f_q(x) = f'_qbar(x) on its obstacle links.  Interface cells are left to
// k_sc_iface.  A segment without any liquid or interface cell is marked
// inactive.
template <int S, int COLL>
__global__ void __launch_bounds__(256) k_sc_bulk(Dev d) {
    using St = Store<S>;
    int cnt[1];
    block_counts<1>(d.counts, {C_SEG}, cnt);
    const int nseg = cnt[0];
    const long long N = d.N;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < nseg; k += nw) {
        const int s = d.seg_list[k];
        const int row = s / d.nsegx;
        const int x = (s - row * d.nsegx) * SEG + lane;
        const int z = row / d.ny, y = row - z * d.ny;
        const bool inb = x < d.nx;
        const int i = inb ? cell_index(d, x, y, z) : 0;
        const uint8_t fl = inb ? d.flags[i] : (uint8_t)T_GAS;
        if (fl & T_LIQ) {
            int src[Q];
            sources(d, x, y, z, src);
            float f[Q];
            if (!(fl & B_NEAR)) {
#pragma unroll
                for (int q = 0; q < Q; ++q) f[q] = St::ld(d.fsrc, (long long)q * N + src[q], q, d);
            } else {
                f[0] = St::ld(d.fsrc, i, 0, d);
#pragma unroll
                for (int q = 1; q < Q; ++q) {
                    const bool wall = (d.flags[src[q]] & T_OBS) != 0;
                    f[q] = wall ? St::ld(d.fsrc, (long long)opp(q) * N + i, opp(q), d)
                                : St::ld(d.fsrc, (long long)q * N + src[q], q, d);
                }
            }
            float rho;
            collide<COLL>(f, d, rho);
#pragma unroll
            for (int q = 0; q < Q; ++q) St::st(d.fdst, (long long)q * N + i, q, f[q], d);
        }
        if (!__any_sync(0xffffffffu, (fl & (T_LIQ | T_IF)) != 0) && lane == 0) {
            d.seg_active[s] = 0;
            d.counts[d.cdirty] = 1;
        }
    }
}

// Interface cells (list), one thread per cell.  Each link is resolved by
// the type of its source cell x - c_q:
//   fluid     f_q(x) = f'_q(x - c_q)                        (Eq. lbe1)
//   gas       f_q(x) = feq_q + feq_qbar - f'_qbar(x)         (Eq. reconstruct)
//             with rho_b = 3 p_g + 6 sigma kappa(x), u_b = u(x, t)
//   obstacle  f_q(x) = f'_qbar(x) (bounce-back), or Eq. reconstruct at a
//             contact-line cell when c_qbar . n_t < 0, n_t the interface normal
//             projected into the wall (Fig. inhomo)
// plus the mass exchange of Eqs. (advection1/2) and the conversion test
// (skipped when the types are frozen).  iface_cell reads kappa(x) and, at
// contact-line cells, the PLIC normal of x -- both the cell's own -- so it may
// run right after the curvature of the same cell, in the same kernel.
template <int S, int COLL>
__device__ __forceinline__ void iface_cell(const Dev &d, int i) {
    using St = Store<S>;
    const long long N = d.N;
    int x, y, z;
    cell_coords(d, i, x, y, z);
    int src[Q];
    sources(d, x, y, z, src);
    const uint8_t fl = d.flags[i];
    float fo[Q], f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) fo[q] = St::ld(d.fsrc, (long long)q * N + i, q, d);
    uint8_t tq[Q];
    bool has_gas = false, has_obs = false;
    float wx = 0.f, wy = 0.f, wz = 0.f;  // sum of vectors x -> obstacle neighbour
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        tq[q] = d.flags[src[q]] & T_MASK;
        has_gas |= (tq[q] & T_GAS) != 0;
        if (tq[q] & T_OBS) {
            has_obs = true;
            wx -= cx(q);
            wy -= cy(q);
            wz -= cz(q);
        }
    }
    // the PDF and fill level of every source cell, loaded unconditionally
    // (in bounds for every cell type; used only on fluid links) so that
    // all of a cell's loads are in flight together
    float fin[Q], phn[Q];
    fin[0] = phn[0] = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        fin[q] = St::ld(d.fsrc, (long long)q * N + src[q], q, d);
        phn[q] = d.phi[src[q]];
    }
    // u_b: velocity of x at time t from its own post-collision PDFs
    float r0 = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        r0 += fo[q];
        jx += cx(q) * fo[q];
        jy += cy(q) * fo[q];
        jz += cz(q) * fo[q];
    }
    const float ux = jx / r0, uy = jy / r0, uz = jz / r0;
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float rho_b = gas_density(d) + d.six_sigma * d.kappa[i];
    const bool corner = has_gas && has_obs;
    float ntx = 0.f, nty = 0.f, ntz = 0.f;
    if (corner) {
        const float4 n4 = d.normal[i];
        const float wl = rsqrtf(wx * wx + wy * wy + wz * wz);
        wx *= wl;
        wy *= wl;
        wz *= wl;
        const float wn = n4.x * wx + n4.y * wy + n4.z * wz;
        ntx = n4.x - wn * wx;
        nty = n4.y - wn * wy;
        ntz = n4.z - wn * wz;
    }
    const float phix = d.phi[i];
    float dm = 0.f;
    f[0] = fo[0];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int qb = opp(q);
        const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
        // feq_q + feq_qbar at (rho_b, u_b): the odd terms cancel
        const float recon = 2.0f * wq(q) * rho_b * (1.0f + 4.5f * cu * cu - uu) - fo[qb];
        const bool fluid = (tq[q] & (T_LIQ | T_IF)) != 0;
        const float kq = (tq[q] & T_LIQ) ? 1.0f : 0.5f * (phix + phn[q]);
        const float outdir = -(cx(q) * ntx + cy(q) * nty + cz(q) * ntz);  // c_qbar . n_t
        const float bound = ((tq[q] & T_OBS) && !(corner && outdir < 0.f)) ? fo[qb] : recon;
        f[q] = fluid ? fin[q] : bound;
        dm += fluid ? kq * (fin[q] - fo[qb]) : 0.f;
    }
    float rho;
    collide<COLL>(f, d, rho);
#pragma unroll
    for (int q = 0; q < Q; ++q) St::st(d.fdst, (long long)q * N + i, q, f[q], d);
    const float m = d.mass[i] + dm;
    d.mass[i] = m;
    d.rho[i] = rho;
    if (d.frozen) return;
    if (m > (1.0f + d.eps) * rho) {
        d.flags[i] = fl | B_TOLIQ;
        d.fill[atomicAdd(d.counts + C_FILL, 1)] = i;
    } else if (m < -d.eps * rho) {
        d.flags[i] = fl | B_TOGAS;
        d.empty[atomicAdd(d.counts + C_EMPTY, 1)] = i;
    }
}

template <int S, int COLL>
__global__ void __launch_bounds__(LIST_BLOCK) k_sc_iface(Dev d) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        iface_cell<S, COLL>(d, d.iflist[k]);
}

// ---- LSQR curvature fused with the interface stream-collide ----------------------
// With the LSQR model the curvature of a cell and its stream-collide run in
// one pass: k_curv_iface_fast fits the cell by the FP32 normal equations
// (as k_lsqr_fast) and, unless the fit defers the cell to the general path,
// goes straight on with the cell's stream-collide, FSL_IFACE_LANES lanes per
// cell; k_curv_iface_slow finishes the deferred cells one thread each (Givens
// fit, FP64 re-solve when ill conditioned, then iface_cell).  In a domain
// without obstacles (no contact lines: a deferral is a rare ill-conditioned
// or degenerate fit) the fused kernel's last block finishes the deferred
// cells and k_curv_iface_slow is not launched.
// iface_cell of one cell changes only that cell's transient flag bits, mass,
// rho and new PDFs, none of which a fit of another cell reads.
// Lattice directions by pair: pair p (0..8) holds q = 2p + 1 with velocity
// c_p and q + 1 with -c_p.  Components packed two bits per pair (1 -> +1,
// 3 -> -1) so that a lane can decode its own pairs without a table.
constexpr unsigned PAIR_CX = 0x1541u;   // p: 0:+1 1:0 2:0 3:+1 4:+1 5:+1 6:+1 7:0 8:0
constexpr unsigned PAIR_CY = 0x14344u;  // p: 0:0 1:+1 2:0 3:+1 4:-1 5:0 6:0 7:+1 8:+1
constexpr unsigned PAIR_CZ = 0x37410u;  // p: 0:0 1:0 2:+1 3:0 4:0 5:+1 6:-1 7:+1 8:-1
__device__ __forceinline__ int pair_c(unsigned packed, int p) {
    const int v = (packed >> (2 * p)) & 3;
    return v == 3 ? -1 : v;
}

// A cell the fast fit deferred: the streaming Givens fit through accessor acc
// (re-solved in FP64 when ill conditioned), then the cell's interface
// stream-collide.
template <int S, int COLL, class Acc>
__device__ __forceinline__ void general_cell(const Dev &d, const Acc &acc, int i) {
    const uint8_t fi = d.flags[i] & (T_MASK | B_NEAR);
    float cond;
    float kap = lsqr_core<float>(acc, fi, cond);
    if (cond * cond > d.fp64_cond) {
        double c2;
        kap = (float)lsqr_core<double>(acc, fi, c2);
        atomicAdd(d.counts + C_FP64, 1);
    }
    d.kappa[i] = kap;
    iface_cell<S, COLL>(d, i);
}

// the same, by one thread reading the block from global memory: the fused
// kernel's own deferred cells in a domain without obstacles (no contact
// lines, so deferrals are rare ill-conditioned fits); out of line, so that the
// fused kernel's registers are not spent on it
template <int S, int COLL>
__device__ __noinline__ void general_cell_grid(const Dev d, int i) {
    int x, y, z;
    cell_coords(d, i, x, y, z);
    const GridAcc acc{d, x, y, z};
    general_cell<S, COLL>(d, acc, i);
}

// L lanes per interface cell (a group), rank r = lane % L.  The fit's 27
// block cells are split t = r, r + L, ...; the 9 direction pairs p = r,
// r + L, ...; the rest population goes to rank L - 1.  Partial sums are
// combined over the group by xor-shuffles in a fixed order.
template <int L>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int L>
__device__ __forceinline__ int group_or(int v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// lanes per cell of the fused fit + stream-collide, and the blocks per SM its
// register budget is held to (one wave of the list on a 256^3 droplet)
#ifndef FSL_IFACE_LANES
#define FSL_IFACE_LANES 2
#endif
constexpr int IFACE_MIN_BLOCKS = FSL_IFACE_LANES == 4 ? 3 : 3;

template <int S, int COLL, int L>
__global__ void __launch_bounds__(LIST_BLOCK, IFACE_MIN_BLOCKS) k_curv_iface_fast(Dev d) {
    pdl_enter();
    using St = Store<S>;
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    const long long N = d.N;
    constexpr int CPW = 32 / L;                 // cells per warp
    constexpr int RS = (27 + L - 1) / L;        // fit rows per lane
    constexpr int PJ = (9 + L - 1) / L;         // direction pairs per lane
    const int lane = threadIdx.x & 31, r = lane % L;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int base = gw * CPW; base < n; base += nwarps * CPW) {  // warp-uniform
        const int k = base + lane / L;
        const bool valid = k < n;
        const int i = d.iflist[valid ? k : base];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        // neighbour coordinates (periodic), picked by select: lane-dependent
        // indices into small arrays would put the arrays in local memory
        const int xm = x == 0 ? d.nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? d.nz - 1 : z - 1, zp = z == d.nz - 1 ? 0 : z + 1;
        auto px = [&](int o) { return o < 0 ? xm : (o > 0 ? xp : x); };
        auto py = [&](int o) { return o < 0 ? ym : (o > 0 ? yp : y); };
        auto pz = [&](int o) { return o < 0 ? zm : (o > 0 ? zp : z); };
        // ---- LSQR fit (FP32 normal equations), rows split over the group
        const float4 c4 = d.normal[i];
        uint8_t fjs[RS];
        float4 q4s[RS];
#pragma unroll
        for (int s7 = 0; s7 < RS; ++s7) {
            const int t = r + L * s7;
            const int tt = t < 27 ? t : 13;
            const int jj = cell_index(d, px(tt % 3 - 1), py((tt / 3) % 3 - 1), pz(tt / 9 - 1));
            fjs[s7] = d.flags[jj];
            q4s[s7] = d.normal[jj];
        }
        const uint8_t fl = d.flags[i];
        const float phix = d.phi[i];
        // ---- the stream-collide's loads (independent of kappa), issued with the fit's
        float fo[PJ][2], fin[PJ][2], phn[PJ][2];
        uint8_t tq[PJ][2];
        float fo0 = 0.f;
        float r0 = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, wx = 0.f, wy = 0.f, wz = 0.f;
        int gas = 0, obs = 0;
#pragma unroll
        for (int j = 0; j < PJ; ++j) {
            const int p = r + L * j;
            const int pp = p < 9 ? p : 0;
            const int ex = pair_c(PAIR_CX, pp), ey = pair_c(PAIR_CY, pp), ez = pair_c(PAIR_CZ, pp);
            const int q = 2 * pp + 1;
            const int sq = cell_index(d, px(-ex), py(-ey), pz(-ez));  // x - c_q
            const int sb = cell_index(d, px(ex), py(ey), pz(ez));     // x + c_q
            fo[j][0] = St::ld(d.fsrc, (long long)q * N + i, q, d);
            fo[j][1] = St::ld(d.fsrc, (long long)(q + 1) * N + i, q + 1, d);
            tq[j][0] = d.flags[sq] & T_MASK;
            tq[j][1] = d.flags[sb] & T_MASK;
            fin[j][0] = St::ld(d.fsrc, (long long)q * N + sq, q, d);
            fin[j][1] = St::ld(d.fsrc, (long long)(q + 1) * N + sb, q + 1, d);
            phn[j][0] = d.phi[sq];
            phn[j][1] = d.phi[sb];
        }
        if (r == L - 1) fo0 = St::ld(d.fsrc, i, 0, d);
        const bool nozero = !(c4.x == 0.f && c4.y == 0.f && c4.z == 0.f);
        FastFrame F;
        lsqr_fast_frame(nozero ? c4 : make_float4(0.f, 0.f, 1.f, 0.f), F);
        float G[15], rv[5];
#pragma unroll
        for (int t = 0; t < 15; ++t) G[t] = 0.f;
#pragma unroll
        for (int t = 0; t < 5; ++t) rv[t] = 0.f;
        int m = 0;
        bool contact = r == 0 && (fl & B_NEAR) != 0;
#pragma unroll
        for (int s7 = 0; s7 < RS; ++s7) {
            const int t = r + L * s7;
            if (t < 27) lsqr_fast_row(t, fjs[s7], q4s[s7], F, G, rv, m, contact);
        }
#pragma unroll
        for (int t = 0; t < 15; ++t) G[t] = group_sum<L>(G[t]);
#pragma unroll
        for (int t = 0; t < 5; ++t) rv[t] = group_sum<L>(rv[t]);
#pragma unroll
        for (int o = 1; o < L; o <<= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        contact = group_or<L>(contact ? 1 : 0) != 0;
        float kap = 0.f;
        const bool ok = nozero ? lsqr_fast_solve(G, rv, m, contact, d.fp64_cond, kap) : true;
        if (!nozero) kap = 0.f;
        const bool defer = valid && !ok;
        const bool act = valid && ok;  // group-uniform
        // ---- interface stream-collide of the cell, direction pairs over the group
#pragma unroll
        for (int j = 0; j < PJ; ++j) {
            const int p = r + L * j;
            if (p < 9) {
                const int ex = pair_c(PAIR_CX, p), ey = pair_c(PAIR_CY, p), ez = pair_c(PAIR_CZ, p);
                r0 += fo[j][0] + fo[j][1];
                const float dj = fo[j][0] - fo[j][1];
                jx += ex * dj;
                jy += ey * dj;
                jz += ez * dj;
                gas |= ((tq[j][0] | tq[j][1]) & T_GAS) ? 1 : 0;
                if (tq[j][0] & T_OBS) { obs = 1; wx -= ex; wy -= ey; wz -= ez; }
                if (tq[j][1] & T_OBS) { obs = 1; wx += ex; wy += ey; wz += ez; }
            }
        }
        if (r == L - 1) r0 += fo0;
        r0 = group_sum<L>(r0);
        jx = group_sum<L>(jx);
        jy = group_sum<L>(jy);
        jz = group_sum<L>(jz);
        wx = group_sum<L>(wx);
        wy = group_sum<L>(wy);
        wz = group_sum<L>(wz);
        gas = group_or<L>(gas);
        obs = group_or<L>(obs);
        const float ux = jx / r0, uy = jy / r0, uz = jz / r0;
        const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
        const float rho_b = gas_density(d) + d.six_sigma * kap;
        const bool corner = gas && obs;
        float ntx = 0.f, nty = 0.f, ntz = 0.f;
        if (corner) {
            const float wl = rsqrtf(wx * wx + wy * wy + wz * wz);
            const float vx = wx * wl, vy = wy * wl, vz = wz * wl;
            const float wn = c4.x * vx + c4.y * vy + c4.z * vz;
            ntx = c4.x - wn * vx;
            nty = c4.y - wn * vy;
            ntz = c4.z - wn * vz;
        }
        float g[PJ][2];
        float dm = 0.f, rg = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int j = 0; j < PJ; ++j) {
            const int p = r + L * j;
            const int pp = p < 9 ? p : 0;
            const int ex = pair_c(PAIR_CX, pp), ey = pair_c(PAIR_CY, pp), ez = pair_c(PAIR_CZ, pp);
            const float w = pp < 3 ? 1.0f / 18.0f : 1.0f / 36.0f;
            const float cu = ex * ux + ey * uy + ez * uz;
            const float base2 = 2.0f * w * rho_b * (1.0f + 4.5f * cu * cu - uu);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float sgn = h == 0 ? 1.0f : -1.0f;  // c = sgn c_p
                const float recon = base2 - fo[j][1 - h];
                const bool fluid = (tq[j][h] & (T_LIQ | T_IF)) != 0;
                const float kq = (tq[j][h] & T_LIQ) ? 1.0f : 0.5f * (phix + phn[j][h]);
                const float outdir = -sgn * (ex * ntx + ey * nty + ez * ntz);  // c_qbar . n_t
                const float bound = ((tq[j][h] & T_OBS) && !(corner && outdir < 0.f)) ? fo[j][1 - h] : recon;
                g[j][h] = fluid ? fin[j][h] : bound;
                dm += (fluid && p < 9) ? kq * (fin[j][h] - fo[j][1 - h]) : 0.f;
            }
            if (p < 9) {
                rg += g[j][0] + g[j][1];
                const float dg = g[j][0] - g[j][1];
                gx += ex * dg;
                gy += ey * dg;
                gz += ez * dg;
            }
        }
        if (r == L - 1) rg += fo0;
        rg = group_sum<L>(rg);
        gx = group_sum<L>(gx);
        gy = group_sum<L>(gy);
        gz = group_sum<L>(gz);
        dm = group_sum<L>(dm);
        // collision (Eq. lbe2) of the cell's own pairs
        const float inv = 1.0f / rg;
        const float vx = gx * inv, vy = gy * inv, vz = gz * inv;
        const float vv = 1.5f * (vx * vx + vy * vy + vz * vz);
#pragma unroll
        for (int j = 0; j < PJ; ++j) {
            const int p = r + L * j;
            const int pp = p < 9 ? p : 0;
            const int ex = pair_c(PAIR_CX, pp), ey = pair_c(PAIR_CY, pp), ez = pair_c(PAIR_CZ, pp);
            const float w = pp < 3 ? 1.0f / 18.0f : 1.0f / 36.0f;
            const int q = 2 * pp + 1;
            const float cu = ex * vx + ey * vy + ez * vz;
            float a0, a1;
            if (COLL == FSL_BGK) {
                const float fe0 = w * rg * (1.0f + 3.0f * cu + 4.5f * cu * cu - vv);
                const float fe1 = w * rg * (1.0f - 3.0f * cu + 4.5f * cu * cu - vv);
                a0 = g[j][0] + d.omega_e * (fe0 - g[j][0]);
                a1 = g[j][1] + d.omega_e * (fe1 - g[j][1]);
            } else {
                const float ep = w * rg * (1.0f + 4.5f * cu * cu - vv);
                const float em = w * rg * 3.0f * cu;
                const float fp = 0.5f * (g[j][0] + g[j][1]), fm = 0.5f * (g[j][0] - g[j][1]);
                const float de = d.omega_e * (fp - ep), dd = d.omega_o * (fm - em);
                a0 = g[j][0] - de - dd;
                a1 = g[j][1] - de + dd;
            }
            if (act && p < 9) {
                St::st(d.fdst, (long long)q * N + i, q, a0, d);
                St::st(d.fdst, (long long)(q + 1) * N + i, q + 1, a1, d);
            }
        }
        if (act && r == L - 1) St::st(d.fdst, i, 0, fo0 + d.omega_e * ((1.0f / 3.0f) * rg * (1.0f - vv) - fo0), d);
        warp_append(d.slow, d.counts + C_SLOW, defer && r == 0, i);
        if (act && r == 0) {
            d.kappa[i] = kap;
            const float mm = d.mass[i] + dm;
            d.mass[i] = mm;
            d.rho[i] = rg;
            if (!d.frozen) {
                if (mm > (1.0f + d.eps) * rg) {
                    d.flags[i] = fl | B_TOLIQ;
                    d.fill[atomicAdd(d.counts + C_FILL, 1)] = i;
                } else if (mm < -d.eps * rg) {
                    d.flags[i] = fl | B_TOGAS;
                    d.empty[atomicAdd(d.counts + C_EMPTY, 1)] = i;
                }
            }
        }
    }
    // without obstacles the last block to finish runs the deferred fits (rare
    // ill-conditioned or degenerate ones), one thread per cell: every block's
    // list appends are fenced before its arrival is counted
    if (d.inline_general) {  // uniform over the grid
        __shared__ int last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(d.counts + C_IFDONE, 1) == (int)gridDim.x - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            const int ns = __ldcg(d.counts + C_SLOW);
            for (int k = threadIdx.x; k < ns; k += blockDim.x) general_cell_grid<S, COLL>(d, __ldcg(d.slow + k));
            if (threadIdx.x == 0) d.counts[C_IFDONE] = 0;
        }
    }
}

// General-path cells (contact-line cells, degenerate or ill-conditioned FP32
// fits): one warp per cell stages the block in shared memory, then one lane
// runs the streaming Givens fit (FP64 when ill conditioned) and the
// interface stream-collide of the cell.
template <int S, int COLL>
__global__ void __launch_bounds__(LIST_BLOCK) k_curv_iface_slow(Dev d) {
    pdl_enter();
    __shared__ uint8_t sfl[LIST_BLOCK / 32][128];
    __shared__ float4 snm[LIST_BLOCK / 32][27];
    int cnt[1];
    block_counts<1>(d.counts, {C_SLOW}, cnt);
    const int n = cnt[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < n; k += nw) {
        const int i = d.slow[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        stage_block(d, x, y, z, lane, sfl[w], snm[w]);
        __syncwarp();
        if (lane == 0) general_cell<S, COLL>(d, StagedAcc{d, sfl[w], snm[w]}, i);
        __syncwarp();
    }
}

// ---- conversion (the paper cites Koerner et al. for it; readings) -------------
//  A  an emptying cell with a filling D3Q19 neighbour stays interface;
//  B  gas neighbours of filling cells and liquid neighbours of emptying cells
//     become interface (deduplicated by an atomic OR on the flag word);
//  C  new cells from gas get f = feq(mean rho, mean u) of their fluid
//     neighbours and m = 0; cells from liquid keep f and get m = rho;
//  D  the excess mass (m - rho of a filled cell, m of an emptied one) is
//     divided equally among the neighbours that are interface after B; the
//     receivers are marked (rmark) and gather it in k_fin_a.  No receiver:
//     added to `lost`.
// One block of 1024 threads with block barriers between the phases: a step
// converts few cells, and one block keeps every phase visible to the next.
// C and D touch disjoint cells (C the new interface cells, D the converted
// ones) and read nothing the other writes, so they share one phase.
constexpr int CONV_BLOCK = 1024;

template <int S>
__global__ void __launch_bounds__(CONV_BLOCK) k_convert(Dev d) {
    pdl_enter();
    using St = Store<S>;
    const int nfill = __ldcg(d.counts + C_FILL), nempty = __ldcg(d.counts + C_EMPTY);
    if (nfill + nempty == 0) return;
    const long long N = d.N;
    // one warp per converted cell, lane q (1..18) for the neighbour x + c_q:
    // all neighbour loads of a cell are in flight together
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const bool act = lane >= 1 && lane < Q;
    const int q = act ? lane : 1;
    // A and B, one pass: a warp takes a converted cell and loads its
    // neighbours' types and segment flags once.  A needs only the cell's own
    // neighbours' B_TOLIQ bits (set before this kernel), and B of a cell only
    // its own A decision and its neighbours' types, so no barrier separates
    // them; the B_NEW bits B sets on other cells' flag words are atomic, and
    // A's clearing of the cell's own B_TOGAS touches only its own byte.
    for (int k = warp; k < nfill + nempty; k += nwarps) {
        const bool isfill = k < nfill;
        const int i = isfill ? d.fill[k] : d.empty[k - nfill];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        const int j = act ? nbr_index(d, x, y, z, cx(q), cy(q), cz(q)) : i;
        const uint8_t fj = act ? __ldcg(d.flags + j) : (uint8_t)0;
        const int sj = seg_of(d, j);
        const uint8_t sa = (act && isfill) ? d.seg_active[sj] : (uint8_t)1;
        if (!isfill && __any_sync(0xffffffffu, act && (fj & B_TOLIQ))) {  // warp-uniform
            if (lane == 0) d.flags[i] &= (uint8_t)~B_TOGAS;  // A: stays interface
            continue;
        }
        if (act && (isfill ? (fj & T_GAS) : (fj & T_LIQ))) {
            unsigned *word = reinterpret_cast<unsigned *>(d.flags + (j & ~3));
            const int sh = (j & 3) * 8;
            const unsigned old = atomicOr(word, (unsigned)B_NEW << sh);
            if (!((old >> sh) & B_NEW)) {
                if (isfill) {
                    d.newgas[atomicAdd(d.counts + C_NEWGAS, 1)] = j;
                    if (!sa) {
                        d.seg_active[sj] = 1;
                        d.counts[d.cdirty] = 1;
                    }
                } else {
                    d.liq2if[atomicAdd(d.counts + C_LIQ2IF, 1)] = j;
                }
            }
        }
    }
    __syncthreads();
    // C (new cells; lane q (1..18) reads neighbour x + c_q) and D (excess of
    // the converted cells) in one phase: item k < ngas + nliq is a new cell,
    // the rest the converted cells
    const int ngas = __ldcg(d.counts + C_NEWGAS), nliq = __ldcg(d.counts + C_LIQ2IF);
    for (int k = warp; k < ngas + nliq + nfill + nempty; k += nwarps) {
        if (k >= ngas + nliq) {
            const int kc = k - ngas - nliq;
            const bool isfill = kc < nfill;
            const int i = isfill ? d.fill[kc] : d.empty[kc - nfill];
            int x, y, z;
            cell_coords(d, i, x, y, z);
            const int j = act ? nbr_index(d, x, y, z, cx(q), cy(q), cz(q)) : i;
            const uint8_t fi = isfill ? (uint8_t)0 : __ldcg(d.flags + i);
            const uint8_t fj = act ? __ldcg(d.flags + j) : (uint8_t)0;
            const float4 ni = d.excess_rule ? d.normal[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float m = lane == 0 ? __ldcg(d.mass + i) : 0.f, r = lane == 0 ? __ldcg(d.rho + i) : 0.f;
            if (!isfill && !(fi & B_TOGAS)) continue;  // warp-uniform
            bool recv = false;
            float wgt = 0.f;
            if (act) {
                recv = ((fj & T_IF) && !(fj & (B_TOLIQ | B_TOGAS))) || (fj & B_NEW);
                if (recv) d.rmark[j] = 1;
                if (recv && d.excess_rule) wgt = excess_weight(ni, isfill, cx(q), cy(q), cz(q));
            }
            const int n = __popc(__ballot_sync(0xffffffffu, recv));
            float W = wgt;  // sum of the receivers' weights, fixed order
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
            if (lane == 0) {
                const float mex = isfill ? m - r : m;
                const bool weighted = d.excess_rule && W > 0.f;
                d.mass[i] = isfill ? r : 0.f;
                d.excess[i] = weighted ? mex / W : (n ? mex / n : 0.f);
                d.exw[i] = weighted ? 1.f : 0.f;
                if (n == 0) atomicAdd(d.lost, (double)mex);
            }
            continue;
        }
        if (k < ngas) {
            const int j = d.newgas[k];
            int x, y, z;
            cell_coords(d, j, x, y, z);
            float r = 0.f, ux = 0.f, uy = 0.f, uz = 0.f, c = 0.f;
            if (act) {  // the neighbour's PDFs are loaded with its type (used only if it is fluid)
                const int l = nbr_index(d, x, y, z, cx(q), cy(q), cz(q));
                const uint8_t fl = __ldcg(d.flags + l);
                float v[Q];
#pragma unroll
                for (int p = 0; p < Q; ++p) v[p] = St::ldcg(d.fdst, (long long)p * N + l, p, d);
                if (fl & (T_LIQ | T_IF)) {
                    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                    for (int p = 0; p < Q; ++p) {
                        r += v[p];
                        jx += cx(p) * v[p];
                        jy += cy(p) * v[p];
                        jz += cz(p) * v[p];
                    }
                    ux = jx / r;
                    uy = jy / r;
                    uz = jz / r;
                    c = 1.f;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r += __shfl_xor_sync(0xffffffffu, r, o);
                ux += __shfl_xor_sync(0xffffffffu, ux, o);
                uy += __shfl_xor_sync(0xffffffffu, uy, o);
                uz += __shfl_xor_sync(0xffffffffu, uz, o);
                c += __shfl_xor_sync(0xffffffffu, c, o);
            }
            const float rb = r / c, vx = ux / c, vy = uy / c, vz = uz / c;
            if (lane < Q) {
                const int p = lane;
                const float uu = 1.5f * (vx * vx + vy * vy + vz * vz);
                const float cu = cx(p) * vx + cy(p) * vy + cz(p) * vz;
                St::st(d.fdst, (long long)p * N + j, p, wq(p) * rb * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu), d);
            }
            if (lane == 0) {
                d.mass[j] = 0.f;
                d.rho[j] = rb;
            }
        } else {
            const int j = d.liq2if[k - ngas];
            float r = lane < Q ? St::ldcg(d.fdst, (long long)lane * N + j, lane, d) : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (lane == 0) {
                d.mass[j] = r;
                d.rho[j] = r;
            }
        }
    }
}

// ---- final update ------------------------------------------------------------
// A: cells that are interface at t+1 (old interface cells that did not convert,
//    and the new ones) set phi = m / rho and form the interface list of t+1;
//    those k_convert marked as receivers first gather the excess mass of their
//    converted neighbours in fixed q order (and clear the mark).
// excess mass of the converted neighbours of receiver i added to its mass m
// (out of line: few cells per step take it, and the list loop stays short)
// (the 18 neighbours' types are loaded before any is used: one round of loads,
// then the converted neighbours' excess in the order of q)
__device__ __noinline__ float gather_excess(const Dev &d, int i, float m) {
    d.rmark[i] = 0;
    int x, y, z;
    cell_coords(d, i, x, y, z);
    int js[Q];
    uint8_t fjs[Q];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        js[q] = nbr_index(d, x, y, z, cx(q), cy(q), cz(q));
        fjs[q] = d.flags[js[q]];
    }
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const uint8_t fj = fjs[q];
        if (!(fj & (B_TOLIQ | B_TOGAS))) continue;
        const int j = js[q];
        // the share of this cell, at -c_q seen from the converted cell j
        const float w =
            d.exw[j] != 0.f ? excess_weight(d.normal[j], (fj & B_TOLIQ) != 0, -cx(q), -cy(q), -cz(q)) : 1.f;
        m += d.excess[j] * w;
    }
    d.mass[i] = m;
    return m;
}

__global__ void __launch_bounds__(LIST_BLOCK) k_fin_a(Dev d) {
    pdl_enter();
    int cnt[6];
    block_counts<6>(d.counts, {d.cif, C_NEWGAS, C_LIQ2IF, C_FILL, C_EMPTY, d.cdirty}, cnt);
    if (blockIdx.x == 0 && threadIdx.x == 0 && cnt[5]) d.counts[C_SEG] = 0;  // filled again by k_fin_b
    const int nold = cnt[0], ngas = cnt[1], nliq = cnt[2];
    const bool any = (cnt[3] + cnt[4]) > 0;
    long long phisum = 0;  // bubble model: fixed-point fill levels of the next interface cells
    warp_uniform_loop(nold + ngas + nliq, [&](int k, bool valid) {
        bool keep = false;
        int i = 0;
        if (valid) {
            i = k < nold ? d.iflist[k] : (k < nold + ngas ? d.newgas[k - nold] : d.liq2if[k - nold - ngas]);
            // the cell's values in one round of loads
            const uint8_t fl = d.flags[i];
            float m = d.mass[i];
            const float rh = d.rho[i];
            const uint8_t rm = any ? d.rmark[i] : (uint8_t)0;
            if (!(k < nold && (fl & (B_TOLIQ | B_TOGAS)))) {
                if (rm) m = gather_excess(d, i, m);  // a converted neighbour shares its excess
                const float ph = m / rh;
                d.phi[i] = ph;
                if (d.bub_i) phisum += __double2ll_rn((double)ph * BUB_FIX);
                keep = true;
            }
        }
        warp_append(d.iflist_next, d.counts + d.cif_next, keep, i);
    });
    if (d.bub_i) {  // block-uniform
        for (int o = 16; o > 0; o >>= 1) phisum += __shfl_down_sync(0xffffffffu, phisum, o);
        __shared__ long long red[LIST_BLOCK / 32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = phisum;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < LIST_BLOCK / 32; ++w) t += red[w];
            if (t) atomicAdd(reinterpret_cast<unsigned long long *>(d.bub_i + 2 + (list_parity(d) ^ 1)),
                             (unsigned long long)t);
        }
    }
}

// B: final types of the converted cells (transient bits cleared), and the
// list of active segments for the next step (block-aggregated compaction),
// rebuilt only when a segment was switched on or off during the step
__global__ void __launch_bounds__(256) k_fin_b(Dev d) {
    pdl_enter();
    int cnt[5];
    block_counts<5>(d.counts, {C_FILL, C_EMPTY, C_NEWGAS, C_LIQ2IF, d.cdirty}, cnt);
    const int nfill = cnt[0], nempty = cnt[1], ngas = cnt[2], nliq = cnt[3];
    const int n = nfill + nempty + ngas + nliq;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (d.bub_i && tid == 0) {  // liquid cells of the next state: filled cells join, cells from liquid leave
        const int par = list_parity(d);
        d.bub_i[par ^ 1] = d.bub_i[par] + nfill - nliq;
    }
    for (int k = tid; k < n; k += nth) {
        if (k < nfill) {
            const int i = d.fill[k];
            d.flags[i] = T_LIQ | (d.flags[i] & B_NEAR);
            d.phi[i] = 1.0f;
        } else if (k < nfill + nempty) {
            const int i = d.empty[k - nfill];
            const uint8_t fl = d.flags[i];
            if (fl & B_TOGAS) {
                d.flags[i] = T_GAS | (fl & B_NEAR);
                d.phi[i] = 0.0f;
                d.mass[i] = 0.0f;
            }
        } else {
            const int j = k < nfill + nempty + ngas ? d.newgas[k - nfill - nempty] : d.liq2if[k - nfill - nempty - ngas];
            d.flags[j] = T_IF | (d.flags[j] & B_NEAR);
        }
    }
    if (!cnt[4]) return;  // the set of active segments did not change (block-uniform)
    // the list again: 16 segment flags per thread (one 16-byte load), a warp
    // scan of the counts and one atomic per warp for the warp's place
    const int lane = threadIdx.x & 31, nchunk = (d.nseg + 15) >> 4;
    for (int base = tid - lane; base < nchunk; base += nth) {  // warp-uniform
        const int c = base + lane;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (c < nchunk) {
            if (16 * c + 16 <= d.nseg) {
                const uint4 v = *reinterpret_cast<const uint4 *>(d.seg_active + 16 * c);
                w[0] = v.x;
                w[1] = v.y;
                w[2] = v.z;
                w[3] = v.w;
            } else {
                for (int b = 0; 16 * c + b < d.nseg; ++b)
                    w[b >> 2] |= (uint32_t)(d.seg_active[16 * c + b] != 0) << (8 * (b & 3));
            }
        }
        uint32_t m = 0u;  // bit b: segment 16 c + b is active
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int b = 0; b < 4; ++b) m |= (((w[k] >> (8 * b)) & 0xffu) != 0u ? 1u : 0u) << (4 * k + b);
        const int cntl = __popc(m);
        int incl = cntl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int wbase = 0;
        if (lane == 31 && incl) wbase = atomicAdd(d.counts + C_SEG, incl);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        int pos = wbase + incl - cntl;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            d.seg_list[pos++] = 16 * c + b;
        }
    }
}

// Final update of a step with frozen types (no conversion, the interface
// list and the active segments stay): phi = m / rho of the interface cells.
__global__ void __launch_bounds__(LIST_BLOCK) k_fin_frozen(Dev d) {
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.iflist[k];
        d.phi[i] = d.mass[i] / d.rho[i];
    }
}

void launch_fin_frozen(const Dev &d, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_fin_frozen, LIST_BLOCK, 4);
    k_fin_frozen<<<g, LIST_BLOCK, 0, s>>>(d);
}

// active segments -> list (warp-ballot compaction); counter zeroed first
__global__ void __launch_bounds__(256) k_seg_compact(Dev d) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = s < d.nseg && d.seg_active[s];
    warp_append(d.seg_list, d.counts + C_SEG, act, s);
}

void launch_seg_compact(const Dev &d, cudaStream_t s) {
    cudaMemsetAsync(d.counts + C_SEG, 0, sizeof(int), s);
    k_seg_compact<<<(d.nseg + 255) / 256, 256, 0, s>>>(d);
}



template <int S, int COLL>
void launch_bulk(const Dev &d, cudaStream_t s) {
    static const int gb = resident_grid((const void *)k_sc_bulk<S, COLL>, 256);
    k_sc_bulk<S, COLL><<<gb, 256, 0, s>>>(d);
}

template <int S, int COLL>
void launch_iface(const Dev &d, cudaStream_t s) {
    static const int gi = list_blocks((const void *)k_sc_iface<S, COLL>, LIST_BLOCK, 4);
    k_sc_iface<S, COLL><<<gi, LIST_BLOCK, 0, s>>>(d);
}

#define FSL_DISPATCH(FN)                                                                          \
    do {                                                                                          \
        const bool trt = d.collision == FSL_TRT;                                                  \
        switch (d.storage) {                                                                      \
        case FSL_F32: trt ? FN<FSL_F32, FSL_TRT>(d, s) : FN<FSL_F32, FSL_BGK>(d, s); break;        \
        case FSL_F16_OFS: trt ? FN<FSL_F16_OFS, FSL_TRT>(d, s) : FN<FSL_F16_OFS, FSL_BGK>(d, s); break; \
        default: trt ? FN<FSL_BF16_OFS, FSL_TRT>(d, s) : FN<FSL_BF16_OFS, FSL_BGK>(d, s); break;   \
        }                                                                                         \
    } while (0)

template <int S, int COLL>
void launch_ci(const Dev &d, cudaStream_t s) {
    static const int gf = list_blocks((const void *)k_curv_iface_fast<S, COLL, FSL_IFACE_LANES>, LIST_BLOCK, 4);
    static const int gs = list_blocks((const void *)k_curv_iface_slow<S, COLL>, LIST_BLOCK, 4);
    launch_pdl(k_curv_iface_fast<S, COLL, FSL_IFACE_LANES>, gf, LIST_BLOCK, s, d);
    if (!d.inline_general) launch_pdl(k_curv_iface_slow<S, COLL>, gs, LIST_BLOCK, s, d);
}

void launch_sc_bulk(const Dev &d, cudaStream_t s) { FSL_DISPATCH(launch_bulk); }
void launch_curv_iface(const Dev &d, cudaStream_t s) { FSL_DISPATCH(launch_ci); }
void launch_sc_iface(const Dev &d, cudaStream_t s) { FSL_DISPATCH(launch_iface); }
#undef FSL_DISPATCH

void launch_stream_collide(const Dev &d, cudaStream_t s) {
    launch_sc_bulk(d, s);
    launch_sc_iface(d, s);
}

void launch_convert(const Dev &d, cudaStream_t s) {
    switch (d.storage) {
    case FSL_F32: launch_pdl(k_convert<FSL_F32>, 1, CONV_BLOCK, s, d); break;
    case FSL_F16_OFS: launch_pdl(k_convert<FSL_F16_OFS>, 1, CONV_BLOCK, s, d); break;
    default: launch_pdl(k_convert<FSL_BF16_OFS>, 1, CONV_BLOCK, s, d); break;
    }
}

void launch_finalize(const Dev &d, cudaStream_t s) {
    static const int ga = list_blocks((const void *)k_fin_a, LIST_BLOCK, 4);
    static const int gb = list_blocks((const void *)k_fin_b, 256, 4);
    launch_pdl(k_fin_a, ga, LIST_BLOCK, s, d);
    launch_pdl(k_fin_b, gb, 256, s, d);
}

}  // namespace fslk
