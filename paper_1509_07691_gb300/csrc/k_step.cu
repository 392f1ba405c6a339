// k_step.cu -- the FSLBM time step (Sec. II): fused pull stream-collide with the
// free-boundary condition and mass exchange, conversion of interface cells
// with excess-mass redistribution, and the final type update with the
// interface list of the next step.
#include "fsl_internal.cuh"

namespace fslk {

constexpr int SC_THREADS = 128;

// BGK / TRT collision in place (Eq. lbe2).  TRT relaxes the even and odd
// parts of each pair (q, opp q) with omega_e = 1/tau and omega_o = 1/tau_o.
template <int COLL>
__device__ __forceinline__ void collide(float f[Q], const Dev &d, float &rho_out) {
    float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        rho += f[q];
        jx += cx(q) * f[q];
        jy += cy(q) * f[q];
        jz += cz(q) * f[q];
    }
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    rho_out = rho;
    if (COLL == FSL_BGK) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float fe = wq(q) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu);
            f[q] += d.omega_e * (fe - f[q]);
        }
    } else {
        f[0] += d.omega_e * (wq(0) * rho * (1.0f - uu) - f[0]);
#pragma unroll
        for (int q = 1; q < Q; q += 2) {
            const int qb = q + 1;
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float ep = wq(q) * rho * (1.0f + 4.5f * cu * cu - uu);
            const float em = wq(q) * rho * 3.0f * cu;
            const float fp = 0.5f * (f[q] + f[qb]), fm = 0.5f * (f[q] - f[qb]);
            const float de = d.omega_e * (fp - ep), dd = d.omega_o * (fm - em);
            f[q] = f[q] - de - dd;
            f[qb] = f[qb] - de + dd;
        }
    }
}

// One thread per cell of an x row.  Gas and obstacle cells do nothing.
// Liquid cells without obstacle neighbours take the plain pull path; the
// others (interface, liquid next to a wall) resolve each link by the type of
// its source cell x - c_q:
//   fluid     f_q(x) = f'_q(x - c_q)                        (Eq. lbe1)
//   gas       f_q(x) = feq_q + feq_qbar - f'_qbar(x)         (Eq. reconstruct)
//             with rho_b = 3 p_g + 6 sigma kappa(x), u_b = u(x, t)
//   obstacle  f_q(x) = f'_qbar(x) (bounce-back), or Eq. reconstruct at a
//             contact-line cell when c_qbar . n_t < 0, n_t the interface normal
//             projected into the wall (Fig. inhomo)
// and interface cells add the mass exchange of Eqs. (advection1/2).
template <int S, int COLL>
__global__ void __launch_bounds__(SC_THREADS) k_stream_collide(Dev d) {
    using St = Store<S>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool inb = x < d.nx;
    const long long N = d.N;
    const long long i = inb ? cell_index(d, x, y, z) : 0;
    const uint8_t fl = inb ? d.flags[i] : (uint8_t)T_GAS;
    bool fill = false, empty = false;

    if (fl & (T_LIQ | T_IF)) {
        const int xs[3] = {x == d.nx - 1 ? 0 : x + 1, x, x == 0 ? d.nx - 1 : x - 1};  // x - c, c = -1,0,1
        const int ys[3] = {y == d.ny - 1 ? 0 : y + 1, y, y == 0 ? d.ny - 1 : y - 1};
        const int zs[3] = {z == d.nz - 1 ? 0 : z + 1, z, z == 0 ? d.nz - 1 : z - 1};
        long long src[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) src[q] = cell_index(d, xs[cx(q) + 1], ys[cy(q) + 1], zs[cz(q) + 1]);

        float f[Q];
        const bool is_if = (fl & T_IF) != 0;
        float dm = 0.f;
        if (!(fl & (T_IF | B_NEAR))) {
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = St::ld(d.fsrc, (long long)q * N + src[q], q, d);
        } else {
            float fo[Q];
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
            const float kap = is_if ? d.kappa[i] : 0.f;
            const float rho_b = d.rho_gas + d.six_sigma * kap;
            const bool corner = is_if && has_gas && has_obs;
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
            const float phix = is_if ? d.phi[i] : 0.f;
            f[0] = fo[0];
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const int qb = opp(q);
                const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
                // feq_q + feq_qbar at (rho_b, u_b): the odd terms cancel
                const float recon = 2.0f * wq(q) * rho_b * (1.0f + 4.5f * cu * cu - uu) - fo[qb];
                if (tq[q] & (T_LIQ | T_IF)) {
                    const float fin = St::ld(d.fsrc, (long long)q * N + src[q], q, d);
                    f[q] = fin;
                    if (is_if) {
                        const float k = (tq[q] & T_LIQ) ? 1.0f : 0.5f * (phix + d.phi[src[q]]);
                        dm += k * (fin - fo[qb]);
                    }
                } else if (tq[q] & T_OBS) {
                    const float outdir = -(cx(q) * ntx + cy(q) * nty + cz(q) * ntz);  // c_qbar . n_t
                    f[q] = (corner && outdir < 0.f) ? recon : fo[qb];
                } else {
                    f[q] = recon;
                }
            }
        }
        float rho;
        collide<COLL>(f, d, rho);
#pragma unroll
        for (int q = 0; q < Q; ++q) St::st(d.fdst, (long long)q * N + i, q, f[q], d);
        if (is_if) {
            const float m = d.mass[i] + dm;
            d.mass[i] = m;
            d.rho[i] = rho;
            fill = m > (1.0f + d.eps) * rho;
            empty = !fill && (m < -d.eps * rho);
            if (fill || empty) d.flags[i] = fl | (fill ? B_TOLIQ : B_TOGAS);
        }
    }
    warp_append(d.fill, d.counts + C_FILL, fill, (int)i);
    warp_append(d.empty, d.counts + C_EMPTY, empty, (int)i);
}

// Conversion (the paper cites Koerner et al. for it; readings):
//  A  an emptying cell with a filling D3Q19 neighbour stays interface;
//  B  gas neighbours of filling cells and liquid neighbours of emptying cells
//     become interface (deduplicated with an atomic OR on the flag word);
//  C  new cells from gas get f = feq(mean rho, mean u) of their fluid
//     neighbours and m = 0; cells from liquid keep f and get m = rho;
//  D  the excess mass (m - rho of a filled cell, m of an emptied one) is
//     divided equally among the neighbours that are interface after B; the
//     receivers gather it in k_finalize.  No receiver: added to `lost`.
// One block: conversions per step are few, and the phases need block barriers.
template <int S>
__global__ void __launch_bounds__(1024) k_convert(Dev d) {
    using St = Store<S>;
    const int nfill = __ldcg(d.counts + C_FILL), nempty = __ldcg(d.counts + C_EMPTY);
    if (nfill + nempty == 0) return;
    const long long N = d.N;
    for (int k = threadIdx.x; k < nempty; k += blockDim.x) {
        const int i = d.empty[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        for (int q = 1; q < Q; ++q)
            if (d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & B_TOLIQ) {
                d.flags[i] &= (uint8_t)~B_TOGAS;
                break;
            }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nfill + nempty; k += blockDim.x) {
        const bool isfill = k < nfill;
        const int i = isfill ? d.fill[k] : d.empty[k - nfill];
        if (!isfill && !(__ldcg(d.flags + i) & B_TOGAS)) continue;
        int x, y, z;
        cell_coords(d, i, x, y, z);
        for (int q = 1; q < Q; ++q) {
            const long long j = nbr_index(d, x, y, z, cx(q), cy(q), cz(q));
            const uint8_t fj = __ldcg(d.flags + j);
            if (isfill ? (fj & T_GAS) : (fj & T_LIQ)) {
                unsigned *word = reinterpret_cast<unsigned *>(d.flags + (j & ~3LL));
                const int sh = (int)(j & 3) * 8;
                const unsigned old = atomicOr(word, (unsigned)B_NEW << sh);
                if (!((old >> sh) & B_NEW)) {
                    if (isfill) d.newgas[atomicAdd(d.counts + C_NEWGAS, 1)] = (int)j;
                    else d.liq2if[atomicAdd(d.counts + C_LIQ2IF, 1)] = (int)j;
                }
            }
        }
    }
    __syncthreads();
    const int ngas = __ldcg(d.counts + C_NEWGAS), nliq = __ldcg(d.counts + C_LIQ2IF);
    for (int k = threadIdx.x; k < ngas + nliq; k += blockDim.x) {
        if (k < ngas) {
            const int j = d.newgas[k];
            int x, y, z;
            cell_coords(d, j, x, y, z);
            float rs = 0.f, us[3] = {0.f, 0.f, 0.f};
            int cnt = 0;
            for (int q = 1; q < Q; ++q) {
                const long long l = nbr_index(d, x, y, z, cx(q), cy(q), cz(q));
                if (!(__ldcg(d.flags + l) & (T_LIQ | T_IF))) continue;
                float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
                for (int p = 0; p < Q; ++p) {
                    const float v = St::ldcg(d.fdst, (long long)p * N + l, p, d);
                    r += v;
                    jx += cx(p) * v;
                    jy += cy(p) * v;
                    jz += cz(p) * v;
                }
                rs += r;
                us[0] += jx / r;
                us[1] += jy / r;
                us[2] += jz / r;
                ++cnt;
            }
            const float rb = rs / cnt, ux = us[0] / cnt, uy = us[1] / cnt, uz = us[2] / cnt;
            const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
            for (int q = 0; q < Q; ++q) {
                const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
                St::st(d.fdst, (long long)q * N + j, q, wq(q) * rb * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu), d);
            }
            d.mass[j] = 0.f;
            d.rho[j] = rb;
        } else {
            const int j = d.liq2if[k - ngas];
            float r = 0.f;
            for (int p = 0; p < Q; ++p) r += St::ldcg(d.fdst, (long long)p * N + j, p, d);
            d.mass[j] = r;
            d.rho[j] = r;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nfill + nempty; k += blockDim.x) {
        const bool isfill = k < nfill;
        const int i = isfill ? d.fill[k] : d.empty[k - nfill];
        if (!isfill && !(__ldcg(d.flags + i) & B_TOGAS)) continue;
        const float m = d.mass[i], r = d.rho[i];
        const float mex = isfill ? m - r : m;
        d.mass[i] = isfill ? r : 0.f;
        int x, y, z;
        cell_coords(d, i, x, y, z);
        int n = 0;
        for (int q = 1; q < Q; ++q) {
            const uint8_t fj = __ldcg(d.flags + nbr_index(d, x, y, z, cx(q), cy(q), cz(q)));
            n += (((fj & T_IF) && !(fj & (B_TOLIQ | B_TOGAS))) || (fj & B_NEW)) ? 1 : 0;
        }
        d.excess[i] = n ? mex / n : 0.f;
        if (n == 0) atomicAdd(d.lost, (double)mex);
    }
}

// Final types of the step and phi = m / rho of interface cells; interface
// cells gather the excess mass of converted neighbours in fixed q order and
// are appended to the interface list of the next step.
__global__ void __launch_bounds__(256) k_finalize(Dev d) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool inb = x < d.nx;
    const long long i = inb ? cell_index(d, x, y, z) : 0;
    const uint8_t fl = inb ? d.flags[i] : (uint8_t)0;
    const bool any = (__ldcg(d.counts + C_FILL) + __ldcg(d.counts + C_EMPTY)) > 0;
    uint8_t t = fl & T_MASK;
    if (fl & B_TOLIQ) t = T_LIQ;
    else if (fl & B_TOGAS) t = T_GAS;
    else if (fl & B_NEW) t = T_IF;
    const bool is_if = inb && t == T_IF;
    if (inb) {
        if (is_if) {
            float m = d.mass[i];
            if (any) {
                for (int q = 1; q < Q; ++q) {
                    const long long j = nbr_index(d, x, y, z, cx(q), cy(q), cz(q));
                    if (d.flags[j] & (B_TOLIQ | B_TOGAS)) m += d.excess[j];
                }
                d.mass[i] = m;
            }
            d.phi[i] = m / d.rho[i];
        } else if (t != (fl & T_MASK)) {
            if (t == T_LIQ) {
                d.phi[i] = 1.0f;
            } else {
                d.phi[i] = 0.0f;
                d.mass[i] = 0.0f;
            }
        }
        d.flags_next[i] = t | (fl & B_NEAR);
    }
    warp_append(d.iflist, d.counts + C_IF, is_if, (int)i);
}

void launch_stream_collide(const Dev &d, cudaStream_t s) {
    dim3 grid((d.nx + SC_THREADS - 1) / SC_THREADS, d.ny, d.nz);
    const bool trt = d.collision == FSL_TRT;
    switch (d.storage) {
    case FSL_F32:
        if (trt) k_stream_collide<FSL_F32, FSL_TRT><<<grid, SC_THREADS, 0, s>>>(d);
        else k_stream_collide<FSL_F32, FSL_BGK><<<grid, SC_THREADS, 0, s>>>(d);
        break;
    case FSL_F16_OFS:
        if (trt) k_stream_collide<FSL_F16_OFS, FSL_TRT><<<grid, SC_THREADS, 0, s>>>(d);
        else k_stream_collide<FSL_F16_OFS, FSL_BGK><<<grid, SC_THREADS, 0, s>>>(d);
        break;
    default:
        if (trt) k_stream_collide<FSL_BF16_OFS, FSL_TRT><<<grid, SC_THREADS, 0, s>>>(d);
        else k_stream_collide<FSL_BF16_OFS, FSL_BGK><<<grid, SC_THREADS, 0, s>>>(d);
        break;
    }
}

void launch_convert(const Dev &d, cudaStream_t s) {
    switch (d.storage) {
    case FSL_F32: k_convert<FSL_F32><<<1, 1024, 0, s>>>(d); break;
    case FSL_F16_OFS: k_convert<FSL_F16_OFS><<<1, 1024, 0, s>>>(d); break;
    default: k_convert<FSL_BF16_OFS><<<1, 1024, 0, s>>>(d); break;
    }
}

void launch_finalize(const Dev &d, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny, d.nz);
    k_finalize<<<grid, 256, 0, s>>>(d);
}

}  // namespace fslk
