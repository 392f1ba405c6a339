// k_init.cu -- initial fill levels by sub-sampling (Sec. III.A), initial cell
// types (Sec. II), refresh of derived data, statistics and the total mass.
#include "fsl_internal.cuh"

namespace fslk {

int resident_grid(const void *kernel, int block, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, smem);
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
}

int list_blocks(const void *kernel, int block, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int want = (sms > 0 ? sms : 1) * per_sm, cap = resident_grid(kernel, block);
    return want < cap ? want : cap;
}

// ---- fill levels -------------------------------------------------------------
// Inside tests in FP64 with explicitly rounded operations (no contraction),
// evaluated in the same order as the sampling formula states, so that every
// sample point is classified as the definition classifies it.
__device__ __forceinline__ double dsq3(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

__device__ bool inside(const fsl_geometry &g, double px, double py, double pz) {
    const double dx = __dsub_rn(px, g.c[0]), dy = __dsub_rn(py, g.c[1]), dz = __dsub_rn(pz, g.c[2]);
    const double r2 = dsq3(dx, dy, dz);
    bool in = false;
    switch (g.kind) {
    case 0: in = r2 <= __dmul_rn(g.R, g.R); break;
    case 1: {
        const double r = __dsqrt_rn(r2);
        if (r == 0.0) { in = true; break; }
        const double mu = __ddiv_rn(dz, r);
        const double p2 = __dsub_rn(__dmul_rn(__dmul_rn(1.5, mu), mu), 0.5);
        in = r <= __dmul_rn(g.R, __dadd_rn(1.0, __dmul_rn(g.eps2, p2)));
        break;
    }
    case 2: in = (r2 <= __dmul_rn(g.R, g.R)) && (pz >= g.zw); break;
    case 3: {
        const double ex = __dsub_rn(px, g.c2[0]), ey = __dsub_rn(py, g.c2[1]), ez = __dsub_rn(pz, g.c2[2]);
        in = (r2 <= __dmul_rn(g.R, g.R)) || (dsq3(ex, ey, ez) <= __dmul_rn(g.R2, g.R2));
        break;
    }
    case 4: {
        const double tp = 6.283185307179586;
        const double h = __dadd_rn(g.h0, __dmul_rn(__dmul_rn(g.amp, sin(__ddiv_rn(__dmul_rn(tp, px), g.wavelength))),
                                                   sin(__ddiv_rn(__dmul_rn(tp, py), g.wavelength))));
        in = pz < h;
        break;
    }
    case 5:
        in = __dadd_rn(__dadd_rn(__dmul_rn(g.n[0], px), __dmul_rn(g.n[1], py)), __dmul_rn(g.n[2], pz)) <= g.d;
        break;
    }
    return g.invert ? !in : in;
}

// -1: whole cell outside, +1: whole cell inside, 0: sample it.  The margins
// (one cell, more than the half diagonal) are conservative.
__device__ int classify(const fsl_geometry &g, double x, double y, double z) {
    const double dx = x - g.c[0], dy = y - g.c[1], dz = z - g.c[2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    int s = 0;
    switch (g.kind) {
    case 0: s = (r + 1.0 < g.R) ? 1 : (r - 1.0 > g.R ? -1 : 0); break;
    case 1: {
        const double e = fabs(g.eps2);
        s = (r + 1.0 < g.R * (1.0 - 0.5 * e)) ? 1 : (r - 1.0 > g.R * (1.0 + e) ? -1 : 0);
        break;
    }
    case 2:
        if (r - 1.0 > g.R || z + 1.0 < g.zw) s = -1;
        else if (r + 1.0 < g.R && z - 1.0 > g.zw) s = 1;
        break;
    case 3: {
        const double ex = x - g.c2[0], ey = y - g.c2[1], ez = z - g.c2[2];
        const double r2 = sqrt(ex * ex + ey * ey + ez * ez);
        if (r + 1.0 < g.R || r2 + 1.0 < g.R2) s = 1;
        else if (r - 1.0 > g.R && r2 - 1.0 > g.R2) s = -1;
        break;
    }
    case 4: {
        const double a = fabs(g.amp);
        s = (z + 1.0 < g.h0 - a) ? 1 : (z - 1.0 > g.h0 + a ? -1 : 0);
        break;
    }
    case 5: {
        const double nl = sqrt(g.n[0] * g.n[0] + g.n[1] * g.n[1] + g.n[2] * g.n[2]);
        const double v = g.n[0] * x + g.n[1] * y + g.n[2] * z - g.d;
        s = (v < -nl) ? 1 : (v > nl ? -1 : 0);
        break;
    }
    }
    return g.invert ? -s : s;
}

__global__ void __launch_bounds__(128) k_fill(fsl_geometry g, int nx, int ny, int nz, float *phi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const long long i = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
    const int c = classify(g, x, y, z);
    if (c != 0) {
        phi[i] = c > 0 ? 1.0f : 0.0f;
        return;
    }
    const int S = g.sub;
    int cnt = 0;
    for (int sz = 0; sz < S; ++sz) {
        const double pz = __dsub_rn(__dadd_rn((double)z, __ddiv_rn(__dadd_rn((double)sz, 0.5), (double)S)), 0.5);
        for (int sy = 0; sy < S; ++sy) {
            const double py = __dsub_rn(__dadd_rn((double)y, __ddiv_rn(__dadd_rn((double)sy, 0.5), (double)S)), 0.5);
            for (int sx = 0; sx < S; ++sx) {
                const double px = __dsub_rn(__dadd_rn((double)x, __ddiv_rn(__dadd_rn((double)sx, 0.5), (double)S)), 0.5);
                cnt += inside(g, px, py, pz) ? 1 : 0;
            }
        }
    }
    phi[i] = (float)((double)cnt / ((double)S * S * S));
}

void launch_fill_geometry(const fsl_params &p, const fsl_geometry &g, float *phi, cudaStream_t s) {
    dim3 grid((p.nx + 127) / 128, p.ny, p.nz);
    k_fill<<<grid, 128, 0, s>>>(g, p.nx, p.ny, p.nz, phi);
}

// ---- initial types (Sec. II) -----------------------------------------------
__global__ void __launch_bounds__(256) k_init_types(Dev d, const uint8_t *obstacle, uint8_t *tmp) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const float p = d.phi[i];
    uint8_t t;
    if (obstacle && obstacle[i]) t = T_OBS;
    else if (p <= 0.f) t = T_GAS;
    else if (p >= 1.f) t = T_LIQ;
    else t = T_IF;
    tmp[i] = t;
}

// liquid cells touching gas become interface; phi, m = phi, f = w_q; interface
// list; active segments
template <int S>
__global__ void __launch_bounds__(256) k_init_state(Dev d, const uint8_t *tmp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const bool inb = x < d.nx;
    const int i = inb ? cell_index(d, x, y, z) : 0;
    bool is_if = false, obs_nbr = false;
    if (inb) {
        uint8_t t = tmp[i];
        bool gas_nbr = false;
        for (int q = 1; q < Q; ++q) {
            const uint8_t u = tmp[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))];
            gas_nbr |= u == T_GAS;
            obs_nbr |= u == T_OBS;
        }
        if (t == T_LIQ && gas_nbr) t = T_IF;
        float p = d.phi[i];
        if (t == T_OBS || t == T_GAS) p = 0.f;
        if (t == T_LIQ) p = 1.f;
        d.phi[i] = p;
        d.mass[i] = (t & (T_LIQ | T_IF)) ? p : 0.f;
        d.flags[i] = t | (obs_nbr ? B_NEAR : 0);
        for (int q = 0; q < Q; ++q) Store<S>::st(d.fdst, (long long)q * d.N + i, q, wq(q), d);
        is_if = t == T_IF;
        if (t & (T_LIQ | T_IF)) d.seg_active[seg_of(d, i)] = 1;
    }
    if (__any_sync(0xffffffffu, obs_nbr) && (threadIdx.x & 31) == 0) d.counts[C_NEAR] = 1;
    warp_append(d.iflist, d.counts + d.cif, is_if, i);
}

void launch_init_types(const Dev &d, const uint8_t *obstacle, uint8_t *tmp, cudaStream_t s) {
    k_init_types<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(d, obstacle, tmp);
}

void launch_init_state(const Dev &d, const uint8_t *tmp, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny, d.nz);
    switch (d.storage) {
    case FSL_F32: k_init_state<FSL_F32><<<grid, 256, 0, s>>>(d, tmp); break;
    case FSL_F16_OFS: k_init_state<FSL_F16_OFS><<<grid, 256, 0, s>>>(d, tmp); break;
    default: k_init_state<FSL_BF16_OFS><<<grid, 256, 0, s>>>(d, tmp); break;
    }
}

// recompute near-obstacle bits, the interface list and the active segments
// after the caller wrote a state (in place: only the near bit changes, and
// readers look at type bits)
__global__ void __launch_bounds__(256) k_refresh(Dev d) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const bool inb = x < d.nx;
    const int i = inb ? cell_index(d, x, y, z) : 0;
    bool is_if = false, obs_nbr = false;
    if (inb) {
        const uint8_t t = d.flags[i] & T_MASK;
        for (int q = 1; q < Q; ++q) obs_nbr |= (d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & T_OBS) != 0;
        d.flags[i] = t | (obs_nbr ? B_NEAR : 0);
        is_if = t == T_IF;
        if (t & (T_LIQ | T_IF)) d.seg_active[seg_of(d, i)] = 1;
    }
    if (__any_sync(0xffffffffu, obs_nbr) && (threadIdx.x & 31) == 0) d.counts[C_NEAR] = 1;
    warp_append(d.iflist, d.counts + d.cif, is_if, i);
}

void launch_refresh(const Dev &d, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny, d.nz);
    k_refresh<<<grid, 256, 0, s>>>(d);
}

// ---- prescribed flow (the advection test of Sec. III.A) -------------------------
// f' = feq(rho, u) at every liquid and interface cell of the active segments,
// so that the next step carries the fill level along a constant flow by the
// mass exchange alone.  One warp per 32-cell segment.
template <int S>
__global__ void __launch_bounds__(256) k_prescribe(Dev d, float rho, float ux, float uy, float uz) {
    int cnt[1];
    block_counts<1>(d.counts, {C_SEG}, cnt);
    const int nseg = cnt[0];
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    for (int k = gw; k < nseg; k += nw) {
        const int s = d.seg_list[k];
        const int row = s / d.nsegx;
        const int x = (s - row * d.nsegx) * SEG + lane;
        if (x >= d.nx) continue;
        const int z = row / d.ny, y = row - z * d.ny;
        const int i = cell_index(d, x, y, z);
        if (!(d.flags[i] & (T_LIQ | T_IF))) continue;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            Store<S>::st(d.fdst, (long long)q * d.N + i, q, wq(q) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu), d);
        }
    }
}

void launch_prescribe(const Dev &d, float rho, float ux, float uy, float uz, cudaStream_t s) {
    static const int g = resident_grid((const void *)k_prescribe<FSL_F32>, 256);
    switch (d.storage) {
    case FSL_F32: k_prescribe<FSL_F32><<<g, 256, 0, s>>>(d, rho, ux, uy, uz); break;
    case FSL_F16_OFS: k_prescribe<FSL_F16_OFS><<<g, 256, 0, s>>>(d, rho, ux, uy, uz); break;
    default: k_prescribe<FSL_BF16_OFS><<<g, 256, 0, s>>>(d, rho, ux, uy, uz); break;
    }
}

// ---- bubble model: liquid cells, non-obstacle cells, fixed-point fill-level sum ----
// of the current state (the entries of the current list parity and [4]; the
// caller zeroes them first).  Block partials, one integer atomic per block and
// quantity, so the totals do not depend on the order of the additions.
__global__ void __launch_bounds__(256) k_bubble_count(Dev d) {
    long long nl = 0, no = 0, sp = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.N; i += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = d.flags[i] & T_MASK;
        nl += t == T_LIQ;
        no += t != T_OBS;
        if (t == T_IF) sp += __double2ll_rn((double)d.phi[i] * BUB_FIX);
    }
    __shared__ long long red[3][8];
    for (int o = 16; o > 0; o >>= 1) {
        nl += __shfl_down_sync(0xffffffffu, nl, o);
        no += __shfl_down_sync(0xffffffffu, no, o);
        sp += __shfl_down_sync(0xffffffffu, sp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = nl;
        red[1][threadIdx.x >> 5] = no;
        red[2][threadIdx.x >> 5] = sp;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        long long t = 0;
        for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
        const int par = list_parity(d);
        const int slot = threadIdx.x == 0 ? par : (threadIdx.x == 1 ? 4 : 2 + par);
        if (t) atomicAdd(reinterpret_cast<unsigned long long *>(d.bub_i + slot), (unsigned long long)t);
    }
}

void launch_bubble_count(const Dev &d, cudaStream_t s) {
    static const int g = resident_grid((const void *)k_bubble_count, 256);
    k_bubble_count<<<g, 256, 0, s>>>(d);
}

// ---- statistics ----------------------------------------------------------------
// stats[0..5]: liquid, interface, gas, obstacle, interface without liquid or gas
// neighbour, liquid touching gas.  One atomic per block and counter.
__global__ void __launch_bounds__(256) k_stats(Dev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int c[6] = {0, 0, 0, 0, 0, 0};
    if (i < d.N) {
        int x, y, z;
        cell_coords(d, i, x, y, z);
        const uint8_t t = d.flags[i] & T_MASK;
        c[0] = t == T_LIQ;
        c[1] = t == T_IF;
        c[2] = t == T_GAS;
        c[3] = t == T_OBS;
        if (t == T_IF || t == T_LIQ) {
            bool hl = false, hg = false;
            for (int q = 1; q < Q; ++q) {
                const uint8_t u = d.flags[nbr_index(d, x, y, z, cx(q), cy(q), cz(q))] & T_MASK;
                hl |= u == T_LIQ;
                hg |= u == T_GAS;
            }
            c[4] = t == T_IF && (!hl || !hg);
            c[5] = t == T_LIQ && hg;
        }
    }
    __shared__ int red[6][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k) {
        int v = c[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        if (s) atomicAdd(reinterpret_cast<unsigned long long *>(d.stats + threadIdx.x), (unsigned long long)s);
    }
}

void launch_stats(const Dev &d, cudaStream_t s) { k_stats<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(d); }

// ---- total mass ----------------------------------------------------------------
// sum over interface cells of m plus sum over liquid cells of rho = sum_q f_q.
// Each block writes one FP64 partial; a single block adds the partials in a
// fixed order, so the result does not depend on scheduling.
constexpr int MASS_THREADS = 256;
constexpr int MASS_BLOCKS = 152 * 8;
int max_partials() { return MASS_BLOCKS; }

template <int S>
__global__ void __launch_bounds__(MASS_THREADS) k_mass_partial(Dev d) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.N; i += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = d.flags[i] & T_MASK;
        if (t == T_IF) {
            acc += d.mass[i];
        } else if (t == T_LIQ) {
            float r = 0.f;
#pragma unroll
            for (int q = 0; q < Q; ++q) r += Store<S>::ld(d.fsrc, (long long)q * d.N + i, q, d);
            acc += r;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[MASS_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < MASS_THREADS / 32; ++w) s += red[w];
        d.partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(MASS_THREADS) k_mass_final(const double *partial, int n, const double *lost, double *out) {
    __shared__ double red[MASS_THREADS];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += partial[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = MASS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0];
        out[1] = *lost;
    }
}

void launch_mass(const Dev &d, double *out, cudaStream_t s) {
    switch (d.storage) {
    case FSL_F32: k_mass_partial<FSL_F32><<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(d); break;
    case FSL_F16_OFS: k_mass_partial<FSL_F16_OFS><<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(d); break;
    default: k_mass_partial<FSL_BF16_OFS><<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(d); break;
    }
    k_mass_final<<<1, MASS_THREADS, 0, s>>>(d.partial, MASS_BLOCKS, d.lost, out);
}

}  // namespace fslk
