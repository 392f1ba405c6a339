// k_adj.cu -- reverse (adjoint) pass of the FSLBM step over a window of time
// steps with frozen cell types, and the curvature Jacobian it needs.
//
// With the types frozen the step is a smooth map of the state (post-collision
// PDFs f, interface mass m, fill level phi = m / rho) and of the parameters
// sigma and theta:
//   kappa  = K(phi; theta)                         LSQR fit, Sec. II.C
//   g_q(x) = f_q(x - c_q)                          fluid source (Eq. lbe1)
//          = f_qbar(x)                             obstacle (bounce-back)
//          = 2 w_q rho_b (1 + 9/2 (c_q.u)^2 - 3/2 u^2) - f_qbar(x)
//                                                  gas source (Eq. reconstruct),
//            rho_b = 3 p_g + 6 sigma kappa(x), u = u(x, t)
//   f(t+1) = C(g)                                  BGK / TRT collision (Eq. lbe2)
//   m(t+1) = m + sum_q k_q (f_q(x - c_q) - f_qbar(x)),  k_q = 1 from a liquid
//            source, (phi(x) + phi(x - c_q)) / 2 from an interface source
//            (Eqs. advection1/2)
//   phi(t+1) = m(t+1) / rho(t+1),  rho(t+1) = sum_q g_q
// The reverse of one step, given the adjoints (F, M, P) of (f, m, phi) at
// t+1, runs as five kernels:
//   k_adj_iface   interface cells: phi(t+1) = m / rho adjoint, collision
//                 adjoint of g, and every dependency of x's own outputs on
//                 x's own inputs (reconstruction, bounce-back, outflow of the
//                 mass exchange, u_b, rho_b -> kappa and sigma)
//   k_adj_bulk    liquid cells: collision adjoint of g
//   k_adj_gather  every fluid cell y: the adjoint of f_r(y) gathered from the
//                 cells that read it (y + c_r streams it; an interface cell
//                 y + c_r also exchanges mass with it), and for interface y
//                 the adjoint of phi(y) through the exchange weights k_q
//   k_adj_curv    interface cells y: adjoint of phi(y) through the curvature
//                 of the interface cells x of the 7x7x7 window around it,
//                 sum_x kbar(x) dkappa_x/dphi_y, and dL/dtheta
//   k_adj_accum   fixed-order sum of the per-block sigma and theta partials
// Gathers (not scatters) keep every sum in a fixed order: the result is
// bit-reproducible.  The curvature Jacobian rows: the normal and PLIC offset
// sensitivities by forward-mode dual numbers through the same per-cell code
// as k_normals (one seed per lane), the fit's sensitivities by one reverse
// sweep of the FP32 normal equations, or, for contact-line and degenerate
// fits, by dual numbers through lsqr_core (curv_common.cuh), one seed per
// thread.
#include "adjoint.cuh"
#include "curv_common.cuh"

namespace fslk {

constexpr int ADJ_BLOCK = 128;

int adj_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (sms > 0 ? sms : 1) * 4;
}

// ---- window bookkeeping ---------------------------------------------------------
// The window's interface list is built from the cell types in cell-index
// order (block counts, one scan, ordered writes), so that every reduction
// over it runs in the same order whatever the order of the step's own list.
constexpr int WIN_BLOCK = 1024;

__global__ void __launch_bounds__(WIN_BLOCK) k_window_count(Dev d, int *bcount) {
    const long long i = (long long)blockIdx.x * WIN_BLOCK + threadIdx.x;
    const bool p = i < d.N && (d.flags[i] & T_MASK) == T_IF;
    const int c = __syncthreads_count(p);
    if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

// exclusive scan of the nb block counts (one block); the total into wcounts
__global__ void __launch_bounds__(WIN_BLOCK) k_window_scan(int *bcount, int nb, int *wcounts) {
    __shared__ int part[WIN_BLOCK];
    const int per = (nb + WIN_BLOCK - 1) / WIN_BLOCK;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int sum = 0;
    for (int b = b0; b < b1; ++b) sum += bcount[b];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < WIN_BLOCK; ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
        wcounts[C_IF0] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        const int v = bcount[b];
        bcount[b] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(WIN_BLOCK) k_window_write(Dev d, const int *boff, int *wlist, int *widx) {
    __shared__ int wsum[WIN_BLOCK / 32];
    const long long i = (long long)blockIdx.x * WIN_BLOCK + threadIdx.x;
    const bool p = i < d.N && (d.flags[i] & T_MASK) == T_IF;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, p);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < WIN_BLOCK / 32; ++w) {
            const int v = wsum[w];
            wsum[w] = run;
            run += v;
        }
    }
    __syncthreads();
    if (p) {
        const int pos = boff[blockIdx.x] + wsum[warp] + __popc(m & ((1u << lane) - 1u));
        wlist[pos] = (int)i;
        widx[i] = pos;
    }
}

// active segments of the step's view (their order does not matter)
__global__ void k_window_segs(Dev d, int *wcounts, int *wseg) {
    int cnt[1];
    block_counts<1>(d.counts, {C_SEG}, cnt);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0) wcounts[C_SEG] = cnt[0];
    for (int k = tid; k < cnt[0]; k += nth) wseg[k] = d.seg_list[k];
}

__global__ void k_window_finish(Dev d, const int *wcounts, const int *wlist) {
    int cnt[1];
    block_counts<1>(wcounts, {C_IF0}, cnt);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0) d.counts[d.cif] = cnt[0];
    for (int k = tid; k < cnt[0]; k += nth) d.iflist[k] = wlist[k];
}

int window_scratch_ints(long long N) { return (int)((N + WIN_BLOCK - 1) / WIN_BLOCK); }

void launch_window_setup(const Dev &src, int *wcounts, int *wlist, int *widx, int *wseg, int *scratch,
                         cudaStream_t s) {
    const int nb = window_scratch_ints(src.N);
    cudaMemsetAsync(widx, 0xff, (size_t)src.N * sizeof(int), s);
    k_window_count<<<nb, WIN_BLOCK, 0, s>>>(src, scratch);
    k_window_scan<<<1, WIN_BLOCK, 0, s>>>(scratch, nb, wcounts);
    k_window_write<<<nb, WIN_BLOCK, 0, s>>>(src, scratch, wlist, widx);
    static const int g = list_blocks((const void *)k_window_segs, 256, 2);
    k_window_segs<<<g, 256, 0, s>>>(src, wcounts, wseg);
}

void launch_window_finish(const Dev &dst, const int *wcounts, const int *wlist, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_window_finish, 256, 2);
    k_window_finish<<<g, 256, 0, s>>>(dst, wcounts, wlist);
}

void launch_frozen_step(const Dev &d, cudaStream_t s) {
    launch_normals(d, s);
    launch_sc_bulk(d, s);
    if (d.curv_model == FSL_CURV_LSQR) {
        launch_curv_iface(d, s);
    } else {
        launch_zero_kappa(d, d.kappa, s);
        launch_sc_iface(d, s);
    }
    launch_fin_frozen(d, s);
}

// ---- helpers --------------------------------------------------------------------
// sum over the block in a fixed order; the result is valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) t += ws[w];
    __syncthreads();
    return t;
}

// Adjoint of the collision f' = C(g) (Eq. lbe2) at g: gb = (dC/dg)^T fb.
// C(g) = L g + w_e e+(rho, j) + w_o e-(j) with the linear part L (relaxation
// of the even and odd parts of each pair q, qbar; symmetric) and the
// equilibrium parts e+_q = w_q (rho + 9/2 (c_q.j)^2 / rho - 3/2 j.j / rho),
// e-_q = 3 w_q c_q.j as functions of rho = sum g and j = sum c g.  BGK is
// the case w_e = w_o.
__device__ __forceinline__ void collide_adj(const float g[Q], const float fb[Q], const Dev &d, float gb[Q]) {
    float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        rho += g[q];
        jx += cx(q) * g[q];
        jy += cy(q) * g[q];
        jz += cz(q) * g[q];
    }
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float u2 = ux * ux + uy * uy + uz * uz;
    const float we = d.omega_e, wo = d.omega_o;
    float A = 0.f, Bx = 0.f, By = 0.f, Bz = 0.f, S = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
        const float t = fb[q] * wq(q);
        A += t * (1.0f - 4.5f * cu * cu + 1.5f * u2);
        const float sc = t * (9.0f * we * cu + 3.0f * wo);
        Bx += sc * cx(q);
        By += sc * cy(q);
        Bz += sc * cz(q);
        S += t;
    }
    A *= we;
    // d/dj of -3/2 j.j / rho over all q: -3 w_e u sum_q fb_q w_q
    Bx -= 3.0f * we * ux * S;
    By -= 3.0f * we * uy * S;
    Bz -= 3.0f * we * uz * S;
    gb[0] = (1.0f - we) * fb[0] + A;
#pragma unroll
    for (int q = 1; q < Q; q += 2) {
        const int qb = q + 1;
        const float sp = 0.5f * (fb[q] + fb[qb]), sm = 0.5f * (fb[q] - fb[qb]);
        const float bc = Bx * cx(q) + By * cy(q) + Bz * cz(q);
        gb[q] = fb[q] - we * sp - wo * sm + A + bc;
        gb[qb] = fb[qb] - we * sp + wo * sm + A - bc;
    }
}

// ---- curvature Jacobian ---------------------------------------------------------
// kappa_x depends on the fill levels through the PLIC normal and offset
// (n_j, a_j) of the interface cells j of its 3x3x3 neighbourhood, and on
// theta through the contact rows.  Two stages:
//   k_normal_jac  per interface cell j: d(n_j, a_j)/dphi over the 5x5x5
//                 window around j (Parker-Youngs stencil, obstacle reflection,
//                 PLIC offset by the implicit function theorem); dual numbers
//                 through the same code as k_normals, one seed per lane
//   k_kappa_rev   per interface cell x: dkappa_x/d(n_j, a_j) for the four
//                 inputs of each interface cell j of the 3x3x3 neighbourhood
//                 by one reverse sweep of the fit (the full model without
//                 contact rows), then the chain rule dkappa_x/dphi_y =
//                 sum_j sum_c dkappa_x/d(n_j,a_j)_c d(n_j,a_j)_c/dphi_y
//                 into the row of x (7x7x7 window slots, theta last)
//   k_kappa_gen   the cells the sweep does not cover (contact rows, the
//                 centre constraint, fewer than five rows, a fit that is not
//                 positive definite or ill conditioned): the same
//                 sensitivities and dkappa_x/dtheta by dual numbers through
//                 lsqr_core with the stored normals as values, one seed per
//                 thread; the same chain rule.
// A cell whose FP32 fit is ill conditioned (cond^2 above fp64_cond, as
// k_lsqr_slow decides) is listed and its second stage redone in Dual<double>.

// Window of half-width R (fill levels and flags) in shared memory, with one
// seeded fill level (window slot `seed`).
template <int R>
struct WinAcc {
    static constexpr int W = 2 * R + 1;
    const float *phi;
    const uint8_t *fl;
    int seed;
    int iters;

    __device__ __forceinline__ static int slot(int dx, int dy, int dz) { return ((dz + R) * W + (dy + R)) * W + (dx + R); }
    __device__ __forceinline__ uint8_t flag(int dx, int dy, int dz) const { return fl[slot(dx, dy, dz)]; }
    __device__ __forceinline__ Dual<float> phi_d(int dx, int dy, int dz) const {
        const int s = slot(dx, dy, dz);
        return Dual<float>(phi[s], s == seed ? 1.0f : 0.0f, 0);
    }
    __device__ __forceinline__ Dual<float> phi_ext(int dx, int dy, int dz) const {
        if (!(flag(dx, dy, dz) & T_OBS)) return phi_d(dx, dy, dz);
        return reflect_value<Dual<float>>([&](int a, int b, int c) { return flag(dx + a, dy + b, dz + c); },
                                          [&](int a, int b, int c) { return phi_d(dx + a, dy + b, dz + c); });
    }
    // normal and PLIC offset of the centre cell, as k_normals computes them
    __device__ __forceinline__ bool centre_normal(Dual<float> n[3], Dual<float> &a) const {
        using DF = Dual<float>;
        if (flag(0, 0, 0) & B_NEAR)
            parker_youngs<DF>([&](int ex, int ey, int ez) { return phi_ext(ex, ey, ez); }, n);
        else
            parker_youngs<DF>([&](int ex, int ey, int ez) { return phi_d(ex, ey, ez); }, n);
        return unit_normal_offset<DF>(n, phi_d(0, 0, 0), iters, a);
    }
};

constexpr int JAC_WARPS = 4;
constexpr int NJ_CELLS = 125;  // 5x5x5 window of d(n_j, a_j)/dphi

__global__ void __launch_bounds__(JAC_WARPS * 32) k_normal_jac(Dev d, Adj a) {
    __shared__ float sphi[JAC_WARPS][NJ_CELLS];
    __shared__ uint8_t sfl[JAC_WARPS][NJ_CELLS + 3];
    __shared__ uint8_t sseed[JAC_WARPS][NJ_CELLS + 3];
    int cnt[1];
    block_counts<1>(d.counts, {C_IF0}, cnt);
    const int n = min(cnt[0], a.cap);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < n; k += nwarps) {
        const int i = a.wlist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        float4 *row = a.nj + (size_t)k * NJ_CELLS;
        for (int sl = lane; sl < NJ_CELLS; sl += 32) {
            const int j = nbr_index(d, x, y, z, sl % 5 - 2, (sl / 5) % 5 - 2, sl / 25 - 2);
            sphi[w][sl] = d.phi[j];
            sfl[w][sl] = d.flags[j];
            row[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        // seeds: interface cells of the 3x3x3 stencil, of the 5x5x5 window
        // at a cell next to an obstacle (reflected fill levels)
        const bool near = (sfl[w][NJ_CELLS / 2] & B_NEAR) != 0;
        int ns = 0;
        for (int base = 0; base < NJ_CELLS; base += 32) {
            const int sl = base + lane;
            const int ox = sl % 5 - 2, oy = (sl / 5) % 5 - 2, oz = sl / 25 - 2;
            const bool inner = ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1;
            const bool p = sl < NJ_CELLS && (sfl[w][sl] & T_IF) && (near || inner);
            const unsigned m = __ballot_sync(0xffffffffu, p);
            if (p) sseed[w][ns + __popc(m & ((1u << lane) - 1u))] = (uint8_t)sl;
            ns += __popc(m);
        }
        __syncwarp();
        for (int base = 0; base < ns; base += 32) {
            const int idx = base + lane;
            const WinAcc<2> acc{sphi[w], sfl[w], idx < ns ? (int)sseed[w][idx] : -1, d.plic_iters};
            Dual<float> nv[3], av;
            const bool ok = acc.centre_normal(nv, av);
            if (ok && idx < ns) row[sseed[w][idx]] = make_float4(nv[0].d, nv[1].d, nv[2].d, av.d);
        }
        __syncwarp();
    }
}

// Accessor of lsqr_core over a cell's neighbourhood staged in shared memory
// (flags of the 5x5x5 block, stored normals of the 3x3x3 block) with the
// stored normals as values and one seeded input: component c of (n_j, a_j)
// of the neighbour j at 3x3x3 slot sj, or theta.
struct SeedAcc {
    const Dev &d;
    const uint8_t *fl;  // slot ((dz+2)*5 + dy+2)*5 + dx+2
    const float4 *nm;   // slot (dz+1)*9 + (dy+1)*3 + dx+1
    int sj, sc;
    bool sth;
    __device__ __forceinline__ uint8_t flag(int dx, int dy, int dz) const {
        return fl[((dz + 2) * 5 + (dy + 2)) * 5 + (dx + 2)];
    }
    template <typename T>
    __device__ __forceinline__ bool normal(int dx, int dy, int dz, T n[3], T &a) const {
        using S = typename scalar_of<T>::type;
        const int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
        const float4 q4 = nm[t];
        if (q4.x == 0.f && q4.y == 0.f && q4.z == 0.f) return false;
        const bool me = t == sj;
        n[0] = T((S)q4.x, (me && sc == 0) ? S(1) : S(0), 0);
        n[1] = T((S)q4.y, (me && sc == 1) ? S(1) : S(0), 0);
        n[2] = T((S)q4.z, (me && sc == 2) ? S(1) : S(0), 0);
        a = T((S)q4.w, (me && sc == 3) ? S(1) : S(0), 0);
        return true;
    }
    template <typename T>
    __device__ __forceinline__ void theta(T &c, T &s) const {
        using S = typename scalar_of<T>::type;
        c = T((S)d.cos_theta_d, sth ? (S)(-d.sin_theta_d) : S(0), 0);
        s = T((S)d.sin_theta_d, sth ? (S)d.cos_theta_d : S(0), 0);
    }
};

constexpr int KJ_SEEDS = 27 * 4 + 1;  // (n_j, a_j) of each 3x3x3 cell, theta

// ---- reverse-mode sensitivities of the FP32 fit ----------------------------------
// Butterfly sum over the warp; both partners of every stage add the same two
// operands, so all lanes end with the same bits.
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ constexpr int pk5(int r, int c) { return r * 5 - r * (r - 1) / 2 + (c - r); }

// Cholesky factor R (upper, packed) of the packed symmetric 5x5 matrix G;
// pd: every pivot positive; cond = (max / min diagonal of R)^2, the condition
// estimate of G the forward fit uses.
__device__ __forceinline__ void chol5(const float G[15], float R[15], bool &pd, float &cond) {
    float dmax = 0.f, dmin = 3.0e38f;
    pd = true;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
#pragma unroll
        for (int c = r; c < 5; ++c) {
            float sum = G[pk5(r, c)];
#pragma unroll
            for (int k = 0; k < r; ++k) sum -= R[pk5(k, r)] * R[pk5(k, c)];
            if (c == r) {
                pd = pd && sum > 0.f;
                const float dd = sqrtf(fmaxf(sum, 1e-30f));
                R[pk5(r, r)] = dd;
                dmax = fmaxf(dmax, dd);
                dmin = fminf(dmin, dd);
            } else {
                R[pk5(r, c)] = sum / R[pk5(r, r)];
            }
        }
    }
    cond = (dmax / dmin) * (dmax / dmin);
}

// x = G^-1 b with G = R^T R
__device__ __forceinline__ void chol5_solve(const float R[15], const float b[5], float x[5]) {
    float y[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        float sum = b[r];
#pragma unroll
        for (int k = 0; k < r; ++k) sum -= R[pk5(k, r)] * y[k];
        y[r] = sum / R[pk5(r, r)];
    }
#pragma unroll
    for (int r = 4; r >= 0; --r) {
        float sum = y[r];
#pragma unroll
        for (int k = r + 1; k < 5; ++k) sum -= R[pk5(r, k)] * x[k];
        x[r] = sum / R[pk5(r, r)];
    }
}

// dkappa/d(n_t, a_t) of the centre cell's LSQR curvature for every slot t of
// its 3x3x3 block, by one reverse sweep instead of one dual evaluation per
// input.  Lane t < 27 holds slot t (flags fj, stored normal and offset q4;
// centre 13).  The fit is the unconstrained full model (Sec. II.C): rows
// (u^2, v^2, uv, u, v) and right-hand side f of the PLIC points in the frame
// (t_u, t_v, n) of the centre normal, solved by the normal equations G x = r,
// kappa by Eq. (anacurv).  The sweep, with bars for sensitivities of kappa:
//   xbar = dkappa/d(A, B, C, H, I), lambda = G^-1 xbar,
//   per row j (residual e_j = f_j - row_j.x):
//     rowbar_j = e_j lambda - (row_j.lambda) x,  fbar_j = row_j.lambda,
//   then through u = d.t_u, v = d.t_v, f = d.n with d = o_j + a_j n_j - a n,
//   and the centre's frame (t_u = w / |w|, t_v = n x t_u) and origin a n.
// Returns false (the same on every lane) where the cell needs the general
// path: a contact-line cell in the block (gradient rows or the centre
// constraint), a zero centre normal, fewer than five rows, or normal
// equations that are not positive definite or worse conditioned than
// fp64_cond.  theta does not enter such a fit.
__device__ bool kappa_reverse(int lane, uint8_t fj, float4 q4, float fp64_cond, float &kap, float4 &g4) {
    const unsigned full = 0xffffffffu;
    const bool isif = lane < 27 && (fj & T_IF);
    if (__any_sync(full, isif && (fj & B_NEAR))) return false;
    float4 c4;
    c4.x = __shfl_sync(full, q4.x, 13);
    c4.y = __shfl_sync(full, q4.y, 13);
    c4.z = __shfl_sync(full, q4.z, 13);
    c4.w = __shfl_sync(full, q4.w, 13);
    if (c4.x == 0.f && c4.y == 0.f && c4.z == 0.f) return false;
    FastFrame F;
    lsqr_fast_frame(c4, F);
    const bool row = isif && lane != 13 && !(q4.x == 0.f && q4.y == 0.f && q4.z == 0.f);
    const float dv[3] = {(float)(lane % 3 - 1) + q4.w * q4.x - F.p[0], (float)((lane / 3) % 3 - 1) + q4.w * q4.y - F.p[1],
                         (float)(lane / 9 - 1) + q4.w * q4.z - F.p[2]};
    const float u = dot3(dv, F.tu), v = dot3(dv, F.tv);
    const float fr = row ? dot3(dv, F.n) : 0.f;
    float a5[5] = {u * u, v * v, u * v, u, v};
#pragma unroll
    for (int c = 0; c < 5; ++c) a5[c] = row ? a5[c] : 0.f;
    float G[15], rv[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
#pragma unroll
        for (int c = r; c < 5; ++c) G[pk5(r, c)] = warp_allsum(a5[r] * a5[c]);
        rv[r] = warp_allsum(a5[r] * fr);
    }
    const int m = __popc(__ballot_sync(full, row));
    float R[15], cond;
    bool pd;
    chol5(G, R, pd, cond);
    if (!(m >= 5 && pd && !(cond > fp64_cond))) return false;
    float x[5];
    chol5_solve(R, rv, x);
    const float A = x[0], B = x[1], C = x[2], H = x[3], I = x[4];
    const float g = 1.0f + H * H + I * I, D = g * sqrtf(g);
    const float Nn = A * (1.0f + I * I) + B * (1.0f + H * H) - C * H * I;
    kap = Nn / D;
    const float xb[5] = {(1.0f + I * I) / D, (1.0f + H * H) / D, -H * I / D,
                         (2.0f * B * H - C * I - 3.0f * Nn * H / g) / D, (2.0f * A * I - C * H - 3.0f * Nn * I / g) / D};
    float lam[5];
    chol5_solve(R, xb, lam);
    // this lane's row
    float e = fr, rl = 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        e -= a5[c] * x[c];
        rl += a5[c] * lam[c];
    }
    float rb[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) rb[c] = row ? e * lam[c] - rl * x[c] : 0.f;
    const float ub = 2.0f * u * rb[0] + v * rb[2] + rb[3];
    const float vb = 2.0f * v * rb[1] + u * rb[2] + rb[4];
    const float fb = row ? rl : 0.f;
    float db[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) db[c] = ub * F.tu[c] + vb * F.tv[c] + fb * F.n[c];
    g4 = row ? make_float4(q4.w * db[0], q4.w * db[1], q4.w * db[2], q4.x * db[0] + q4.y * db[1] + q4.z * db[2])
             : make_float4(0.f, 0.f, 0.f, 0.f);
    // the centre's frame and origin
    float tub[3], tvb[3], nb[3], pb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        tub[c] = warp_allsum(row ? ub * dv[c] : 0.f);
        tvb[c] = warp_allsum(row ? vb * dv[c] : 0.f);
        nb[c] = warp_allsum(row ? fb * dv[c] : 0.f);
        pb[c] = -warp_allsum(db[c]);
    }
    const float *n = F.n, *tu = F.tu;
    nb[0] += tu[1] * tvb[2] - tu[2] * tvb[1];  // t_v = n x t_u
    nb[1] += tu[2] * tvb[0] - tu[0] * tvb[2];
    nb[2] += tu[0] * tvb[1] - tu[1] * tvb[0];
    tub[0] += tvb[1] * n[2] - tvb[2] * n[1];
    tub[1] += tvb[2] * n[0] - tvb[0] * n[2];
    tub[2] += tvb[0] * n[1] - tvb[1] * n[0];
    int k = 0;  // the frame's case, as lsqr_fast_frame picks it
    if (fabsf(n[1]) < fabsf(n[0])) k = 1;
    if (fabsf(n[2]) < fabsf(n[k])) k = 2;
    float wv[3];
    if (k == 0) { wv[0] = 0.f; wv[1] = -n[2]; wv[2] = n[1]; }
    else if (k == 1) { wv[0] = n[2]; wv[1] = 0.f; wv[2] = -n[0]; }
    else { wv[0] = -n[1]; wv[1] = n[0]; wv[2] = 0.f; }
    const float wl = sqrtf(dot3(wv, wv)), tt = dot3(tu, tub);
    float wb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) wb[c] = (tub[c] - tu[c] * tt) / wl;
    if (k == 0) { nb[2] -= wb[1]; nb[1] += wb[2]; }
    else if (k == 1) { nb[2] += wb[0]; nb[0] -= wb[2]; }
    else { nb[1] -= wb[0]; nb[0] += wb[1]; }
    const float ab = dot3(pb, n);
#pragma unroll
    for (int c = 0; c < 3; ++c) nb[c] += c4.w * pb[c];
    if (lane == 13) g4 = make_float4(nb[0], nb[1], nb[2], ab);
    return true;
}

// Chain rule into the row of x: each used cell j of the 3x3x3 block adds
// sum_c dkappa_x/d(n_j,a_j)_c d(n_j,a_j)_c/dphi over the 5x5x5 window around j
// (a block of the 7x7x7 row) into acc7.  K holds the four sensitivities of the
// cell at 3x3x3 slot tj from K[pos[tj]]; the slots tj0, tj0 + step, ... are
// this warp's, in ascending order, so every entry sums in a fixed order.
__device__ __forceinline__ void chain_rows(const Adj &a, const int *idx, const int *pos, const float *K, float *acc7,
                                           int tj0, int step, int lane) {
    for (int sl = lane; sl < JAC_CELLS; sl += 32) acc7[sl] = 0.f;
    __syncwarp();
    for (int tj = tj0; tj < 27; tj += step) {
        const int jk = idx[tj];
        if (jk < 0) continue;
        const int p = pos[tj];
        const float k0 = K[p], k1 = K[p + 1], k2 = K[p + 2], k3 = K[p + 3];
        const float4 *nrow = a.nj + (size_t)jk * NJ_CELLS;
        const int jx = tj % 3, jy = (tj / 3) % 3, jz = tj / 9;  // 7x7x7 slot of the corner of j's 5x5x5 window
        float4 v[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int r = lane + 32 * h;
            v[h] = r < NJ_CELLS ? nrow[r] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int r = lane + 32 * h;
            if (r < NJ_CELLS) {
                const int sl = ((jz + r / 25) * 7 + (jy + (r / 5) % 5)) * 7 + (jx + r % 5);
                acc7[sl] += k0 * v[h].x + k1 * v[h].y + k2 * v[h].z + k3 * v[h].w;
            }
        }
        __syncwarp();
    }
}

// The seeds of cell x (lanes of one warp, lane t < 27 holding 3x3x3 slot t
// with flags fj and stored normal q4): the four inputs of every interface
// cell of the block with a nonzero normal and a window-list position, then
// theta.  Fills idx / pos (per slot) and seed (codes 4 t + c, 108 = theta);
// returns the number of seeds.
__device__ __forceinline__ int seed_list(const Adj &a, int lane, int jw, uint8_t fj, float4 q4, int *idx, int *pos,
                                         uint8_t *seed) {
    bool use = false;
    int jdx = -1;
    if (lane < 27) {
        use = (fj & T_IF) && !(q4.x == 0.f && q4.y == 0.f && q4.z == 0.f);
        jdx = use ? a.widx[jw] : -1;
        use = use && jdx >= 0 && jdx < a.cap;
    }
    const unsigned m = __ballot_sync(0xffffffffu, use);
    const int nu = __popc(m);
    if (lane < 27) {
        const int p = use ? 4 * __popc(m & ((1u << lane) - 1u)) : -1;
        idx[lane] = use ? jdx : -1;
        pos[lane] = p;
        if (use)
#pragma unroll
            for (int c = 0; c < 4; ++c) seed[p + c] = (uint8_t)(lane * 4 + c);
    }
    if (lane == 0) seed[4 * nu] = (uint8_t)(27 * 4);
    return 4 * nu + 1;
}

// Warp per interface cell of the window: the reverse sweep; cells it does
// not cover go to the general list (C_ADJGEN).
__global__ void __launch_bounds__(JAC_WARPS * 32) k_kappa_rev(Dev d, Adj a) {
    __shared__ uint8_t sseed[JAC_WARPS][KJ_SEEDS + 3];
    __shared__ float sK[JAC_WARPS][KJ_SEEDS + 3];
    __shared__ int sidx[JAC_WARPS][27];  // window-list position of the 3x3x3 cells used, -1 otherwise
    __shared__ int spos[JAC_WARPS][27];  // their first entry in sK
    __shared__ float sacc[JAC_WARPS][JAC_CELLS + 1];
    int cnt[1];
    block_counts<1>(d.counts, {C_IF0}, cnt);
    const int n = min(cnt[0], a.cap);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < n; k += nwarps) {
        const int i = a.wlist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        uint8_t fj = 0;
        float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int jw = 0;
        if (lane < 27) {
            jw = nbr_index(d, x, y, z, lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1);
            fj = d.flags[jw];
            q4 = d.normal[jw];
        }
        const int ns = seed_list(a, lane, jw, fj, q4, sidx[w], spos[w], sseed[w]);
        __syncwarp();
        float kr;
        float4 g4;
        if (!kappa_reverse(lane, fj, q4, d.fp64_cond, kr, g4)) {
            if (lane == 0) a.glist[atomicAdd(d.counts + C_ADJGEN, 1)] = k;
            __syncwarp();
            continue;
        }
        if (lane < 27 && sidx[w][lane] >= 0) {
            const int p = spos[w][lane];
            sK[w][p] = g4.x;
            sK[w][p + 1] = g4.y;
            sK[w][p + 2] = g4.z;
            sK[w][p + 3] = g4.w;
        }
        if (lane == 0) {
            sK[w][ns - 1] = 0.f;  // theta enters no such fit
            a.jval[k] = kr;
        }
        __syncwarp();
        chain_rows(a, sidx[w], spos[w], sK[w], sacc[w], 0, 1, lane);
        float *jrow = a.jac + (size_t)k * JAC_STRIDE;
        for (int sl = lane; sl < JAC_CELLS; sl += 32) jrow[sl] = sacc[w][sl];
        if (lane == 0) jrow[JAC_CELLS] = sK[w][ns - 1];
        __syncwarp();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && cnt[0] > a.cap) set_status(d.status, FSL_ECAPACITY);
}

// Block per cell of the general list (contact-line cells, degenerate or
// ill-conditioned fits) in FP32 duals, or of the FP64 list in FP64 duals:
// the neighbourhood staged in shared memory, one dual evaluation of
// lsqr_core per seed (at most 109 seeds, one per thread), the chain rule
// split over the warps by slot (partial rows summed in warp order).  An FP32
// fit that is ill conditioned (cond^2 above fp64_cond, as k_lsqr_slow
// decides) moves the cell to the FP64 list.
constexpr int GEN_WARPS = 4;
static_assert(GEN_WARPS * 32 >= KJ_SEEDS, "one seed per thread");

template <typename T, bool FP64>
__global__ void __launch_bounds__(GEN_WARPS * 32) k_kappa_gen(Dev d, Adj a) {
    __shared__ uint8_t sfl[128];
    __shared__ float4 snm[27];
    __shared__ uint8_t sseed[KJ_SEEDS + 3];
    __shared__ float sK[KJ_SEEDS + 3];
    __shared__ int sidx[27], spos[27];
    __shared__ int sns;
    __shared__ float sacc[GEN_WARPS][JAC_CELLS + 1];
    int cnt[1];
    block_counts<1>(d.counts, {FP64 ? C_ADJ64 : C_ADJGEN}, cnt);
    const int n = min(cnt[0], a.cap);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int k = FP64 ? a.dlist[t] : a.glist[t];
        const int i = a.wlist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        const uint8_t fi = d.flags[i];
        if (threadIdx.x < 125) {
            const int e = threadIdx.x;
            sfl[e] = d.flags[nbr_index(d, x, y, z, e % 5 - 2, (e / 5) % 5 - 2, e / 25 - 2)];
        }
        if (w == 0) {
            uint8_t fj = 0;
            float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
            int jw = 0;
            if (lane < 27) {
                jw = nbr_index(d, x, y, z, lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1);
                fj = d.flags[jw];
                q4 = d.normal[jw];
                snm[lane] = q4;
            }
            const int ns = seed_list(a, lane, jw, fj, q4, sidx, spos, sseed);
            if (lane == 0) sns = ns;
        }
        __syncthreads();
        const int ns = sns;
        const int code = (int)threadIdx.x < ns ? (int)sseed[threadIdx.x] : -1;
        const SeedAcc acc{d, sfl, snm, code >= 0 && code < 108 ? code >> 2 : -1, code & 3, code == 108};
        T cond;
        const T kap = lsqr_core<T>(acc, fi, cond);
        if ((int)threadIdx.x < ns) sK[threadIdx.x] = (float)kap.d;
        if (threadIdx.x == 0) a.jval[k] = (float)kap.v;
        // the condition of the fit does not depend on the seed: the same on every thread
        if (__syncthreads_or(!FP64 && (float)(cond.v * cond.v) > d.fp64_cond)) {
            if (threadIdx.x == 0) a.dlist[atomicAdd(d.counts + C_ADJ64, 1)] = k;
            continue;
        }
        chain_rows(a, sidx, spos, sK, sacc[w], w, GEN_WARPS, lane);
        __syncthreads();
        float *jrow = a.jac + (size_t)k * JAC_STRIDE;
        for (int sl = threadIdx.x; sl < JAC_CELLS; sl += blockDim.x) {
            float v = sacc[0][sl];
#pragma unroll
            for (int ww = 1; ww < GEN_WARPS; ++ww) v += sacc[ww][sl];
            jrow[sl] = v;
        }
        if (threadIdx.x == 0) jrow[JAC_CELLS] = sK[ns - 1];
        __syncthreads();  // shared memory is reused by the next cell
    }
}

void launch_kappa_jacobian(const Dev &d, const Adj &a, cudaStream_t s) {
    static const int gn = list_blocks((const void *)k_normal_jac, JAC_WARPS * 32, 4);
    static const int g = list_blocks((const void *)k_kappa_rev, JAC_WARPS * 32, 4);
    static const int g32 = list_blocks((const void *)k_kappa_gen<Dual<float>, false>, GEN_WARPS * 32, 4);
    static const int g64 = list_blocks((const void *)k_kappa_gen<Dual<double>, true>, GEN_WARPS * 32, 2);
    cudaMemsetAsync(d.counts + C_ADJ64, 0, sizeof(int), s);
    cudaMemsetAsync(d.counts + C_ADJGEN, 0, sizeof(int), s);
    k_normal_jac<<<gn, JAC_WARPS * 32, 0, s>>>(d, a);
    k_kappa_rev<<<g, JAC_WARPS * 32, 0, s>>>(d, a);
    k_kappa_gen<Dual<float>, false><<<g32, GEN_WARPS * 32, 0, s>>>(d, a);
    k_kappa_gen<Dual<double>, true><<<g64, GEN_WARPS * 32, 0, s>>>(d, a);
}

// ---- reverse of the stream-collide, boundary condition and mass exchange ---------
// source of direction q of cell (x, y, z): x - c_q (periodic)
__device__ __forceinline__ void adj_sources(const Dev &d, int x, int y, int z, int src[Q]) {
    const int xs[3] = {x == d.nx - 1 ? 0 : x + 1, x, x == 0 ? d.nx - 1 : x - 1};
    const int ys[3] = {y == d.ny - 1 ? 0 : y + 1, y, y == 0 ? d.ny - 1 : y - 1};
    const int zs[3] = {z == d.nz - 1 ? 0 : z + 1, z, z == 0 ? d.nz - 1 : z - 1};
#pragma unroll
    for (int q = 0; q < Q; ++q) src[q] = cell_index(d, xs[cx(q) + 1], ys[cy(q) + 1], zs[cz(q) + 1]);
}

// Interface cells (window list), one thread per cell; recomputes the
// forward step of the cell (as k_sc_iface) and reverses it.  Writes the
// adjoint of the pre-collision PDFs (gb), the cell's own contribution to the
// adjoint of its post-collision PDFs at t (fb_out), the adjoint of m(t+1)
// after the phi = m / rho link (mb, in place: it is also the adjoint of m(t)
// before phi(t) is accounted for), kbar (kb) and the block's sigma partial.
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_iface(Dev d, Adj a) {
    int cnt[1];
    block_counts<1>(d.counts, {C_IF0}, cnt);
    const int n = cnt[0];
    const long long N = d.N;
    const float *fs = static_cast<const float *>(d.fsrc);
    double sig = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = a.wlist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        int src[Q];
        adj_sources(d, x, y, z, src);
        float fo[Q], g[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) fo[q] = __ldg(fs + (long long)q * N + i);
        uint8_t tq[Q];
        bool has_gas = false, has_obs = false;
        float wx = 0.f, wy = 0.f, wz = 0.f;
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
        const float kap = d.kappa[i];
        const float rho_b = d.rho_gas + d.six_sigma * kap;
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
        // forward: g, the link kinds, the exchange weights, dm
        unsigned fluid = 0u, recon = 0u;
        float kw[Q];
        float dm = 0.f;
        g[0] = fo[0];
        kw[0] = 0.f;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const int qb = opp(q);
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float rc = 2.0f * wq(q) * rho_b * (1.0f + 4.5f * cu * cu - uu) - fo[qb];
            kw[q] = 0.f;
            if (tq[q] & (T_LIQ | T_IF)) {
                const float fin = __ldg(fs + (long long)q * N + src[q]);
                g[q] = fin;
                kw[q] = (tq[q] & T_LIQ) ? 1.0f : 0.5f * (phix + d.phi[src[q]]);
                dm += kw[q] * (fin - fo[qb]);
                fluid |= 1u << q;
            } else if (tq[q] & T_OBS) {
                const float outdir = -(cx(q) * ntx + cy(q) * nty + cz(q) * ntz);
                if (corner && outdir < 0.f) {
                    g[q] = rc;
                    recon |= 1u << q;
                } else {
                    g[q] = fo[qb];
                }
            } else {
                g[q] = rc;
                recon |= 1u << q;
            }
        }
        float rho1 = 0.f;
#pragma unroll
        for (int q = 0; q < Q; ++q) rho1 += g[q];
        const float m1 = d.mass[i] + dm;
        // reverse: phi(t+1) = m(t+1) / rho(t+1)
        float fb[Q], gb[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) fb[q] = a.fb_in[(long long)q * N + i];
        const float pb1 = a.pb[i];
        const float mbar = a.mb[i] + pb1 / rho1;
        const float rhobar = -pb1 * m1 / (rho1 * rho1);
        collide_adj(g, fb, d, gb);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            gb[q] += rhobar;
            a.gb[(long long)q * N + i] = gb[q];
        }
        // reverse of the links: own PDFs at t, rho_b, u_b
        float own[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) own[q] = 0.f;
        own[0] = gb[0];
        float rbb = 0.f, ubx = 0.f, uby = 0.f, ubz = 0.f;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const int qb = opp(q);
            if (fluid & (1u << q)) {
                own[qb] -= kw[q] * mbar;
            } else if (recon & (1u << q)) {
                const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
                own[qb] -= gb[q];
                rbb += gb[q] * 2.0f * wq(q) * (1.0f + 4.5f * cu * cu - uu);
                const float s = gb[q] * 2.0f * wq(q) * rho_b;
                ubx += s * (9.0f * cu * cx(q) - 3.0f * ux);
                uby += s * (9.0f * cu * cy(q) - 3.0f * uy);
                ubz += s * (9.0f * cu * cz(q) - 3.0f * uz);
            } else {
                own[qb] += gb[q];
            }
        }
        // u = j / r0 of the own PDFs: du/dfo_r = (c_r - u) / r0
        const float ir0 = 1.0f / r0;
#pragma unroll
        for (int r = 0; r < Q; ++r)
            own[r] += ((cx(r) - ux) * ubx + (cy(r) - uy) * uby + (cz(r) - uz) * ubz) * ir0;
#pragma unroll
        for (int r = 0; r < Q; ++r) a.fb_out[(long long)r * N + i] = own[r];
        a.mb[i] = mbar;
        a.kb[i] = d.six_sigma * rbb;
        sig += 6.0 * (double)kap * (double)rbb;
    }
    const double t = block_sum(sig);
    if (threadIdx.x == 0) a.part[blockIdx.x] = t;
}

// Liquid cells of the active segments: recomputed pull (bounce-back at wall
// links) and the collision adjoint.
__global__ void __launch_bounds__(256) k_adj_bulk(Dev d, Adj a) {
    int cnt[1];
    block_counts<1>(d.counts, {C_SEG}, cnt);
    const int nseg = cnt[0];
    const long long N = d.N;
    const float *fs = static_cast<const float *>(d.fsrc);
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < nseg; k += nw) {
        const int s = d.seg_list[k];
        const int row = s / d.nsegx;
        const int x = (s - row * d.nsegx) * SEG + lane;
        const int z = row / d.ny, y = row - z * d.ny;
        if (x >= d.nx) continue;
        const int i = cell_index(d, x, y, z);
        const uint8_t fl = d.flags[i];
        if (!(fl & T_LIQ)) continue;
        int src[Q];
        adj_sources(d, x, y, z, src);
        float g[Q], fb[Q], gb[Q];
        g[0] = __ldg(fs + i);
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const bool wall = (fl & B_NEAR) && (d.flags[src[q]] & T_OBS);
            g[q] = wall ? __ldg(fs + (long long)opp(q) * N + i) : __ldg(fs + (long long)q * N + src[q]);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) fb[q] = a.fb_in[(long long)q * N + i];
        collide_adj(g, fb, d, gb);
#pragma unroll
        for (int q = 0; q < Q; ++q) a.gb[(long long)q * N + i] = gb[q];
    }
}

// Every fluid cell y of the active segments: the adjoint of f_r(y, t) is
// gathered from its readers.  The cell y + c_r (fluid) pulls it as its g_r;
// an interface cell y + c_r also takes k_r (f_r(y) - ...) into its mass; a
// liquid y at an obstacle link takes it back as g_rbar(y).  Interface y add
// their own part (k_adj_iface) and get the exchange-weight part of the
// adjoint of phi(y): 1/2 sum over interface sources y - c_p of
// (mbar(y) - mbar(y - c_p)) (f_p(y - c_p) - f_pbar(y)).
__global__ void __launch_bounds__(256) k_adj_gather(Dev d, Adj a) {
    int cnt[1];
    block_counts<1>(d.counts, {C_SEG}, cnt);
    const int nseg = cnt[0];
    const long long N = d.N;
    const float *fs = static_cast<const float *>(d.fsrc);
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k = gw; k < nseg; k += nw) {
        const int s = d.seg_list[k];
        const int row = s / d.nsegx;
        const int x = (s - row * d.nsegx) * SEG + lane;
        const int z = row / d.ny, y = row - z * d.ny;
        if (x >= d.nx) continue;
        const int i = cell_index(d, x, y, z);
        const uint8_t fl = d.flags[i];
        if (!(fl & (T_LIQ | T_IF))) continue;
        const bool isif = (fl & T_IF) != 0;
        int src[Q];
        adj_sources(d, x, y, z, src);  // src[opp(r)] = y + c_r
        const float phiy = isif ? d.phi[i] : 1.0f;
        const float mby = isif ? a.mb[i] : 0.f;
        float pbar = 0.f;
        {
            const float v = isif ? 0.f : a.gb[i];
            a.fb_out[i] = isif ? a.fb_out[i] + v : v;
        }
#pragma unroll
        for (int r = 1; r < Q; ++r) {
            const int rb = opp(r);
            const int xn = src[rb];
            const uint8_t tx = d.flags[xn];
            float v = 0.f;
            if (tx & (T_LIQ | T_IF)) {
                v = a.gb[(long long)r * N + xn];
                if (tx & T_IF) v += (isif ? 0.5f * (d.phi[xn] + phiy) : 1.0f) * a.mb[xn];
            } else if ((tx & T_OBS) && !isif) {
                v = a.gb[(long long)rb * N + i];
            }
            const long long o = (long long)r * N + i;
            a.fb_out[o] = isif ? a.fb_out[o] + v : v;
            // exchange weight of the link from the source y - c_r (direction r)
            if (isif && (d.flags[src[r]] & T_IF)) {
                const int sr = src[r];
                pbar += (mby - a.mb[sr]) * (__ldg(fs + (long long)r * N + sr) - __ldg(fs + (long long)rb * N + i));
            }
        }
        if (isif) a.pb[i] = 0.5f * pbar;
    }
}

// Interface cells y (window list), one warp each: the curvature part of the
// adjoint of phi(y), sum over the interface cells x of the 7x7x7 window of
// kbar(x) dkappa_x/dphi_y (row of x, slot of y - x), and the block's theta
// partial kbar(y) dkappa_y/dtheta.
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_curv(Dev d, Adj a) {
    int cnt[1];
    block_counts<1>(d.counts, {C_IF0}, cnt);
    const int n = cnt[0];
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    double th = 0.0;
    for (int k = gw; k < n; k += nwarps) {
        const int i = a.wlist[k];
        int x, y, z;
        cell_coords(d, i, x, y, z);
        float acc = 0.f;
        for (int sl = lane; sl < JAC_CELLS; sl += 32) {
            const int j = nbr_index(d, x, y, z, sl % 7 - 3, (sl / 7) % 7 - 3, sl / 49 - 3);
            if (!(d.flags[j] & T_IF)) continue;
            const int kx = a.widx[j];
            if (kx < 0 || kx >= a.cap) continue;
            acc += a.kb[j] * a.jac[(size_t)kx * JAC_STRIDE + (JAC_CELLS - 1 - sl)];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            a.pb[i] += acc;
            if (k < a.cap) th += (double)a.kb[i] * (double)a.jac[(size_t)k * JAC_STRIDE + JAC_CELLS];
        }
    }
    const double t = block_sum(th);
    if (threadIdx.x == 0) a.part[a.nblk + blockIdx.x] = t;
}

// acc[0] += sum of the sigma partials, acc[1] += sum of the theta partials
// (fixed order)
__global__ void __launch_bounds__(256) k_adj_accum(Adj a, int with_theta) {
    double s = 0.0, t = 0.0;
    for (int b = threadIdx.x; b < a.nblk; b += blockDim.x) {
        s += a.part[b];
        if (with_theta) t += a.part[a.nblk + b];
    }
    s = block_sum(s);
    t = block_sum(t);
    if (threadIdx.x == 0) {
        a.acc[0] += s;
        a.acc[1] += t;
    }
}

// adjoint of phi at the window's end: the interface entries of dL/dphi
__global__ void k_adjoint_seed(Dev d, Adj a, const float *dphi) {
    int cnt[1];
    block_counts<1>(d.counts, {C_IF0}, cnt);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt[0]; k += gridDim.x * blockDim.x) {
        const int i = a.wlist[k];
        a.pb[i] = dphi[i];
    }
}

void launch_adjoint_seed(const Dev &d, const Adj &a, const float *dL_dphi, cudaStream_t s) {
    static const int g = list_blocks((const void *)k_adjoint_seed, 256, 2);
    k_adjoint_seed<<<g, 256, 0, s>>>(d, a, dL_dphi);
}

void launch_adjoint_step(const Dev &d, const Adj &a, cudaStream_t s) {
    const bool lsqr = d.curv_model == FSL_CURV_LSQR;
    if (lsqr) launch_kappa_jacobian(d, a, s);
    static const int gb = resident_grid((const void *)k_adj_bulk, 256);
    static const int gg = resident_grid((const void *)k_adj_gather, 256);
    k_adj_iface<<<a.nblk, ADJ_BLOCK, 0, s>>>(d, a);
    k_adj_bulk<<<gb, 256, 0, s>>>(d, a);
    k_adj_gather<<<gg, 256, 0, s>>>(d, a);
    if (lsqr) k_adj_curv<<<a.nblk, ADJ_BLOCK, 0, s>>>(d, a);
    k_adj_accum<<<1, 256, 0, s>>>(a, lsqr ? 1 : 0);
}

}  // namespace fslk
