// fsl_internal.cuh -- device-side building blocks shared by the FSLBM kernels
// (lattice, cell flags, PDF storage encodings, list appends, kernel argument
// block).  Internal to libfsl; the public ABI is include/fsl.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fsl.h"

namespace fslk {

constexpr int Q = 19;

// D3Q19 lattice (Sec. II), same order as the public header.
__host__ __device__ __forceinline__ constexpr int cx(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
         : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cy(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
         : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cz(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
         : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ __forceinline__ constexpr float wq(int q) {
    return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// cell flag bits: type (public), near-obstacle (public, static), transient (internal)
enum : uint8_t {
    T_LIQ = FSL_LIQUID,
    T_IF = FSL_INTERFACE,
    T_GAS = FSL_GAS,
    T_OBS = FSL_OBSTACLE,
    T_MASK = FSL_TYPE_MASK,
    B_NEAR = FSL_NEAR_OBSTACLE,
    B_TOLIQ = 32,  // interface cell that fills this step
    B_TOGAS = 64,  // interface cell that empties this step
    B_NEW = 128,   // gas or liquid cell that becomes interface this step
};

// device counters in the workspace: interface-list lengths of the two list
// buffers, conversion lists, FP64 LSQR re-solves, active segments, and the
// two "segment set changed" flags (one per step parity: a step sets its own,
// clears the next step's, and rebuilds the segment list only if it is set)
enum { C_IF0 = 0, C_IF1 = 1, C_FILL = 2, C_EMPTY = 3, C_NEWGAS = 4, C_LIQ2IF = 5, C_FP64 = 6, C_SEG = 7, C_SLOW = 8,
       C_MLP = 9, C_MLPKEEP = 10, C_ADJ64 = 11, C_SEGD0 = 12, C_SEGD1 = 13, C_ADJGEN = 14, C_NEAR = 15,
       C_IFDONE = 16, C_NCOUNT = 17 };
// C_NEAR is 1 when some cell has an obstacle neighbour (set with the
// near-obstacle bits at initialisation and refresh; no step changes it);
// C_IFDONE counts the blocks of the fused fit + interface kernel that have
// finished (the last one resets it)

// the grid is walked in x-row segments of SEG cells (one warp each); a
// segment is active while it holds a liquid or interface cell
constexpr int SEG = 32;

// status word values (sticky; first error wins)
__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }

// Programmatic dependent launch along the serial chain of a step.  A kernel
// started with launch_pdl may be dispatched while its predecessor on the
// stream is still running: it calls pdl_wait() before anything else (the wait
// returns once the predecessor grid has completed and its writes are
// visible), then pdl_trigger() so that its own successor can be dispatched
// early in turn.  Both are no-ops in a kernel launched the ordinary way.
#ifndef FSL_PDL
#define FSL_PDL 1
#endif
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), int grid, int block, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = FSL_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// kernel argument block (passed by value)
struct Dev {
    int nx, ny, nz;
    long long N;
    const void *fsrc;  // post-collision PDFs at t
    void *fdst;        // post-collision PDFs at t+1
    uint8_t *flags;    // cell types (+ transient bits during a step), updated in place
    float *mass, *phi, *kappa, *rho, *excess;
    float *exw;        // 1: the converted cell's excess is shared by normal weights (else equally)
    float4 *normal;
    int *iflist;       // interface cells at t
    int *iflist_next;  // interface cells at t+1 (built by the step)
    int cif, cif_next; // their counters
    int cdirty, cdirty_next;  // segment-set-changed flags of this step and the next
    int *fill, *empty, *newgas, *liq2if;
    int *slow;         // interface cells whose LSQR fit takes the general path
    uint8_t *seg_active;
    uint8_t *rmark;    // 1: the cell receives excess mass in this step's final update (0 between steps)
    int *seg_list;
    int nsegx, nseg;
    int *counts;
    double *lost;
    int *status;
    double *partial;
    long long *stats;
    // method parameters
    int collision, storage, plic_iters, curv_model;
    int frozen;              // 1: cell types frozen (no conversion test; adjoint windows)
    int excess_rule;         // 0 equal excess shares, 1 normal-weighted shares
    float omega_e, omega_o;  // 1/tau_even, 1/tau_odd
    float rho_gas, six_sigma, eps;
    float cos_theta, sin_theta;
    float scale, inv_scale;  // 16-bit offset storage
    float fp64_cond;
    // 1: no cell has an obstacle neighbour, so no fit has a contact line and
    // the fused fit + interface kernel finishes its few deferred fits itself
    // (its last block to finish runs them)
    int inline_general;
    double cos_theta_d, sin_theta_d;
    // learned curvature (FSL_CURV_MLP): packed parameters, judge tolerance
    const uint8_t *mlp_params;
    float mlp_rel;
    // bubble model (gas pressure from the gas volume), off when bub_rho is null:
    // bub_i[0..1] liquid cells of the state of each list parity, bub_i[2..3]
    // sum of phi over its interface cells in fixed point (2^-32), bub_i[4]
    // non-obstacle cells; bub_d[0..1] = p0, V0; *bub_rho = 3 p_g of the step
    long long *bub_i;
    double *bub_d;
    float *bub_rho;
};

// fixed-point scale of the bubble model's fill-level sum (integer atomics keep
// the sum independent of the order of the additions)
constexpr double BUB_FIX = 4294967296.0;

// 3 p_g of this step: the bubble model's value, else the constant parameter
__device__ __forceinline__ float gas_density(const Dev &d) { return d.bub_rho ? __ldcg(d.bub_rho) : d.rho_gas; }

// weight of the receiver at x + c of the excess mass of a converted cell with
// interface normal n (into the liquid): a filled cell gives to the gas side,
// an emptied one to the liquid side
__device__ __forceinline__ float excess_weight(const float4 n, bool filled, int ccx, int ccy, int ccz) {
    const float nc = n.x * ccx + n.y * ccy + n.z * ccz;
    return fmaxf(0.f, filled ? -nc : nc);
}

// list parity of the step that d describes (0 or 1)
__device__ __forceinline__ int list_parity(const Dev &d) { return d.cif - C_IF0; }

// Work at the start of a step (or of a curvature pass), by one thread, before
// any kernel of the step appends to a list: zero the step's counters and the
// counter of the list the final update builds, and with the bubble model set
// this step's gas density 3 p_g = 3 p0 V0 / V from the gas volume V =
// non-obstacle cells - liquid cells - interface fill levels of the state the
// step starts from.
__device__ __forceinline__ void step_prologue(const Dev &d) {
    const int zero[9] = {C_FILL, C_EMPTY, C_NEWGAS, C_LIQ2IF, C_SLOW, C_FP64, C_MLP, C_MLPKEEP, C_IFDONE};
#pragma unroll
    for (int k = 0; k < 9; ++k) d.counts[zero[k]] = 0;
    d.counts[d.cif_next] = 0;
    d.counts[d.cdirty_next] = 0;
    if (d.bub_i) {
        const int par = list_parity(d);
        const double V = (double)(d.bub_i[4] - d.bub_i[par]) - (double)d.bub_i[2 + par] / BUB_FIX;
        *d.bub_rho = V > 0.0 ? (float)(3.0 * d.bub_d[0] * d.bub_d[1] / V) : d.rho_gas;
        d.bub_i[2 + (par ^ 1)] = 0;  // the next state's sum, accumulated by the final update
    }
}

// ---- PDF storage -----------------------------------------------------------
template <int S>
struct Store;
template <>
struct Store<FSL_F32> {
    using T = float;
    __device__ static __forceinline__ float ld(const void *p, long long k, int q, const Dev &) {
        return __ldg(static_cast<const float *>(p) + k);
    }
    __device__ static __forceinline__ float ldcg(const void *p, long long k, int q, const Dev &) {
        return __ldcg(static_cast<const float *>(p) + k);
    }
    __device__ static __forceinline__ void st(void *p, long long k, int q, float v, const Dev &) {
        static_cast<float *>(p)[k] = v;
    }
};
template <>
struct Store<FSL_F16_OFS> {
    using T = __half;
    __device__ static __forceinline__ float ld(const void *p, long long k, int q, const Dev &d) {
        return fmaf(__half2float(__ldg(static_cast<const __half *>(p) + k)), d.inv_scale, wq(q));
    }
    __device__ static __forceinline__ float ldcg(const void *p, long long k, int q, const Dev &d) {
        return fmaf(__half2float(__ldcg(static_cast<const __half *>(p) + k)), d.inv_scale, wq(q));
    }
    __device__ static __forceinline__ void st(void *p, long long k, int q, float v, const Dev &d) {
        static_cast<__half *>(p)[k] = __float2half_rn((v - wq(q)) * d.scale);
    }
};
template <>
struct Store<FSL_BF16_OFS> {
    using T = __nv_bfloat16;
    __device__ static __forceinline__ float ld(const void *p, long long k, int q, const Dev &d) {
        return fmaf(__bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(p) + k)), d.inv_scale, wq(q));
    }
    __device__ static __forceinline__ float ldcg(const void *p, long long k, int q, const Dev &d) {
        return fmaf(__bfloat162float(__ldcg(static_cast<const __nv_bfloat16 *>(p) + k)), d.inv_scale, wq(q));
    }
    __device__ static __forceinline__ void st(void *p, long long k, int q, float v, const Dev &d) {
        static_cast<__nv_bfloat16 *>(p)[k] = __float2bfloat16_rn((v - wq(q)) * d.scale);
    }
};

// ---- indexing ----------------------------------------------------------------
__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// cell indices fit in int32 (N < 2^31 is checked at init); only q*N offsets
// into the PDF arrays need 64 bits
__device__ __forceinline__ int cell_index(const Dev &d, int x, int y, int z) { return x + d.nx * (y + d.ny * z); }

__device__ __forceinline__ int nbr_index(const Dev &d, int x, int y, int z, int dx, int dy, int dz) {
    return cell_index(d, wrap(x + dx, d.nx), wrap(y + dy, d.ny), wrap(z + dz, d.nz));
}

__device__ __forceinline__ void cell_coords(const Dev &d, int i, int &x, int &y, int &z) {
    const int row = i / d.nx;
    x = i - row * d.nx;
    z = row / d.ny;
    y = row - z * d.ny;
}

// Warp-aggregated append of `value` to `list` when `pred` holds.  Every lane of
// the warp must call it (no lane may have exited).
__device__ __forceinline__ void warp_append(int *list, int *count, bool pred, int value) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// Device-side list lengths read once per block (by the first threads, from
// L2) and broadcast through shared memory: every warp reading a counter
// itself would queue thousands of requests on the one L2 slice that holds
// it.  Call once per kernel, from all threads, before any early exit.
template <int K>
__device__ __forceinline__ void block_counts(const int *counts, const int (&idx)[K], int (&out)[K]) {
    __shared__ int sh[K];
    if (threadIdx.x < K) sh[threadIdx.x] = __ldcg(counts + idx[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh[k];
}

// Block-aggregated append: one global atomic per block.  Every thread of the
// block must call it (block-uniform control flow; blockDim.x <= 1024).
__device__ __forceinline__ void block_append(int *list, int *count, bool pred, int value) {
    __shared__ int warp_cnt[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
        for (int w = 0; w < nwarp; ++w) {
            const int c = warp_cnt[w];
            warp_cnt[w] = total;
            total += c;
        }
        base = total ? atomicAdd(count, total) : 0;
    }
    __syncthreads();
    if (pred) list[base + warp_cnt[warp] + __popc(m & ((1u << lane) - 1u))] = value;
    __syncthreads();
}

// Loop of a list kernel with a warp-uniform trip count, so that warp_append can
// be used inside: calls body(k, valid) for k = base + lane.
template <typename Body>
__device__ __forceinline__ void warp_uniform_loop(int n, Body body) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int base = gwarp * 32; base < n; base += nwarps * 32) body(base + lane, base + lane < n);
}

__device__ __forceinline__ int seg_of(const Dev &d, int i) {
    const int row = i / d.nx;
    return (i - row * d.nx) / SEG + d.nsegx * row;
}

// ---- launch wrappers (defined in the .cu files) -------------------------------
void launch_fill_geometry(const fsl_params &p, const fsl_geometry &g, float *phi, cudaStream_t s);
void launch_init_types(const Dev &d, const uint8_t *obstacle, uint8_t *tmp, cudaStream_t s);
void launch_init_state(const Dev &d, const uint8_t *tmp, cudaStream_t s);
void launch_refresh(const Dev &d, cudaStream_t s);
// f' = feq(rho, u) at the liquid and interface cells of the buffer d.fdst
void launch_prescribe(const Dev &d, float rho, float ux, float uy, float uz, cudaStream_t s);
void launch_seg_compact(const Dev &d, cudaStream_t s);
void launch_stats(const Dev &d, cudaStream_t s);
void launch_mass(const Dev &d, double *out, cudaStream_t s);
void launch_stream_collide(const Dev &d, cudaStream_t s);
void launch_sc_bulk(const Dev &d, cudaStream_t s);
void launch_sc_iface(const Dev &d, cudaStream_t s);
// LSQR curvature and interface stream-collide in one pass (after launch_normals)
void launch_curv_iface(const Dev &d, cudaStream_t s);
void launch_convert(const Dev &d, cudaStream_t s);
void launch_finalize(const Dev &d, cudaStream_t s);
void launch_normals(const Dev &d, cudaStream_t s);
void launch_lsqr(const Dev &d, float *kappa_out, cudaStream_t s);
void launch_fd(const Dev &d, float *kappa_out, cudaStream_t s);
void launch_tr(const Dev &d, float *kappa_out, cudaStream_t s);
void launch_zero_kappa(const Dev &d, float *kappa_out, cudaStream_t s);
void launch_mlp_curv(const Dev &d, float *kappa_out, cudaStream_t s);
// batch forward of the MLP on the tcgen05 tensor cores (k_mlp_tc.cu)
int launch_mlp_forward_tc(const uint8_t *params, const __nv_bfloat16 *X, int n, float *y, float *z1, float *z2,
                          cudaStream_t s);
int mlp_tc_status(bool reset);
// one training step's forward, deltas and gradient partials on the tensor cores,
// one CTA per 128 rows of the batch (rows perm[row0 ..] of X, or row0 .. when
// perm is null); part holds mlp_tile_partial_floats(n) floats, lpart one double per tile
size_t mlp_tile_partial_floats(int n);
int launch_mlp_train_tile(const uint8_t *params, const __nv_bfloat16 *X, const float *target, const int64_t *perm,
                          long long row0, int n, long long n_all, float *part, double *lpart, cudaStream_t s);
void launch_fin_frozen(const Dev &d, cudaStream_t s);
// bubble model: liquid cells, non-obstacle cells and the fixed-point fill-level
// sum of the current state into d.bub_i (entries of the current parity and [4])
void launch_bubble_count(const Dev &d, cudaStream_t s);


int max_partials();
// blocks of `block` threads of `kernel` that are resident on the whole GPU at once
int resident_grid(const void *kernel, int block, size_t smem = 0);
// grid of the list kernels: `per_sm` blocks per SM, capped at the resident grid
int list_blocks(const void *kernel, int block, int per_sm);

}  // namespace fslk
