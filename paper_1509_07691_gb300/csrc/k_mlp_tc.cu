// k_mlp_tc.cu -- the learned-curvature MLP (125 -> 128 -> 128 -> 1, GELU,
// BF16 weights, FP32 accumulate; see k_mlp.cu) on the 5th-generation tensor
// cores: tcgen05.mma with both operands in shared memory and the FP32
// accumulators in tensor memory (TMEM).  Three kernels: the forward pass over
// a batch of stencils (below), the training step of a 128-row tile, and the
// in-step estimate over the interface list.
//
// One CTA (8 warps) per 128-row tile of the batch, persistent over tiles:
//   layer 1  D1[128 x 128] = X[128 x 128] W1^T   (8 MMAs, M = N = 128, K = 16)
//   epilogue tcgen05.ld of D1 (warp w reads TMEM lanes 32 (w % 4) .. + 31, the
//            column half w / 4), + b1, GELU, BF16 -> H[128 x 128] in shared
//            memory, the A operand of layer 2
//   layer 2  D2 = H W2^T, epilogue + b2, GELU, dot with w3, + b3 -> y
// Operands are stored K-major in the canonical no-swizzle layout: core
// matrices of 8 rows x 16 bytes (8 BF16 along K), core (r8, k8) of a
// 128 x 128 tile at byte (r8 * 16 + k8) * 128.  Completion of the MMAs is
// signalled to an mbarrier by tcgen05.commit; every wait on it is bounded
// and, when it runs out, records FSL_ETIMEOUT, skips the remaining tiles and
// still frees the tensor memory.
#include <math.h>

#include "fsl_internal.cuh"
#include "mlp_common.cuh"

namespace fslk {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TILE = 128;
constexpr int TMEM_COLS = 256;                 // D1 in columns 0..127, D2 in 128..255
constexpr uint32_t CORE_K = 128;               // byte stride between core matrices along K
constexpr uint32_t CORE_MN = 16 * 128;         // byte stride between 8-row groups
constexpr int MB_BIAS_TC = 32896 * 2;          // byte offset of the FP32 biases in the packed block
constexpr long long WAIT_LIMIT = 1ll << 26;    // try_wait polls before a wait gives up

struct TcSmem {
    __nv_bfloat16 W1[TILE * TILE];
    __nv_bfloat16 W2[TILE * TILE];
    __nv_bfloat16 X[TILE * TILE];
    __nv_bfloat16 H[TILE * TILE];
    float b1[TILE], b2[TILE], w3[TILE];
    float ypart[TILE];
    float b3;
    uint32_t tmem_base;
    unsigned long long mbar;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a 128 x 128 K-major tile in the canonical layout
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)(r >> 3) * CORE_MN + (uint32_t)(k >> 3) * CORE_K + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (>> 4), descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ void mbar_init(unsigned long long *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ float gelu_tc(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// copy a row-major [128][128] BF16 matrix (row stride ld elements) into the
// canonical tile layout, 16 bytes at a time; rows >= nrows are zero
__device__ __forceinline__ void load_tile(char *tile, const __nv_bfloat16 *src, long long ld, int nrows) {
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {
        const int r = c >> 4, k8 = c & 15;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < nrows) v = *reinterpret_cast<const uint4 *>(src + (long long)r * ld + k8 * 8);
        *reinterpret_cast<uint4 *>(tile + tile_off(r, k8 * 8)) = v;
    }
}

}  // namespace

// Descriptors: leading byte offset = stride between core matrices along K,
// stride byte offset = stride between 8-row groups (the outputs are checked
// against the FP64 oracle network in the tests).
template <bool STORE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_forward_tc(const uint8_t *params, const __nv_bfloat16 *X, int n,
                                                                  float *y, float *z1, float *z2, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &s = *reinterpret_cast<TcSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lbo = CORE_K, sbo = CORE_MN;
    // weights, biases
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(params);
    const float *bias = reinterpret_cast<const float *>(params + MB_BIAS_TC);
    load_tile(reinterpret_cast<char *>(s.W1), wb, TILE, TILE);
    load_tile(reinterpret_cast<char *>(s.W2), wb + TILE * TILE, TILE, TILE);
    for (int e = threadIdx.x; e < TILE; e += blockDim.x) {
        s.b1[e] = bias[e];
        s.b2[e] = bias[TILE + e];
        s.w3[e] = __bfloat162float(wb[2 * TILE * TILE + e]);
    }
    if (threadIdx.x == 0) {
        s.b3 = bias[2 * TILE];
        s.abort = 0;
        mbar_init(&s.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
    const int row = 32 * (warp & 3) + lane;                         // tile row of this thread
    const int col0 = 64 * (warp >> 2);                              // its column half
    const uint32_t aX = smem_u32(s.X), aH = smem_u32(s.H), aW1 = smem_u32(s.W1), aW2 = smem_u32(s.W2);
    uint32_t phase = 0;
    for (long long t0 = (long long)blockIdx.x * TILE; t0 < n; t0 += (long long)gridDim.x * TILE) {
        const int rows = (int)min((long long)TILE, n - t0);
        load_tile(reinterpret_cast<char *>(s.X), X + t0 * TILE, TILE, rows);
        proxy_fence();
        __syncthreads();
        // ---- layer 1
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk)
                tc_mma(tmem, smem_desc(aX + kk * 2 * CORE_K, lbo, sbo), smem_desc(aW1 + kk * 2 * CORE_K, lbo, sbo),
                       kk > 0);
            tc_commit(&s.mbar);
        }
        if (__syncthreads_or(mbar_wait(&s.mbar, phase) ? 0 : 1)) {
            if (threadIdx.x == 0) set_status(status, FSL_ETIMEOUT);
            break;
        }
        phase ^= 1;
        tc_fence_after();
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + lane_base + c, v);
            uint32_t h[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float za = v[e] + s.b1[c + e], zb = v[e + 1] + s.b1[c + e + 1];
                if (STORE && row < rows) *reinterpret_cast<float2 *>(z1 + (t0 + row) * TILE + c + e) = make_float2(za, zb);
                h[e >> 1] = pack2(gelu_tc(za), gelu_tc(zb));
            }
            *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(s.H) + tile_off(row, c)) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(s.H) + tile_off(row, c + 8)) = make_uint4(h[4], h[5], h[6], h[7]);
        }
        tc_fence_before();
        proxy_fence();
        __syncthreads();
        // ---- layer 2
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk)
                tc_mma(tmem + TILE, smem_desc(aH + kk * 2 * CORE_K, lbo, sbo), smem_desc(aW2 + kk * 2 * CORE_K, lbo, sbo),
                       kk > 0);
            tc_commit(&s.mbar);
        }
        if (__syncthreads_or(mbar_wait(&s.mbar, phase) ? 0 : 1)) {
            if (threadIdx.x == 0) set_status(status, FSL_ETIMEOUT);
            break;
        }
        phase ^= 1;
        tc_fence_after();
        float yp = 0.f;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + TILE + lane_base + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float za = v[e] + s.b2[c + e], zb = v[e + 1] + s.b2[c + e + 1];
                if (STORE && row < rows) *reinterpret_cast<float2 *>(z2 + (t0 + row) * TILE + c + e) = make_float2(za, zb);
                yp += gelu_tc(za) * s.w3[c + e] + gelu_tc(zb) * s.w3[c + e + 1];
            }
        }
        if (warp >= 4) s.ypart[row] = yp;
        tc_fence_before();
        __syncthreads();
        if (warp < 4 && row < rows) y[t0 + row] = yp + s.ypart[row] + s.b3;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---- the learned curvature inside the step, on the tensor cores -----------------
// One CTA (16 warps) per SM, persistent over 128-cell tiles of the interface
// list.  Warp w takes rows 8w .. 8w+7 of a tile: lane r < 8 finds cell r's
// canonical order from its 3x3x3 fill levels, then the warp gathers the 5x5x5
// fill levels of four cells at a time straight into the canonical BF16 rows
// of X (x = 2 phi - 1).  The two layers run as in k_mlp_forward_tc (MMAs into
// TMEM, GELU epilogues; thread (row, column quarter) reads 32 accumulator
// columns), the four quarters' parts of y are summed in order, and the LSQR
// value already in kappa_out judges: the network's value is kept where
// |y - k_lsqr| <= rel |k_lsqr| and no obstacle cell lies in the stencil.
constexpr int CV_THREADS = 512;

struct CvSmem {
    __nv_bfloat16 W1[TILE * TILE];
    __nv_bfloat16 W2[TILE * TILE];
    __nv_bfloat16 X[TILE * TILE];
    __nv_bfloat16 H[TILE * TILE];
    float b1[TILE], b2[TILE], w3[TILE];
    float ypart[4][TILE];
    int cell[TILE];  // interface cell of each row, -1 past the end of the list
    int wall[TILE];  // 1: an obstacle cell in the row's stencil
    float b3;
    uint32_t tmem_base;
    unsigned long long mbar;
};

__global__ void __launch_bounds__(CV_THREADS, 1) k_mlp_curv_tc(Dev d, float *kappa_out, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    CvSmem &s = *reinterpret_cast<CvSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(d.mlp_params);
    const float *bias = reinterpret_cast<const float *>(d.mlp_params + MB_BIAS_TC);
    load_tile(reinterpret_cast<char *>(s.W1), wb, TILE, TILE);
    load_tile(reinterpret_cast<char *>(s.W2), wb + TILE * TILE, TILE, TILE);
    for (int e = threadIdx.x; e < TILE; e += blockDim.x) {
        s.b1[e] = bias[e];
        s.b2[e] = bias[TILE + e];
        s.w3[e] = __bfloat162float(wb[2 * TILE * TILE + e]);
    }
    if (threadIdx.x == 0) {
        s.b3 = bias[2 * TILE];
        mbar_init(&s.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    const int q4 = warp & 3, cq = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;  // this warp's TMEM lanes
    const int row = 32 * q4 + lane;                         // tile row of this thread in the epilogues
    const int col0 = 32 * cq;                               // its 32 accumulator columns
    const uint32_t aX = smem_u32(s.X), aH = smem_u32(s.H), aW1 = smem_u32(s.W1), aW2 = smem_u32(s.W2);
    char *Xb = reinterpret_cast<char *>(s.X);
    uint32_t phase = 0;
    int evaluated = 0, kept = 0;
    for (long long t0 = (long long)blockIdx.x * TILE; t0 < n; t0 += (long long)gridDim.x * TILE) {
        // ---- gather: rows r0 .. r0 + 7 of this warp
        const int r0 = warp * 8;
        int cx0 = 0, cy0 = 0, cz0 = 0, ci = -1;
        CanonAffine ca{0, {0, 0, 0}};
        if (lane < 8 && t0 + r0 + lane < n) {
            ci = d.iflist[t0 + r0 + lane];
            cell_coords(d, ci, cx0, cy0, cz0);
            ca = canon_affine(
                canon_at([&](int dx, int dy, int dz) { return d.phi[nbr_index(d, cx0, cy0, cz0, dx, dy, dz)]; }));
        }
        if (lane < 8) s.cell[r0 + lane] = ci;
        unsigned obsm = 0u;
#pragma unroll 4
        for (int r = 0; r < 8; ++r) {
            const int x = __shfl_sync(0xffffffffu, cx0, r), y = __shfl_sync(0xffffffffu, cy0, r),
                      z = __shfl_sync(0xffffffffu, cz0, r);
            const int cb = __shfl_sync(0xffffffffu, ca.base, r), s0 = __shfl_sync(0xffffffffu, ca.s[0], r),
                      s1 = __shfl_sync(0xffffffffu, ca.s[1], r), s2 = __shfl_sync(0xffffffffu, ca.s[2], r);
            const bool rv = t0 + r0 + r < n;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = lane + 32 * t;
                if (e < 125) {
                    float v = 0.f;
                    if (rv) {
                        const int j = nbr_index(d, x, y, z, e / 25 - 2, (e / 5) % 5 - 2, e % 5 - 2);
                        v = d.phi[j];
                        obsm |= (d.flags[j] & T_OBS) ? (1u << r) : 0u;
                    }
                    const int k = cb + (e / 25) * s0 + ((e / 5) % 5) * s1 + (e % 5) * s2;
                    *reinterpret_cast<__nv_bfloat16 *>(Xb + tile_off(r0 + r, k)) = __float2bfloat16_rn(2.0f * v - 1.0f);
                } else {
                    *reinterpret_cast<__nv_bfloat16 *>(Xb + tile_off(r0 + r, e)) = __float2bfloat16_rn(0.f);
                }
            }
        }
        obsm = __reduce_or_sync(0xffffffffu, obsm);
        if (lane < 8) s.wall[r0 + lane] = (obsm >> lane) & 1u;
        proxy_fence();
        __syncthreads();
        // ---- layer 1
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk)
                tc_mma(tmem, smem_desc(aX + kk * 2 * CORE_K, CORE_K, CORE_MN),
                       smem_desc(aW1 + kk * 2 * CORE_K, CORE_K, CORE_MN), kk > 0);
            tc_commit(&s.mbar);
        }
        if (__syncthreads_or(mbar_wait(&s.mbar, phase) ? 0 : 1)) {
            if (threadIdx.x == 0) set_status(status, FSL_ETIMEOUT);
            break;
        }
        phase ^= 1;
        tc_fence_after();
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + lane_base + c, v);
            uint32_t h[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2)
                h[e >> 1] = pack2(gelu_tc(v[e] + s.b1[c + e]), gelu_tc(v[e + 1] + s.b1[c + e + 1]));
            char *Hb = reinterpret_cast<char *>(s.H);
            *reinterpret_cast<uint4 *>(Hb + tile_off(row, c)) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(Hb + tile_off(row, c + 8)) = make_uint4(h[4], h[5], h[6], h[7]);
        }
        tc_fence_before();
        proxy_fence();
        __syncthreads();
        // ---- layer 2
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk)
                tc_mma(tmem + TILE, smem_desc(aH + kk * 2 * CORE_K, CORE_K, CORE_MN),
                       smem_desc(aW2 + kk * 2 * CORE_K, CORE_K, CORE_MN), kk > 0);
            tc_commit(&s.mbar);
        }
        if (__syncthreads_or(mbar_wait(&s.mbar, phase) ? 0 : 1)) {
            if (threadIdx.x == 0) set_status(status, FSL_ETIMEOUT);
            break;
        }
        phase ^= 1;
        tc_fence_after();
        float yp = 0.f;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + TILE + lane_base + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 2)
                yp += gelu_tc(v[e] + s.b2[c + e]) * s.w3[c + e] + gelu_tc(v[e + 1] + s.b2[c + e + 1]) * s.w3[c + e + 1];
        }
        s.ypart[cq][row] = yp;
        tc_fence_before();
        __syncthreads();
        // ---- the judge
        if (cq == 0) {
            const int i = s.cell[row];
            if (i >= 0 && !s.wall[row]) {
                const float y = ((s.ypart[0][row] + s.ypart[1][row]) + s.ypart[2][row]) + s.ypart[3][row] + s.b3;
                const float kls = kappa_out[i];
                ++evaluated;
                if (fabsf(y - kls) <= d.mlp_rel * fabsf(kls)) {
                    kappa_out[i] = y;
                    ++kept;
                }
            }
        }
        __syncthreads();  // X, H, the row tables and ypart are rewritten by the next tile
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
        kept += __shfl_xor_sync(0xffffffffu, kept, o);
    }
    if (lane == 0 && evaluated) {
        atomicAdd(d.counts + C_MLP, evaluated);
        atomicAdd(d.counts + C_MLPKEEP, kept);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}
// derivative of the GELU (erf form)
__device__ __forceinline__ float gelu_grad_tc(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ---- one training step on the tensor cores, one CTA per 128-row tile --------------
// Forward, loss, deltas and the weight-gradient partials of a tile in one
// kernel: five 128 x 128 x 128 MMA groups on operands kept in shared memory,
// accumulators in TMEM, and the elementwise work in the epilogues between
// them.  Five operand tiles (T0..T4, 32 KB each) change roles as the step
// goes on:
//   load   T0 = X[b][i], T4 = X^T[i][b] (rows gathered through perm),
//          T1 = W1[o][i], T2 = W2[o][h], T3 = W2^T[h][o]
//   L1     D[0..127]   = T0 T1^T            z1 = D + b1
//   E1     T0 = h1[b][h] = bf16(gelu(z1)),  T1 = h1^T[h][b]
//   L2     D[128..255] = T0 T2^T            z2 = D + b2, y = gelu(z2) . w3 + b3
//   E2     d3 = 2 (y - t) / ((t^2 + 7e-5) n), d2 = d3 w3 gelu'(z2) (FP32);
//          T0 = bf16(d2)[b][o], T2 = bf16(d2)^T[o][b]
//   delta  D[256..383] = T0 T3^T  (= d2 W2)  d1 = D gelu'(z1) (FP32), T3 = bf16(d1)^T[o][b]
//   wgrad  D[384..511] = T3 T4^T  (= d1^T X, dW1),  D[128..255] = T2 T1^T  (= d2^T h1, dW2)
//   E4     the tile's partials to part[tile] (PART_STRIDE floats: dW1, dW2,
//          then the column sums of d1, d2, d3 gelu(z2) and d3, that is db1,
//          db2, dw3, db3 at [0]); the tile's loss terms (FP32 terms, FP64 sum
//          in row order) to lpart[tile].
// The operand layouts are those of the forward, delta and weight-gradient
// kernels above (K-major tiles, transposes written element by element).  Column
// sums reduce over the 32 rows of a warp by a fixed shuffle tree and over the
// four row quarters in order.  Rows past the batch end are zero (their deltas
// are 0).  Every MMA wait is bounded; a timeout records FSL_ETIMEOUT, skips the
// rest and still frees the tensor memory.
constexpr int PART_STRIDE = 2 * TILE * TILE + 4 * TILE;
constexpr int FT_THREADS = 512;  // 16 warps: four per TMEM lane quarter, 32 columns each

// Sum over the 32 lanes of a warp of 16 values per lane, scattered: lane l
// returns the total of value l % 16.  A fixed butterfly: each stage a lane
// keeps half of its partial sums and adds its partner's copy of them (8, 4, 2,
// 1 exchanges), then the two lane halves are added.
__device__ __forceinline__ float colsum16(const float (&v)[16]) {
    const int lane = threadIdx.x & 31;
    float a[8], b[4], c[2];
    const bool h8 = (lane & 8) != 0, h4 = (lane & 4) != 0, h2 = (lane & 2) != 0, h1 = (lane & 1) != 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        a[j] = (h8 ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, h8 ? v[j] : v[j + 8], 8);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        b[j] = (h4 ? a[j + 4] : a[j]) + __shfl_xor_sync(0xffffffffu, h4 ? a[j] : a[j + 4], 4);
#pragma unroll
    for (int j = 0; j < 2; ++j)
        c[j] = (h2 ? b[j + 2] : b[j]) + __shfl_xor_sync(0xffffffffu, h2 ? b[j] : b[j + 2], 2);
    const float d = (h1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h1 ? c[0] : c[1], 1);
    return d + __shfl_xor_sync(0xffffffffu, d, 16);
}

struct FtSmem {
    __nv_bfloat16 T[5][TILE * TILE];
    float b1[TILE], b2[TILE], w3[TILE];
    float tgt[TILE], d3[TILE], ypart[4][TILE], lterm[TILE];
    int valid[TILE];
    float colred[4][4][TILE];  // [row quarter][db1, db2, dw3, db3][column]
    float b3;
    uint32_t tmem_base;
    unsigned long long mbar;
};

__global__ void __launch_bounds__(FT_THREADS, 1)
    k_mlp_train_tile(const uint8_t *params, const __nv_bfloat16 *X, const float *target, const int64_t *perm,
                     long long row0, int n, long long n_all, float *part, double *lpart, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FtSmem &s = *reinterpret_cast<FtSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const long long t0 = (long long)tile * TILE;
    const int rows = (int)min((long long)TILE, (long long)n - t0);
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(params);
    const float *bias = reinterpret_cast<const float *>(params + MB_BIAS_TC);
    char *T0 = reinterpret_cast<char *>(s.T[0]), *T1 = reinterpret_cast<char *>(s.T[1]);
    char *T2 = reinterpret_cast<char *>(s.T[2]), *T3 = reinterpret_cast<char *>(s.T[3]);
    char *T4 = reinterpret_cast<char *>(s.T[4]);
    auto source = [&](int r) -> long long {  // stencil row of tile row r, or -1
        if (r >= rows) return -1;
        const long long k = row0 + t0 + r;
        const long long src = perm ? perm[k] : k;
        return (src >= 0 && src < n_all) ? src : -1;
    };
    // ---- load: X and X^T, W1, W2, W2^T, vectors, targets.  The 32 lanes of a
    // warp take 32 rows of one 8-column group: the transposed 2-byte stores
    // then fall on distinct banks (two lanes per 4-byte word).
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {
        const int r = (c & 31) + 32 * ((c >> 9) & 3), k8 = ((c >> 5) & 15) * 8;
        const long long src = source(r);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (src >= 0) v = *reinterpret_cast<const uint4 *>(X + src * TILE + k8);
        *reinterpret_cast<uint4 *>(T0 + tile_off(r, k8)) = v;
        const __nv_bfloat16 *e8 = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int e = 0; e < 8; ++e) *reinterpret_cast<__nv_bfloat16 *>(T4 + tile_off(k8 + e, r)) = e8[e];
    }
    load_tile(T1, wb, TILE, TILE);
    load_tile(T2, wb + TILE * TILE, TILE, TILE);
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {  // T3[h][o] = W2[o][h]
        const int o = (c & 31) + 32 * ((c >> 9) & 3), h8 = ((c >> 5) & 15) * 8;
        const uint4 v = *reinterpret_cast<const uint4 *>(wb + TILE * TILE + o * TILE + h8);
        const __nv_bfloat16 *e8 = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int e = 0; e < 8; ++e) *reinterpret_cast<__nv_bfloat16 *>(T3 + tile_off(h8 + e, o)) = e8[e];
    }
    if (threadIdx.x < TILE) {
        const int e = threadIdx.x;
        s.b1[e] = bias[e];
        s.b2[e] = bias[TILE + e];
        s.w3[e] = __bfloat162float(wb[2 * TILE * TILE + e]);
        const long long src = source(e);
        s.valid[e] = src >= 0;
        s.tgt[e] = src >= 0 ? target[src] : 0.f;
    }
    if (threadIdx.x == 0) {
        s.b3 = bias[2 * TILE];
        mbar_init(&s.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    const int q4 = warp & 3;                                      // row quarter
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;         // this warp's TMEM lanes
    const int row = 32 * q4 + lane;                               // tile row (and, for dW, output o) of this thread
    const int cq = warp >> 2;                                     // its column quarter
    const int col0 = 32 * cq;
    const uint32_t a0 = smem_u32(T0), a1 = smem_u32(T1), a2 = smem_u32(T2), a3 = smem_u32(T3), a4 = smem_u32(T4);
    uint32_t phase = 0;
    bool ok = true;
    auto mma_group = [&](uint32_t dcol, uint32_t aA, uint32_t aB) {
#pragma unroll
        for (int kk = 0; kk < TILE / 16; ++kk)
            tc_mma(tmem + dcol, smem_desc(aA + kk * 2 * CORE_K, CORE_K, CORE_MN),
                   smem_desc(aB + kk * 2 * CORE_K, CORE_K, CORE_MN), kk > 0);
    };
    auto wait_mma = [&]() {
        if (__syncthreads_or(mbar_wait(&s.mbar, phase) ? 0 : 1)) {
            if (threadIdx.x == 0) set_status(status, FSL_ETIMEOUT);
            ok = false;
        }
        phase ^= 1;
        tc_fence_after();
    };
    auto handoff = [&]() {  // epilogue writes to shared memory and TMEM reads done before the next MMAs
        tc_fence_before();
        proxy_fence();
        __syncthreads();
    };
    auto colsum = [&](float v) {  // sum over the 32 rows of this warp, fixed tree
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    // ---- L1
    if (threadIdx.x == 0) {
        tc_fence_after();
        mma_group(0, a0, a1);
        tc_commit(&s.mbar);
    }
    wait_mma();
    if (ok) {  // E1: h1 and h1^T
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + lane_base + c, v);
            uint32_t h[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float ga = gelu_tc(v[e] + s.b1[c + e]), gb = gelu_tc(v[e + 1] + s.b1[c + e + 1]);
                h[e >> 1] = pack2(ga, gb);
                *reinterpret_cast<__nv_bfloat16 *>(T1 + tile_off(c + e, row)) = __float2bfloat16_rn(ga);
                *reinterpret_cast<__nv_bfloat16 *>(T1 + tile_off(c + e + 1, row)) = __float2bfloat16_rn(gb);
            }
            *reinterpret_cast<uint4 *>(T0 + tile_off(row, c)) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(T0 + tile_off(row, c + 8)) = make_uint4(h[4], h[5], h[6], h[7]);
        }
    }
    handoff();
    // ---- L2
    if (ok && threadIdx.x == 0) {
        tc_fence_after();
        mma_group(TILE, a0, a2);
        tc_commit(&s.mbar);
    }
    if (ok) wait_mma();
    if (ok) {  // E2: y, loss term, d3
        float yp = 0.f;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + TILE + lane_base + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float za = v[e] + s.b2[c + e], zb = v[e + 1] + s.b2[c + e + 1];
                yp += gelu_tc(za) * s.w3[c + e] + gelu_tc(zb) * s.w3[c + e + 1];
            }
        }
        s.ypart[cq][row] = yp;
        __syncthreads();
        if (cq == 0) {
            const float y = ((s.ypart[0][row] + s.ypart[1][row]) + s.ypart[2][row]) + s.ypart[3][row] + s.b3;
            const float tt = s.tgt[row], er = y - tt;
            const bool vr = s.valid[row] != 0;
            s.d3[row] = vr ? 2.0f * er / ((tt * tt + 7e-5f) * (float)n) : 0.f;
            s.lterm[row] = vr ? er * er / (tt * tt + 7e-5f) : 0.f;
        }
        __syncthreads();
        // d2 (FP32 for the vector sums, BF16 into T0 and, transposed, T2)
        const float d3r = s.d3[row];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16], dv[16], wv[16];
            tc_ld16(tmem + TILE + lane_base + c, v);
            uint32_t h[8];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float z = v[e] + s.b2[c + e];
                dv[e] = d3r * s.w3[c + e] * gelu_grad_tc(z);
                wv[e] = d3r * gelu_tc(z);
                *reinterpret_cast<__nv_bfloat16 *>(T2 + tile_off(c + e, row)) = __float2bfloat16_rn(dv[e]);
            }
#pragma unroll
            for (int e = 0; e < 16; e += 2) h[e >> 1] = pack2(dv[e], dv[e + 1]);
            *reinterpret_cast<uint4 *>(T0 + tile_off(row, c)) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(T0 + tile_off(row, c + 8)) = make_uint4(h[4], h[5], h[6], h[7]);
            const float sd = colsum16(dv), sw = colsum16(wv);
            if (lane < 16) {
                s.colred[q4][1][c + lane] = sd;
                s.colred[q4][2][c + lane] = sw;
            }
        }
        const float s3 = colsum(d3r);
        if (lane == 0 && cq == 0) s.colred[q4][3][0] = s3;
    }
    handoff();
    // ---- delta: d2 W2
    if (ok && threadIdx.x == 0) {
        tc_fence_after();
        mma_group(2 * TILE, a0, a3);
        tc_commit(&s.mbar);
    }
    if (ok) wait_mma();
    if (ok) {  // E3: d1 = (d2 W2) gelu'(z1); d1^T into T3
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16], z[16], dv[16];
            tc_ld16(tmem + 2 * TILE + lane_base + c, v);
            tc_ld16(tmem + lane_base + c, z);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                dv[e] = v[e] * gelu_grad_tc(z[e] + s.b1[c + e]);
                *reinterpret_cast<__nv_bfloat16 *>(T3 + tile_off(c + e, row)) = __float2bfloat16_rn(dv[e]);
            }
            const float sd = colsum16(dv);
            if (lane < 16) s.colred[q4][0][c + lane] = sd;
        }
    }
    handoff();
    // ---- weight gradients: dW1 = d1^T X, dW2 = d2^T h1
    if (ok && threadIdx.x == 0) {
        tc_fence_after();
        mma_group(3 * TILE, a3, a4);
        mma_group(TILE, a2, a1);
        tc_commit(&s.mbar);
    }
    if (ok) wait_mma();
    if (ok) {  // E4: partials of the tile
        float *P1 = part + (size_t)tile * PART_STRIDE + (size_t)row * TILE;
        float *P2 = P1 + TILE * TILE;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + 3 * TILE + lane_base + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 4) *reinterpret_cast<float4 *>(P1 + c + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            tc_ld16(tmem + TILE + lane_base + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 4) *reinterpret_cast<float4 *>(P2 + c + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        }
        if (threadIdx.x < TILE) {
            const int c = threadIdx.x;
            float *V = part + (size_t)tile * PART_STRIDE + 2 * TILE * TILE;
#pragma unroll
            for (int k = 0; k < 3; ++k) V[k * TILE + c] = ((s.colred[0][k][c] + s.colred[1][k][c]) + s.colred[2][k][c]) + s.colred[3][k][c];
            V[3 * TILE + c] = c == 0 ? ((s.colred[0][3][0] + s.colred[1][3][0]) + s.colred[2][3][0]) + s.colred[3][3][0] : 0.f;
        }
        if (threadIdx.x == 0) {
            double l = 0.0;
            for (int r = 0; r < TILE; ++r) l += (double)s.lterm[r];
            lpart[tile] = l;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

size_t mlp_tc_smem() { return sizeof(TcSmem) + 1024; }

// sticky status of the tensor-core kernels (a bounded wait that ran out)
__device__ int g_mlp_tc_status;

namespace {
int *status_ptr() {  // device address of g_mlp_tc_status, looked up once per device
    static int *ptr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!ptr[dev] && cudaGetSymbolAddress((void **)&ptr[dev], g_mlp_tc_status) != cudaSuccess) ptr[dev] = nullptr;
    return ptr[dev];
}
}  // namespace

// launch on at most one CTA per SM (the tiles and the weights take about
// 133 KB of shared memory), persistent over the 128-row tiles
int launch_mlp_forward_tc(const uint8_t *params, const __nv_bfloat16 *X, int n, float *y, float *z1, float *z2,
                          cudaStream_t s) {
    int *st = status_ptr();
    if (!st) return FSL_ECUDA;
    const size_t sm = mlp_tc_smem();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + TILE - 1) / TILE;
    const int grid = tiles < sms ? (tiles > 0 ? tiles : 1) : sms;
    if (z1) {
        if (cudaFuncSetAttribute(k_mlp_forward_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return FSL_ECUDA;
        k_mlp_forward_tc<true><<<grid, TC_THREADS, sm, s>>>(params, X, n, y, z1, z2, st);
    } else {
        if (cudaFuncSetAttribute(k_mlp_forward_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return FSL_ECUDA;
        k_mlp_forward_tc<false><<<grid, TC_THREADS, sm, s>>>(params, X, n, y, z1, z2, st);
    }
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

size_t mlp_tile_partial_floats(int n) { return (size_t)((n + TILE - 1) / TILE) * PART_STRIDE; }

// one training-step tile kernel per 128 rows of the batch (one CTA per SM at
// about 170 KB of shared memory and 512 TMEM columns)
int launch_mlp_train_tile(const uint8_t *params, const __nv_bfloat16 *X, const float *target, const int64_t *perm,
                          long long row0, int n, long long n_all, float *part, double *lpart, cudaStream_t s) {
    int *st = status_ptr();
    if (!st) return FSL_ECUDA;
    const size_t sm = sizeof(FtSmem) + 1024;
    if (cudaFuncSetAttribute(k_mlp_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return FSL_ECUDA;
    k_mlp_train_tile<<<(n + TILE - 1) / TILE, FT_THREADS, sm, s>>>(params, X, target, perm, row0, n, n_all, part, lpart,
                                                                   st);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

// the learned curvature of the step's interface cells on the tensor cores: one
// CTA per SM (about 135 KB of shared memory, 256 TMEM columns), persistent
// over the 128-cell tiles of the list (its length is read on the device)
int launch_mlp_curv_tc(const Dev &d, float *kappa_out, cudaStream_t s) {
    int *st = status_ptr();
    if (!st) return FSL_ECUDA;
    const size_t sm = sizeof(CvSmem) + 1024;
    static const bool attr =
        cudaFuncSetAttribute(k_mlp_curv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess;
    if (!attr) return FSL_ECUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_mlp_curv_tc<<<sms > 0 ? sms : 1, CV_THREADS, sm, s>>>(d, kappa_out, st);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int mlp_tc_status(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_mlp_tc_status, sizeof v) != cudaSuccess) return FSL_ECUDA;
    if (reset) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_mlp_tc_status, &zero, sizeof zero) != cudaSuccess) return FSL_ECUDA;
    }
    return v;
}

}  // namespace fslk
