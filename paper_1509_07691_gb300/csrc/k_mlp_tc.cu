// k_mlp_tc.cu -- forward pass of the learned-curvature MLP (125 -> 128 -> 128
// -> 1, GELU, BF16 weights, FP32 accumulate; see k_mlp.cu) over a batch of
// stencils on the 5th-generation tensor cores: tcgen05.mma with both operands
// in shared memory and the FP32 accumulators in tensor memory (TMEM).
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
// stride byte offset = stride between 8-row groups (checked against the
// mma.sync network: identical pre-activations).
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

// ---- weight gradients on the tensor cores -------------------------------------
// dW1[o][i] = sum_b d1[b][o] x[b][i] and dW2[o][i] = sum_b d2[b][o] h1[b][i]
// (h1 = bf16(gelu(z1)), as the forward feeds layer 2): one CTA per 128-sample
// chunk of the batch and matrix, an MMA group with M = o, N = i, K = b over
// the chunk (both operands staged transposed into the K-major tile, in BF16),
// the 128 x 128 partial written to partial[mat][chunk]; k_mlp_wreduce sums
// the chunks in a fixed order.
struct WgSmem {
    __nv_bfloat16 A[TILE * TILE];
    __nv_bfloat16 B[TILE * TILE];
    uint32_t tmem_base;
    unsigned long long mbar;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_wgrad_tc(const __nv_bfloat16 *X, const float *z1, const float *d1,
                                                               const float *d2, int n, float *partial, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    WgSmem &s = *reinterpret_cast<WgSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mat = blockIdx.y, chunk = blockIdx.x, nchunk = gridDim.x;
    const long long b0 = (long long)chunk * TILE;
    const int rows = (int)min((long long)TILE, n - b0);
    const float *D = mat == 0 ? d1 : d2;
    char *At = reinterpret_cast<char *>(s.A), *Bt = reinterpret_cast<char *>(s.B);
    // A[o][b] = D[b0 + b][o], B[i][b] = x or h1 at [b0 + b][i]: thread per (b, 8 columns)
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {
        const int b = c >> 4, c8 = (c & 15) * 8;
        float av[8], bv[8];
        if (b < rows) {
            const float4 a0 = *reinterpret_cast<const float4 *>(D + (b0 + b) * TILE + c8);
            const float4 a1 = *reinterpret_cast<const float4 *>(D + (b0 + b) * TILE + c8 + 4);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w; av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            if (mat == 0) {
#pragma unroll
                for (int e = 0; e < 8; ++e) bv[e] = __bfloat162float(X[(b0 + b) * TILE + c8 + e]);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) bv[e] = gelu_tc(z1[(b0 + b) * TILE + c8 + e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) av[e] = bv[e] = 0.f;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            *reinterpret_cast<__nv_bfloat16 *>(At + tile_off(c8 + e, b)) = __float2bfloat16_rn(av[e]);
            *reinterpret_cast<__nv_bfloat16 *>(Bt + tile_off(c8 + e, b)) = __float2bfloat16_rn(bv[e]);
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&s.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(TILE)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t aA = smem_u32(s.A), aB = smem_u32(s.B);
#pragma unroll
        for (int kk = 0; kk < TILE / 16; ++kk)
            tc_mma(tmem, smem_desc(aA + kk * 2 * CORE_K, CORE_K, CORE_MN), smem_desc(aB + kk * 2 * CORE_K, CORE_K, CORE_MN),
                   kk > 0);
        tc_commit(&s.mbar);
    }
    const bool ok = !__syncthreads_or(mbar_wait(&s.mbar, 0) ? 0 : 1);
    if (ok) {
        tc_fence_after();
        const int o = 32 * (warp & 3) + lane, col0 = 64 * (warp >> 2);
        float *P = partial + ((size_t)mat * nchunk + chunk) * TILE * TILE + (size_t)o * TILE;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c, v);
#pragma unroll
            for (int e = 0; e < 16; e += 4) *reinterpret_cast<float4 *>(P + c + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        }
    } else if (threadIdx.x == 0) {
        set_status(status, FSL_ETIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TILE) : "memory");
}

// ---- deltas on the tensor cores ------------------------------------------------
// d3 = dL/dy = 2 (y - t) / ((t^2 + 7e-5) n), d2 = d3 w3 gelu'(z2) (FP32, as
// stored for the weight and bias gradients), d1 = (d2 W2) gelu'(z1) with the
// product d2 W2 as an MMA: M = sample b, N = i, K = o, d2 rounded to BF16,
// W2 staged transposed (B[i][o] = W2[o][i]).  One CTA per 128-sample chunk.
__device__ __forceinline__ float gelu_grad_tc(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

struct DtSmem {
    __nv_bfloat16 A[TILE * TILE];
    __nv_bfloat16 B[TILE * TILE];
    float w3[TILE];
    float d3[TILE];
    uint32_t tmem_base;
    unsigned long long mbar;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_delta_tc(const uint8_t *params, const float *y, const float *target,
                                                               int n, const float *z1, const float *z2, float *d1,
                                                               float *d2, float *d3, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    DtSmem &s = *reinterpret_cast<DtSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long b0 = (long long)blockIdx.x * TILE;
    const int rows = (int)min((long long)TILE, n - b0);
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(params);
    char *At = reinterpret_cast<char *>(s.A), *Bt = reinterpret_cast<char *>(s.B);
    if (threadIdx.x < TILE) {
        const int b = threadIdx.x;
        s.w3[b] = __bfloat162float(wb[2 * TILE * TILE + b]);
        float v = 0.f;
        if (b < rows) {
            const float tt = target[b0 + b];
            v = 2.0f * (y[b0 + b] - tt) / ((tt * tt + 7e-5f) * (float)n);
            d3[b0 + b] = v;
        }
        s.d3[b] = v;
    }
    // B[i][o] = W2[o][i]: thread per (o, 8 consecutive i)
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {
        const int o = c >> 4, i8 = (c & 15) * 8;
        const uint4 v = *reinterpret_cast<const uint4 *>(wb + TILE * TILE + o * TILE + i8);
        const __nv_bfloat16 *e8 = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int e = 0; e < 8; ++e) *reinterpret_cast<__nv_bfloat16 *>(Bt + tile_off(i8 + e, o)) = e8[e];
    }
    __syncthreads();
    // d2 (FP32 to memory, BF16 into A[b][o])
    for (int c = threadIdx.x; c < TILE * TILE / 8; c += blockDim.x) {
        const int b = c >> 4, o8 = (c & 15) * 8;
        uint32_t h[4];
        if (b < rows) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = s.d3[b] * s.w3[o8 + e] * gelu_grad_tc(z2[(b0 + b) * TILE + o8 + e]);
            *reinterpret_cast<float4 *>(d2 + (b0 + b) * TILE + o8) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4 *>(d2 + (b0 + b) * TILE + o8 + 4) = make_float4(v[4], v[5], v[6], v[7]);
#pragma unroll
            for (int e = 0; e < 4; ++e) h[e] = pack2(v[2 * e], v[2 * e + 1]);
        } else {
            h[0] = h[1] = h[2] = h[3] = 0u;
        }
        *reinterpret_cast<uint4 *>(At + tile_off(b, o8)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
    if (threadIdx.x == 0) {
        mbar_init(&s.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(TILE)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t aA = smem_u32(s.A), aB = smem_u32(s.B);
#pragma unroll
        for (int kk = 0; kk < TILE / 16; ++kk)
            tc_mma(tmem, smem_desc(aA + kk * 2 * CORE_K, CORE_K, CORE_MN), smem_desc(aB + kk * 2 * CORE_K, CORE_K, CORE_MN),
                   kk > 0);
        tc_commit(&s.mbar);
    }
    const bool ok = !__syncthreads_or(mbar_wait(&s.mbar, 0) ? 0 : 1);
    if (ok) {
        tc_fence_after();
        const int b = 32 * (warp & 3) + lane, col0 = 64 * (warp >> 2);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = col0 + 16 * cc;
            float v[16];
            tc_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c, v);
            if (b < rows) {
                const float *zr = z1 + (b0 + b) * TILE + c;
                float *dr = d1 + (b0 + b) * TILE + c;
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                    *reinterpret_cast<float4 *>(dr + e) =
                        make_float4(v[e] * gelu_grad_tc(zr[e]), v[e + 1] * gelu_grad_tc(zr[e + 1]),
                                    v[e + 2] * gelu_grad_tc(zr[e + 2]), v[e + 3] * gelu_grad_tc(zr[e + 3]));
            }
        }
    } else if (threadIdx.x == 0) {
        set_status(status, FSL_ETIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TILE) : "memory");
}

// grad[off + e] = sum over chunks of partial[mat][chunk][e], chunks in order
__global__ void __launch_bounds__(256) k_mlp_wreduce(const float *partial, int nchunk, float *gW1, float *gW2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * TILE * TILE) return;
    const int mat = e / (TILE * TILE), k = e % (TILE * TILE);
    const float *P = partial + (size_t)mat * nchunk * TILE * TILE + k;
    float acc = 0.f;
    for (int c = 0; c < nchunk; ++c) acc += P[(size_t)c * TILE * TILE];
    (mat == 0 ? gW1 : gW2)[k] = acc;
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

size_t mlp_wgrad_partial_floats(int n) { return (size_t)2 * ((n + TILE - 1) / TILE) * TILE * TILE; }

int launch_mlp_wgrad_tc(const __nv_bfloat16 *X, const float *z1, const float *d1, const float *d2, int n, float *partial,
                        float *gW1, float *gW2, cudaStream_t s) {
    int *st = status_ptr();
    if (!st) return FSL_ECUDA;
    const int nchunk = (n + TILE - 1) / TILE;
    const size_t sm = sizeof(WgSmem) + 1024;
    if (cudaFuncSetAttribute(k_mlp_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return FSL_ECUDA;
    k_mlp_wgrad_tc<<<dim3(nchunk, 2), TC_THREADS, sm, s>>>(X, z1, d1, d2, n, partial, st);
    k_mlp_wreduce<<<(2 * TILE * TILE + 255) / 256, 256, 0, s>>>(partial, nchunk, gW1, gW2);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int launch_mlp_delta_tc(const uint8_t *params, const float *y, const float *target, int n, const float *z1,
                        const float *z2, float *d1, float *d2, float *d3, cudaStream_t s) {
    int *st = status_ptr();
    if (!st) return FSL_ECUDA;
    const size_t sm = sizeof(DtSmem) + 1024;
    if (cudaFuncSetAttribute(k_mlp_delta_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return FSL_ECUDA;
    k_mlp_delta_tc<<<(n + TILE - 1) / TILE, TC_THREADS, sm, s>>>(params, y, target, n, z1, z2, d1, d2, d3, st);
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
