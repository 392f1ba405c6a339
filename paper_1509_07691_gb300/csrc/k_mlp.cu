// k_mlp.cu -- learned curvature on the 5x5x5 fill-level stencil: training
// stencils, the MLP 125 -> 128 -> 128 -> 1 (GELU) with BF16 weights, its FP32
// backward and Adam, and the in-step estimate that keeps the LSQR fit
// (Sec. II.C) as judge and fallback.  The batch forward (training, checks)
// runs on the tcgen05 tensor cores (k_mlp_tc.cu); the in-step estimate, which
// gathers 16 stencils per warp from the grid, on mma.sync m16n8k16 here.
//
// Network (packed parameter block, see include/fsl.h):
//   x = bf16(2 phi - 1) over the canonical stencil (125 values, 3 zero pads)
//   z1 = W1 x + b1, h1 = bf16(gelu(z1)), z2 = W2 h1 + b2, h2 = gelu(z2),
//   y = w3 . h2 + b3 = kappa dx;   gelu(x) = x Phi(x) (erf form)
// Canonical stencil: axes flipped so the Parker-Youngs normal of the middle
// cell has non-negative components, then ordered by decreasing |n_k|.
#include <math.h>

#include "fsl_internal.cuh"

namespace fslk {

constexpr int MK = 128;     // padded input width, hidden width
constexpr int WPAD = 136;   // bf16 row stride of the shared-memory tiles
constexpr int MB_BF = 32896;  // bf16 elements of W1 | W2 | w3
constexpr size_t MB_BIAS = (size_t)MB_BF * 2;  // byte offset of the FP32 biases (256-aligned)
// FP32 master / gradient / moment layout
constexpr int M_W1 = 0, M_W2 = 16384, M_W3 = 32768, M_B1 = 32896, M_B2 = 33024, M_B3 = 33152, M_COUNT = 33153;
static_assert(M_W1 == 0 && M_W2 == M_W1 + MK * MK && M_W3 == M_W2 + MK * MK && M_B1 == MB_BF && M_B2 == M_B1 + MK &&
                  M_B3 == M_B2 + MK && M_COUNT == M_B3 + 1,
              "master layout: W1, W2, w3, b1, b2, b3 (the tile partials use the same order)");
constexpr int MLP_WARPS = 4, MLP_ROWS = 16 * MLP_WARPS;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// D = A B + D for A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct MlpSmem {  // size a multiple of 16 bytes: the activation tiles follow it
    __nv_bfloat16 W1[MK * WPAD];
    __nv_bfloat16 W2[MK * WPAD];
    float b1[MK], b2[MK], w3[MK];
    float b3, pad_[3];
};
static_assert(sizeof(MlpSmem) % 16 == 0, "shared-memory tiles after MlpSmem must stay 16-byte aligned");

// cooperative copy of the packed parameters into shared memory
__device__ void load_weights(MlpSmem &s, const uint8_t *params) {
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(params);
    const float *bias = reinterpret_cast<const float *>(params + MB_BIAS);
    for (int e = threadIdx.x; e < MK * MK / 2; e += blockDim.x) {
        const int r = (2 * e) / MK, c = (2 * e) % MK;
        *reinterpret_cast<uint32_t *>(&s.W1[r * WPAD + c]) = reinterpret_cast<const uint32_t *>(wb)[e];
        *reinterpret_cast<uint32_t *>(&s.W2[r * WPAD + c]) = reinterpret_cast<const uint32_t *>(wb + MK * MK)[e];
    }
    for (int e = threadIdx.x; e < MK; e += blockDim.x) {
        s.b1[e] = bias[e];
        s.b2[e] = bias[MK + e];
        s.w3[e] = __bfloat162float(wb[2 * MK * MK + e]);
    }
    if (threadIdx.x == 0) s.b3 = bias[2 * MK];
}

// One warp: the 16 rows of Xw ([16][WPAD], bf16) through the network.  Lanes
// with (lane & 3) == 0 return y of rows lane/4 (y_lo) and lane/4 + 8 (y_hi).
// With z1/z2 given (training), the pre-activations of the rows r < nvalid are
// stored at z[(row0 + r) * 128 + col].
template <bool STORE>
__device__ void warp_mlp(const MlpSmem &s, const __nv_bfloat16 *Xw, float &y_lo, float &y_hi, float *z1, float *z2,
                         long long row0, int nvalid) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const int k0 = kt * 16 + 2 * t;
        const uint32_t a[4] = {ld32(Xw + g * WPAD + k0), ld32(Xw + (g + 8) * WPAD + k0), ld32(Xw + g * WPAD + k0 + 8),
                               ld32(Xw + (g + 8) * WPAD + k0 + 8)};
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const __nv_bfloat16 *w = s.W1 + (nt * 8 + g) * WPAD + k0;
            mma_bf16(acc[nt], a, ld32(w), ld32(w + 8));
        }
    }
    // bias, GELU, BF16: the C fragments of n-tiles 2j, 2j+1 are the A fragment of k-tile j
    uint32_t h1[8][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float za = acc[nt][0] + s.b1[col], zb = acc[nt][1] + s.b1[col + 1];
        const float zc = acc[nt][2] + s.b1[col], zd = acc[nt][3] + s.b1[col + 1];
        if (STORE) {
            if (g < nvalid) *reinterpret_cast<float2 *>(z1 + (row0 + g) * MK + col) = make_float2(za, zb);
            if (g + 8 < nvalid) *reinterpret_cast<float2 *>(z1 + (row0 + g + 8) * MK + col) = make_float2(zc, zd);
        }
        const uint32_t lo = pack_bf16(gelu(za), gelu(zb)), hi = pack_bf16(gelu(zc), gelu(zd));
        if ((nt & 1) == 0) {
            h1[nt >> 1][0] = lo;
            h1[nt >> 1][1] = hi;
        } else {
            h1[nt >> 1][2] = lo;
            h1[nt >> 1][3] = hi;
        }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const int k0 = kt * 16 + 2 * t;
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const __nv_bfloat16 *w = s.W2 + (nt * 8 + g) * WPAD + k0;
            mma_bf16(acc[nt], h1[kt], ld32(w), ld32(w + 8));
        }
    }
    float ylo = 0.f, yhi = 0.f;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float za = acc[nt][0] + s.b2[col], zb = acc[nt][1] + s.b2[col + 1];
        const float zc = acc[nt][2] + s.b2[col], zd = acc[nt][3] + s.b2[col + 1];
        if (STORE) {
            if (g < nvalid) *reinterpret_cast<float2 *>(z2 + (row0 + g) * MK + col) = make_float2(za, zb);
            if (g + 8 < nvalid) *reinterpret_cast<float2 *>(z2 + (row0 + g + 8) * MK + col) = make_float2(zc, zd);
        }
        ylo += gelu(za) * s.w3[col] + gelu(zb) * s.w3[col + 1];
        yhi += gelu(zc) * s.w3[col] + gelu(zd) * s.w3[col + 1];
    }
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 1);
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 2);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 1);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 2);
    y_lo = ylo + s.b3;
    y_hi = yhi + s.b3;
}



// ---- training: gradient reduction and Adam --------------------------------------
// (forward, deltas and the per-tile gradient partials run on the tensor cores
// in k_mlp_train_tile, k_mlp_tc.cu)
// Sum of the per-tile partials of k_mlp_train_tile in tile order into the
// gradient (master layout), and, with master != null, the Adam step on it in
// the same thread (as k_mlp_adam).  Thread 0 also sums the tiles' loss terms.
constexpr int PART_STRIDE = 2 * MK * MK + 4 * MK;  // floats of one tile's partials

__global__ void __launch_bounds__(256) k_mlp_tile_reduce(const float *part, const double *lpart, int ntiles, int n,
                                                         float *grad, float *loss,
                                                         uint8_t *params, float *master, float *m, float *v, float lr,
                                                         float bc1, float bc2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0 && loss) {
        double l = 0.0;
        for (int t = 0; t < ntiles; ++t) l += lpart[t];
        loss[0] = (float)(l / n);
    }
    if (e >= M_COUNT) return;
    float acc = 0.f;
    if (e < M_W3) {
        const int mat = e / (MK * MK), k = e % (MK * MK);
        const float *P = part + (size_t)mat * MK * MK + k;
        for (int t = 0; t < ntiles; ++t) acc += P[(size_t)t * PART_STRIDE];
    } else {
        int vec, c = 0;
        if (e < M_B1) { vec = 2; c = e - M_W3; }
        else if (e < M_B2) { vec = 0; c = e - M_B1; }
        else if (e < M_B3) { vec = 1; c = e - M_B2; }
        else { vec = 3; }
        const float *P = part + (size_t)2 * MK * MK + (size_t)vec * MK + c;
        for (int t = 0; t < ntiles; ++t) acc += P[(size_t)t * PART_STRIDE];
    }
    if (grad) grad[e] = acc;
    if (master) {
        __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(params);
        float *bias = reinterpret_cast<float *>(params + MB_BIAS);
        const float mm = 0.9f * m[e] + 0.1f * acc, vv = 0.999f * v[e] + 0.001f * acc * acc;
        m[e] = mm;
        v[e] = vv;
        const float w = master[e] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
        master[e] = w;
        if (e < M_B1) wb[e] = __float2bfloat16_rn(w);
        else bias[e - M_B1] = w;
    }
}

// master parameters -> packed BF16 weights and FP32 biases
__global__ void __launch_bounds__(256) k_mlp_pack(const float *master, uint8_t *params) {
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(params);
    float *bias = reinterpret_cast<float *>(params + MB_BIAS);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M_COUNT; e += gridDim.x * blockDim.x) {
        if (e < M_B1) wb[e] = __float2bfloat16_rn(master[e]);
        else bias[e - M_B1] = master[e];
    }
}

// ---- training stencils ---------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform_at(unsigned long long seed, unsigned long long k) {
    return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

// canonical placement of a 5x5x5 stencil s[(i*5 + j)*5 + k] (x = i, y = j, z = k):
// returns, for each raw element, its index in the canonical ordering
struct Canon {
    int flip[3], order[3];
};
__device__ Canon canon_of(const float *s) {
    float n[3] = {0.f, 0.f, 0.f};
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                const float v = s[((2 + dx) * 5 + 2 + dy) * 5 + 2 + dz];
                if (dx) n[0] += dx * (dy == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dy) n[1] += dy * (dx == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dz) n[2] += dz * (dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1) * v;
            }
    Canon c;
    for (int k = 0; k < 3; ++k) c.flip[k] = n[k] < 0.f;
    // order axes by decreasing |n|, lower index first on ties
    const float a0 = fabsf(n[0]), a1 = fabsf(n[1]), a2 = fabsf(n[2]);
    int o0 = 0, o1 = 1, o2 = 2;
    float m0 = a0, m1 = a1, m2 = a2, tf;
    int ti;
    if (m1 > m0) { tf = m0; m0 = m1; m1 = tf; ti = o0; o0 = o1; o1 = ti; }
    if (m2 > m1) { tf = m1; m1 = m2; m2 = tf; ti = o1; o1 = o2; o2 = ti; }
    if (m1 > m0) { tf = m0; m0 = m1; m1 = tf; ti = o0; o0 = o1; o1 = ti; }
    c.order[0] = o0;
    c.order[1] = o1;
    c.order[2] = o2;
    return c;
}
__device__ __forceinline__ int canon_index(const Canon &c, int e) {
    int r[3] = {e / 25, (e / 5) % 5, e % 5};
    for (int k = 0; k < 3; ++k)
        if (c.flip[k]) r[k] = 4 - r[k];
    return r[c.order[0]] * 25 + r[c.order[1]] * 5 + r[c.order[2]];
}
// The same map as an affine function of the raw coordinates (r0, r1, r2) =
// (e / 25, e / 5 % 5, e % 5): canonical = base + r0 s0 + r1 s1 + r2 s2, with
// s_k = +-(the weight 25, 5 or 1 of the place axis k takes) and the flips
// folded into base.  Per stencil the four numbers, per element three
// multiply-adds.
struct CanonAffine {
    int base, s[3];
};
__device__ __forceinline__ CanonAffine canon_affine(const Canon &c) {
    CanonAffine a;
    a.base = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int w = c.order[0] == k ? 25 : (c.order[1] == k ? 5 : 1);
        a.s[k] = c.flip[k] ? -w : w;
        a.base += c.flip[k] ? 4 * w : 0;
    }
    return a;
}

// mean curvature at the point of the ellipsoid sum (y/a)^2 = 1 (body frame)
// nearest to o (body frame): x_k = a_k^2 o_k / (a_k^2 + t), bisection on t
__device__ double nearest_mean_curvature(const double a[3], const double o[3]) {
    double lo = -fmin(a[0] * a[0], fmin(a[1] * a[1], a[2] * a[2])) * (1.0 - 1e-15);
    double hi = fmax(1.0, fmax(fabs(o[0]), fmax(fabs(o[1]), fabs(o[2]))) * fmax(a[0], fmax(a[1], a[2])));
    auto gfun = [&](double t) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double q = a[k] * o[k] / (a[k] * a[k] + t);
            s += q * q;
        }
        return s - 1.0;
    };
    for (int it = 0; it < 64 && gfun(hi) > 0.0; ++it) hi *= 2.0;
    for (int it = 0; it < 100; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (gfun(mid) > 0.0) lo = mid;
        else hi = mid;
    }
    const double t = 0.5 * (lo + hi);
    double gr[3], hs[3], gn2 = 0.0, trh = 0.0, ghg = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double x = a[k] * a[k] * o[k] / (a[k] * a[k] + t);
        gr[k] = 2.0 * x / (a[k] * a[k]);
        hs[k] = 2.0 / (a[k] * a[k]);
        gn2 += gr[k] * gr[k];
        trh += hs[k];
        ghg += gr[k] * gr[k] * hs[k];
    }
    const double gn = sqrt(gn2);
    return (gn2 * trh - ghg) / (2.0 * gn2 * gn);
}

// one block per stencil: thread e < 125 samples cell e
__global__ void __launch_bounds__(128) k_mlp_stencils(int n, const float *axes, const float *quat, const float *dir,
                                                      const float *delta, const int *invert, int sub, float noise,
                                                      unsigned long long noise_seed, __nv_bfloat16 *X, float *target) {
    __shared__ float Rm[9], C[3], ax[3];
    __shared__ float st[125];
    __shared__ Canon cs;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const double w = quat[4 * k], x = quat[4 * k + 1], y = quat[4 * k + 2], z = quat[4 * k + 3];
            const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                                 2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                                 2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
            const double a[3] = {axes[3 * k], axes[3 * k + 1], axes[3 * k + 2]};
            const double d[3] = {dir[3 * k], dir[3 * k + 1], dir[3 * k + 2]};
            const double sc = 1.0 / sqrt((d[0] / a[0]) * (d[0] / a[0]) + (d[1] / a[1]) * (d[1] / a[1]) +
                                         (d[2] / a[2]) * (d[2] / a[2]));
            double c[3], o[3];
            for (int r = 0; r < 3; ++r) {
                c[r] = delta[3 * k + r] - (R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2]) * sc;
                C[r] = (float)c[r];
                ax[r] = (float)a[r];
            }
            for (int e = 0; e < 9; ++e) Rm[e] = (float)R[e];
            for (int r = 0; r < 3; ++r) o[r] = -(R[r] * c[0] + R[3 + r] * c[1] + R[6 + r] * c[2]);  // R^T (0 - C)
            const double H = nearest_mean_curvature(a, o);
            target[k] = (float)(invert[k] ? -H : H);
        }
        __syncthreads();
        const int e = threadIdx.x;
        if (e < 125) {
            const int i = e / 25 - 2, j = (e / 5) % 5 - 2, l = e % 5 - 2;
            const float inv_a0 = 1.0f / ax[0], inv_a1 = 1.0f / ax[1], inv_a2 = 1.0f / ax[2];
            const float h = 1.0f / sub;
            int cnt = 0;
            for (int sx = 0; sx < sub; ++sx) {
                const float px = i + (sx + 0.5f) * h - 0.5f - C[0];
                for (int sy = 0; sy < sub; ++sy) {
                    const float py = j + (sy + 0.5f) * h - 0.5f - C[1];
                    for (int sz = 0; sz < sub; ++sz) {
                        const float pz = l + (sz + 0.5f) * h - 0.5f - C[2];
                        const float y0 = (Rm[0] * px + Rm[3] * py + Rm[6] * pz) * inv_a0;
                        const float y1 = (Rm[1] * px + Rm[4] * py + Rm[7] * pz) * inv_a1;
                        const float y2 = (Rm[2] * px + Rm[5] * py + Rm[8] * pz) * inv_a2;
                        cnt += (y0 * y0 + y1 * y1 + y2 * y2 <= 1.0f) ? 1 : 0;
                    }
                }
            }
            const int tot = sub * sub * sub;
            float phi = (float)(invert[k] ? tot - cnt : cnt) / (float)tot;
            if (noise > 0.f && phi > 0.f && phi < 1.f) {
                const unsigned long long idx = (unsigned long long)k * 125ULL + e;
                const double u1 = uniform_at(noise_seed, 2 * idx), u2 = uniform_at(noise_seed, 2 * idx + 1);
                const float nrm = (float)(sqrt(-2.0 * log1p(-u1)) * cos(6.283185307179586 * u2));
                phi = fminf(fmaxf(phi + noise * nrm, 0.f), 1.f);
            }
            st[e] = phi;
        }
        __syncthreads();
        if (threadIdx.x == 0) cs = canon_of(st);
        __syncthreads();
        if (e < 125) X[k * MK + canon_index(cs, e)] = __float2bfloat16_rn(2.0f * st[e] - 1.0f);
        else X[k * MK + e] = __float2bfloat16_rn(0.f);
    }
}

// ---- in-step learned curvature ---------------------------------------------------
// One warp per 16 interface cells: gather the 5x5x5 fill levels (periodic),
// canonical order, network, then the LSQR value already in kappa_out judges:
// the network's value is kept where |k_mlp - k_lsqr| <= rel |k_lsqr| and no
// obstacle cell lies in the stencil; otherwise the LSQR value stays.
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_curv(Dev d, float *kappa_out) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(smem_raw);
    __nv_bfloat16 *Xs = reinterpret_cast<__nv_bfloat16 *>(smem_raw + sizeof(MlpSmem));
    float *raw = reinterpret_cast<float *>(Xs + MLP_ROWS * WPAD);  // [MLP_ROWS][128]
    __shared__ CanonAffine cw[MLP_ROWS];
    __shared__ int wall[MLP_ROWS];
    int cnt[1];
    block_counts<1>(d.counts, {d.cif}, cnt);
    const int n = cnt[0];
    load_weights(s, d.mlp_params);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __nv_bfloat16 *Xw = Xs + warp * 16 * WPAD;
    float *rw = raw + warp * 16 * MK;
    int evaluated = 0, kept = 0;
    for (int base = blockIdx.x * MLP_ROWS + warp * 16; base < n; base += gridDim.x * MLP_ROWS) {
        const int nvalid = n - base < 16 ? n - base : 16;
        // the 16 cells' coordinates (lane r holds cell r), then their 5x5x5
        // gathers four cells at a time, so that 32 loads per lane are in flight
        int cx0 = 0, cy0 = 0, cz0 = 0;
        if (lane < nvalid) cell_coords(d, d.iflist[base + lane], cx0, cy0, cz0);
        unsigned obsm = 0u;  // bit r: an obstacle cell in row r's stencil (this lane's elements)
#pragma unroll 4
        for (int r = 0; r < 16; ++r) {
            const int x = __shfl_sync(0xffffffffu, cx0, r), y = __shfl_sync(0xffffffffu, cy0, r),
                      z = __shfl_sync(0xffffffffu, cz0, r);
            if (r < nvalid) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = lane + 32 * t;
                    if (e < 125) {
                        const int j = nbr_index(d, x, y, z, e / 25 - 2, (e / 5) % 5 - 2, e % 5 - 2);
                        rw[r * MK + e] = d.phi[j];
                        obsm |= (d.flags[j] & T_OBS) ? (1u << r) : 0u;
                    }
                }
            }
        }
        obsm = __reduce_or_sync(0xffffffffu, obsm);
        if (lane < 16) wall[warp * 16 + lane] = (obsm >> lane) & 1u;
        __syncwarp();
        if (lane < 16) cw[warp * 16 + lane] = canon_affine(canon_of(rw + lane * MK));
        __syncwarp();
        for (int r = 0; r < 16; ++r) {
            const CanonAffine c = cw[warp * 16 + r];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = lane + 32 * t;
                if (e < 125)
                    Xw[r * WPAD + c.base + (e / 25) * c.s[0] + ((e / 5) % 5) * c.s[1] + (e % 5) * c.s[2]] =
                        __float2bfloat16_rn(2.0f * rw[r * MK + e] - 1.0f);
                else
                    Xw[r * WPAD + e] = __float2bfloat16_rn(0.f);
            }
        }
        __syncwarp();
        float ylo, yhi;
        warp_mlp<false>(s, Xw, ylo, yhi, nullptr, nullptr, 0, 0);
        if ((lane & 3) == 0) {
            const int g = lane >> 2;
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                if (r < nvalid && !wall[warp * 16 + r]) {
                    const int i = d.iflist[base + r];
                    const float kls = kappa_out[i], km = h ? yhi : ylo;
                    ++evaluated;
                    if (fabsf(km - kls) <= d.mlp_rel * fabsf(kls)) {
                        kappa_out[i] = km;
                        ++kept;
                    }
                }
            }
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
        kept += __shfl_xor_sync(0xffffffffu, kept, o);
    }
    if (lane == 0 && evaluated) {
        atomicAdd(d.counts + C_MLP, evaluated);
        atomicAdd(d.counts + C_MLPKEEP, kept);
    }
}

size_t mlp_forward_smem() { return sizeof(MlpSmem) + (size_t)MLP_ROWS * WPAD * 2; }
size_t mlp_curv_smem() { return mlp_forward_smem() + (size_t)MLP_ROWS * MK * 4; }

int mlp_grid(const void *kernel, int block, size_t smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return resident_grid(kernel, block, smem);
}

void launch_mlp_curv(const Dev &d, float *kappa_out, cudaStream_t s) {
    static const int g = mlp_grid((const void *)k_mlp_curv, 32 * MLP_WARPS, mlp_curv_smem());
    k_mlp_curv<<<g, 32 * MLP_WARPS, mlp_curv_smem(), s>>>(d, kappa_out);
}

}  // namespace fslk

using namespace fslk;

extern "C" {

size_t fsl_mlp_param_bytes(void) { return MB_BIAS + (size_t)(2 * MK + 1) * sizeof(float); }
int fsl_mlp_master_count(void) { return M_COUNT; }

// training workspace (bytes, each part 256-aligned): the gradient (master
// layout), the per-tile partials of the tile kernel and the tiles' loss sums
static size_t up256(size_t v) { return (v + 255) / 256 * 256; }
struct TrainWs {
    size_t grad, part, lpart, total;
};
static TrainWs train_ws(int n) {
    TrainWs w;
    size_t o = 0;
    w.grad = o; o = up256(o + (size_t)M_COUNT * sizeof(float));
    w.part = o; o = up256(o + mlp_tile_partial_floats(n) * sizeof(float));
    w.lpart = o; o = up256(o + (size_t)((n + MK - 1) / MK) * sizeof(double));
    w.total = o;
    return w;
}

size_t fsl_mlp_train_workspace(int n) {
    if (n <= 0) return 0;
    return train_ws(n).total + 1024;
}

int fsl_mlp_stencils(int n, const float *axes, const float *quat, const float *dir, const float *delta,
                     const int32_t *invert, int sub, float noise, uint64_t noise_seed, void *X, float *target,
                     void *stream) {
    if (n < 0 || !axes || !quat || !dir || !delta || !invert || !X || !target || sub < 1 || sub > 32 || noise < 0.f)
        return FSL_EINVAL;
    if (n == 0) return FSL_OK;
    const int grid = n < 65536 ? n : 65536;
    k_mlp_stencils<<<grid, 128, 0, (cudaStream_t)stream>>>(n, axes, quat, dir, delta, invert, sub, noise, noise_seed,
                                                          static_cast<__nv_bfloat16 *>(X), target);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_mlp_forward(const void *params, const void *X, int n, float *y, float *z1, float *z2, void *stream) {
    if (!params || !X || !y || n < 0 || ((z1 == nullptr) != (z2 == nullptr))) return FSL_EINVAL;
    if (n == 0) return FSL_OK;
    return launch_mlp_forward_tc(static_cast<const uint8_t *>(params), static_cast<const __nv_bfloat16 *>(X), n, y, z1,
                                 z2, (cudaStream_t)stream);
}

int fsl_mlp_status(int reset) { return mlp_tc_status(reset != 0); }

// One training step's gradient (and with master non-null the Adam step): the
// tile kernel over the batch rows perm[row0 .. row0 + n) of X (rows row0 ..
// when perm is null), then the fixed-order reduction of its partials.
static int mlp_step(const void *params, const void *X, const float *target, const int64_t *perm, long long row0, int n,
                    long long n_all, float *loss_dev, void *workspace, float *grad_out, void *params_rw, float *master,
                    float *m, float *v, float lr, int step, cudaStream_t s) {
    char *ws = static_cast<char *>(workspace);
    const TrainWs L = train_ws(n);
    float *part = reinterpret_cast<float *>(ws + L.part);
    double *lpart = reinterpret_cast<double *>(ws + L.lpart);
    const int rc = launch_mlp_train_tile(static_cast<const uint8_t *>(params), static_cast<const __nv_bfloat16 *>(X),
                                         target, perm, row0, n, n_all, part, lpart, s);
    if (rc != FSL_OK) return rc;
    const float bc1 = master ? (float)(1.0 - pow(0.9, step)) : 1.f, bc2 = master ? (float)(1.0 - pow(0.999, step)) : 1.f;
    k_mlp_tile_reduce<<<(M_COUNT + 255) / 256, 256, 0, s>>>(part, lpart, (n + MK - 1) / MK, n, grad_out, loss_dev,
                                                           static_cast<uint8_t *>(params_rw), master, m, v, lr, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_mlp_gradients(const void *params, const void *X, const float *target, int n, float *grad, float *loss_dev,
                      void *workspace, void *stream) {
    if (!params || !X || !target || !grad || !workspace || n <= 0) return FSL_EINVAL;
    if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(workspace) % 256) return FSL_EINVAL;
    return mlp_step(params, X, target, nullptr, 0, n, n, loss_dev, workspace, grad, nullptr, nullptr, nullptr, nullptr,
                    0.f, 1, (cudaStream_t)stream);
}

int fsl_mlp_train_step(void *params, float *master, float *m, float *v, const void *X, const float *target, int n,
                       float lr, int step, float *loss_dev, void *workspace, void *stream) {
    if (!params || !master || !m || !v || !X || !target || !workspace || n <= 0 || step < 1 || !(lr > 0.f))
        return FSL_EINVAL;
    if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(workspace) % 256) return FSL_EINVAL;
    return mlp_step(params, X, target, nullptr, 0, n, n, loss_dev, workspace, nullptr, params, master, m, v, lr, step,
                    (cudaStream_t)stream);
}

// the epoch loop reads its batches through the permutation inside the tile
// kernel: the epoch workspace is the training workspace of one batch
size_t fsl_mlp_epoch_workspace(int batch) {
    if (batch <= 0) return 0;
    return fsl_mlp_train_workspace(batch);
}

int fsl_mlp_train_epoch(void *params, float *master, float *m, float *v, const void *X, const float *target,
                        const int64_t *perm, int n, int batch, float lr, int step0, float *losses_dev,
                        void *workspace, void *stream) {
    if (!params || !master || !m || !v || !X || !target || !perm || !workspace || batch < 1 || n < batch ||
        step0 < 0 || !(lr > 0.f))
        return FSL_EINVAL;
    if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(workspace) % 256) return FSL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = n / batch;
    for (int b = 0; b < nb; ++b) {
        const int rc = mlp_step(params, X, target, perm, (long long)b * batch, batch, n,
                                losses_dev ? losses_dev + b : nullptr, workspace, nullptr, params, master, m, v, lr,
                                step0 + b + 1, s);
        if (rc != FSL_OK) return rc;
    }
    return FSL_OK;
}

int fsl_mlp_pack(const float *master, void *params, void *stream) {
    if (!master || !params) return FSL_EINVAL;
    k_mlp_pack<<<(M_COUNT + 255) / 256, 256, 0, (cudaStream_t)stream>>>(master, static_cast<uint8_t *>(params));
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

}  // extern "C"
