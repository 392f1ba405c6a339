// k_mlp.cu -- learned curvature on the 5x5x5 fill-level stencil: training
// stencils, the MLP 125 -> 128 -> 128 -> 1 (GELU) with BF16 weights, its FP32
// backward and Adam, and the in-step estimate that keeps the LSQR fit
// (Sec. II.C) as judge and fallback.  Every network evaluation -- the batch
// forward, the training step and the in-step estimate -- runs on the tcgen05
// tensor cores (k_mlp_tc.cu); this file holds the training stencils, the
// gradient reduction with Adam, and the C entry points.
//
// Network (packed parameter block, see include/fsl.h):
//   x = bf16(2 phi - 1) over the canonical stencil (125 values, 3 zero pads)
//   z1 = W1 x + b1, h1 = bf16(gelu(z1)), z2 = W2 h1 + b2, h2 = gelu(z2),
//   y = w3 . h2 + b3 = kappa dx;   gelu(x) = x Phi(x) (erf form)
// Canonical stencil: axes flipped so the Parker-Youngs normal of the middle
// cell has non-negative components, then ordered by decreasing |n_k|.
#include <math.h>

#include "fsl_internal.cuh"
#include "mlp_common.cuh"

namespace fslk {

constexpr int MK = 128;     // padded input width, hidden width
constexpr int MB_BF = 32896;  // bf16 elements of W1 | W2 | w3
constexpr size_t MB_BIAS = (size_t)MB_BF * 2;  // byte offset of the FP32 biases (256-aligned)
// FP32 master / gradient / moment layout
constexpr int M_W1 = 0, M_W2 = 16384, M_W3 = 32768, M_B1 = 32896, M_B2 = 33024, M_B3 = 33152, M_COUNT = 33153;
static_assert(M_W1 == 0 && M_W2 == M_W1 + MK * MK && M_W3 == M_W2 + MK * MK && M_B1 == MB_BF && M_B2 == M_B1 + MK &&
                  M_B3 == M_B2 + MK && M_COUNT == M_B3 + 1,
              "master layout: W1, W2, w3, b1, b2, b3 (the tile partials use the same order)");


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

// ---- in-step learned curvature (the network on the tensor cores, k_mlp_tc.cu) ----
void launch_mlp_curv(const Dev &d, float *kappa_out, cudaStream_t s) {
    launch_mlp_curv_tc(d, kappa_out, s);
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
