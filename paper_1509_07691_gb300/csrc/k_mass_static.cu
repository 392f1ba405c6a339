// k_mass_static.cu -- total mass of a state for callers that cannot allocate
// device memory: the per-block partial sums go to a fixed array in the
// library's own device memory instead of a caller-provided workspace.
//
// Who needs it: code embedded in a host application that owns every byte of
// device memory (its own caching allocator or a hard memory budget, so a
// cudaMalloc behind its back is not allowed), and monitoring code inside a
// time-critical loop that cannot afford an allocation and the device
// synchronisation it implies.  They pass the state buffers and one output
// double; nothing is allocated.
//
// The array lives in every device that loads the library, until the process
// exits.  In host code its name is only a host-side stand-in, so its device
// address is looked up once per device (cudaGetSymbolAddress, with that
// device current) and cached.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fsl_internal.cuh"

namespace fslk {

constexpr int MS_THREADS = 256;
constexpr long long MS_CELLS_PER_BLOCK = FSL_MASS_STATIC_CELLS_PER_BLOCK;
constexpr int MS_MAX_DEVICES = 64;

// one FP64 partial per block of MS_CELLS_PER_BLOCK cells; every slot the
// reduction reads is written by the same call first, so nothing needs clearing
static __device__ __align__(256) double g_mass_partials[FSL_MASS_STATIC_MAX_BLOCKS];

template <int S>
__global__ void __launch_bounds__(MS_THREADS) k_mass_static_partial(Dev d, double *partials) {
    const long long begin = (long long)blockIdx.x * MS_CELLS_PER_BLOCK;
    const long long end = begin + MS_CELLS_PER_BLOCK < d.N ? begin + MS_CELLS_PER_BLOCK : d.N;
    double acc = 0.0;
    for (long long i = begin + threadIdx.x; i < end; i += blockDim.x) {
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
    __shared__ double red[MS_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < MS_THREADS / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// one block adds the partials in a fixed order
__global__ void __launch_bounds__(MS_THREADS) k_mass_static_final(const double *partials, int n, double *out) {
    __shared__ double red[MS_THREADS];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = MS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// device address of g_mass_partials on the current device (looked up once)
double *static_partials() {
    static std::mutex mu;
    static double *addr[MS_MAX_DEVICES] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MS_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) return nullptr;
        addr[dev] = static_cast<double *>(p);
    }
    return addr[dev];
}

}  // namespace fslk

using namespace fslk;

extern "C" int fsl_mass_static(const fsl_params *params, const void *f, const uint8_t *flags, const float *mass,
                               double *total_dev, void *stream) {
    if (!params || !f || !flags || !mass || !total_dev) return FSL_EINVAL;
    if (params->nx < 1 || params->ny < 1 || params->nz < 1) return FSL_EINVAL;
    if (params->storage < FSL_F32 || params->storage > FSL_BF16_OFS) return FSL_EINVAL;
    if (params->storage != FSL_F32 && (params->storage_shift < 0 || params->storage_shift > 24)) return FSL_EINVAL;
    const long long N = (long long)params->nx * params->ny * params->nz;
    if (N > FSL_MASS_STATIC_MAX_CELLS) return FSL_EINVAL;  // more partials than the fixed array holds
    const int nb = (int)((N + MS_CELLS_PER_BLOCK - 1) / MS_CELLS_PER_BLOCK);
    double *partials = static_partials();
    if (!partials) return FSL_ECUDA;
    Dev d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.fsrc = f;
    d.flags = const_cast<uint8_t *>(flags);
    d.mass = const_cast<float *>(mass);
    d.storage = params->storage;
    d.scale = (float)ldexp(1.0, params->storage == FSL_F32 ? 0 : params->storage_shift);
    d.inv_scale = 1.0f / d.scale;
    cudaStream_t s = (cudaStream_t)stream;
    switch (params->storage) {
    case FSL_F32: k_mass_static_partial<FSL_F32><<<nb, MS_THREADS, 0, s>>>(d, partials); break;
    case FSL_F16_OFS: k_mass_static_partial<FSL_F16_OFS><<<nb, MS_THREADS, 0, s>>>(d, partials); break;
    default: k_mass_static_partial<FSL_BF16_OFS><<<nb, MS_THREADS, 0, s>>>(d, partials); break;
    }
    k_mass_static_final<<<1, MS_THREADS, 0, s>>>(partials, nb, total_dev);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}
