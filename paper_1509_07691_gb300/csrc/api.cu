// api.cu -- the C ABI of include/fsl.h: parameter checks, workspace layout,
// step sequencing and CUDA-graph replay.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "fsl_internal.cuh"

using namespace fslk;

struct fsl_ctx {
    fsl_params p;
    fsl_fields fields;
    cudaStream_t stream;     // caller's stream
    cudaStream_t cap_stream; // private streams used only to record graphs
    cudaStream_t cap_side;   // (the bulk stream-collide runs on a parallel branch)
    cudaEvent_t fork, join;
    int parity;
    Dev base;                // pointers and parameters common to both parities
    cudaGraphExec_t graph[2];
    double *mass_out;        // 2 doubles in the workspace
    double *host_mass;       // pinned, 2 doubles
    long long *host_stats;   // pinned
};

namespace {

constexpr size_t ALIGN = 256;
size_t up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t normal, rho, excess, iflist0, iflist1, fill, empty, newgas, liq2if, slow, seg_active, seg_list, counts,
        lost, status, partial, stats, mass_out, total;
};

size_t nseg_of(const fsl_params &p) { return (size_t)((p.nx + SEG - 1) / SEG) * p.ny * p.nz; }

Layout layout(const fsl_params &p) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    Layout L;
    size_t o = 0;
    L.normal = o; o += up(N * sizeof(float4));
    L.rho = o; o += up(N * sizeof(float));
    L.excess = o; o += up(N * sizeof(float));
    L.iflist0 = o; o += up(N * sizeof(int));
    L.iflist1 = o; o += up(N * sizeof(int));
    L.fill = o; o += up(N * sizeof(int));
    L.empty = o; o += up(N * sizeof(int));
    L.newgas = o; o += up(N * sizeof(int));
    L.liq2if = o; o += up(N * sizeof(int));
    L.slow = o; o += up(N * sizeof(int));
    L.seg_active = o; o += up(nseg_of(p));
    L.seg_list = o; o += up(nseg_of(p) * sizeof(int));
    L.counts = o; o += up(C_NCOUNT * sizeof(int));
    L.lost = o; o += up(sizeof(double));
    L.status = o; o += up(sizeof(int));
    L.partial = o; o += up((size_t)max_partials() * sizeof(double));
    L.stats = o; o += up(16 * sizeof(long long));
    L.mass_out = o; o += up(2 * sizeof(double));
    L.total = o;
    return L;
}

bool valid_params(const fsl_params *p) {
    if (!p) return false;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3) return false;
    const double N = (double)p->nx * p->ny * p->nz;
    if (N >= 2147483647.0) return false;  // cell indices are int32 in the lists
    if (p->nx > 65535 * 256 || p->ny > 65535 || p->nz > 65535) return false;
    if (p->collision != FSL_BGK && p->collision != FSL_TRT) return false;
    if (p->curv_model < FSL_CURV_LSQR || p->curv_model > FSL_CURV_MLP) return false;
    if (p->storage < FSL_F32 || p->storage > FSL_BF16_OFS) return false;
    if (p->storage != FSL_F32 && (p->storage_shift < 0 || p->storage_shift > 24)) return false;
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return false;
    if (p->collision == FSL_TRT && !(p->magic > 0.0)) return false;
    if (p->plic_iters < 1 || p->plic_iters > 64) return false;
    if (!isfinite(p->sigma) || !isfinite(p->p_gas) || !isfinite(p->theta) || !(p->eps_convert >= 0.0)) return false;
    if (!(p->lsqr_fp64_cond > 1.0)) return false;
    return true;
}

bool aligned(const void *ptr) { return ptr && ((uintptr_t)ptr % ALIGN) == 0; }

Dev make_dev(const fsl_params &p, const fsl_fields &f) {
    const Layout L = layout(p);
    char *ws = static_cast<char *>(f.workspace);
    Dev d;
    memset(&d, 0, sizeof d);
    d.nx = p.nx;
    d.ny = p.ny;
    d.nz = p.nz;
    d.N = (long long)p.nx * p.ny * p.nz;
    d.mass = f.mass;
    d.phi = f.phi;
    d.kappa = f.kappa;
    d.normal = reinterpret_cast<float4 *>(ws + L.normal);
    d.rho = reinterpret_cast<float *>(ws + L.rho);
    d.excess = reinterpret_cast<float *>(ws + L.excess);
    d.iflist = reinterpret_cast<int *>(ws + L.iflist0);
    d.iflist_next = reinterpret_cast<int *>(ws + L.iflist1);
    d.seg_active = reinterpret_cast<uint8_t *>(ws + L.seg_active);
    d.seg_list = reinterpret_cast<int *>(ws + L.seg_list);
    d.nsegx = (p.nx + SEG - 1) / SEG;
    d.nseg = (int)nseg_of(p);
    d.fill = reinterpret_cast<int *>(ws + L.fill);
    d.empty = reinterpret_cast<int *>(ws + L.empty);
    d.newgas = reinterpret_cast<int *>(ws + L.newgas);
    d.liq2if = reinterpret_cast<int *>(ws + L.liq2if);
    d.slow = reinterpret_cast<int *>(ws + L.slow);
    d.counts = reinterpret_cast<int *>(ws + L.counts);
    d.lost = reinterpret_cast<double *>(ws + L.lost);
    d.status = reinterpret_cast<int *>(ws + L.status);
    d.partial = reinterpret_cast<double *>(ws + L.partial);
    d.stats = reinterpret_cast<long long *>(ws + L.stats);
    d.collision = p.collision;
    d.storage = p.storage;
    d.plic_iters = p.plic_iters;
    d.curv_model = p.curv_model;
    const double tau_o = p.collision == FSL_TRT ? 0.5 + p.magic / (p.tau - 0.5) : p.tau;
    d.omega_e = (float)(1.0 / p.tau);
    d.omega_o = (float)(1.0 / tau_o);
    d.rho_gas = (float)(3.0 * p.p_gas);
    d.six_sigma = (float)(6.0 * p.sigma);
    d.eps = (float)p.eps_convert;
    d.cos_theta = (float)cos(p.theta);
    d.sin_theta = (float)sin(p.theta);
    d.cos_theta_d = cos(p.theta);
    d.sin_theta_d = sin(p.theta);
    d.scale = (float)ldexp(1.0, p.storage == FSL_F32 ? 0 : p.storage_shift);
    d.inv_scale = 1.0f / d.scale;
    d.fp64_cond = (float)p.lsqr_fp64_cond;
    return d;
}

// Parity p: PDFs f[p] -> f[1-p], interface list p -> 1-p.  The cell types
// live in fields.flags[0] and are updated in place; fields.flags[1] is scratch.
Dev dev_for(const fsl_ctx *c, int parity) {
    Dev d = c->base;
    const Layout L = layout(c->p);
    char *ws = static_cast<char *>(c->fields.workspace);
    int *lists[2] = {reinterpret_cast<int *>(ws + L.iflist0), reinterpret_cast<int *>(ws + L.iflist1)};
    d.fsrc = c->fields.f[parity];
    d.fdst = c->fields.f[parity ^ 1];
    d.flags = c->fields.flags[0];
    d.iflist = lists[parity];
    d.iflist_next = lists[parity ^ 1];
    d.cif = C_IF0 + parity;
    d.cif_next = C_IF0 + (parity ^ 1);
    return d;
}

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) return FSL_ECUDA; \
    } while (0)

// enqueue the curvature of the current state into kappa_out
void enqueue_curvature(const Dev &d, int model, float *kappa_out, cudaStream_t s) {
    launch_normals(d, s);
    if (model == FSL_CURV_LSQR || model == FSL_CURV_MLP) launch_lsqr(d, kappa_out, s);
    else if (model == FSL_CURV_FD) launch_fd(d, kappa_out, s);
    else launch_zero_kappa(d, kappa_out, s);
    if (model == FSL_CURV_MLP) launch_mlp_curv(d, kappa_out, s);
}

// One time step from parity p (see fsl_step), recorded as a graph with two
// branches: the liquid stream-collide does not need the curvature, so it runs
// beside normals -> LSQR -> interface stream-collide; both join before the
// conversion.  The counters of the step are zeroed by its first kernel.
int enqueue_step_graph(const fsl_ctx *c, int parity) {
    const Dev d = dev_for(c, parity);
    cudaStream_t s = c->cap_stream, side = c->cap_side;
    CK(cudaEventRecord(c->fork, s));
    CK(cudaStreamWaitEvent(side, c->fork, 0));
    launch_sc_bulk(d, side);
    CK(cudaEventRecord(c->join, side));
    enqueue_curvature(d, c->p.curv_model, d.kappa, s);
    launch_sc_iface(d, s);
    CK(cudaStreamWaitEvent(s, c->join, 0));
    launch_convert(d, s);
    launch_finalize(d, s);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int record_graph(fsl_ctx *c, int parity) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_step_graph(c, parity);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != FSL_OK || e != cudaSuccess) return FSL_ECUDA;
    e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

}  // namespace

extern "C" {

size_t fsl_workspace_size(const fsl_params *params) {
    if (!valid_params(params)) return 0;
    return layout(*params).total;
}

int fsl_fill_geometry(const fsl_params *params, const fsl_geometry *geom, float *phi_dev, void *stream) {
    if (!valid_params(params) || !geom || !phi_dev) return FSL_EINVAL;
    if (geom->kind < 0 || geom->kind > 5 || geom->sub < 1 || geom->sub > 64) return FSL_EINVAL;
    launch_fill_geometry(*params, *geom, phi_dev, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_init(const fsl_params *params, const fsl_fields *fields, const float *phi0, int phi0_where,
             const uint8_t *obstacle, int obstacle_where, void *stream, fsl_ctx **out) {
    if (!out) return FSL_EINVAL;
    *out = nullptr;
    if (!valid_params(params) || !fields) return FSL_EINVAL;
    if (!aligned(fields->f[0]) || !aligned(fields->f[1]) || !aligned(fields->flags[0]) || !aligned(fields->flags[1]) ||
        !aligned(fields->mass) || !aligned(fields->phi) || !aligned(fields->kappa) || !aligned(fields->workspace))
        return FSL_EINVAL;
    if ((phi0_where != FSL_NONE && !phi0) || (obstacle_where != FSL_NONE && !obstacle)) return FSL_EINVAL;
    fsl_ctx *c = new (std::nothrow) fsl_ctx;
    if (!c) return FSL_EINVAL;
    memset(c, 0, sizeof *c);
    c->p = *params;
    c->fields = *fields;
    c->stream = (cudaStream_t)stream;
    c->base = make_dev(c->p, c->fields);
    const Layout L = layout(c->p);
    c->mass_out = reinterpret_cast<double *>(static_cast<char *>(fields->workspace) + L.mass_out);
    int rc = FSL_ECUDA;
    do {
        if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) break;
        if (cudaStreamCreateWithFlags(&c->cap_side, cudaStreamNonBlocking) != cudaSuccess) break;
        if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) break;
        if (cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) break;
        if (cudaMallocHost((void **)&c->host_mass, 2 * sizeof(double)) != cudaSuccess) break;
        if (cudaMallocHost((void **)&c->host_stats, 16 * sizeof(long long)) != cudaSuccess) break;
        const size_t N = (size_t)c->base.N;
        cudaStream_t s = c->stream;
        if (phi0_where != FSL_NONE &&
            cudaMemcpyAsync(fields->phi, phi0, N * sizeof(float), cudaMemcpyDefault, s) != cudaSuccess)
            break;
        // obstacle mask staged in flags[0]; types computed into flags[1]
        const uint8_t *obs = nullptr;
        if (obstacle_where != FSL_NONE) {
            if (cudaMemcpyAsync(fields->flags[0], obstacle, N, cudaMemcpyDefault, s) != cudaSuccess) break;
            obs = fields->flags[0];
        }
        if (cudaMemsetAsync(c->base.counts, 0, C_NCOUNT * sizeof(int), s) != cudaSuccess) break;
        if (cudaMemsetAsync(c->base.lost, 0, sizeof(double), s) != cudaSuccess) break;
        if (cudaMemsetAsync(c->base.status, 0, sizeof(int), s) != cudaSuccess) break;
        if (cudaMemsetAsync(c->base.normal, 0, N * sizeof(float4), s) != cudaSuccess) break;
        if (cudaMemsetAsync(fields->kappa, 0, N * sizeof(float), s) != cudaSuccess) break;
        if (cudaMemsetAsync(c->base.seg_active, 0, c->base.nseg, s) != cudaSuccess) break;
        Dev d = dev_for(c, 1);  // fdst = f[0]
        launch_init_types(d, obs, fields->flags[1], s);
        Dev d0 = dev_for(c, 0);
        d0.fdst = fields->f[0];
        launch_init_state(d0, fields->flags[1], s);
        launch_seg_compact(d0, s);
        if (cudaGetLastError() != cudaSuccess) break;
        c->parity = 0;
        rc = FSL_OK;
    } while (0);
    if (rc != FSL_OK) {
        fsl_destroy(c);
        return rc;
    }
    *out = c;
    return FSL_OK;
}

int fsl_refresh(fsl_ctx *c) {
    if (!c) return FSL_EINVAL;
    Dev d = dev_for(c, c->parity);
    CK(cudaMemsetAsync(d.counts, 0, C_NCOUNT * sizeof(int), c->stream));
    CK(cudaMemsetAsync(d.seg_active, 0, d.nseg, c->stream));
    launch_refresh(d, c->stream);
    launch_seg_compact(d, c->stream);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_step(fsl_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return FSL_EINVAL;
    if (c->p.curv_model == FSL_CURV_MLP && !c->base.mlp_params) return FSL_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (!c->graph[c->parity]) {
            const int rc = record_graph(c, c->parity);
            if (rc != FSL_OK) return rc;
        }
        CK(cudaGraphLaunch(c->graph[c->parity], c->stream));
        c->parity ^= 1;
    }
    return FSL_OK;
}

int fsl_step_profile(fsl_ctx *c, float ms_out[6]) {
    if (!c || !ms_out) return FSL_EINVAL;
    cudaEvent_t ev[7];
    for (int k = 0; k < 7; ++k)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) return FSL_ECUDA;
    const Dev d = dev_for(c, c->parity);
    cudaStream_t s = c->stream;
    int rc = FSL_ECUDA;
    do {
        if (cudaEventRecord(ev[0], s) != cudaSuccess) break;
        launch_normals(d, s);
        if (cudaEventRecord(ev[1], s) != cudaSuccess) break;
        if (c->p.curv_model == FSL_CURV_LSQR || c->p.curv_model == FSL_CURV_MLP) launch_lsqr(d, d.kappa, s);
        else if (c->p.curv_model == FSL_CURV_FD) launch_fd(d, d.kappa, s);
        else launch_zero_kappa(d, d.kappa, s);
        if (c->p.curv_model == FSL_CURV_MLP) launch_mlp_curv(d, d.kappa, s);
        if (cudaEventRecord(ev[2], s) != cudaSuccess) break;
        launch_sc_bulk(d, s);
        if (cudaEventRecord(ev[3], s) != cudaSuccess) break;
        launch_sc_iface(d, s);
        if (cudaEventRecord(ev[4], s) != cudaSuccess) break;
        launch_convert(d, s);
        if (cudaEventRecord(ev[5], s) != cudaSuccess) break;
        launch_finalize(d, s);
        if (cudaEventRecord(ev[6], s) != cudaSuccess) break;
        if (cudaEventSynchronize(ev[6]) != cudaSuccess) break;
        for (int k = 0; k < 6; ++k) cudaEventElapsedTime(&ms_out[k], ev[k], ev[k + 1]);
        c->parity ^= 1;
        rc = FSL_OK;
    } while (0);
    for (int k = 0; k < 7; ++k) cudaEventDestroy(ev[k]);
    return rc;
}

int fsl_curvature(fsl_ctx *c, int model, float *kappa_out) {
    if (!c || !kappa_out || model < FSL_CURV_LSQR || model > FSL_CURV_MLP) return FSL_EINVAL;
    if (model == FSL_CURV_MLP && !c->base.mlp_params) return FSL_EINVAL;
    const Dev d = dev_for(c, c->parity);
    enqueue_curvature(d, model, kappa_out, c->stream);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_mass(fsl_ctx *c, double *total_mass, double *lost_mass) {
    if (!c) return FSL_EINVAL;
    const Dev d = dev_for(c, c->parity);
    launch_mass(d, c->mass_out, c->stream);
    CK(cudaMemcpyAsync(c->host_mass, c->mass_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (total_mass) *total_mass = c->host_mass[0];
    if (lost_mass) *lost_mass = c->host_mass[1];
    return FSL_OK;
}

int fsl_mlp_attach(fsl_ctx *c, const void *params, double fallback_rel) {
    if (!c || !params || !(fallback_rel >= 0.0)) return FSL_EINVAL;
    c->base.mlp_params = static_cast<const uint8_t *>(params);
    c->base.mlp_rel = (float)fallback_rel;
    // recorded graphs hold the old parameters
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
    return FSL_OK;
}

int fsl_stats(fsl_ctx *c, int64_t counts_out[10]) {
    if (!c || !counts_out) return FSL_EINVAL;
    const Dev d = dev_for(c, c->parity);
    CK(cudaMemsetAsync(d.stats, 0, 16 * sizeof(long long), c->stream));
    launch_stats(d, c->stream);
    CK(cudaMemcpyAsync(c->host_stats, d.stats, 6 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    int cnt[C_NCOUNT];
    CK(cudaMemcpyAsync(cnt, d.counts, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 6; ++k) counts_out[k] = c->host_stats[k];
    counts_out[6] = cnt[C_FP64];
    counts_out[7] = cnt[C_IF0 + c->parity];
    counts_out[8] = cnt[C_MLP];
    counts_out[9] = cnt[C_MLPKEEP];
    return FSL_OK;
}

int fsl_parity(const fsl_ctx *c) { return c ? c->parity : FSL_EINVAL; }

int fsl_status(fsl_ctx *c) {
    if (!c) return FSL_EINVAL;
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->base.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return st;
}

const char *fsl_strerror(int code) {
    switch (code) {
    case FSL_OK: return "ok";
    case FSL_EINVAL: return "invalid parameter, shape or pointer";
    case FSL_ECUDA: return "CUDA runtime error";
    case FSL_ECAPACITY: return "device list capacity exceeded";
    case FSL_ETIMEOUT: return "bounded device wait timed out";
    case FSL_ENAN: return "non-finite value in the state";
    case FSL_EUNSUPPORTED: return "unsupported option";
    default: return "unknown error";
    }
}

void fsl_destroy(fsl_ctx *c) {
    if (!c) return;
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_side) cudaStreamDestroy(c->cap_side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->host_mass) cudaFreeHost(c->host_mass);
    if (c->host_stats) cudaFreeHost(c->host_stats);
    delete c;
}

}  // extern "C"
