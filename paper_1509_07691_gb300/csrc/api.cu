// api.cu -- the C ABI of include/fsl.h: parameter checks, workspace layout,
// step sequencing and CUDA-graph replay.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <new>

#include "adjoint.cuh"
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
    double *host_mass;       // pinned, 4 doubles (mass, lost; dL/dsigma, dL/dtheta)
    long long *host_stats;   // pinned
    int *host_count;         // pinned, 1 int
    int bubble;              // bubble model on (fsl_set_bubble)
    // the last adjoint window (fsl_window_forward)
    void *adj_ws;
    int adj_window, adj_ckpt, adj_cap, adj_valid;
};

namespace {

constexpr size_t ALIGN = 256;
size_t up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t normal, rho, excess, exw, rmark, iflist0, iflist1, fill, empty, newgas, liq2if, slow, seg_active, seg_list, counts,
        lost, status, partial, stats, mass_out, bubble, total;
};

size_t nseg_of(const fsl_params &p) { return (size_t)((p.nx + SEG - 1) / SEG) * p.ny * p.nz; }

Layout layout(const fsl_params &p) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    Layout L;
    size_t o = 0;
    L.normal = o; o += up(N * sizeof(float4));
    L.rho = o; o += up(N * sizeof(float));
    L.excess = o; o += up(N * sizeof(float));
    L.exw = o; o += up(N * sizeof(float));
    L.rmark = o; o += up(N);
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
    L.bubble = o; o += up(8 * sizeof(long long) + 2 * sizeof(double) + sizeof(float));
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
    if (p->curv_model < FSL_CURV_LSQR || p->curv_model > FSL_CURV_TR) return false;
    if (p->storage < FSL_F32 || p->storage > FSL_BF16_OFS) return false;
    if (p->storage != FSL_F32 && (p->storage_shift < 0 || p->storage_shift > 24)) return false;
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return false;
    if (p->collision == FSL_TRT && !(p->magic > 0.0)) return false;
    if (p->plic_iters < 1 || p->plic_iters > 64) return false;
    if (!isfinite(p->sigma) || !isfinite(p->p_gas) || !isfinite(p->theta) || !(p->eps_convert >= 0.0)) return false;
    if (!(p->lsqr_fp64_cond > 1.0)) return false;
    if (p->excess_rule != 0 && p->excess_rule != 1) return false;
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
    d.exw = reinterpret_cast<float *>(ws + L.exw);
    d.excess_rule = p.excess_rule;
    d.rmark = reinterpret_cast<uint8_t *>(ws + L.rmark);
    d.iflist = reinterpret_cast<int *>(ws + L.iflist0);
    d.iflist_next = reinterpret_cast<int *>(ws + L.iflist1);
    d.seg_active = reinterpret_cast<uint8_t *>(ws + L.seg_active);
    d.seg_list = reinterpret_cast<int *>(ws + L.seg_list);
    d.nsegx = (p.nx + SEG - 1) / SEG;
    d.nseg = (int)nseg_of(p);
    // counter slots of list parity 0 (dev_for and the window view set their own)
    d.cif = C_IF0;
    d.cif_next = C_IF1;
    d.cdirty = C_SEGD0;
    d.cdirty_next = C_SEGD1;
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
    d.cdirty = C_SEGD0 + parity;
    d.cdirty_next = C_SEGD0 + (parity ^ 1);
    return d;
}

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) return FSL_ECUDA; \
    } while (0)

// After the near-obstacle bits were (re)computed: with no cell next to an
// obstacle no fit has a contact line, and the fused fit + interface kernel
// finishes the few fits it defers itself (the general-path kernel is not
// launched).  Recorded graphs of the other kind are dropped.
int read_near(fsl_ctx *c) {
    CK(cudaMemcpyAsync(c->host_count, c->base.counts + C_NEAR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int inl = *c->host_count == 0 ? 1 : 0;
    if (inl != c->base.inline_general)
        for (int k = 0; k < 2; ++k)
            if (c->graph[k]) {
                cudaGraphExecDestroy(c->graph[k]);
                c->graph[k] = nullptr;
            }
    c->base.inline_general = inl;
    return FSL_OK;
}

// enqueue the curvature of the current state into kappa_out
void enqueue_curvature(const Dev &d, int model, float *kappa_out, cudaStream_t s) {
    launch_normals(d, s);
    if (model == FSL_CURV_LSQR || model == FSL_CURV_MLP) launch_lsqr(d, kappa_out, s);
    else if (model == FSL_CURV_FD) launch_fd(d, kappa_out, s);
    else if (model == FSL_CURV_TR) launch_tr(d, kappa_out, s);
    else launch_zero_kappa(d, kappa_out, s);
    if (model == FSL_CURV_MLP) launch_mlp_curv(d, kappa_out, s);
}

// One time step from parity p (see fsl_step), recorded as a graph with two
// branches: the liquid stream-collide does not need the curvature, so it runs
// beside normals -> LSQR -> interface stream-collide; both join before the
// conversion.  The counters of the step are zeroed by its first kernel.  The
// kernels after the first of each branch start with a programmatic-launch
// wait, so each is dispatched while its predecessor drains.
int enqueue_step_graph(const fsl_ctx *c, int parity) {
    const Dev d = dev_for(c, parity);
    cudaStream_t s = c->cap_stream, side = c->cap_side;
    CK(cudaEventRecord(c->fork, s));
    CK(cudaStreamWaitEvent(side, c->fork, 0));
    launch_sc_bulk(d, side);
    CK(cudaEventRecord(c->join, side));
    if (c->p.curv_model == FSL_CURV_LSQR) {
        launch_normals(d, s);
        launch_curv_iface(d, s);
    } else {
        enqueue_curvature(d, c->p.curv_model, d.kappa, s);
        launch_sc_iface(d, s);
    }
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

// ---- adjoint workspace -------------------------------------------------------------
// Every array is 256-byte aligned.  Checkpoint s holds (f', m, phi) of step
// s*K; in-segment slot t (1..K) the same of step t of a recomputed segment,
// and curvature/normal slot t (0..K-1) the values step t used.
constexpr int ADJ_MAX_PARTIALS = 4096;

struct AdjLayout {
    size_t wcounts, wlist, widx, wseg, wscr, ckpt, slot, kn, fb0, fb1, gb, mb, pb, kb, jac, jval, dlist, glist, nj, part, acc,
        total;
    size_t state_bytes;  // one (f', m, phi) record
    size_t kn_bytes;     // one (kappa, normal) record
    int nseg_ckpt;
};

AdjLayout adj_layout(const fsl_params &p, int W, int K, int cap) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    AdjLayout A;
    A.state_bytes = up(19 * N * sizeof(float)) + 2 * up(N * sizeof(float));
    A.kn_bytes = up(N * sizeof(float)) + up(N * sizeof(float4));
    A.nseg_ckpt = (W + K - 1) / K;
    size_t o = 0;
    A.wcounts = o; o += up(C_NCOUNT * sizeof(int));
    A.wlist = o; o += up(N * sizeof(int));
    A.widx = o; o += up(N * sizeof(int));
    A.wseg = o; o += up(nseg_of(p) * sizeof(int));
    A.wscr = o; o += up((size_t)window_scratch_ints((long long)N) * sizeof(int));
    A.ckpt = o; o += (size_t)A.nseg_ckpt * A.state_bytes;
    A.slot = o; o += (size_t)K * A.state_bytes;
    A.kn = o; o += (size_t)K * A.kn_bytes;
    A.fb0 = o; o += up(19 * N * sizeof(float));
    A.fb1 = o; o += up(19 * N * sizeof(float));
    A.gb = o; o += up(19 * N * sizeof(float));
    A.mb = o; o += up(N * sizeof(float));
    A.pb = o; o += up(N * sizeof(float));
    A.kb = o; o += up(N * sizeof(float));
    A.jac = o; o += up((size_t)cap * JAC_STRIDE * sizeof(float));
    A.jval = o; o += up((size_t)cap * sizeof(float));
    A.dlist = o; o += up((size_t)cap * sizeof(int));
    A.glist = o; o += up((size_t)cap * sizeof(int));
    A.nj = o; o += up((size_t)cap * 125 * sizeof(float4));
    A.part = o; o += up(2 * ADJ_MAX_PARTIALS * sizeof(double));
    A.acc = o; o += up(2 * sizeof(double));
    A.total = o;
    return A;
}

// (f', m, phi) pointers of a record at byte offset off
struct StatePtrs {
    float *f, *m, *phi;
};
StatePtrs state_at(char *ws, size_t off, size_t N) {
    StatePtrs r;
    r.f = reinterpret_cast<float *>(ws + off);
    r.m = reinterpret_cast<float *>(ws + off + up(19 * N * sizeof(float)));
    r.phi = reinterpret_cast<float *>(ws + off + up(19 * N * sizeof(float)) + up(N * sizeof(float)));
    return r;
}

bool adjoint_supported(const fsl_params &p) {
    return p.storage == FSL_F32 && (p.curv_model == FSL_CURV_LSQR || p.curv_model == FSL_CURV_NONE) && p.nx >= 7 &&
           p.ny >= 7 && p.nz >= 7;
}

// Kernel view of a window: frozen types, the window's own interface list,
// active segments and counters (the context's lists are not touched).
Dev window_dev(const fsl_ctx *c, char *ws, const AdjLayout &A) {
    Dev d = c->base;
    d.flags = c->fields.flags[0];
    d.counts = reinterpret_cast<int *>(ws + A.wcounts);
    d.iflist = reinterpret_cast<int *>(ws + A.wlist);
    d.iflist_next = nullptr;
    d.cif = C_IF0;
    d.cif_next = C_IF1;
    d.cdirty = C_SEGD0;
    d.cdirty_next = C_SEGD1;
    d.seg_list = reinterpret_cast<int *>(ws + A.wseg);
    d.frozen = 1;
    return d;
}

Adj adj_args(char *ws, const AdjLayout &A, int cap) {
    Adj a;
    memset(&a, 0, sizeof a);
    a.wlist = reinterpret_cast<const int *>(ws + A.wlist);
    a.widx = reinterpret_cast<const int *>(ws + A.widx);
    a.cap = cap;
    a.jac = reinterpret_cast<float *>(ws + A.jac);
    a.jval = reinterpret_cast<float *>(ws + A.jval);
    a.dlist = reinterpret_cast<int *>(ws + A.dlist);
    a.glist = reinterpret_cast<int *>(ws + A.glist);
    a.nj = reinterpret_cast<float4 *>(ws + A.nj);
    a.gb = reinterpret_cast<float *>(ws + A.gb);
    a.mb = reinterpret_cast<float *>(ws + A.mb);
    a.pb = reinterpret_cast<float *>(ws + A.pb);
    a.kb = reinterpret_cast<float *>(ws + A.kb);
    a.part = reinterpret_cast<double *>(ws + A.part);
    a.acc = reinterpret_cast<double *>(ws + A.acc);
    const int nb = adj_blocks();
    a.nblk = nb < ADJ_MAX_PARTIALS ? nb : ADJ_MAX_PARTIALS;
    return a;
}

// window setup from the context's current lists; returns the interface count
int window_setup(fsl_ctx *c, char *ws, const AdjLayout &A, int *n_out) {
    const Dev src = dev_for(c, c->parity);
    int *wc = reinterpret_cast<int *>(ws + A.wcounts);
    CK(cudaMemsetAsync(wc, 0, C_NCOUNT * sizeof(int), c->stream));
    launch_window_setup(src, wc, reinterpret_cast<int *>(ws + A.wlist), reinterpret_cast<int *>(ws + A.widx),
                        reinterpret_cast<int *>(ws + A.wseg), reinterpret_cast<int *>(ws + A.wscr), c->stream);
    CK(cudaMemcpyAsync(c->host_count, wc + C_IF0, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *n_out = *c->host_count;
    return FSL_OK;
}

// checkpoint file layout and staging (fsl_save / fsl_load)

struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, nz, storage, storage_shift;
    int32_t pad;
    double lost;
    fsl_params params;
};

size_t pdf_elem_bytes(int storage) { return storage == FSL_F32 ? 4 : 2; }

// one device buffer <-> file through a host staging buffer; false on any error
bool dev_to_file(FILE *fp, const void *dev, size_t bytes, cudaStream_t s) {
    void *h = malloc(bytes ? bytes : 1);
    if (!h) return false;
    bool ok = cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess && fwrite(h, 1, bytes, fp) == bytes;
    free(h);
    return ok;
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
        if (cudaMallocHost((void **)&c->host_mass, 4 * sizeof(double)) != cudaSuccess) break;
        if (cudaMallocHost((void **)&c->host_count, sizeof(int)) != cudaSuccess) break;
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
        if (cudaMemsetAsync(c->base.rmark, 0, N, s) != cudaSuccess) break;
        Dev d = dev_for(c, 1);  // fdst = f[0]
        launch_init_types(d, obs, fields->flags[1], s);
        Dev d0 = dev_for(c, 0);
        d0.fdst = fields->f[0];
        launch_init_state(d0, fields->flags[1], s);
        launch_seg_compact(d0, s);
        // the second buffer starts as a copy, so every cell of both buffers
        // holds a defined value (w_q away from the fluid) from here on
        const size_t fbytes = (size_t)Q * N * pdf_elem_bytes(c->p.storage);
        if (cudaMemcpyAsync(fields->f[1], fields->f[0], fbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) break;
        if (cudaGetLastError() != cudaSuccess) break;
        if (read_near(c) != FSL_OK) break;
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
    c->adj_valid = 0;
    Dev d = dev_for(c, c->parity);
    CK(cudaMemsetAsync(d.counts, 0, C_NCOUNT * sizeof(int), c->stream));
    CK(cudaMemsetAsync(d.seg_active, 0, d.nseg, c->stream));
    CK(cudaMemsetAsync(d.rmark, 0, d.N, c->stream));
    launch_refresh(d, c->stream);
    launch_seg_compact(d, c->stream);
    if (c->bubble) {  // the caller may have changed the liquid volume: recount it
        CK(cudaMemsetAsync(c->base.bub_i, 0, 5 * sizeof(long long), c->stream));
        launch_bubble_count(d, c->stream);
    }
    CK(cudaGetLastError());
    return read_near(c);
}

int fsl_step(fsl_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return FSL_EINVAL;
    if (nsteps > 0) c->adj_valid = 0;
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
    c->adj_valid = 0;
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
        const bool fused = c->p.curv_model == FSL_CURV_LSQR;
        if (fused) launch_curv_iface(d, s);  // curvature + interface stream-collide
        else if (c->p.curv_model == FSL_CURV_MLP) launch_lsqr(d, d.kappa, s);
        else if (c->p.curv_model == FSL_CURV_FD) launch_fd(d, d.kappa, s);
        else if (c->p.curv_model == FSL_CURV_TR) launch_tr(d, d.kappa, s);
        else launch_zero_kappa(d, d.kappa, s);
        if (c->p.curv_model == FSL_CURV_MLP) launch_mlp_curv(d, d.kappa, s);
        if (cudaEventRecord(ev[2], s) != cudaSuccess) break;
        launch_sc_bulk(d, s);
        if (cudaEventRecord(ev[3], s) != cudaSuccess) break;
        if (!fused) launch_sc_iface(d, s);
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
    if (!c || !kappa_out || model < FSL_CURV_LSQR || model > FSL_CURV_TR) return FSL_EINVAL;
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

// gas volume of the current state from the bubble counters (synchronising)
static int bubble_volume(fsl_ctx *c, double *V) {
    long long b[5];
    CK(cudaMemcpyAsync(b, c->base.bub_i, sizeof b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int par = c->parity;
    *V = (double)(b[4] - b[par]) - (double)b[2 + par] / BUB_FIX;
    return FSL_OK;
}

int fsl_set_bubble(fsl_ctx *c, double p0, double V0) {
    if (!c || !isfinite(p0) || !isfinite(V0) || p0 < 0.0) return FSL_EINVAL;
    for (int k = 0; k < 2; ++k)  // recorded graphs hold the old kernel arguments
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
    c->adj_valid = 0;
    if (p0 == 0.0) {
        c->bubble = 0;
        c->base.bub_i = nullptr;
        c->base.bub_d = nullptr;
        c->base.bub_rho = nullptr;
        return FSL_OK;
    }
    const Layout L = layout(c->p);
    char *bw = static_cast<char *>(c->fields.workspace) + L.bubble;
    c->base.bub_i = reinterpret_cast<long long *>(bw);
    c->base.bub_d = reinterpret_cast<double *>(bw + 8 * sizeof(long long));
    c->base.bub_rho = reinterpret_cast<float *>(bw + 8 * sizeof(long long) + 2 * sizeof(double));
    c->bubble = 1;
    const Dev d = dev_for(c, c->parity);
    CK(cudaMemsetAsync(c->base.bub_i, 0, 8 * sizeof(long long), c->stream));
    launch_bubble_count(d, c->stream);
    double V = 0.0;
    const int rc = bubble_volume(c, &V);
    if (rc != FSL_OK) return rc;
    const double pd[2] = {p0, V0 > 0.0 ? V0 : V};
    if (!(pd[1] > 0.0)) return FSL_EINVAL;  // no gas in the state
    const float r0 = (float)(3.0 * p0 * pd[1] / V);
    CK(cudaMemcpyAsync(c->base.bub_d, pd, sizeof pd, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->base.bub_rho, &r0, sizeof r0, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FSL_OK;
}

int fsl_bubble(fsl_ctx *c, double *volume, double *p_gas) {
    if (!c || !c->bubble) return FSL_EINVAL;
    double V = 0.0;
    const int rc = bubble_volume(c, &V);
    if (rc != FSL_OK) return rc;
    double pd[2];
    CK(cudaMemcpy(pd, c->base.bub_d, sizeof pd, cudaMemcpyDeviceToHost));
    if (volume) *volume = V;
    if (p_gas) *p_gas = V > 0.0 ? pd[0] * pd[1] / V : c->p.p_gas;
    return FSL_OK;
}

int fsl_prescribe_flow(fsl_ctx *c, double rho, double ux, double uy, double uz) {
    if (!c || !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) return FSL_EINVAL;
    Dev d = dev_for(c, c->parity);
    d.fdst = c->fields.f[c->parity];  // the current buffer: what the next step streams from
    launch_prescribe(d, (float)rho, (float)ux, (float)uy, (float)uz, c->stream);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_conversions(fsl_ctx *c, int64_t counts_out[4], int32_t *cells_out, int64_t capacity) {
    if (!c || !counts_out || (cells_out && capacity < 0)) return FSL_EINVAL;
    const Dev d = dev_for(c, c->parity);
    int cnt[C_NCOUNT];
    CK(cudaMemcpyAsync(cnt, d.counts, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int *lists[4] = {d.fill, d.empty, d.newgas, d.liq2if};
    const int n[4] = {cnt[C_FILL], cnt[C_EMPTY], cnt[C_NEWGAS], cnt[C_LIQ2IF]};
    std::vector<int32_t> v[4];
    for (int k = 0; k < 4; ++k) {
        if (n[k] < 0 || n[k] > c->base.N) return FSL_ECUDA;
        v[k].resize((size_t)n[k]);
        if (n[k]) CK(cudaMemcpy(v[k].data(), lists[k], (size_t)n[k] * sizeof(int), cudaMemcpyDeviceToHost));
    }
    // an emptying candidate that a filling neighbour kept at the interface is
    // not emptied: keep the candidates whose type after the step is gas
    std::vector<int32_t> emptied;
    for (int32_t i : v[1]) {
        uint8_t f = 0;
        CK(cudaMemcpy(&f, c->fields.flags[0] + i, 1, cudaMemcpyDeviceToHost));
        if ((f & T_MASK) == T_GAS) emptied.push_back(i);
    }
    v[1].swap(emptied);
    int64_t total = 0;
    for (int k = 0; k < 4; ++k) {
        std::sort(v[k].begin(), v[k].end());
        counts_out[k] = (int64_t)v[k].size();
        total += counts_out[k];
    }
    if (!cells_out) return FSL_OK;
    if (total > capacity) return FSL_ECAPACITY;
    for (int k = 0; k < 4; ++k) {
        memcpy(cells_out, v[k].data(), v[k].size() * sizeof(int32_t));
        cells_out += v[k].size();
    }
    return FSL_OK;
}

size_t fsl_adjoint_workspace_size(const fsl_params *params, int window, int ckpt_every, int max_interface) {
    if (!valid_params(params) || window < 1 || ckpt_every < 1 || max_interface < 1) return 0;
    const int K = ckpt_every < window ? ckpt_every : window;
    return adj_layout(*params, window, K, max_interface).total;
}

int fsl_set_surface(fsl_ctx *c, double sigma, double theta) {
    if (!c || !isfinite(sigma) || !isfinite(theta)) return FSL_EINVAL;
    c->p.sigma = sigma;
    c->p.theta = theta;
    c->base.six_sigma = (float)(6.0 * sigma);
    c->base.cos_theta = (float)cos(theta);
    c->base.sin_theta = (float)sin(theta);
    c->base.cos_theta_d = cos(theta);
    c->base.sin_theta_d = sin(theta);
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
    c->adj_valid = 0;
    return FSL_OK;
}

int fsl_window_forward(fsl_ctx *c, int window, int ckpt_every, int max_interface, void *adj_ws, size_t adj_bytes) {
    if (!c || window < 1 || ckpt_every < 1 || max_interface < 1 || !aligned(adj_ws)) return FSL_EINVAL;
    if (!adjoint_supported(c->p) || c->bubble) return FSL_EUNSUPPORTED;
    const int K = ckpt_every < window ? ckpt_every : window;
    const AdjLayout A = adj_layout(c->p, window, K, max_interface);
    if (adj_bytes < A.total) return FSL_EINVAL;
    c->adj_valid = 0;
    char *ws = static_cast<char *>(adj_ws);
    const size_t N = (size_t)c->base.N;
    int nif = 0;
    const int rc = window_setup(c, ws, A, &nif);
    if (rc != FSL_OK) return rc;
    if (nif > max_interface) return FSL_ECAPACITY;
    Dev d = window_dev(c, ws, A);
    int par = c->parity;
    for (int t = 0; t < window; ++t) {
        if (t % K == 0) {
            const StatePtrs ck = state_at(ws, A.ckpt + (size_t)(t / K) * A.state_bytes, N);
            CK(cudaMemcpyAsync(ck.f, c->fields.f[par], 19 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
            CK(cudaMemcpyAsync(ck.m, c->fields.mass, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
            CK(cudaMemcpyAsync(ck.phi, c->fields.phi, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        }
        d.fsrc = c->fields.f[par];
        d.fdst = c->fields.f[par ^ 1];
        d.mass = c->fields.mass;
        d.phi = c->fields.phi;
        d.kappa = c->fields.kappa;
        d.normal = c->base.normal;
        launch_frozen_step(d, c->stream);
        par ^= 1;
    }
    launch_window_finish(dev_for(c, par), reinterpret_cast<int *>(ws + A.wcounts),
                         reinterpret_cast<int *>(ws + A.wlist), c->stream);
    if (cudaGetLastError() != cudaSuccess) return FSL_ECUDA;
    c->parity = par;
    c->adj_ws = adj_ws;
    c->adj_window = window;
    c->adj_ckpt = K;
    c->adj_cap = max_interface;
    c->adj_valid = 1;
    return FSL_OK;
}

int fsl_window_adjoint(fsl_ctx *c, const float *dL_dphi, double *dL_dsigma, double *dL_dtheta, float *dL_dphi0,
                       float *dL_dmass0, float *dL_df0) {
    if (!c || !dL_dphi || !c->adj_valid) return FSL_EINVAL;
    const int W = c->adj_window, K = c->adj_ckpt;
    const AdjLayout A = adj_layout(c->p, W, K, c->adj_cap);
    char *ws = static_cast<char *>(c->adj_ws);
    const size_t N = (size_t)c->base.N;
    cudaStream_t st = c->stream;
    Adj a = adj_args(ws, A, c->adj_cap);
    float *fb[2] = {reinterpret_cast<float *>(ws + A.fb0), reinterpret_cast<float *>(ws + A.fb1)};
    CK(cudaMemsetAsync(fb[0], 0, 19 * N * sizeof(float), st));
    CK(cudaMemsetAsync(fb[1], 0, 19 * N * sizeof(float), st));
    CK(cudaMemsetAsync(a.mb, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(a.pb, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(a.kb, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(a.acc, 0, 2 * sizeof(double), st));
    Dev w = window_dev(c, ws, A);
    launch_adjoint_seed(w, a, dL_dphi, st);
    int cur = 0;  // fb[cur] holds the adjoint of f' at the step after the one being reversed
    for (int sgm = A.nseg_ckpt - 1; sgm >= 0; --sgm) {
        const int len = (W - sgm * K) < K ? (W - sgm * K) : K;
        const StatePtrs ck = state_at(ws, A.ckpt + (size_t)sgm * A.state_bytes, N);
        auto state = [&](int t) { return t == 0 ? ck : state_at(ws, A.slot + (size_t)(t - 1) * A.state_bytes, N); };
        auto kn = [&](int t, float **kap, float4 **nrm) {
            char *b = ws + A.kn + (size_t)t * A.kn_bytes;
            *kap = reinterpret_cast<float *>(b);
            *nrm = reinterpret_cast<float4 *>(b + up(N * sizeof(float)));
        };
        // recompute the segment, keeping every state
        for (int t = 0; t < len; ++t) {
            const StatePtrs s0 = state(t), s1 = state(t + 1);
            CK(cudaMemcpyAsync(s1.m, s0.m, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(s1.phi, s0.phi, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
            Dev d = w;
            d.fsrc = s0.f;
            d.fdst = s1.f;
            d.mass = s1.m;
            d.phi = s1.phi;
            kn(t, &d.kappa, &d.normal);
            launch_frozen_step(d, st);
        }
        // reverse it
        for (int t = len - 1; t >= 0; --t) {
            const StatePtrs s0 = state(t);
            Dev d = w;
            d.fsrc = s0.f;
            d.fdst = nullptr;
            d.mass = s0.m;
            d.phi = s0.phi;
            kn(t, &d.kappa, &d.normal);
            a.fb_in = fb[cur];
            a.fb_out = fb[cur ^ 1];
            launch_adjoint_step(d, a, st);
            cur ^= 1;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return FSL_ECUDA;
    if (dL_dphi0) CK(cudaMemcpyAsync(dL_dphi0, a.pb, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (dL_dmass0) CK(cudaMemcpyAsync(dL_dmass0, a.mb, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (dL_df0) CK(cudaMemcpyAsync(dL_df0, fb[cur], 19 * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->host_mass + 2, a.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (dL_dsigma) *dL_dsigma = c->host_mass[2];
    if (dL_dtheta) *dL_dtheta = c->host_mass[3];
    int status = 0;
    CK(cudaMemcpy(&status, c->base.status, sizeof(int), cudaMemcpyDeviceToHost));
    return status ? status : FSL_OK;
}

int fsl_kappa_jacobian(fsl_ctx *c, void *adj_ws, size_t adj_bytes, int max_interface, float *jac_out,
                       int32_t *cells_out, float *kappa_out, int *n_out) {
    if (!c || max_interface < 1 || !aligned(adj_ws) || !jac_out || !cells_out || !kappa_out || !n_out)
        return FSL_EINVAL;
    if (!adjoint_supported(c->p)) return FSL_EUNSUPPORTED;
    const AdjLayout A = adj_layout(c->p, 1, 1, max_interface);
    if (adj_bytes < A.total) return FSL_EINVAL;
    char *ws = static_cast<char *>(adj_ws);
    if (adj_ws == c->adj_ws) c->adj_valid = 0;  // the window's buffers are reused
    int nif = 0;
    const int rc = window_setup(c, ws, A, &nif);
    if (rc != FSL_OK) return rc;
    *n_out = nif;
    if (nif > max_interface) return FSL_ECAPACITY;
    Adj a = adj_args(ws, A, max_interface);
    a.jac = jac_out;
    a.jval = kappa_out;
    Dev d = window_dev(c, ws, A);
    d.phi = c->fields.phi;
    d.normal = c->base.normal;
    launch_normals(d, c->stream);  // the fit reads the normals of this state
    launch_kappa_jacobian(d, a, c->stream);
    CK(cudaMemcpyAsync(cells_out, a.wlist, (size_t)nif * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ECUDA;
}

int fsl_parity(const fsl_ctx *c) { return c ? c->parity : FSL_EINVAL; }

int fsl_status(fsl_ctx *c) {
    if (!c) return FSL_EINVAL;
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->base.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return st;
}

// ---- checkpoint / resume -------------------------------------------------------
int fsl_save(fsl_ctx *c, const char *path) {
    if (!c || !path) return FSL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FSL_ECUDA;
    const size_t N = (size_t)c->p.nx * c->p.ny * c->p.nz;
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "FSLCKPT1", 8);
    h.version = 2;  // 2: fsl_params with excess_rule
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.nz = c->p.nz;
    h.storage = c->p.storage;
    h.storage_shift = c->p.storage_shift;
    h.params = c->p;
    if (cudaMemcpy(&h.lost, c->base.lost, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return FSL_ECUDA;
    // cell types without the near-obstacle and transient bits
    uint8_t *fl = static_cast<uint8_t *>(malloc(N ? N : 1));
    if (!fl) return FSL_EIO;
    if (cudaMemcpy(fl, c->fields.flags[0], N, cudaMemcpyDeviceToHost) != cudaSuccess) {
        free(fl);
        return FSL_ECUDA;
    }
    for (size_t i = 0; i < N; ++i) fl[i] &= T_MASK;
    FILE *fp = fopen(path, "wb");
    if (!fp) {
        free(fl);
        return FSL_EIO;
    }
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1;
    ok = ok && dev_to_file(fp, c->fields.f[c->parity], (size_t)Q * N * pdf_elem_bytes(c->p.storage), c->stream);
    ok = ok && fwrite(fl, 1, N, fp) == N;
    ok = ok && dev_to_file(fp, c->fields.mass, N * sizeof(float), c->stream);
    ok = ok && dev_to_file(fp, c->fields.phi, N * sizeof(float), c->stream);
    free(fl);
    if (fclose(fp) != 0) ok = false;
    return ok ? FSL_OK : FSL_EIO;
}

int fsl_load(fsl_ctx *c, const char *path) {
    if (!c || !path) return FSL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FSL_ECUDA;
    const size_t N = (size_t)c->p.nx * c->p.ny * c->p.nz;
    const size_t fbytes = (size_t)Q * N * pdf_elem_bytes(c->p.storage);
    // the whole file is read and checked before any device buffer changes, so
    // a failed load leaves the context's state as it was
    const size_t body = fbytes + N + 2 * N * sizeof(float);
    FILE *fp = fopen(path, "rb");
    if (!fp) return FSL_EIO;
    CkptHeader h;
    bool ok = fread(&h, sizeof h, 1, fp) == 1 && memcmp(h.magic, "FSLCKPT1", 8) == 0 && h.version == 2 &&
              h.nx == c->p.nx && h.ny == c->p.ny && h.nz == c->p.nz && h.storage == c->p.storage &&
              h.storage_shift == c->p.storage_shift;
    char *buf = ok ? static_cast<char *>(malloc(body ? body : 1)) : nullptr;
    ok = ok && buf && fread(buf, 1, body, fp) == body && fgetc(fp) == EOF;  // exact length
    fclose(fp);
    if (!ok) {
        free(buf);
        return FSL_EIO;
    }
    cudaStream_t s = c->stream;
    const char *src = buf;
    bool cu = cudaMemcpyAsync(c->fields.f[c->parity], src, fbytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    src += fbytes;
    cu = cu && cudaMemcpyAsync(c->fields.flags[0], src, N, cudaMemcpyHostToDevice, s) == cudaSuccess;
    src += N;
    cu = cu && cudaMemcpyAsync(c->fields.mass, src, N * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess;
    src += N * sizeof(float);
    cu = cu && cudaMemcpyAsync(c->fields.phi, src, N * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess;
    cu = cu && cudaMemcpyAsync(c->base.lost, &h.lost, sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
    cu = cu && cudaStreamSynchronize(s) == cudaSuccess;  // the staging buffer is freed below
    free(buf);
    if (!cu) return FSL_ECUDA;
    const int rc = fsl_refresh(c);
    if (rc != FSL_OK) return rc;
    return cudaStreamSynchronize(s) == cudaSuccess ? FSL_OK : FSL_ECUDA;
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
    case FSL_EIO: return "checkpoint file error or mismatch";
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
    if (c->host_count) cudaFreeHost(c->host_count);
    delete c;
}

}  // extern "C"
