/*
 * fsl.h -- C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann step
 * with least-squares and finite-difference curvature (Bogner, Ruede, Harting,
 * arXiv 1509.07691).
 *
 * Memory and ownership
 *   All field buffers are caller-owned device memory (for instance torch
 *   tensors), described by fsl_fields.  The library borrows them for the
 *   lifetime of the context and never frees them.  It allocates nothing on
 *   the device itself: every piece of scratch lives in the caller's
 *   workspace buffer (size from fsl_workspace_size).
 *
 * Layout (shared with any checker: plain arrays, x fastest)
 *   cell index   i = x + nx*(y + ny*z), 0 <= i < N = nx*ny*nz.  All three axes
 *                wrap periodically; walls are cells of type FSL_OBSTACLE.
 *   PDFs         f[q*N + i], q in the D3Q19 order
 *                  q  : 0  1  2  3  4  5  6  7  8  9 10 11 12 13 14 15 16 17 18
 *                  cx : 0  1 -1  0  0  0  0  1 -1  1 -1  1 -1  1 -1  0  0  0  0
 *                  cy : 0  0  0  1 -1  0  0  1 -1 -1  1  0  0  0  0  1 -1  1 -1
 *                  cz : 0  0  0  0  0  1 -1  0  0  0  0  1 -1 -1  1  1 -1 -1  1
 *                stored as float (FSL_F32), or as (f - w_q) * 2^storage_shift in
 *                IEEE half (FSL_F16_OFS) or bfloat16 (FSL_BF16_OFS).
 *                Between steps the current buffer holds post-collision values f'
 *                at liquid and interface cells.  fsl_init writes w_q into every
 *                cell of both buffers; a non-fluid cell keeps w_q or the last
 *                value written while it was fluid, and no step reads it.
 *   flags        one byte per cell: bits 0..3 the cell type (one of the FSL_*
 *                type values below), bit 4 FSL_NEAR_OBSTACLE (set by the
 *                library: the cell has an obstacle D3Q19 neighbour), bits 5..7
 *                zero between steps.  The buffers hold N bytes rounded up to a
 *                multiple of 4.
 *   mass, phi    float per cell: mass m and fill level phi = m / rho (meaningful
 *                at interface cells; phi = 1 at liquid, 0 at gas cells).
 *   kappa        float per cell: the curvature last computed (interface cells).
 *
 * Streams and synchronisation
 *   Every call enqueues its work on the stream given to fsl_init and returns
 *   without waiting, except the calls marked "synchronising".
 *
 * Errors
 *   Functions return FSL_OK (0) or a negative code.  Device-side failures set
 *   a sticky status word that fsl_status reads.  A context is not thread
 *   safe: use one context per host thread and stream.
 */
#ifndef FSL_H
#define FSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSL_OK 0
#define FSL_EINVAL (-1)       /* invalid parameter, shape or pointer */
#define FSL_ECUDA (-2)        /* a CUDA runtime call failed */
#define FSL_ECAPACITY (-3)    /* a device list overflowed (state not advanced) */
#define FSL_ETIMEOUT (-4)     /* a bounded device wait gave up */
#define FSL_ENAN (-5)         /* non-finite value found in the state */
#define FSL_EUNSUPPORTED (-6) /* option not available in this build */
#define FSL_EIO (-7)          /* checkpoint file unreadable, unwritable or not matching the context */

/* cell types (Sec. II: liquid, interface, gas cells; walls are obstacle cells) */
#define FSL_LIQUID 1
#define FSL_INTERFACE 2
#define FSL_GAS 4
#define FSL_OBSTACLE 8
#define FSL_TYPE_MASK 15
#define FSL_NEAR_OBSTACLE 16

typedef struct fsl_ctx fsl_ctx; /* opaque */

enum fsl_collision { FSL_BGK = 0, FSL_TRT = 1 };
enum fsl_curv_model { FSL_CURV_LSQR = 0, FSL_CURV_FD = 1, FSL_CURV_NONE = 2, FSL_CURV_MLP = 3, FSL_CURV_TR = 4 };
enum fsl_storage { FSL_F32 = 0, FSL_F16_OFS = 1, FSL_BF16_OFS = 2 };
enum fsl_where { FSL_NONE = 0, FSL_HOST = 1, FSL_DEVICE = 2 };

/* Parameters of the method (Sec. II).  All lattice units. */
typedef struct fsl_params {
    int32_t nx, ny, nz;     /* grid; each >= 3 */
    int32_t collision;      /* FSL_BGK or FSL_TRT (two relaxation times) */
    int32_t curv_model;     /* model used inside fsl_step */
    int32_t storage;        /* fsl_storage of the PDF buffers */
    int32_t storage_shift;  /* power-of-two scale of 16-bit offsets (e.g. 8) */
    int32_t plic_iters;     /* Newton steps of the PLIC offset in its cubic branch (e.g. 4) */
    double tau;             /* relaxation time, nu = (tau - 1/2)/3; > 1/2 */
    double magic;           /* TRT Lambda = (tau - 1/2)(tau_odd - 1/2), e.g. 3/16 */
    double sigma;           /* surface tension */
    double p_gas;           /* gas pressure p_g (1/3 gives rho_b = 1 at sigma = 0) */
    double theta;           /* equilibrium contact angle theta_eq, radians */
    double eps_convert;     /* conversion threshold eps, e.g. 1e-3 */
    double lsqr_fp64_cond;  /* condition estimate of the LSQR normal equations A^T A,
                               (max R_jj / min R_jj)^2 of its FP32 factor, above which
                               the cell is re-solved in FP64 (e.g. 1e6) */
    int32_t excess_rule;    /* excess mass of converted cells (the conversion rules the
                               paper cites from Koerner et al.): 0 equal shares among the
                               interface neighbours after conversion; 1 shares weighted
                               by the cell's interface normal n (into the liquid): a
                               filled cell gives max(0, -n.c_q), an emptied one
                               max(0, n.c_q) to the receiver at x + c_q, equal shares
                               if every weight is 0 */
    int32_t pad_;
} fsl_params;

/* Caller-owned device buffers (all 256-byte aligned). */
typedef struct fsl_fields {
    void *f[2];          /* 19*N PDFs each, element type per params.storage */
    uint8_t *flags[2];   /* N bytes rounded up to a multiple of 4, each; flags[0]
                            holds the cell types, flags[1] is scratch */
    float *mass;         /* N */
    float *phi;          /* N */
    float *kappa;        /* N */
    void *workspace;     /* fsl_workspace_size(params) bytes */
} fsl_fields;

/* Geometry of the initial fill levels (Sec. III.A: each cell is sub-divided
 * sub^3 times and phi is the fraction of sub-cell centres inside the shape). */
typedef struct fsl_geometry {
    int32_t kind;     /* 0 sphere |x-c| <= R; 1 P2-perturbed sphere
                         r <= R (1 + eps2 P2(cos th)); 2 spherical cap: sphere and
                         z >= zw; 3 union of spheres (c, R) and (c2, R2);
                         4 pool z < h0 + amp sin(2 pi x/L) sin(2 pi y/L);
                         5 half-space n.x <= d */
    int32_t invert;   /* 1: liquid outside the shape (a bubble) */
    int32_t sub;      /* sub-samples per axis, 1..64 */
    int32_t pad_;
    double c[3], R, eps2;
    double c2[3], R2;
    double zw;
    double n[3], d;
    double h0, amp, wavelength;
} fsl_geometry;

/* Bytes of workspace the context needs for these parameters. */
size_t fsl_workspace_size(const fsl_params *params);

/* Fill levels of a geometry by sub-sampling (Sec. III.A), written to phi_dev
 * (N floats, device).  Sample points are x + (s + 1/2)/sub - 1/2 in each axis;
 * inside tests run in FP64 without contraction.  Asynchronous on `stream`. */
int fsl_fill_geometry(const fsl_params *params, const fsl_geometry *geom, float *phi_dev, void *stream);

/* Create a context and set up the initial state (Sec. II):
 *   phi0       fill levels (N floats) on the host (FSL_HOST), on the device
 *              (FSL_DEVICE), or FSL_NONE to take fields->phi as it is;
 *   obstacle   N bytes, nonzero = obstacle cell, host or device, or FSL_NONE;
 * then types from phi (phi <= 0 gas, >= 1 liquid, else interface; every
 * liquid cell with a gas neighbour becomes interface), f = w_q, m = phi, and
 * the interface list.  fields->f[0] and flags[0] hold the state afterwards;
 * fields->f[1] is a copy of fields->f[0].
 * Queued on `stream` (a cudaStream_t, or NULL for the default stream); returns
 * after that stream has drained, having read back whether any cell has an
 * obstacle neighbour (a domain without one runs its rare general-path LSQR
 * fits inside the fused step kernel instead of a kernel of their own). */
int fsl_init(const fsl_params *params, const fsl_fields *fields, const float *phi0, int phi0_where,
             const uint8_t *obstacle, int obstacle_where, void *stream, struct fsl_ctx **out);

/* The caller wrote a state directly into f[parity], flags[0] (type bits),
 * mass and phi: recompute the near-obstacle bits, the interface list and the
 * active row segments.
 * Synchronising: returns after the context's stream has drained (it reads
 * back whether any cell has an obstacle neighbour, as fsl_init). */
int fsl_refresh(struct fsl_ctx *ctx);

/* Checkpoint and resume (a service of this library; the paper has no
 * counterpart).  fsl_save writes the state of the context after all work
 * queued on its stream: a header (magic "FSLCKPT1", format version 2, nx, ny,
 * nz, storage, storage_shift, the lost-mass counter, the context's
 * fsl_params), then the current PDF buffer f[parity] (19 N values in the
 * storage type, f[q N + i]), the cell types (N bytes, type bits only), mass
 * and phi (N floats each).  fsl_load reads such a file into a context with
 * the same nx, ny, nz, storage and storage_shift (FSL_EIO otherwise; the
 * other parameters of the loading context apply from then on), writes the
 * state into the current buffers, restores the lost-mass counter and
 * rebuilds the near-obstacle bits, interface list and active segments (as
 * fsl_refresh).  fsl_load reads and checks the whole file (header fields and
 * exact length) in host memory before it writes any device buffer, so a
 * failed load (FSL_EIO) leaves the context's state unchanged.  Both are
 * synchronising and stage data in host memory they allocate and free.
 * FSL_EINVAL for NULL arguments, FSL_EIO for file errors. */
int fsl_save(struct fsl_ctx *ctx, const char *path);
int fsl_load(struct fsl_ctx *ctx, const char *path);

/* Advance nsteps time steps (Sec. II): curvature kappa(t) of every interface
 * cell by params.curv_model; pull stream with Eq. (reconstruct) at gas links
 * (rho_b = 3 p_g + 6 sigma kappa, u_b = u(x,t)) and at contact-line obstacle
 * links whose outgoing direction points against the interface normal projected
 * into the wall, bounce-back at other obstacle links; mass exchange Eqs.
 * (advection1/2); BGK/TRT collision; conversion of interface cells with
 * m > (1+eps) rho or m < -eps rho, neighbourhood fix and equal sharing of the
 * excess mass among interface neighbours.  The step sequence is recorded as
 * a CUDA graph on first use.  Asynchronous. */
int fsl_step(struct fsl_ctx *ctx, int nsteps);

/* Curvature of the current state by `model` (Sec. II.A FD with K8 smoothing
 * and wetting normals, Eq. contactNormal; Sec. II.C LSQR paraboloid fit to
 * PLIC points with contact-point rows/constraints, Eq. contactConstraint;
 * Sec. II.B TR: a triangle fan of the PLIC points of the 3x3x3 block around
 * the centre point, ordered by angle in its tangent plane, and the mean of
 * the directional curvatures 2h/|p|^2 weighted by the areas of the fan
 * triangles at each edge, without a wetting treatment), written to kappa_out
 * (N floats, device; interface cells only; may be fields->kappa).
 * Asynchronous. */
int fsl_curvature(struct fsl_ctx *ctx, int model, float *kappa_out);

/* Total mass sum_interface m + sum_liquid rho, and the mass lost by
 * conversions with no interface neighbour.  Block partial sums in FP64 are
 * added in a fixed order.  Synchronising. */
int fsl_mass(struct fsl_ctx *ctx, double *total_mass, double *lost_mass);

/* counts_out[0..9]: liquid, interface, gas, obstacle cells, interface cells
 * without a liquid or without a gas neighbour, liquid cells touching gas,
 * LSQR cells solved in FP64 (last curvature pass), interface list length,
 * cells the learned curvature evaluated and cells where its value was kept
 * (last FSL_CURV_MLP pass).  Synchronising. */
int fsl_stats(struct fsl_ctx *ctx, int64_t counts_out[10]);

/* Bubble model (Sec. III.A: the gas is not simulated; its pressure follows
 * the gas volume).  With p0 > 0 the gas pressure of every step is
 * p_g = p0 V0 / V (isothermal ideal gas), V the gas volume of the state the
 * step starts from: non-obstacle cells minus liquid cells minus the sum of
 * the interface fill levels (gas cells count 1, interface cells 1 - phi).
 * V0 > 0 sets the reference volume, V0 <= 0 takes the current one.  The
 * volume is counted from the state here and by fsl_refresh / fsl_load, and
 * tracked by the step's own kernels in between (integer fixed-point sums, so
 * it does not depend on the order of additions).  It is one total: several
 * separate bubbles share one pressure.  p0 = 0 switches the model off
 * (params.p_gas applies again).  Adjoint windows are unsupported while it is
 * on.  Synchronising; FSL_EINVAL for p0 < 0 or a state without gas. */
int fsl_set_bubble(struct fsl_ctx *ctx, double p0, double V0);

/* Gas volume of the current state and the gas pressure the next step uses
 * (bubble model on; FSL_EINVAL otherwise).  Synchronising. */
int fsl_bubble(struct fsl_ctx *ctx, double *volume, double *p_gas);

/* Prescribed flow for the advection test of Sec. III.A (Tab. advection):
 * sets the current post-collision PDFs of every liquid and interface cell to
 * the equilibrium feq(rho, u) (standard second-order D3Q19 form), so that the
 * next fsl_step moves the fill level through the mass exchange of Eqs.
 * (advection1/2) and the conversions in a constant flow; calling it before
 * every step keeps the lattice Boltzmann data constant.  rho > 0.
 * Asynchronous. */
int fsl_prescribe_flow(struct fsl_ctx *ctx, double rho, double ux, double uy, double uz);

/* Conversions of the last fsl_step (Sec. II; the rules the paper cites from
 * Koerner et al., see fsl_step): counts_out[0..3] = cells that filled
 * (interface -> liquid), emptied (interface -> gas; a candidate kept at the
 * interface by a filling neighbour is not counted), became interface from
 * gas, and became interface from liquid.  If cells_out is not NULL the cell
 * indices of the four sets follow one another there, each set in ascending
 * order (host memory, capacity entries; FSL_ECAPACITY if they do not fit).
 * Valid until the next fsl_step or fsl_curvature; zero after fsl_init,
 * fsl_refresh and fsl_load.  Synchronising. */
int fsl_conversions(struct fsl_ctx *ctx, int64_t counts_out[4], int32_t *cells_out, int64_t capacity);

/* One time step like fsl_step(ctx, 1), launched kernel by kernel (no graph,
 * phases in sequence) with CUDA events on the context's stream between its
 * phases; ms_out[0..5] receive the device time of: normals + PLIC, curvature,
 * liquid stream-collide, interface stream-collide, conversion, finalize.  With
 * the LSQR model the curvature and the interface stream-collide run fused (one
 * pass per cell): their time is in ms_out[1] and ms_out[3] is the empty
 * interval.  For profiling.  Synchronising. */
int fsl_step_profile(struct fsl_ctx *ctx, float ms_out[6]);

/* Total mass of a state (sum of m over interface cells plus sum of rho over
 * liquid cells) for callers that cannot allocate device memory: a host
 * application that owns all device memory through its own allocator or a
 * fixed budget, or monitoring code in a time-critical loop that must not pay
 * for an allocation.  The paper has no counterpart; it is a service of this
 * library.  The caller passes the state (f: the current PDF buffer, storage
 * per params; flags; mass) and one device double for the result.  Nothing is
 * allocated: the block partial sums go to a fixed FP64 array of
 * FSL_MASS_STATIC_MAX_BLOCKS entries (32 KiB) that every GPU loading the
 * library holds until the process exits.  Grids with more than
 * FSL_MASS_STATIC_MAX_CELLS cells are rejected with FSL_EINVAL.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress with
 * that device current); make that first call before any stream capture.
 * Every call uses the same array, so calls whose kernels overlap on the GPU
 * (for instance on two streams without ordering) race and give wrong sums.
 * Asynchronous on `stream`; the result is in total_dev when the stream reaches it. */
#define FSL_MASS_STATIC_CELLS_PER_BLOCK 65536
#define FSL_MASS_STATIC_MAX_BLOCKS 4096
#define FSL_MASS_STATIC_MAX_CELLS 268435456LL
int fsl_mass_static(const fsl_params *params, const void *f, const uint8_t *flags, const float *mass,
                    double *total_dev, void *stream);

/* ---- Learned curvature (extension beyond the paper: an MLP estimate of the
 * curvature from the 5x5x5 fill-level stencil, with the LSQR fit of Sec. II.C
 * as judge and fallback) ------------------------------------------------------
 * Network: x = bf16(2 phi - 1) over the canonical stencil (axes flipped so the
 * Parker-Youngs normal of the middle cell is non-negative, then ordered by
 * decreasing |n_k|; 125 values, 3 zero pads), z1 = W1 x + b1,
 * h1 = bf16(gelu(z1)), z2 = W2 h1 + b2, y = w3 . gelu(z2) + b3 = kappa dx,
 * gelu(x) = x Phi(x).  BF16 weights, FP32 accumulation on the tensor cores.
 * Packed parameter block (device, fsl_mlp_param_bytes() bytes): bf16 W1[128][128]
 * (row = hidden unit), bf16 W2[128][128], bf16 w3[128], then at byte 65792
 * float b1[128], b2[128], b3.  FP32 master layout (fsl_mlp_master_count()
 * floats, also used for gradients and Adam moments): W1, W2, w3, b1, b2, b3. */
size_t fsl_mlp_param_bytes(void);
int fsl_mlp_master_count(void);

/* Training stencils: for each of n shape parameter sets (device arrays: axes
 * [n][3] semi-axes, quat [n][4] (w,x,y,z), dir [n][3] body-frame direction of
 * the surface point placed at the middle cell, delta [n][3] its offset from
 * the middle cell's centre, invert [n] 1 = liquid outside), the 5x5x5 fill
 * levels by sub^3 sub-sampling, Gaussian noise of s.d. `noise` on partially
 * filled cells (splitmix64 at counters 2k, 2k+1 for stencil cell k of sample s,
 * k = 125 s + cell, Box-Muller; clipped to [0, 1]), written as canonical BF16
 * rows X [n][128], and the target: mean curvature at the surface point nearest
 * the middle cell's centre (negative for liquid outside).  Asynchronous. */
int fsl_mlp_stencils(int n, const float *axes, const float *quat, const float *dir, const float *delta,
                     const int32_t *invert, int sub, float noise, uint64_t noise_seed, void *X, float *target,
                     void *stream);

/* y [n] = network(X [n][128] bf16); with z1, z2 (each [n][128] floats) the
 * pre-activations are kept for the backward pass.  Runs on the tcgen05 tensor
 * cores (both layers as 128 x 128 x 128 BF16 MMAs per 128-row tile, FP32
 * accumulators in tensor memory); uses about 133 KB of shared memory per SM.
 * Asynchronous; fsl_mlp_status reports a wait that ran out. */
int fsl_mlp_forward(const void *params, const void *X, int n, float *y, float *z1, float *z2, void *stream);

/* Sticky status of the tensor-core MLP kernels of this device: FSL_OK, or
 * FSL_ETIMEOUT if a bounded wait for the tensor cores ran out (the tiles not
 * finished are left unwritten).  reset != 0 clears it.  Synchronising. */
int fsl_mlp_status(int reset);

/* Bytes of workspace the training calls need for a batch of n. */
size_t fsl_mlp_train_workspace(int n);

/* Gradients (master layout) of loss = (1/n) sum w (y - t)^2, w = 1/(t^2 + 7e-5),
 * and the loss itself (one float, device; may be NULL).  The weight gradients
 * dW1 = d1^T x and dW2 = d2^T h1 run on the tcgen05 tensor cores with the
 * deltas rounded to BF16 and FP32 accumulation, one 128-sample chunk per CTA,
 * the chunks summed in a fixed order; the deltas and bias gradients in FP32.
 * Asynchronous. */
int fsl_mlp_gradients(const void *params, const void *X, const float *target, int n, float *grad, float *loss_dev,
                      void *workspace, void *stream);

/* One training step: gradients, then Adam (beta 0.9 / 0.999, eps 1e-8, bias
 * correction with step counted from 1) on the FP32 master weights, and the
 * packed BF16 parameters refreshed from them.  Asynchronous. */
int fsl_mlp_train_step(void *params, float *master, float *m, float *v, const void *X, const float *target, int n,
                       float lr, int step, float *loss_dev, void *workspace, void *stream);

/* Bytes of workspace fsl_mlp_train_epoch needs for batches of `batch` rows. */
size_t fsl_mlp_epoch_workspace(int batch);

/* One pass over a training set, the batch loop inside the library: for
 * b = 0 .. n/batch - 1 (a ragged tail is left out) the rows
 * perm[b*batch .. (b+1)*batch) of X ([n][128] BF16 rows, device, 16-byte
 * aligned) and of target (n floats, device) are gathered on the device and the
 * step of fsl_mlp_train_step is taken with step counter step0 + b + 1.  perm:
 * n int64 row indices on the device (a permutation for one epoch; an index
 * outside [0, n) gathers a zero row and target 0).  losses_dev: NULL or n/batch
 * floats (device) receiving each batch's loss.  workspace:
 * fsl_mlp_epoch_workspace(batch) bytes, 256-byte aligned.  FSL_EINVAL for
 * NULL pointers, batch < 1, n < batch, step0 < 0, lr <= 0 or misaligned
 * pointers.  Asynchronous. */
int fsl_mlp_train_epoch(void *params, float *master, float *m, float *v, const void *X, const float *target,
                        const int64_t *perm, int n, int batch, float lr, int step0, float *losses_dev,
                        void *workspace, void *stream);

/* Packed parameters from FP32 master weights (BF16 rounding).  Asynchronous. */
int fsl_mlp_pack(const float *master, void *params, void *stream);

/* Use the network in the context (curvature model FSL_CURV_MLP): after the LSQR
 * fit of every interface cell, the network's value replaces it where
 * |kappa_mlp - kappa_lsqr| <= fallback_rel |kappa_lsqr| and the stencil holds no
 * obstacle cell.  The parameters stay caller-owned.  Resets recorded graphs. */
int fsl_mlp_attach(struct fsl_ctx *ctx, const void *params, double fallback_rel);

/* ---- Adjoint windows (extension beyond the paper: gradients of a loss on the
 * fill level with respect to sigma and theta, through a window of steps with
 * frozen cell types) -----------------------------------------------------------
 * With the types frozen (no conversion test, no excess mass; the interface
 * list stays that of the window's first step) the step is a smooth map of the
 * state (f', m, phi) and of sigma (the Laplace term 2 sigma kappa of the
 * free-boundary condition, Eq. reconstruct) and theta (the contact normal of
 * the LSQR fit, Sec. II.C, Eq. contactNormal).  fsl_window_forward runs W such
 * steps and keeps a checkpoint of (f', m, phi) every K steps;
 * fsl_window_adjoint takes dL/dphi at the end of the window and returns
 * dL/dsigma and dL/dtheta (theta in radians) by the exact reverse of the
 * FP32 step: each K-step segment is recomputed from its checkpoint (all K
 * states kept), then reversed step by step.  Needs FSL_F32 storage, the LSQR
 * curvature (or FSL_CURV_NONE) and a grid of at least 7 cells per axis.
 *
 * Adjoint workspace: caller-owned device memory of
 * fsl_adjoint_workspace_size(params, W, K, max_interface) bytes (256-byte
 * aligned); max_interface bounds the interface cells of the window (one
 * curvature Jacobian row of FSL_JAC_STRIDE floats each).  The workspace must
 * stay untouched between the forward and the adjoint call. */
#define FSL_JAC_STRIDE 344 /* 7x7x7 window slots (dz+3)*49+(dy+3)*7+(dx+3), then theta */
size_t fsl_adjoint_workspace_size(const fsl_params *params, int window, int ckpt_every, int max_interface);

/* Change sigma and theta (radians) of the context.  Resets recorded graphs and
 * ends the current adjoint window. */
int fsl_set_surface(struct fsl_ctx *ctx, double sigma, double theta);

/* W steps with frozen cell types from the current state, checkpoints every K
 * steps into the adjoint workspace.  Afterwards the context holds the state
 * of step W; fsl_step continues from it (conversions resume).  Reads the
 * interface count once (synchronising); FSL_ECAPACITY if it exceeds
 * max_interface (nothing advanced). */
int fsl_window_forward(struct fsl_ctx *ctx, int window, int ckpt_every, int max_interface, void *adj_workspace,
                       size_t adj_bytes);

/* Reverse pass over the last window.  dL_dphi (device, N floats): dL/dphi at
 * the window's end; only interface entries are read (phi is constant at other
 * cells).  dL_dsigma, dL_dtheta: host doubles.  Optional device outputs
 * (NULL to skip), all at the window's start with phi, m and f' taken as
 * independent inputs: dL_dphi0 and dL_dmass0 (N floats, interface entries,
 * 0 elsewhere), dL_df0 (19 N floats, fluid cells, 0 elsewhere).
 * Synchronising.  The window stays valid (the call may be repeated with
 * another dL_dphi) until the context steps, refreshes or changes sigma/theta. */
int fsl_window_adjoint(struct fsl_ctx *ctx, const float *dL_dphi, double *dL_dsigma, double *dL_dtheta,
                       float *dL_dphi0, float *dL_dmass0, float *dL_df0);

/* Curvature Jacobian of the current state: for each interface cell x (order
 * in cells_out), row jac_out[k*FSL_JAC_STRIDE ...] = dkappa_x/dphi_y over the
 * interface cells y of the 7x7x7 window around x (slots of other cells are
 * not written) and dkappa_x/dtheta last; kappa_out[k] = kappa_x of the same
 * evaluation (forward-mode dual numbers through the LSQR fit).  Device
 * outputs of max_interface rows; adj_workspace as for a window of 1 step.
 * *n_out = interface cells (synchronising; FSL_ECAPACITY above max_interface). */
int fsl_kappa_jacobian(struct fsl_ctx *ctx, void *adj_workspace, size_t adj_bytes, int max_interface, float *jac_out,
                       int32_t *cells_out, float *kappa_out, int *n_out);

/* Which buffer (0 or 1) of fields->f holds the current PDFs. */
int fsl_parity(const struct fsl_ctx *ctx);

/* Sticky device status (FSL_OK or an error code).  Synchronising. */
int fsl_status(struct fsl_ctx *ctx);

const char *fsl_strerror(int code);

/* Release host-side resources and CUDA graphs (not the caller's buffers). */
void fsl_destroy(struct fsl_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif
