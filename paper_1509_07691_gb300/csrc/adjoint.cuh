// adjoint.cuh -- argument block and launch wrappers of the reverse pass over
// a window of time steps with frozen cell types (k_adj.cu).  Internal to
// libfsl; the public calls are fsl_window_forward / fsl_window_adjoint.
#pragma once

#include "fsl_internal.cuh"

namespace fslk {

// Curvature Jacobian rows: dkappa_x / dphi_y for the cells y of the 7x7x7
// window around x (slot (dz+3)*49 + (dy+3)*7 + (dx+3)), dkappa_x / dtheta last.
constexpr int JAC_W = 7;
constexpr int JAC_CELLS = JAC_W * JAC_W * JAC_W;  // 343
constexpr int JAC_STRIDE = JAC_CELLS + 1;         // + theta
constexpr int JAC_CENTRE = JAC_CELLS / 2;         // slot of offset (0, 0, 0)

struct Adj {
    const int *wlist;    // interface cells of the window (fixed for the window)
    const int *widx;     // cell -> position in wlist, -1 for other cells
    int cap;             // rows of jac
    float *jac;          // [cap][JAC_STRIDE]
    float *jval;         // [cap] kappa value of the Jacobian pass
    int *dlist;          // wlist positions whose Jacobian is redone in FP64
    int *glist;          // wlist positions whose Jacobian takes the dual-number path
    float4 *nj;          // [cap][125] d(n, a)/dphi over the 5x5x5 window of each interface cell
    const float *fb_in;  // adjoint of the post-collision PDFs at t+1 [19 N]
    float *fb_out;       // adjoint of the post-collision PDFs at t   [19 N]
    float *gb;           // adjoint of the pre-collision PDFs of step t [19 N]
    float *mb;           // adjoint of the interface mass   (t+1 on entry, t on exit) [N]
    float *pb;           // adjoint of the fill level       (t+1 on entry, t on exit) [N]
    float *kb;           // adjoint of the curvature of step t [N]
    double *part;        // per-block partial sums: [0, nblk) sigma, [nblk, 2 nblk) theta
    double *acc;         // running dL/dsigma, dL/dtheta
    int nblk;
};

// blocks of the adjoint list kernels (each writes one partial per block)
int adj_blocks();

// One frozen-type time step: curvature (LSQR or none), stream-collide with the
// free-boundary condition and mass exchange, phi = m / rho.
void launch_frozen_step(const Dev &d, cudaStream_t s);
// Adjoint of phi at the window's end from dL/dphi (interface entries).
void launch_adjoint_seed(const Dev &d, const Adj &a, const float *dL_dphi, cudaStream_t s);
// Reverse of one frozen-type step (state of step t in d), accumulating into acc.
void launch_adjoint_step(const Dev &d, const Adj &a, cudaStream_t s);
// Curvature Jacobian rows of the window's interface cells at the state in d.
void launch_kappa_jacobian(const Dev &d, const Adj &a, cudaStream_t s);
// Window bookkeeping: the interface cells of the view `src` in cell-index
// order (list and cell -> position index) and a copy of its active segments,
// into the window's own buffers; scratch holds window_scratch_ints(N) ints.
int window_scratch_ints(long long N);
void launch_window_setup(const Dev &src, int *wcounts, int *wlist, int *widx, int *wseg, int *scratch,
                         cudaStream_t s);
// Copy the window's interface list back into the step-parity view `dst`.
void launch_window_finish(const Dev &dst, const int *wcounts, const int *wlist, cudaStream_t s);

}  // namespace fslk
