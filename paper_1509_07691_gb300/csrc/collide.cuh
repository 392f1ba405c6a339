// collide.cuh -- the BGK / TRT collision of one cell (Eq. lbe2), shared by the
// liquid stream-collide kernels (k_step.cu, k_bulk_tma.cu) so that both give
// the same bits.  Internal to libfsl.
#pragma once

#include "fsl_internal.cuh"

namespace fslk {

// BGK / TRT collision in place (Eq. lbe2).  TRT relaxes the even and odd
// parts of each pair (q, opp q) with omega_e = 1/tau and omega_o = 1/tau_o.
template <int COLL>
__device__ __forceinline__ void collide(float f[Q], const Dev &d, float &rho_out) {
    float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        rho += f[q];
        jx += cx(q) * f[q];
        jy += cy(q) * f[q];
        jz += cz(q) * f[q];
    }
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    rho_out = rho;
    if (COLL == FSL_BGK) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float fe = wq(q) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu);
            f[q] += d.omega_e * (fe - f[q]);
        }
    } else {
        f[0] += d.omega_e * (wq(0) * rho * (1.0f - uu) - f[0]);
#pragma unroll
        for (int q = 1; q < Q; q += 2) {
            const int qb = q + 1;
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float ep = wq(q) * rho * (1.0f + 4.5f * cu * cu - uu);
            const float em = wq(q) * rho * 3.0f * cu;
            const float fp = 0.5f * (f[q] + f[qb]), fm = 0.5f * (f[q] - f[qb]);
            const float de = d.omega_e * (fp - ep), dd = d.omega_o * (fm - em);
            f[q] = f[q] - de - dd;
            f[qb] = f[qb] - de + dd;
        }
    }
}

}  // namespace fslk
