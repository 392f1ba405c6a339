// mlp_common.cuh -- canonical order of a 5x5x5 fill-level stencil for the
// learned curvature (reading M1): the stencil is flipped so that the
// central-difference normal points into the positive octant and its axes are
// ordered by decreasing |n|, so that the network sees one of the 48 cube
// symmetries of every stencil.  Shared by the training stencil generator
// (k_mlp.cu) and the in-step network (k_mlp_tc.cu); and the launcher of the
// latter.  Internal to libfsl.
#pragma once

#include "fsl_internal.cuh"

namespace fslk {

// canonical placement of a 5x5x5 stencil s[(i*5 + j)*5 + k] (x = i, y = j, z = k):
// returns, for each raw element, its index in the canonical ordering
struct Canon {
    int flip[3], order[3];
};
template <typename Get>
__device__ __forceinline__ Canon canon_at(Get get) {
    float n[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz) {
                const float v = get(dx, dy, dz);
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
__device__ __forceinline__ Canon canon_of(const float *s) {
    return canon_at([&](int dx, int dy, int dz) { return s[((2 + dx) * 5 + 2 + dy) * 5 + 2 + dz]; });
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

// The learned curvature of the step's interface cells (k_mlp_tc.cu): network
// on the tensor cores, judged by the LSQR value in kappa_out.
int launch_mlp_curv_tc(const Dev &d, float *kappa_out, cudaStream_t s);

}  // namespace fslk
