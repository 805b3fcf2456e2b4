// smi_box.h -- the dynamic computing box (Sec. 4.1), evaluated identically
// by the kernels and by the host's byte accounting.
#pragma once

#include <cmath>

#include "smi_internal.h"

namespace smi {

#ifdef __CUDACC__
#define SMI_HD __host__ __device__ __forceinline__
#else
#define SMI_HD inline
#endif

SMI_HD double box_mul(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}

SMI_HD double box_div(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}

// Box after n elapsed steps around the stencil extent ext = {lo0, lo1, lo2,
// hi0, hi1, hi2}: the wavefront has travelled at most vmax (n+1) dt, so each
// face moves out by r_n = ceil(vmax dt (n+1) / h) + 2N + ri cells (2N for the
// two half-step stencils, ri for the injection width), clipped to the
// extended grid.  FP64 with round-to-nearest products in a fixed order, so
// host and device agree bit for bit.  n < 0: empty box (hi < lo).
SMI_HD void box_bounds(const Grid &g, const int *ext, int n, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) {
        if (n < 0) {
            lo[a] = 0;
            hi[a] = -1;
        } else if (a >= g.ndim) {
            lo[a] = 0;
            hi[a] = 0;
        } else if (!g.use_box) {
            lo[a] = 0;
            hi[a] = g.ne[a] - 1;
        } else {
            double r = box_mul(g.vdt, (double)(n + 1));
            r = box_div(r, g.h[a]);
            const int rn = (int)ceil(r) + 2 * g.N + g.ri;
            const int l = ext[a] - rn, h = ext[3 + a] + rn;
            lo[a] = l < 0 ? 0 : l;
            hi[a] = h > g.ne[a] - 1 ? g.ne[a] - 1 : h;
        }
    }
    // free surface: the nodes more than N above the surface are never updated
    if (n >= 0 && g.freesurf && lo[0] < g.L[0] - g.N) lo[0] = g.L[0] - g.N;
}

// Points of the box [lo, hi] (0 if empty).
SMI_HD long long box_points(const int lo[3], const int hi[3])
{
    long long v = 1;
    for (int a = 0; a < 3; a++) v *= hi[a] >= lo[a] ? (long long)(hi[a] - lo[a] + 1) : 0LL;
    return v;
}

// Box of shot s after n steps (n >= -1) from a table filled by box_bounds.
SMI_HD void box_at(const int *tab, int nt1, int s, int n, int lo[3], int hi[3])
{
    const int *e = tab + ((long long)s * nt1 + (n + 1)) * 6;
    lo[0] = e[0];
    lo[1] = e[1];
    lo[2] = e[2];
    hi[0] = e[3];
    hi[1] = e[4];
    hi[2] = e[5];
}

}  // namespace smi
