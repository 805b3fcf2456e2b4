// smi_kernels.cu -- CUDA kernels of libsmi (sm_103a): staggered-grid
// velocity/pressure updates with slab-only CPML, source injection, receiver
// gather, boundary-band save/restore, residual/misfit, the exact discrete
// adjoint in "same solver" form, source-field reconstruction fused with
// imaging/gradient accumulation, and the device-side computing box.
//
// Every stencil kernel is bounded by the computing box of its shot (Sec.
// 4.1), computed on the device from the step counter; threads stride over
// the box's points.  Stencil reads outside the extended grid are zero.
#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "smi_internal.h"
#include "smi_box.h"

namespace smi {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocksX = 152 * 16;

__device__ __forceinline__ long long gidx(const Grid &g, int i1, int i2, int i3)
{
    return (long long)i1 + (long long)g.px * ((long long)i2 + (long long)g.ne[1] * i3);
}

__device__ __forceinline__ long long gstride(const Grid &g, int a)
{
    return a == 0 ? 1LL : (a == 1 ? (long long)g.px : (long long)g.px * g.ne[1]);
}

// CPML slab membership along axis a: nodes 0..nb-1 and ne-nb-1..ne-1 (the
// latter covers the first v node of the high layer).
__device__ __forceinline__ bool in_slab(const Grid &g, int a, int j)
{
    return j < g.nb || j >= g.ne[a] - g.nb - 1;
}

// Index into the slab array of axis a (axis a compressed to S = 2nb+1).
__device__ __forceinline__ long long slab_index(const Grid &g, int a, int i1, int i2, int i3)
{
    if (a == 0) {
        int js = i1 < g.nb ? i1 : i1 - (g.ne[0] - 2 * g.nb - 1);
        return (long long)js + (long long)g.S * ((long long)i2 + (long long)g.ne[1] * i3);
    }
    if (a == 1) {
        int js = i2 < g.nb ? i2 : i2 - (g.ne[1] - 2 * g.nb - 1);
        return (long long)i1 + (long long)g.ne[0] * ((long long)js + (long long)g.S * i3);
    }
    int js = i3 < g.nb ? i3 : i3 - (g.ne[2] - 2 * g.nb - 1);
    return (long long)i1 + (long long)g.ne[0] * ((long long)i2 + (long long)g.ne[1] * js);
}

__device__ __forceinline__ float buoyancy(const Grid &g, int a, int ia, long long k, float rho0)
{
    return (ia + 1 < g.ne[a]) ? 2.0f / (rho0 + g.rho[k + gstride(g, a)]) : 1.0f / rho0;
}

struct BoxIter {
    int lo[3], hi[3];
    int w0, w1;
    long long vol;
    __device__ void set(const int l[3], const int h[3])
    {
        for (int a = 0; a < 3; a++) { lo[a] = l[a]; hi[a] = h[a]; }
        w0 = hi[0] - lo[0] + 1;
        w1 = hi[1] - lo[1] + 1;
        const int w2 = hi[2] - lo[2] + 1;
        vol = (w0 > 0 && w1 > 0 && w2 > 0) ? (long long)w0 * w1 * w2 : 0;
    }
    __device__ void at(long long q, int i[3]) const
    {
        i[0] = lo[0] + (int)(q % w0);
        long long r = q / w0;
        i[1] = lo[1] + (int)(r % w1);
        i[2] = lo[2] + (int)(r / w1);
    }
};

__device__ __forceinline__ bool inside(const int i[3], const int lo[3], const int hi[3])
{
    return i[0] >= lo[0] && i[0] <= hi[0] && i[1] >= lo[1] && i[1] <= hi[1] && i[2] >= lo[2] &&
           i[2] <= hi[2];
}

// ---------------------------------------------------------------------------
// Forward velocity update (Sec. 2.1): v_a -= dt b_a (D_a p + psi_a), with the
// slab memory variable psi_a <- b psi_a + a D_a p updated first.
template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads) k_fwd_v(Grid g, Batch b, Fields f, int it)
{
    const int s = blockIdx.y;
    int lo[3], hi[3];
    box_at(b.tab_src, b.nt1, s, it, lo, hi);
    BoxIter bi;
    bi.set(lo, hi);
    const float *p = f.p + s * g.ntot;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        const float rho0 = g.rho[k];
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            const long long st = gstride(g, a);
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) {
                const float pp = (i[a] + l < g.ne[a]) ? p[k + l * st] : 0.0f;
                const float pm = (i[a] - l + 1 >= 0) ? p[k - (l - 1) * st] : 0.0f;
                D += g.c[a][l - 1] * (pp - pm);
            }
            if (in_slab(g, a, i[a])) {
                const long long si = s * g.slab_n[a] + slab_index(g, a, i[0], i[1], i[2]);
                const float psi = g.cvb[a][i[a]] * f.psip[a][si] + g.cva[a][i[a]] * D;
                f.psip[a][si] = psi;
                D += psi;
            }
            f.v[a][s * g.ntot + k] -= g.dt * buoyancy(g, a, i[a], k, rho0) * D;
        }
    }
}

// Forward pressure update: p -= dt kappa sum_a (D_a v_a + psi_a).
template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads) k_fwd_p(Grid g, Batch b, Fields f, int it)
{
    const int s = blockIdx.y;
    int lo[3], hi[3];
    box_at(b.tab_src, b.nt1, s, it, lo, hi);
    BoxIter bi;
    bi.set(lo, hi);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        float div = 0.0f;
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            const long long st = gstride(g, a);
            const float *v = f.v[a] + s * g.ntot;
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) {
                const float vp = (i[a] + l - 1 < g.ne[a]) ? v[k + (l - 1) * st] : 0.0f;
                const float vm = (i[a] - l >= 0) ? v[k - l * st] : 0.0f;
                D += g.c[a][l - 1] * (vp - vm);
            }
            if (in_slab(g, a, i[a])) {
                const long long si = s * g.slab_n[a] + slab_index(g, a, i[0], i[1], i[2]);
                const float psi = g.cpb[a][i[a]] * f.psiv[a][si] + g.cpa[a][i[a]] * D;
                f.psiv[a][si] = psi;
                D += psi;
            }
            div += D;
        }
        f.p[s * g.ntot + k] -= g.dt * g.K[k] * div;
    }
}

// ---------------------------------------------------------------------------
// Exact discrete adjoint in "same solver" form.  With lambda_p = kappa pbar
// and lambda_v = -b vbar (pbar, vbar the adjoints of p, v), the transpose of
// the forward step becomes, in reverse time:
//   V: lv_a -= dt b_a D_a[(1 + Ap_a) lp + Ap_a phi_a];   phi_a <- Bp_a (phi_a + lp)
//   P: lp   -= dt kappa sum_a D_a[(1 + Av_a) lv_a + Av_a chi_a];  chi_a <- Bv_a (chi_a + lv_a)
// (A, B the CPML a/b on the p grid (Ap, Bp) or v grid (Av, Bv)); in the
// interior this is the forward scheme itself (Sec. 2.2: the adjoint shares
// the forward solver).  phi lives on the p grid (stored in psiv), chi on
// the v grid (stored in psip).  The chi update of a reverse step is applied
// at the start of the next V kernel (it is pointwise), the phi update in the
// P kernel before lp changes.  m = reverse steps elapsed (box of the
// receivers, Sec. 4.1).
template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads) k_adj_v(Grid g, Batch b, Fields f, int m)
{
    const int s = blockIdx.y;
    int lo[3], hi[3];
    box_at(b.tab_rec, b.nt1, s, m, lo, hi);
    BoxIter bi;
    bi.set(lo, hi);
    const float *lp = f.p + s * g.ntot;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        const float rho0 = g.rho[k];
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            const long long st = gstride(g, a);
            float *lv = f.v[a] + s * g.ntot;
            if (in_slab(g, a, i[a])) {             // deferred chi update
                const long long si = s * g.slab_n[a] + slab_index(g, a, i[0], i[1], i[2]);
                f.psip[a][si] = g.cvb[a][i[a]] * (f.psip[a][si] + lv[k]);
            }
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) {
                float qv[2];
                const int off[2] = {l, 1 - l};
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    int j[3] = {i[0], i[1], i[2]};
                    j[a] += off[e];
                    float val = 0.0f;
                    if (j[a] >= 0 && j[a] < g.ne[a]) {
                        const long long kk = k + off[e] * st;
                        val = lp[kk];
                        if (in_slab(g, a, j[a])) {
                            const float A = g.cpa[a][j[a]];
                            const long long sj = s * g.slab_n[a] + slab_index(g, a, j[0], j[1], j[2]);
                            val += A * (val + f.psiv[a][sj]);
                        }
                    }
                    qv[e] = val;
                }
                D += g.c[a][l - 1] * (qv[0] - qv[1]);
            }
            lv[k] -= g.dt * buoyancy(g, a, i[a], k, rho0) * D;
        }
    }
}

template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads) k_adj_p(Grid g, Batch b, Fields f, int m)
{
    const int s = blockIdx.y;
    int lo[3], hi[3];
    box_at(b.tab_rec, b.nt1, s, m, lo, hi);
    BoxIter bi;
    bi.set(lo, hi);
    float *lp = f.p + s * g.ntot;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        const float lpk = lp[k];
        float div = 0.0f;
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            const long long st = gstride(g, a);
            const float *lv = f.v[a] + s * g.ntot;
            if (in_slab(g, a, i[a])) {             // phi update with lp before this step
                const long long si = s * g.slab_n[a] + slab_index(g, a, i[0], i[1], i[2]);
                f.psiv[a][si] = g.cpb[a][i[a]] * (f.psiv[a][si] + lpk);
            }
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) {
                float rv[2];
                const int off[2] = {l - 1, -l};
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    int j[3] = {i[0], i[1], i[2]};
                    j[a] += off[e];
                    float val = 0.0f;
                    if (j[a] >= 0 && j[a] < g.ne[a]) {
                        const long long kk = k + off[e] * st;
                        val = lv[kk];
                        if (in_slab(g, a, j[a])) {
                            const float A = g.cva[a][j[a]];
                            const long long sj = s * g.slab_n[a] + slab_index(g, a, j[0], j[1], j[2]);
                            val += A * (val + f.psip[a][sj]);
                        }
                    }
                    rv[e] = val;
                }
                D += g.c[a][l - 1] * (rv[0] - rv[1]);
            }
            div += D;
        }
        lp[k] = lpk - g.dt * g.K[k] * div;
    }
}

// ---------------------------------------------------------------------------
// Transposed CPML terms of the adjoint, applied over the slabs only, before
// the interior adjoint kernels (which then run the plain forward scheme).
// Axis a, band of nodes whose stencil reaches the axis-a CPML layer:
//   V (lam_v update): lv_a -= dt b_a D_a[eta_a],  eta_a = Ap_a (lp + phi_a),
//                     after the deferred chi_a <- Bv_a (chi_a + lv_a);
//   P (lam_p update): lp -= dt kappa D_a[zeta_a], zeta_a = Av_a (lv_a + chi_a),
//                     after phi_a <- Bp_a (phi_a + lp).
// Region: the receiver box (m reverse steps) within nb+N+1 nodes of either
// end of axis a.
// Thread -> node of the axis-AX band: wl = nb + N + 1 nodes at each end of
// the axis (they cover every node whose stencil reaches that CPML layer),
// other axes over the grid; nodes outside the receiver box are skipped.
template <int N, int AX>
__device__ __forceinline__ bool corr_node(const Grid &g, const Batch &b, const int *tab, int m, int &s, int i[3], int wl)
{
    const int zdim = (AX == 2) ? 2 * wl : g.ne[2];
    s = blockIdx.z / zdim;
    const int tz = blockIdx.z - s * zdim;
    const int tx = blockIdx.x * 32 + threadIdx.x, ty = blockIdx.y * 8 + threadIdx.y;
    int j;
    if (AX == 0) { j = tx; i[1] = ty; i[2] = tz; }
    else if (AX == 1) { i[0] = tx; j = ty; i[2] = tz; }
    else { i[0] = tx; i[1] = ty; j = tz; }
    if (j >= 2 * wl) return false;
    i[AX] = j < wl ? j : g.ne[AX] - 2 * wl + j;
    if (i[AX] < 0 || (j >= wl && i[AX] < wl)) return false;     // bands overlap on a short axis
    int lo[3], hi[3];
    box_at(tab, b.nt1, s, m, lo, hi);
    return i[0] >= lo[0] && i[0] <= hi[0] && i[1] >= lo[1] && i[1] <= hi[1] && i[2] >= lo[2] && i[2] <= hi[2];
}

// js of node j of a CPML slab (slab arrays compress their axis to 2 nb + 1).
__device__ __forceinline__ int slab_j(const Grid &g, int a, int j) { return j < g.nb ? j : j - (g.ne[a] - 2 * g.nb - 1); }

// Offset and stride of axis AX's slab index at node i with i[AX] replaced.
template <int AX>
__device__ __forceinline__ void slab_base(const Grid &g, const int i[3], long long &base, long long &stride)
{
    if (AX == 0) { base = (long long)g.S * ((long long)i[1] + (long long)g.ne[1] * i[2]); stride = 1; }
    else if (AX == 1) { base = (long long)i[0] + (long long)g.ne[0] * g.S * i[2]; stride = g.ne[0]; }
    else { base = (long long)i[0] + (long long)g.ne[0] * i[1]; stride = (long long)g.ne[0] * g.ne[1]; }
}

template <int N, int AX>
__global__ void __launch_bounds__(256) k_corr_v(Grid g, Batch b, Fields f, int m)
{
    int s, i[3];
    if (!corr_node<N, AX>(g, b, b.tab_rec, m, s, i, g.nb + N + 1)) return;
    const long long k = gidx(g, i[0], i[1], i[2]), st = gstride(g, AX);
    long long sb, ss;
    slab_base<AX>(g, i, sb, ss);
    sb += (long long)s * g.slab_n[AX];
    const float *lp = f.p + s * g.ntot;
    float *lv = f.v[AX] + s * g.ntot;
    const int ia = i[AX];
    if (in_slab(g, AX, ia)) {                  // deferred chi update with lv before this step
        float *ch = f.psip[AX] + sb + slab_j(g, AX, ia) * ss;
        *ch = g.cvb[AX][ia] * (*ch + lv[k]);
    }
    float E = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; l++) {
        float h[2];
        const int off[2] = {l, 1 - l};
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int j = ia + off[e];
            h[e] = 0.0f;
            if (j >= 0 && j < g.ne[AX] && in_slab(g, AX, j)) {
                const float A = __ldg(g.cpa[AX] + j);
                if (A != 0.0f) h[e] = A * (lp[k + off[e] * st] + f.psiv[AX][sb + slab_j(g, AX, j) * ss]);
            }
        }
        E += g.c[AX][l - 1] * (h[0] - h[1]);
    }
    if (E != 0.0f) lv[k] -= g.dt * buoyancy(g, AX, ia, k, g.rho[k]) * E;
}

template <int N, int AX>
__global__ void __launch_bounds__(256) k_corr_phi(Grid g, Batch b, Fields f, int m)
{
    int s, i[3];
    if (!corr_node<N, AX>(g, b, b.tab_rec, m, s, i, g.nb + N + 1)) return;
    const int ia = i[AX];
    if (!in_slab(g, AX, ia)) return;
    long long sb, ss;
    slab_base<AX>(g, i, sb, ss);
    float *ph = f.psiv[AX] + (long long)s * g.slab_n[AX] + sb + slab_j(g, AX, ia) * ss;
    *ph = g.cpb[AX][ia] * (*ph + f.p[s * g.ntot + gidx(g, i[0], i[1], i[2])]);
}

template <int N, int AX>
__global__ void __launch_bounds__(256) k_corr_p(Grid g, Batch b, Fields f, int m)
{
    int s, i[3];
    if (!corr_node<N, AX>(g, b, b.tab_rec, m, s, i, g.nb + N + 1)) return;
    const long long k = gidx(g, i[0], i[1], i[2]), st = gstride(g, AX);
    long long sb, ss;
    slab_base<AX>(g, i, sb, ss);
    sb += (long long)s * g.slab_n[AX];
    const float *lv = f.v[AX] + s * g.ntot;
    const int ia = i[AX];
    float F = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; l++) {
        float h[2];
        const int off[2] = {l - 1, -l};
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int j = ia + off[e];
            h[e] = 0.0f;
            if (j >= 0 && j < g.ne[AX] && in_slab(g, AX, j)) {
                const float A = __ldg(g.cva[AX] + j);
                if (A != 0.0f) h[e] = A * (lv[k + off[e] * st] + f.psip[AX][sb + slab_j(g, AX, j) * ss]);
            }
        }
        F += g.c[AX][l - 1] * (h[0] - h[1]);
    }
    if (F != 0.0f) f.p[s * g.ntot + k] -= g.dt * g.K[k] * F;
}

// ---------------------------------------------------------------------------
// Source-field reconstruction (Sec. 4.2, Algorithm 2 reverse loop) fused with
// the imaging / gradient accumulation, over the physical nodes of the
// forward box of step it:
//   acc += lp * div v^{it+1/2}  (gradient)   or  lp * p^{it+1}  (image)
//   p^{it} = p^{it+1} + dt kappa div v^{it+1/2} - dt stf[it] w / dV
// Nodes outside the box of step it-1 are set to zero (they were zero
// before step it).  lp is the adjoint pressure after the receivers of step
// it were injected.
template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads)
k_recon_p(Grid g, Batch b, Fields f, const float *lpall, float *acc, int mode, const float *stf,
          int it, float src_scale)
{
    const int s = blockIdx.y;
    int lo[3], hi[3], plo[3], phi[3];
    box_at(b.tab_src, b.nt1, s, it, lo, hi);
    box_at(b.tab_src, b.nt1, s, it - 1, plo, phi);
    for (int a = 0; a < 3; a++) {
        lo[a] = max(lo[a], g.L[a]);
        hi[a] = min(hi[a], g.H[a]);
    }
    BoxIter bi;
    bi.set(lo, hi);
    float *p = f.p + s * g.ntot;
    const float *lp = lpall + s * g.ntot;
    const Stencil &sst = b.src[s];
    const float amp = src_scale * stf[it];
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        float dv = 0.0f;
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            const long long st = gstride(g, a);
            const float *v = f.v[a] + s * g.ntot;
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) D += g.c[a][l - 1] * (v[k + (l - 1) * st] - v[k - l * st]);
            dv += D;
        }
        const float pk = p[k];
        const long long kp = (long long)(i[0] - g.L[0]) +
                             (long long)(g.H[0] - g.L[0] + 1) *
                                 ((long long)(i[1] - g.L[1]) + (long long)(g.H[1] - g.L[1] + 1) * (i[2] - g.L[2]));
        acc[s * g.nphys + kp] += lp[k] * (mode == 0 ? dv : pk);
        float pn = pk + g.dt * g.K[k] * dv;
        bool in_src = true;
        float w = 1.0f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int t = i[a] - sst.first[a];
            in_src = in_src && t >= 0 && t < sst.cnt[a];
            if (in_src) w *= sst.w[a][t];
        }
        if (in_src) pn -= amp * w;
        if (!inside(i, plo, phi)) pn = 0.0f;
        p[k] = pn;
    }
}

// v_a^{it-1/2} = v_a^{it+1/2} + dt b_a D_a p^{it} on L_a+N-1 .. H_a-N along a
// (other axes over the physical nodes), inside the forward box of step it.
template <int NDIM, int N>
__global__ void __launch_bounds__(kThreads) k_recon_v(Grid g, Batch b, Fields f, int it)
{
    const int s = blockIdx.y;
    int lo[3], hi[3], plo[3], phi[3];
    box_at(b.tab_src, b.nt1, s, it, lo, hi);
    box_at(b.tab_src, b.nt1, s, it - 1, plo, phi);
    for (int a = 0; a < 3; a++) {
        lo[a] = max(lo[a], g.L[a]);
        hi[a] = min(hi[a], g.H[a]);
    }
    BoxIter bi;
    bi.set(lo, hi);
    const float *p = f.p + s * g.ntot;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < bi.vol;
         q += (long long)gridDim.x * blockDim.x) {
        int i[3];
        bi.at(q, i);
        const long long k = gidx(g, i[0], i[1], i[2]);
        const bool keep = inside(i, plo, phi);
        const float rho0 = g.rho[k];
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            if (i[a] < g.L[a] + N - 1 || i[a] > g.H[a] - N) continue;
            const long long st = gstride(g, a);
            float D = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++) D += g.c[a][l - 1] * (p[k + l * st] - p[k - (l - 1) * st]);
            float *v = f.v[a] + s * g.ntot;
            v[k] = keep ? v[k] + g.dt * buoyancy(g, a, i[a], k, rho0) * D : 0.0f;
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void k_inject_source(Grid g, Batch b, float *p, const float *stf, int it, float scale)
{
    const int s = blockIdx.x;
    const Stencil &st = b.src[s];
    const int n = st.cnt[0] * st.cnt[1] * st.cnt[2];
    const float amp = scale * stf[it];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int a0 = t % st.cnt[0], r = t / st.cnt[0];
        const int a1 = r % st.cnt[1], a2 = r / st.cnt[1];
        const float w = st.w[0][a0] * st.w[1][a1] * st.w[2][a2];
        p[s * g.ntot + gidx(g, st.first[0] + a0, st.first[1] + a1, st.first[2] + a2)] += amp * w;
    }
}

__global__ void k_gather(Grid g, Batch b, const float *p, float *seis, const long long *seis_off,
                         int it)
{
    const int s = blockIdx.y;
    const int nr = b.rec_off[s + 1] - b.rec_off[s];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const Stencil &st = b.rec[b.rec_off[s] + r];
    const float *ps = p + s * g.ntot;
    float sum = 0.0f;
    for (int a2 = 0; a2 < st.cnt[2]; a2++)
        for (int a1 = 0; a1 < st.cnt[1]; a1++)
            for (int a0 = 0; a0 < st.cnt[0]; a0++)
                sum += st.w[0][a0] * st.w[1][a1] * st.w[2][a2] *
                       ps[gidx(g, st.first[0] + a0, st.first[1] + a1, st.first[2] + a2)];
    seis[seis_off[s] + (long long)it * nr + r] = sum;
}

// Adjoint source (Algorithm 2): lp += kappa w_r res at the receiver stencils.
__global__ void k_adj_inject(Grid g, Batch b, float *lp, const float *res, const long long *seis_off,
                             int it)
{
    const int s = blockIdx.y;
    const int nr = b.rec_off[s + 1] - b.rec_off[s];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const Stencil &st = b.rec[b.rec_off[s] + r];
    const float val = res[seis_off[s] + (long long)it * nr + r];
    float *ls = lp + s * g.ntot;
    for (int a2 = 0; a2 < st.cnt[2]; a2++)
        for (int a1 = 0; a1 < st.cnt[1]; a1++)
            for (int a0 = 0; a0 < st.cnt[0]; a0++) {
                const long long k = gidx(g, st.first[0] + a0, st.first[1] + a1, st.first[2] + a2);
                atomicAdd(ls + k, g.K[k] * st.w[0][a0] * st.w[1][a1] * st.w[2][a2] * val);
            }
}

// ---------------------------------------------------------------------------
// Boundary bands: value t of a step maps to (axis, side, node).
__device__ __forceinline__ bool band_node(const Bands &bd, int ndim, long long t, int &a, int &sd,
                                          int i[3])
{
    for (a = 0; a < ndim; a++)
        for (sd = 0; sd < 2; sd++) {
            const long long o = bd.off[a][sd];
            const int *lo = bd.lo[a][sd], *hi = bd.hi[a][sd];
            const long long w0 = hi[0] - lo[0] + 1, w1 = hi[1] - lo[1] + 1, w2 = hi[2] - lo[2] + 1;
            const long long n = w0 * w1 * w2;
            if (t >= o && t < o + n) {
                const long long u = t - o;
                i[0] = lo[0] + (int)(u % w0);
                i[1] = lo[1] + (int)((u / w0) % w1);
                i[2] = lo[2] + (int)(u / (w0 * w1));
                return true;
            }
        }
    return false;
}

__global__ void k_band_absmax(Grid g, Fields f, Bands bd, unsigned *amax)
{
    const int s = blockIdx.y;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bd.count) return;
    int a, sd, i[3];
    if (!band_node(bd, g.ndim, t, a, sd, i)) return;
    const float v = fabsf(f.v[a][s * g.ntot + gidx(g, i[0], i[1], i[2])]);
    atomicMax(amax + s * 6 + a * 2 + sd, __float_as_uint(v));
}

__global__ void k_band_save(Grid g, Fields f, Bands bd, int it, const unsigned *amax)
{
    const int s = blockIdx.y;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bd.count) return;
    int a, sd, i[3];
    if (!band_node(bd, g.ndim, t, a, sd, i)) return;
    const float v = f.v[a][s * g.ntot + gidx(g, i[0], i[1], i[2])];
    const long long o = ((long long)s * bd.nt + it) * bd.count + t;
    if (bd.prec == SMI_PREC_F32) {
        static_cast<float *>(bd.data)[o] = v;
        return;
    }
    // 16-bit storage scaled per (step, axis, side): the largest magnitude
    // maps to 2^14 (FP16) or 1 (BF16).
    const float m = __uint_as_float(amax[s * 6 + a * 2 + sd]);
    const float target = bd.prec == SMI_PREC_F16 ? 16384.0f : 1.0f;
    const float scale = m > 0.0f ? m / target : 0.0f;
    if (t == bd.off[a][sd]) bd.scale[((long long)s * bd.nt + it) * 6 + a * 2 + sd] = scale;
    const float x = scale > 0.0f ? v / scale : 0.0f;
    if (bd.prec == SMI_PREC_F16) static_cast<__half *>(bd.data)[o] = __float2half_rn(x);
    else static_cast<__nv_bfloat16 *>(bd.data)[o] = __float2bfloat16_rn(x);
}

__global__ void k_band_restore(Grid g, Fields f, Bands bd, int it)
{
    const int s = blockIdx.y;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bd.count) return;
    int a, sd, i[3];
    if (!band_node(bd, g.ndim, t, a, sd, i)) return;
    const long long o = ((long long)s * bd.nt + it) * bd.count + t;
    float v;
    if (bd.prec == SMI_PREC_F32) {
        v = static_cast<const float *>(bd.data)[o];
    } else {
        const float scale = bd.scale[((long long)s * bd.nt + it) * 6 + a * 2 + sd];
        const float x = bd.prec == SMI_PREC_F16 ? __half2float(static_cast<const __half *>(bd.data)[o])
                                                : __bfloat162float(static_cast<const __nv_bfloat16 *>(bd.data)[o]);
        v = x * scale;
    }
    f.v[a][s * g.ntot + gidx(g, i[0], i[1], i[2])] = v;
}

// ---------------------------------------------------------------------------
// Residual (mode 0: u - d, mode 1: d) and per-block partial sums of
// 1/2 (u - d)^2 in FP64 (Eq. objfwi).
__global__ void k_residual(const float *u, const float *d, long long n, int mode, float *res,
                           double *partials)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float r = u[t] - d[t];
        res[t] = mode == 0 ? r : d[t];
        acc += 0.5 * (double)r * (double)r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double *partials, int n, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; i++) s += partials[i];
    *out += s;
}

// out[x] (+)= sum_s acc[s][x], shots added in order (deterministic).
__global__ void k_reduce_shots(const float *acc, long long n, int nshot, float *out, int accumulate)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        float s = accumulate ? out[t] : 0.0f;
        for (int k = 0; k < nshot; k++) s += acc[k * n + t];
        out[t] = s;
    }
}

// dJ/dVp = 2 rho Vp dJ/dkappa with dJ/dkappa = -dt sum lp div v / kappa and
// kappa = rho Vp^2: -2 dt sum(lp div v) / Vp.
__global__ void k_finalize_grad(long long n, const float *vp, float dt, float *gr)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        gr[t] = -2.0f * dt * gr[t] / vp[t];
}

__global__ void k_nonfinite(const float *x, long long n, unsigned *flag)
{
    bool bad = false;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[t]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

__global__ void k_extend_model(Grid g, const float *vp, const float *rho, int n1, int n2, int n3,
                               float *K, float *rho_e)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < g.ntot;
         t += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(t % g.px);
        const int i2 = (int)((t / g.px) % g.ne[1]);
        const int i3 = (int)(t / ((long long)g.px * g.ne[1]));
        if (i1 >= g.ne[0]) {            // row padding
            rho_e[t] = 0.0f;
            K[t] = 0.0f;
            continue;
        }
        const int j1 = min(max(i1 - g.L[0], 0), n1 - 1);
        const int j2 = min(max(i2 - g.L[1], 0), n2 - 1);
        const int j3 = min(max(i3 - g.L[2], 0), n3 - 1);
        const long long kp = (long long)j1 + (long long)n1 * ((long long)j2 + (long long)n2 * j3);
        const float r = rho[kp], c = vp[kp];
        rho_e[t] = r;
        K[t] = r * c * c;
    }
}

__global__ void k_minmax_init(unsigned *tmp)
{
    tmp[0] = 0x7f800000u;   // +inf
    tmp[1] = 0u;
}

// min/max of positive floats via their ordered bit patterns (NaN or <= 0
// entries force min to 0 so that the host rejects the model).
__global__ void k_minmax(const float *x, long long n, unsigned *tmp)
{
    unsigned lo = 0x7f800000u, hi = 0u;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float v = x[t];
        const unsigned u = (v > 0.0f && isfinite(v)) ? __float_as_uint(v) : 0u;
        lo = min(lo, u);
        hi = max(hi, u);
    }
    atomicMin(tmp, lo);
    atomicMax(tmp + 1, hi);
}

__global__ void k_minmax_out(const unsigned *tmp, float *out2)
{
    out2[0] = __uint_as_float(tmp[0]);
    out2[1] = __uint_as_float(tmp[1]);
}

__global__ void k_box_fill(Grid g, const int *ext, int nshot, int nt, int *tab)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nshot * (nt + 1)) return;
    const int s = (int)(t / (nt + 1)), n = (int)(t % (nt + 1)) - 1;
    int lo[3], hi[3];
    box_bounds(g, ext + 6 * s, n, lo, hi);
    for (int a = 0; a < 3; a++) {
        tab[t * 6 + a] = lo[a];
        tab[t * 6 + 3 + a] = hi[a];
    }
}

__global__ void k_box_table(Grid g, const int *ext, int n0, int count, int *lo, int *hi)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    box_bounds(g, ext, n0 + c, lo + 3 * c, hi + 3 * c);
}

inline cudaStream_t S(const LaunchCtx &lc) { return static_cast<cudaStream_t>(lc.stream); }

inline int blocks_for(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)(b < kMaxBlocksX ? b : kMaxBlocksX);
}

}  // namespace

// ---------------------------------------------------------------------------
#define SMI_DISPATCH(KERNEL, GRID, ...)                                                    \
    do {                                                                                   \
        if (g.ndim == 2 && g.N == 2) KERNEL<2, 2><<<GRID, kThreads, 0, S(lc)>>>(__VA_ARGS__); \
        else if (g.ndim == 2 && g.N == 4) KERNEL<2, 4><<<GRID, kThreads, 0, S(lc)>>>(__VA_ARGS__); \
        else if (g.ndim == 3 && g.N == 2) KERNEL<3, 2><<<GRID, kThreads, 0, S(lc)>>>(__VA_ARGS__); \
        else KERNEL<3, 4><<<GRID, kThreads, 0, S(lc)>>>(__VA_ARGS__);                       \
        ++*lc.launches;                                                                    \
    } while (0)

void launch_fwd_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it)
{
    dim3 grid(blocks_for(g.ntot), b.nshot);
    SMI_DISPATCH(k_fwd_v, grid, g, b, f, it);
}

void launch_fwd_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it)
{
    dim3 grid(blocks_for(g.ntot), b.nshot);
    SMI_DISPATCH(k_fwd_p, grid, g, b, f, it);
}

void launch_adj_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m)
{
    dim3 grid(blocks_for(g.ntot), b.nshot);
    SMI_DISPATCH(k_adj_v, grid, g, b, f, m);
}

void launch_adj_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m)
{
    dim3 grid(blocks_for(g.ntot), b.nshot);
    SMI_DISPATCH(k_adj_p, grid, g, b, f, m);
}

void launch_recon_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, const float *lp,
                    float *acc, int mode, const float *stf, int it, float src_scale)
{
    dim3 grid(blocks_for(g.nphys), b.nshot);
    SMI_DISPATCH(k_recon_p, grid, g, b, f, lp, acc, mode, stf, it, src_scale);
}

void launch_recon_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it)
{
    dim3 grid(blocks_for(g.nphys), b.nshot);
    SMI_DISPATCH(k_recon_v, grid, g, b, f, it);
}

// Forward CPML over the slabs only (Sec. 2.1, Komatitsch & Martin CPML),
// added to the interior update that the main kernels apply everywhere:
//   V: psi_a <- Bv_a psi_a + Av_a D_a p;  v_a -= dt b_a psi_a
//   P: psi_a <- Bp_a psi_a + Ap_a D_a v_a; p -= dt kappa psi_a
// over the forward box (step it); nodes outside the axis-AX slab skip.
template <int N, int AX>
__global__ void __launch_bounds__(256) k_fcorr_v(Grid g, Batch b, Fields f, int it)
{
    int s, i[3];
    if (!corr_node<N, AX>(g, b, b.tab_src, it, s, i, g.nb + 1)) return;
    const int ia = i[AX];
    if (!in_slab(g, AX, ia)) return;
    const long long k = gidx(g, i[0], i[1], i[2]), st = gstride(g, AX);
    const float *p = f.p + s * g.ntot;
    float D = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; l++) {
        const float pp = (ia + l < g.ne[AX]) ? p[k + l * st] : 0.0f;
        const float pm = (ia - l + 1 >= 0) ? p[k - (l - 1) * st] : 0.0f;
        D += g.c[AX][l - 1] * (pp - pm);
    }
    long long sb, ss;
    slab_base<AX>(g, i, sb, ss);
    float *ps = f.psip[AX] + (long long)s * g.slab_n[AX] + sb + slab_j(g, AX, ia) * ss;
    const float psi = g.cvb[AX][ia] * *ps + g.cva[AX][ia] * D;
    *ps = psi;
    f.v[AX][s * g.ntot + k] -= g.dt * buoyancy(g, AX, ia, k, g.rho[k]) * psi;
}

template <int N, int AX>
__global__ void __launch_bounds__(256) k_fcorr_p(Grid g, Batch b, Fields f, int it)
{
    int s, i[3];
    if (!corr_node<N, AX>(g, b, b.tab_src, it, s, i, g.nb + 1)) return;
    const int ia = i[AX];
    if (!in_slab(g, AX, ia)) return;
    const long long k = gidx(g, i[0], i[1], i[2]), st = gstride(g, AX);
    const float *v = f.v[AX] + s * g.ntot;
    float D = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; l++) {
        const float vp = (ia + l - 1 < g.ne[AX]) ? v[k + (l - 1) * st] : 0.0f;
        const float vm = (ia - l >= 0) ? v[k - l * st] : 0.0f;
        D += g.c[AX][l - 1] * (vp - vm);
    }
    long long sb, ss;
    slab_base<AX>(g, i, sb, ss);
    float *ps = f.psiv[AX] + (long long)s * g.slab_n[AX] + sb + slab_j(g, AX, ia) * ss;
    const float psi = g.cpb[AX][ia] * *ps + g.cpa[AX][ia] * D;
    *ps = psi;
    f.p[s * g.ntot + k] -= g.dt * g.K[k] * psi;
}

template <int N, int AX>
void corr_launch(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, int which)
{
    const int wl = which >= 3 ? g.nb + 1 : g.nb + N + 1;
    dim3 grid(AX == 0 ? (2 * wl + 31) / 32 : (g.ne[0] + 31) / 32, AX == 1 ? (2 * wl + 7) / 8 : (g.ne[1] + 7) / 8,
              (AX == 2 ? 2 * wl : g.ne[2]) * b.nshot);
    dim3 block(32, 8);
    if (which == 0) k_corr_v<N, AX><<<grid, block, 0, S(lc)>>>(g, b, f, m);
    else if (which == 1) k_corr_phi<N, AX><<<grid, block, 0, S(lc)>>>(g, b, f, m);
    else if (which == 2) k_corr_p<N, AX><<<grid, block, 0, S(lc)>>>(g, b, f, m);
    else if (which == 3) k_fcorr_v<N, AX><<<grid, block, 0, S(lc)>>>(g, b, f, m);
    else k_fcorr_p<N, AX><<<grid, block, 0, S(lc)>>>(g, b, f, m);
    ++*lc.launches;
}

template <int N>
void corr_axes(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, int which)
{
    corr_launch<N, 0>(lc, g, b, f, m, which);
    corr_launch<N, 1>(lc, g, b, f, m, which);
    if (g.ndim == 3) corr_launch<N, 2>(lc, g, b, f, m, which);
}

void launch_adj_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, bool vel)
{
    // velocity part: the axes touch disjoint arrays.  Pressure part: every
    // phi update reads lp before any axis changes it, then one launch per
    // axis (each updates lp).
    if (vel) {
        if (g.N == 2) corr_axes<2>(lc, g, b, f, m, 0);
        else corr_axes<4>(lc, g, b, f, m, 0);
        return;
    }
    if (g.N == 2) {
        corr_axes<2>(lc, g, b, f, m, 1);
        corr_axes<2>(lc, g, b, f, m, 2);
    } else {
        corr_axes<4>(lc, g, b, f, m, 1);
        corr_axes<4>(lc, g, b, f, m, 2);
    }
}

void launch_fwd_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, bool vel)
{
    // velocity: axes touch disjoint arrays; pressure: one launch per axis,
    // each updating p in the slab of its axis
    if (g.N == 2) corr_axes<2>(lc, g, b, f, it, vel ? 3 : 4);
    else corr_axes<4>(lc, g, b, f, it, vel ? 3 : 4);
}

void launch_inject_source(const LaunchCtx &lc, const Grid &g, const Batch &b, float *p,
                          const float *stf, int it, float scale)
{
    k_inject_source<<<b.nshot, 128, 0, S(lc)>>>(g, b, p, stf, it, scale);
    ++*lc.launches;
}

void launch_gather(const LaunchCtx &lc, const Grid &g, const Batch &b, const float *p, float *seis,
                   const long long *seis_off, int nt, int it)
{
    (void)nt;
    dim3 grid((b.max_rec + 127) / 128, b.nshot);
    k_gather<<<grid, 128, 0, S(lc)>>>(g, b, p, seis, seis_off, it);
    ++*lc.launches;
}

void launch_adj_inject(const LaunchCtx &lc, const Grid &g, const Batch &b, float *lp, const float *res,
                       const long long *seis_off, int nt, int it)
{
    (void)nt;
    dim3 grid((b.max_rec + 127) / 128, b.nshot);
    k_adj_inject<<<grid, 128, 0, S(lc)>>>(g, b, lp, res, seis_off, it);
    ++*lc.launches;
}

void launch_save_bands(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, Bands bd, int it,
                       unsigned *absmax_tmp)
{
    dim3 grid((unsigned)((bd.count + kThreads - 1) / kThreads), b.nshot);
    if (bd.prec != SMI_PREC_F32) {
        cudaMemsetAsync(absmax_tmp, 0, sizeof(unsigned) * 6 * b.nshot, S(lc));
        k_band_absmax<<<grid, kThreads, 0, S(lc)>>>(g, f, bd, absmax_tmp);
        ++*lc.launches;
    }
    k_band_save<<<grid, kThreads, 0, S(lc)>>>(g, f, bd, it, absmax_tmp);
    ++*lc.launches;
}

void launch_restore_bands(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, Bands bd, int it)
{
    dim3 grid((unsigned)((bd.count + kThreads - 1) / kThreads), b.nshot);
    k_band_restore<<<grid, kThreads, 0, S(lc)>>>(g, f, bd, it);
    ++*lc.launches;
}

void launch_residual(const LaunchCtx &lc, const float *seis, const float *dobs, long long n, int mode,
                     float *res, double *partials, int npart)
{
    k_residual<<<npart, kThreads, 0, S(lc)>>>(seis, dobs, n, mode, res, partials);
    ++*lc.launches;
}

void launch_sum_partials(const LaunchCtx &lc, const double *partials, int npart, double *out)
{
    k_sum_partials<<<1, 32, 0, S(lc)>>>(partials, npart, out);
    ++*lc.launches;
}

void launch_reduce_shots(const LaunchCtx &lc, const Grid &g, const float *acc, int nshot, float *out,
                         int accumulate)
{
    k_reduce_shots<<<blocks_for(g.nphys), kThreads, 0, S(lc)>>>(acc, g.nphys, nshot, out, accumulate);
    ++*lc.launches;
}

void launch_finalize_grad(const LaunchCtx &lc, long long n, const float *vp, float dt, float *gr)
{
    k_finalize_grad<<<blocks_for(n), kThreads, 0, S(lc)>>>(n, vp, dt, gr);
    ++*lc.launches;
}

void launch_nonfinite(const LaunchCtx &lc, const float *x, long long n, unsigned *flag)
{
    k_nonfinite<<<blocks_for(n), kThreads, 0, S(lc)>>>(x, n, flag);
    ++*lc.launches;
}

void launch_extend_model(const LaunchCtx &lc, const Grid &g, const float *vp, const float *rho, int n1,
                         int n2, int n3, float *K, float *rho_e)
{
    k_extend_model<<<blocks_for(g.ntot), kThreads, 0, S(lc)>>>(g, vp, rho, n1, n2, n3, K, rho_e);
    ++*lc.launches;
}

void launch_minmax(const LaunchCtx &lc, const float *vp, long long n, float *out2, unsigned *tmp)
{
    k_minmax_init<<<1, 1, 0, S(lc)>>>(tmp);
    k_minmax<<<blocks_for(n), kThreads, 0, S(lc)>>>(vp, n, tmp);
    k_minmax_out<<<1, 1, 0, S(lc)>>>(tmp, out2);
    *lc.launches += 3;
}

void launch_zero(const LaunchCtx &lc, void *ptr, size_t bytes)
{
    cudaMemsetAsync(ptr, 0, bytes, S(lc));
}

void launch_box_fill(const LaunchCtx &lc, const Grid &g, const int *ext, int nshot, int nt, int *tab)
{
    const long long n = (long long)nshot * (nt + 1);
    k_box_fill<<<(unsigned)((n + 127) / 128), 128, 0, S(lc)>>>(g, ext, nshot, nt, tab);
    ++*lc.launches;
}

void launch_box_table(const LaunchCtx &lc, const Grid &g, const int *ext, int n0, int count, int *lo,
                      int *hi)
{
    k_box_table<<<(count + 127) / 128, 128, 0, S(lc)>>>(g, ext, n0, count, lo, hi);
    ++*lc.launches;
}

}  // namespace smi
