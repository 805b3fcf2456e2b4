// smi_stencil2d.cu -- 2D staggered-grid stencil kernels (sm_103a).
//
// Two kernels advance one half of a leap-frog step each (Sec. 2.1 update
// equations): k2_v updates v_z and v_x from p, k2_p updates p from them.
// Modes:
//   FWD  forward update on the computing box of the source, with the CPML
//        memory variables (Sec. 2.1, Komatitsch & Martin) inline;
//   ADJ  the exact discrete adjoint in "same solver" form on the box of the
//        receivers: the interior scheme applied to operands that carry the
//        transposed CPML terms -- in the slabs D_a acts on
//        lp + Ap_a (lp + phi_a) (velocity kernel) or
//        lv_a + Av_a (lv_a + chi_a) (pressure kernel) instead of the plain
//        field -- and the memory variables chi_a, phi_a updated at the
//        thread's own nodes;
//   REC        source-field reconstruction backwards in time (Sec. 4.2) on
//              the physical domain inside the forward box of the step,
//              fused with the imaging / gradient accumulation in k2_p;
//              nodes outside the previous step's box are set to zero.
//
// A block is 8 x 32 threads over a 32 (z) x 32 (x) tile of the batch's box
// union (blockIdx.z = shot); a thread owns 4 consecutive z nodes of one x
// column as one float4.  z-derivatives use a 12-value window (three float4
// loads), x-derivatives one float4 per tap; neighbours come through L1.
// Rows are padded to px (a multiple of 8) and the padding holds zeros, so a
// float4 that reaches past the last z node reads the scheme's zero values.
// Offsets inside one shot's arrays are 32-bit (fewer than 2^31 points).
#include <cuda_runtime.h>

#include <algorithm>

#include "smi_box.h"
#include "smi_internal.h"

namespace smi {

namespace {

enum { FWD = 0, ADJ = 1, REC = 2 };

// Resident 256-thread blocks per SM the register budget must allow: 4
// (64 registers, a few spilled) for the forward and adjoint kernels, 3 for
// reconstruction.  The kernels are load-latency bound; on the 301 x 1001
// 40-shot gradient the budget moved the step from 37.5 (no bound, 88-96
// registers, 3 blocks) to 49.3 Gpt-updates/s.
__host__ __device__ constexpr int k2_min_blocks(int mode) { return mode == 2 ? 3 : 4; }

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void put(float (&a)[4], float4 v) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ bool in_range(int v, int lo, int hi) { return v >= lo && v <= hi; }

// Quad of field q at (oz..oz+3, x): zero outside the grid.
__device__ __forceinline__ void quad(const Grid &g, const float *q, int oz, int x, float (&a)[4])
{
    if (oz < 0 || oz >= g.px || x < 0 || x >= g.ne[1]) {
        a[0] = a[1] = a[2] = a[3] = 0.0f;
        return;
    }
    put(a, ld4(q + oz + g.px * x));
}

// The node block of this thread and the update box of its shot (REC: the
// forward box within the physical domain, plus the previous step's box).
struct Node2 {
    int s, oz, ox;
    bool mx, mz[4], any;
    int plo[3], phi[3];
};

template <int MODE>
__device__ __forceinline__ bool node2(const Grid &g, const Batch &b, int step, int z0, int x0, Node2 &n)
{
    n.s = blockIdx.z;
    n.oz = z0 + 32 * blockIdx.x + 4 * threadIdx.x;
    n.ox = x0 + 32 * blockIdx.y + threadIdx.y;
    if (n.oz >= g.ne[0] || n.ox >= g.ne[1]) return false;
    int lo[3], hi[3];
    box_at(MODE == ADJ ? b.tab_rec : b.tab_src, b.nt1, n.s, step, lo, hi);
    if (MODE == REC) {
        for (int a = 0; a < 2; a++) {
            lo[a] = max(lo[a], g.L[a]);
            hi[a] = min(hi[a], g.H[a]);
        }
        box_at(b.tab_src, b.nt1, n.s, step - 1, n.plo, n.phi);
    }
    n.mx = in_range(n.ox, lo[1], hi[1]);
    n.any = false;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        n.mz[r] = n.mx && in_range(n.oz + r, lo[0], hi[0]);
        n.any = n.any || n.mz[r];
    }
    return n.any;
}

__device__ __forceinline__ float buoy2(float r0, float r1, bool last)
{
    // fast reciprocal-based division: a few ulp, far below the FP32 scheme error
    return last ? __fdividef(1.0f, r0) : __fdividef(2.0f, r0 + r1);
}

// CPML slabs: nodes 0..nb-1 and ne-nb-1..ne-1 of an axis (the latter covers
// the first v node of the high layer).  Slab arrays of one shot: axis z at
// js + S x, axis x at z + ne_z js (js = index inside the slab).
__device__ __forceinline__ bool slab2(const Grid &g, int a, int j) { return j < g.nb || j >= g.ne[a] - g.nb - 1; }
__device__ __forceinline__ int js2(const Grid &g, int a, int j) { return j < g.nb ? j : j - (g.ne[a] - 2 * g.nb - 1); }
__device__ __forceinline__ int zslab_idx(const Grid &g, int z, int x) { return js2(g, 0, z) + g.S * x; }
__device__ __forceinline__ int xslab_idx(const Grid &g, int z, int x) { return z + g.ne[0] * js2(g, 1, x); }

// ADJ: operand q -> q + A (q + m) at the slab nodes of a z window W
// (W[e] at z = oz - 4 + e, column x) and of the x taps, m the memory
// variable of the axis (shot's slab arrays mz_s, mx_s), A = coefficient
// table of the axis.
template <int N>
__device__ __forceinline__ void adj_operand(const Grid &g, int oz, int ox, float (&W)[12], float (&Xp)[N][4],
                                            float (&Xm)[N][4], int xp0, int xm0, const float *Az,
                                            const float *Ax, const float *mz_s, const float *mx_s)
{
    if (oz - 4 < g.nb || oz + 7 >= g.ne[0] - g.nb - 1) {       // window reaches a z slab
#pragma unroll
        for (int e = 0; e < 12; e++) {
            const int z = oz - 4 + e;
            if (z >= 0 && z < g.ne[0] && slab2(g, 0, z)) W[e] += Az[z] * (W[e] + mz_s[zslab_idx(g, z, ox)]);
        }
    }
#pragma unroll
    for (int l = 1; l <= N; l++) {
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const int x = side == 0 ? ox + xp0 + l : ox + xm0 - l;
            float(&X)[4] = side == 0 ? Xp[l - 1] : Xm[l - 1];
            if (x < 0 || x >= g.ne[1] || !slab2(g, 1, x)) continue;
            const float A = Ax[x];
#pragma unroll
            for (int r = 0; r < 4; r++)
                if (oz + r < g.ne[0]) X[r] += A * (X[r] + mx_s[xslab_idx(g, oz + r, x)]);
        }
    }
}

// FWD: v_a -= dt b_a (D_a p + psi_a), psi_a <- Bv psi_a + Av D_a p in the
// slabs.  ADJ: chi_a <- Bv (chi_a + lv_a) at own slab nodes, then
// lv_a -= dt b_a D_a[lp + Ap_a (lp + phi_a)].  REC: v_a += dt b_a D_a p on
// L_a+N-1 .. H_a-N along a (elsewhere v_a keeps its saved value), zero
// outside the previous box.
template <int N, int MODE>
__global__ void __launch_bounds__(256, k2_min_blocks(MODE)) k2_v(Grid g, Batch b, Fields f, int step, int z0, int x0)
{
    Node2 n;
    if (!node2<MODE>(g, b, step, z0, x0, n)) return;
    const long long sh = (long long)n.s * g.ntot;
    const float *p = f.p + sh;
    const int oz = n.oz, ox = n.ox, k = oz + g.px * ox;
    float W[12];
    {
        float a[4], c[4], d[4];
        quad(g, p, oz - 4, ox, a);
        quad(g, p, oz, ox, c);
        quad(g, p, oz + 4, ox, d);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            W[r] = a[r];
            W[4 + r] = c[r];
            W[8 + r] = d[r];
        }
    }
    float Xp[N][4], Xm[N][4];                 // p at ox + l and ox - l + 1
#pragma unroll
    for (int l = 1; l <= N; l++) {
        quad(g, p, oz, ox + l, Xp[l - 1]);
        if (l == 1) {
#pragma unroll
            for (int r = 0; r < 4; r++) Xm[0][r] = W[4 + r];
        } else {
            quad(g, p, oz, ox - l + 1, Xm[l - 1]);
        }
    }
    if (MODE == ADJ)
        adj_operand<N>(g, oz, ox, W, Xp, Xm, 0, 1, g.cpa[0], g.cpa[1], f.psiv[0] + n.s * g.slab_n[0],
                       f.psiv[1] + n.s * g.slab_n[1]);
    float rho0[4], rx[4], vz[4], vx[4];
    put(rho0, ld4(g.rho + k));
    const bool lastx = ox + 1 >= g.ne[1];
    if (!lastx) put(rx, ld4(g.rho + k + g.px));
    const float rz4 = oz + 4 < g.ne[0] ? g.rho[k + 4] : 0.0f;
    put(vz, ld4(f.v[0] + sh + k));
    put(vx, ld4(f.v[1] + sh + k));
    bool keep[4];
    if (MODE == REC) {
#pragma unroll
        for (int r = 0; r < 4; r++)
            keep[r] = in_range(oz + r, n.plo[0], n.phi[0]) && in_range(ox, n.plo[1], n.phi[1]);
    }
    const bool rxm = in_range(ox, g.L[1] + N - 1, g.H[1] - N);
    const bool sx = MODE != REC && slab2(g, 1, ox);
    float *mz_s = f.psip[0] + n.s * g.slab_n[0], *mx_s = f.psip[1] + n.s * g.slab_n[1];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (!n.mz[r]) continue;
        float dz = 0.0f, dx = 0.0f;
#pragma unroll
        for (int l = 1; l <= N; l++) {
            dz += g.c[0][l - 1] * (W[4 + r + l] - W[4 + r - l + 1]);
            dx += g.c[1][l - 1] * (Xp[l - 1][r] - Xm[l - 1][r]);
        }
        const int z = oz + r;
        const float bz = buoy2(rho0[r], r < 3 ? rho0[r + 1] : rz4, z + 1 >= g.ne[0]);
        const float bx = buoy2(rho0[r], lastx ? 0.0f : rx[r], lastx);
        if (MODE == REC) {
            if (in_range(z, g.L[0] + N - 1, g.H[0] - N)) vz[r] = keep[r] ? vz[r] + g.dt * bz * dz : 0.0f;
            if (rxm) vx[r] = keep[r] ? vx[r] + g.dt * bx * dx : 0.0f;
            continue;
        }
        if (slab2(g, 0, z)) {
            float &m = mz_s[zslab_idx(g, z, ox)];
            if (MODE == FWD) {
                const float ps = g.cvb[0][z] * m + g.cva[0][z] * dz;
                m = ps;
                dz += ps;
            } else {
                m = g.cvb[0][z] * (m + vz[r]);            // deferred chi update, lv before this step
            }
        }
        if (sx) {
            float &m = mx_s[xslab_idx(g, z, ox)];
            if (MODE == FWD) {
                const float ps = g.cvb[1][ox] * m + g.cva[1][ox] * dx;
                m = ps;
                dx += ps;
            } else {
                m = g.cvb[1][ox] * (m + vx[r]);
            }
        }
        vz[r] -= g.dt * bz * dz;
        vx[r] -= g.dt * bx * dx;
    }
    *reinterpret_cast<float4 *>(f.v[0] + sh + k) = make_float4(vz[0], vz[1], vz[2], vz[3]);
    *reinterpret_cast<float4 *>(f.v[1] + sh + k) = make_float4(vx[0], vx[1], vx[2], vx[3]);
}

// FWD: p -= dt kappa sum_a (D_a v_a + psi_a), psi_a <- Bp psi_a + Ap D_a v_a
// in the slabs, then (stf not null) p += dt stf w / dV at the source stencil.  ADJ: phi_a <- Bp (phi_a + lp) at own slab nodes (lp before
// this step), then lp -= dt kappa sum_a D_a[lv_a + Av_a (lv_a + chi_a)].
// REC: acc += lp * (div v | p^{it+1}) (and, img_mode 2, the illumination
// p^2 into the second half of acc), p^{it} = p^{it+1} + dt kappa div v -
// dt stf w / dV, zero outside the previous box.
template <int N, int MODE>
__global__ void __launch_bounds__(256, k2_min_blocks(MODE)) k2_p(Grid g, Batch b, Fields f, int step, int z0, int x0, const float *lpall,
                                            float *acc, int img_mode, const float *stf, float src_scale)
{
    Node2 n;
    if (!node2<MODE>(g, b, step, z0, x0, n)) return;
    const long long sh = (long long)n.s * g.ntot;
    const float *vzf = f.v[0] + sh, *vxf = f.v[1] + sh;
    const int oz = n.oz, ox = n.ox, k = oz + g.px * ox;
    float W[12];
    {
        float a[4], c[4], d[4];
        quad(g, vzf, oz - 4, ox, a);
        quad(g, vzf, oz, ox, c);
        quad(g, vzf, oz + 4, ox, d);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            W[r] = a[r];
            W[4 + r] = c[r];
            W[8 + r] = d[r];
        }
    }
    float Xp[N][4], Xm[N][4];                 // v_x at ox + l - 1 and ox - l
#pragma unroll
    for (int l = 1; l <= N; l++) {
        quad(g, vxf, oz, ox + l - 1, Xp[l - 1]);
        quad(g, vxf, oz, ox - l, Xm[l - 1]);
    }
    if (MODE == ADJ)
        adj_operand<N>(g, oz, ox, W, Xp, Xm, -1, 0, g.cva[0], g.cva[1], f.psip[0] + n.s * g.slab_n[0],
                       f.psip[1] + n.s * g.slab_n[1]);
    float pv[4], Kv[4];
    put(pv, ld4(f.p + sh + k));
    put(Kv, ld4(g.K + k));
    float lpv[4];
    if (MODE == REC) put(lpv, ld4(lpall + sh + k));
    const bool sx = MODE != REC && slab2(g, 1, ox);
    float *mz_s = f.psiv[0] + n.s * g.slab_n[0], *mx_s = f.psiv[1] + n.s * g.slab_n[1];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (!n.mz[r]) continue;
        float dz = 0.0f, dx = 0.0f;
#pragma unroll
        for (int l = 1; l <= N; l++) {
            dz += g.c[0][l - 1] * (W[4 + r + l - 1] - W[4 + r - l]);
            dx += g.c[1][l - 1] * (Xp[l - 1][r] - Xm[l - 1][r]);
        }
        const int z = oz + r;
        if (MODE == REC) {
            const float div = dz + dx;
            const long long kp = (long long)n.s * g.nphys + (z - g.L[0]) +
                                 (long long)(g.H[0] - g.L[0] + 1) * (ox - g.L[1]);
            acc[kp] += lpv[r] * (img_mode == 0 ? div : pv[r]);
            if (img_mode == 2) acc[(long long)b.nshot * g.nphys + kp] += pv[r] * pv[r];   // illumination
            float pn = pv[r] + g.dt * Kv[r] * div;
            const Stencil &st = b.src[n.s];
            const int t0 = z - st.first[0], t1 = ox - st.first[1];
            if (t0 >= 0 && t0 < st.cnt[0] && t1 >= 0 && t1 < st.cnt[1])
                pn -= src_scale * stf[step] * st.w[0][t0] * st.w[1][t1] * st.w[2][0];
            const bool keep = in_range(z, n.plo[0], n.phi[0]) && in_range(ox, n.plo[1], n.phi[1]);
            pv[r] = keep ? pn : 0.0f;
            continue;
        }
        if (slab2(g, 0, z)) {
            float &m = mz_s[zslab_idx(g, z, ox)];
            if (MODE == FWD) {
                const float ps = g.cpb[0][z] * m + g.cpa[0][z] * dz;
                m = ps;
                dz += ps;
            } else {
                m = g.cpb[0][z] * (m + pv[r]);            // phi update, lp before this step
            }
        }
        if (sx) {
            float &m = mx_s[xslab_idx(g, z, ox)];
            if (MODE == FWD) {
                const float ps = g.cpb[1][ox] * m + g.cpa[1][ox] * dx;
                m = ps;
                dx += ps;
            } else {
                m = g.cpb[1][ox] * (m + pv[r]);
            }
        }
        pv[r] -= g.dt * Kv[r] * (dz + dx);
        if (MODE == FWD && stf) {                // source injection of this step (Algorithm 2)
            const Stencil &st = b.src[n.s];
            const int t0 = z - st.first[0], t1 = ox - st.first[1];
            if (t0 >= 0 && t0 < st.cnt[0] && t1 >= 0 && t1 < st.cnt[1])
                pv[r] += src_scale * stf[step] * st.w[0][t0] * st.w[1][t1] * st.w[2][0];
        }
    }
    *reinterpret_cast<float4 *>(f.p + sh + k) = make_float4(pv[0], pv[1], pv[2], pv[3]);
}

// Tile grid over the box union [lo, hi] (z start rounded down to 4).
dim3 grid2(const int lo[3], const int hi[3], int nshot, int &z0, int &x0)
{
    z0 = lo[0] & ~3;
    x0 = lo[1];
    const int nz = hi[0] - z0 + 1, nx = hi[1] - x0 + 1;
    if (nz <= 0 || nx <= 0) return dim3(0, 0, 0);
    return dim3((nz + 31) / 32, (nx + 31) / 32, nshot);
}

}  // namespace

bool stencil2d_supported(const Grid &g) { return g.ndim == 2 && (g.N == 2 || g.N == 4) && g.ntot < (1LL << 31); }

void launch2_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int step, int mode, const int lo[3],
               const int hi[3])
{
    int z0, x0;
    const dim3 grid = grid2(lo, hi, b.nshot, z0, x0);
    if (grid.x == 0) return;
    const dim3 block(8, 32);
    cudaStream_t st = static_cast<cudaStream_t>(lc.stream);
    if (g.N == 2) {
        if (mode == FWD) k2_v<2, FWD><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
        else if (mode == ADJ) k2_v<2, ADJ><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
        else k2_v<2, REC><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
    } else {
        if (mode == FWD) k2_v<4, FWD><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
        else if (mode == ADJ) k2_v<4, ADJ><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
        else k2_v<4, REC><<<grid, block, 0, st>>>(g, b, f, step, z0, x0);
    }
    ++*lc.launches;
}

void launch2_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int step, int mode, const int lo[3],
               const int hi[3], const float *lp, float *acc, int img_mode, const float *stf, float src_scale)
{
    int z0, x0;
    const dim3 grid = grid2(lo, hi, b.nshot, z0, x0);
    if (grid.x == 0) return;
    const dim3 block(8, 32);
    cudaStream_t st = static_cast<cudaStream_t>(lc.stream);
    if (g.N == 2) {
        if (mode == FWD) k2_p<2, FWD><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
        else if (mode == ADJ) k2_p<2, ADJ><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
        else k2_p<2, REC><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
    } else {
        if (mode == FWD) k2_p<4, FWD><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
        else if (mode == ADJ) k2_p<4, ADJ><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
        else k2_p<4, REC><<<grid, block, 0, st>>>(g, b, f, step, z0, x0, lp, acc, img_mode, stf, src_scale);
    }
    ++*lc.launches;
}

}  // namespace smi
