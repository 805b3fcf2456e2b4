// smi_fused3d.cu -- single-pass 3D staggered-grid step for sm_103a: the
// velocity update and the pressure update of one leap-frog step (Sec. 2.1
// update equations) in one kernel, with the CPML terms of all three axes
// applied inline (forward, and exactly transposed for the adjoint in its
// "same solver" form, Sec. 2.2 / Eq. adj).
//
// Why one pass: a two-pass step writes v and reads it back (56 B a point);
// here v^{n+1/2} is produced and consumed on chip, so the algorithmic traffic
// is 40 B a point (p, v_z, v_x, v_y, kappa, rho in; p, v out).  In practice
// p is loaded twice (its halo tiles at its own plane, and 2N-1 planes earlier
// for the v_y queue) and rho in three geometries, and those re-reads do not
// all hit in L2: about 50 B a point reach DRAM in interior tiles.
//
// Status: an opt-in kernel family (SMI_KERNELS_FUSED).  On GB300 it runs
// slower than the two-pass kernels with the CPML band kernels: it issues at
// 35-40 % with 7-10 warps resident (both register queues, the halo
// recomputation and the CPML work sit on each thread).
//
// How: persistent CTAs walk 32 (z) x 16 (x) tile columns times y-chunks of
// the computing box (Sec. 4.1).  For the p-plane y a CTA computes
//   - v_z on its tile widened by the N-1 / N nodes along z that D_z v_z
//     needs, and v_x widened along x likewise (halo nodes are recomputed by
//     every tile that needs them), into shared memory;
//   - v_y on plane y+N-1 into a register queue (D_y v_y at p-plane y needs
//     v_y on planes y-N .. y+N-1);
//   - p on plane y from those.
// Inputs arrive by TMA (cp.async.bulk.tensor) into a ring of shared-memory
// slots, two planes deep, guarded by mbarriers; the p values that feed the
// v_y derivative ride in a second register queue (planes y .. y+2N-1).
//
// Because halo nodes of v (and of the CPML memory variables) are recomputed
// from old values that the neighbouring tile overwrites, the state is double
// buffered: the kernel reads buffer `cur` and writes buffer `nxt`, only at
// its own nodes and only inside the box.  Boxes grow monotonically in the
// forward and adjoint runs, so both buffers hold zeros outside the box and
// the result equals the in-place scheme exactly.
//
// CPML (z and x memory variables full-size, y memory variables in the y
// slab layout): forward psi <- B psi + A D, added to the derivative; adjoint
// (lambda form) D_a acts on (1 + Ap) lp + Ap phi at p nodes and the pressure
// part on R = (1 + Av) lv + Av chi at v nodes, with chi <- Bv (chi + lv_old)
// and phi <- Bp (phi + lp_old).  Tiles whose stencils reach a z or x slab
// take the CPML branch (CTA-uniform); the others run the plain scheme.
//
// Every mbarrier wait is bounded; a CTA that gives up sets bit 0 of the
// error word, drains its own copies (bounded) and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "smi_box.h"
#include "smi_fused3d.h"
#include "smi_internal.h"
#include "smi_stencil3d.h"
#include "smi_tile3d.h"

#ifndef SMI_FD1
#define SMI_FD1 2            // ring depth (planes) of the fused kernel
#endif
#ifndef SMI_FMINB
#define SMI_FMINB 3          // resident CTAs per SM the register budget must allow
#endif
#ifndef SMI_FUNROLL
#define SMI_FUNROLL 1        // y planes per unrolled group (the body is large: keep it in the instruction cache)
#endif

namespace smi {
namespace s3 {

constexpr int FD1 = SMI_FD1;
constexpr int FCORE = TZ * TX;

// Shared-memory slot of one p-plane y (floats; every piece a multiple of 32).
// Band tiles add the CPML memory variables of plane y: the p-grid ones (z:
// psiv[0], x: psiv[1]) in the geometry of the p tiles and the v-grid ones (z:
// psip[0], x: psip[1]) in that of the old v_z / v_x tiles.
template <int N, bool BAND = false> struct FLay {
    static constexpr int PB_X = TX + 4 * N - 2;   // p rows x0-2N+1 .. x0+TX+2N-2 (for D_x at the v_x halo)
    static constexpr int VX_X = TX + 2 * N - 1;   // v_x rows x0-N .. x0+TX+N-2
    static constexpr int RB_X = TX + 2 * N;       // rho rows x0-N .. x0+TX+N-1
    static constexpr int PA = 0;                  // p, z0-8 .. z0+39 (48) x tile x
    static constexpr int PB = PA + 48 * TX;       // p, tile z x PB_X rows
    static constexpr int VZ = PB + 32 * PB_X;     // v_z old, z0-4 .. z0+35 (40) x tile x
    static constexpr int VX = VZ + 40 * TX;       // v_x old, tile z x VX_X rows
    static constexpr int RA = VX + 32 * VX_X;     // rho, z0-4 .. z0+39 (44) x tile x
    static constexpr int RB = RA + 44 * TX;       // rho, tile z x RB_X rows
    static constexpr int KC = RB + 32 * RB_X;     // kappa, plane y
    static constexpr int P0 = KC + FCORE;         // p old, plane y
    static constexpr int VY = P0 + FCORE;         // v_y old, plane y+N-1
    static constexpr int RY = VY + FCORE;         // rho, plane y+N
    static constexpr int PQ = RY + FCORE;         // p old, plane y+2N-1 (enters the queue)
    static constexpr int ZA = PQ + FCORE;         // band: z memory variable on the p grid, PA geometry
    static constexpr int XB = ZA + 48 * TX;       // band: x memory variable on the p grid, PB geometry
    static constexpr int ZV = XB + 32 * PB_X;     // band: z memory variable on the v grid, VZ geometry
    static constexpr int XV = ZV + 40 * TX;       // band: x memory variable on the v grid, VX geometry
    static constexpr int SLOT = BAND ? XV + 32 * VX_X : ZA;
    static constexpr unsigned BYTES = (unsigned)ZA * 4u;            // fields and model (every tile)
    static constexpr unsigned ZBYTES = (unsigned)(48 * TX + 40 * TX) * 4u;      // z memory variables
    static constexpr unsigned XBYTES = (unsigned)(32 * PB_X + 32 * VX_X) * 4u;  // x memory variables
    static constexpr int VZN = 40 * TX;           // new v_z (adjoint: R_z), z0-4 .. z0+35
    static constexpr int VXN = 32 * VX_X;         // new v_x (adjoint: R_x), VX_X rows
    static constexpr int SMEM = (FD1 * SLOT + VZN + VXN) * 4;
    static_assert(PB % 32 == 0 && VZ % 32 == 0 && VX % 32 == 0 && RA % 32 == 0 && RB % 32 == 0 && KC % 32 == 0 &&
                      ZA % 32 == 0 && XB % 32 == 0 && ZV % 32 == 0 && XV % 32 == 0 && SLOT % 32 == 0,
                  "slot pieces must stay 128-byte aligned for TMA");
};

// Own-node offsets: field arrays and full-size z / x memory variables share
// the padded layout; 32-bit within one shot.
__device__ __forceinline__ int foff(const Grid &g, int z, int x, int y) { return z + g.px * (x + g.ne[1] * y); }

template <class T> __device__ __forceinline__ void ld4(float (&a)[4], const T *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
__device__ __forceinline__ void st4(float *p, const float (&a)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
}
__device__ __forceinline__ void sts4(float *p, const float (&a)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
}

// Per-tile context shared by the quad routines.
struct FCtx {
    int s, z0, x0;
    int lo[3], hi[3];
    long long sh;           // offset of the shot's arrays (within one shot offsets are 32-bit)
    bool zb, xb;            // tile whose stencils reach a z / x slab
};

// ---------------------------------------------------------------------------
// v_z on the quad of z nodes z..z+3 at column x of plane y.  Returns the new
// values (out-of-box nodes keep their old values) and, in the adjoint, the
// pressure-part operand R_z = lv + Av (lv + chi); own quads write v (and the
// memory variable) to nxt.
template <int N, int MODE, bool BAND>
__device__ __forceinline__ void vz_quad(const Grid &g, const FCtx &c, const FTabs &tb, const float *slot, int z,
                                        int cx, const bool (&m)[4], bool wr, long long o, const Fields &nxt,
                                        float (&out)[4])
{
    using Lay = FLay<N, BAND>;
    const int zi = z - c.z0 + 4;                   // index in the 40/44-row layouts
    float W[12];
    {
        const float *row = slot + Lay::PA + cx * 48 + zi;
        float4 a0 = lds4(row), a1 = lds4(row + 4), a2 = lds4(row + 8);
        W[0] = a0.x; W[1] = a0.y; W[2] = a0.z; W[3] = a0.w;
        W[4] = a1.x; W[5] = a1.y; W[6] = a1.z; W[7] = a1.w;
        W[8] = a2.x; W[9] = a2.y; W[10] = a2.z; W[11] = a2.w;
    }
    const bool sq = BAND && c.zb && zquad_slab(g, z);      // the quad itself has slab nodes
    if (MODE == ADJ && BAND && c.zb && (z - 4 < g.nb || z + 7 >= g.ne[0] - g.nb - 1)) {
        // transposed CPML operand over the window: lp + Ap (lp + phi) at slab nodes
        const float *ph = slot + Lay::ZA + cx * 48 + zi;
#pragma unroll
        for (int i = 0; i < 12; i++) W[i] += tb.z[0][zi + i] * (W[i] + ph[i]);
    }
    float rz[5], v[4];
    {
        const float *rr = slot + Lay::RA + cx * 44 + zi;
        float4 r0 = lds4(rr);
        rz[0] = r0.x; rz[1] = r0.y; rz[2] = r0.z; rz[3] = r0.w; rz[4] = rr[4];
        put(v, lds4(slot + Lay::VZ + cx * 40 + zi));
    }
    float D[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        float d = 0.f;
#pragma unroll
        for (int l = 1; l <= N; l++) d += g.c[0][l - 1] * (W[4 + r + l] - W[4 + r - l + 1]);
        D[r] = d;
    }
    float mem[4] = {0.f, 0.f, 0.f, 0.f};
    if (sq) put(mem, lds4(slot + Lay::ZV + cx * 40 + zi));
    float nv[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        // interior tiles never hold the last node of the axis (1 / rho there)
        const float bz = BAND ? buoy(rz[r], rz[r + 1], z + r + 1 >= g.ne[0]) : __fdividef(2.0f, rz[r] + rz[r + 1]);
        const int t = zi + 4 + r;                  // table index of node z+r
        const bool sl = sq && slab_at(g, 0, z + r);
        if (MODE == FWD) {
            float dd = D[r];
            if (sl && m[r]) {
                mem[r] = tb.z[3][t] * mem[r] + tb.z[2][t] * dd;
                dd += mem[r];
            }
            nv[r] = m[r] ? v[r] - g.dt * bz * dd : v[r];
            out[r] = nv[r];
        } else {
            if (sl && m[r]) mem[r] = tb.z[3][t] * (mem[r] + v[r]);     // chi with lv before this step
            nv[r] = m[r] ? v[r] - g.dt * bz * D[r] : v[r];
            out[r] = sl ? nv[r] + tb.z[2][t] * (nv[r] + mem[r]) : nv[r];
        }
    }
    if (wr) {
        st4(nxt.v[0] + o, nv);
        if (sq) st4(nxt.psip[0] + o, mem);
    }
}

// v_x on the quad z..z+3 at column x (x0-N <= x <= x0+TX+N-2) of plane y.
template <int N, int MODE, bool BAND>
__device__ __forceinline__ void vx_quad(const Grid &g, const FCtx &c, const FTabs &tb, const float *slot, int zc,
                                        int x, const bool (&m)[4], bool wr, long long o, const Fields &nxt,
                                        float (&out)[4])
{
    using Lay = FLay<N, BAND>;
    const int xr = x - c.x0 + N;                   // row in the VX / RB layouts
    float Xr[2 * N][4];                            // p at x-N+1 .. x+N
#pragma unroll
    for (int t = 0; t < 2 * N; t++) put(Xr[t], lds4(slot + Lay::PB + (xr + t) * 32 + zc));
    if (MODE == ADJ && BAND && c.xb) {
        // transposed CPML operand at the taps (Ap = 0 off the slab)
#pragma unroll
        for (int t = 0; t < 2 * N; t++) {
            const float A = tb.x[0][xr + t + 8 - 2 * N + 1];
            if (A != 0.f) {
                float ph[4];
                put(ph, lds4(slot + Lay::XB + (xr + t) * 32 + zc));
#pragma unroll
                for (int r = 0; r < 4; r++) Xr[t][r] += A * (Xr[t][r] + ph[r]);
            }
        }
    }
    float r0[4], r1[4], v[4];
    put(r0, lds4(slot + Lay::RB + xr * 32 + zc));
    put(r1, lds4(slot + Lay::RB + (xr + 1) * 32 + zc));
    put(v, lds4(slot + Lay::VX + xr * 32 + zc));
    float D[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        float d = 0.f;
#pragma unroll
        for (int l = 1; l <= N; l++) d += g.c[1][l - 1] * (Xr[N - 1 + l][r] - Xr[N - l][r]);
        D[r] = d;
    }
    const bool sx = BAND && c.xb && in_range(x, 0, g.ne[1] - 1) && slab_at(g, 1, x);
    float mem[4] = {0.f, 0.f, 0.f, 0.f};
    if (sx) put(mem, lds4(slot + Lay::XV + xr * 32 + zc));
    const int t = x - c.x0 + 8;
    const bool lastx = BAND && x + 1 >= g.ne[1];
    float nv[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const float bx = BAND ? buoy(r0[r], r1[r], lastx) : __fdividef(2.0f, r0[r] + r1[r]);
        if (MODE == FWD) {
            float dd = D[r];
            if (sx && m[r]) {
                mem[r] = tb.x[3][t] * mem[r] + tb.x[2][t] * dd;
                dd += mem[r];
            }
            nv[r] = m[r] ? v[r] - g.dt * bx * dd : v[r];
            out[r] = nv[r];
        } else {
            if (sx && m[r]) mem[r] = tb.x[3][t] * (mem[r] + v[r]);
            nv[r] = m[r] ? v[r] - g.dt * bx * D[r] : v[r];
            out[r] = sx ? nv[r] + tb.x[2][t] * (nv[r] + mem[r]) : nv[r];
        }
    }
    if (wr) {
        st4(nxt.v[1] + o, nv);
        if (sx) st4(nxt.psip[1] + o, mem);
    }
}

// v_y on the own quad at plane yv from its derivative D (of p, or in the
// adjoint of the transposed operand), with the y-slab CPML; out = the queue
// entry (v, or in the adjoint R_y).  Writes nxt when the plane is the
// tile's own (write) and the column lies inside the box.
template <int MODE>
__device__ __forceinline__ void vy_update(const Grid &g, const FCtx &c, int oz, int ox, int yv, bool memq, bool write,
                                          float (&D)[4], const float (&rho0)[4], const float (&rho1)[4],
                                          const float (&v)[4], const Fields &cur, const Fields &nxt, float (&out)[4])
{
    const bool ingrid = yv >= 0 && yv < g.ne[2];
    const bool mxy = in_range(ox, c.lo[1], c.hi[1]) && in_range(yv, c.lo[2], c.hi[2]);
    bool m[4];
#pragma unroll
    for (int r = 0; r < 4; r++) m[r] = mxy && in_range(oz + r, c.lo[0], c.hi[0]);
    const bool sl = memq && ingrid && yslab(g, yv);
    float mem[4] = {0.f, 0.f, 0.f, 0.f};
    long long yo = 0;
    float A = 0.f, B = 0.f;
    if (sl) {
        yo = yslab_off(g, c.s, oz, ox, yv);
        ld4(mem, cur.psip[2] + yo);
        A = g.cva[2][yv];
        B = g.cvb[2][yv];
    }
    const bool lasty = yv + 1 >= g.ne[2];
    float nv[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const float by = buoy(rho0[r], rho1[r], lasty);
        if (MODE == FWD) {
            float dd = D[r];
            if (sl && m[r]) {
                mem[r] = B * mem[r] + A * dd;
                dd += mem[r];
            }
            nv[r] = m[r] ? v[r] - g.dt * by * dd : v[r];
            out[r] = nv[r];
        } else {
            if (sl && m[r]) mem[r] = B * (mem[r] + v[r]);
            nv[r] = m[r] ? v[r] - g.dt * by * D[r] : v[r];
            out[r] = sl ? nv[r] + A * (nv[r] + mem[r]) : nv[r];
        }
    }
    if (write && memq && ingrid && mxy) {
        st4(nxt.v[2] + c.sh + foff(g, oz, ox, yv), nv);
        if (sl) st4(nxt.psip[2] + yo, mem);
    }
}

// p on the own quad at plane y from the three derivatives of v (adjoint:
// of the R operands), with the CPML terms of the three axes.  m: the quad's
// box mask (all false: nothing is updated and nxt keeps its equal value).
template <int N, int MODE, bool BAND>
__device__ __forceinline__ void p_update(const Grid &g, const FCtx &c, const FTabs &tb, const float *slot, int oz,
                                         int ox, int y, int txi, int tzi, const bool (&m)[4], long long o,
                                         float (&dz)[4], float (&dx)[4], float (&dy)[4], const float (&pold)[4],
                                         const float (&K)[4], const Fields &cur, const Fields &nxt)
{
    using Lay = FLay<N, BAND>;
    if (!(m[0] || m[1] || m[2] || m[3])) return;
    if (BAND && c.zb && zquad_slab(g, oz)) {     // z memory variable at the quad's slab nodes
        float mem[4];
        put(mem, lds4(slot + Lay::ZA + txi * 48 + 4 * tzi + 8));
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int t = 4 * tzi + 8 + r;
            if (!(m[r] && slab_at(g, 0, oz + r))) continue;
            if (MODE == FWD) {
                mem[r] = tb.z[1][t] * mem[r] + tb.z[0][t] * dz[r];
                dz[r] += mem[r];
            } else {
                mem[r] = tb.z[1][t] * (mem[r] + pold[r]);
            }
        }
        st4(nxt.psiv[0] + o, mem);
    }
    if (BAND && c.xb && slab_at(g, 1, ox)) {
        float mem[4];
        put(mem, lds4(slot + Lay::XB + (txi + 2 * N - 1) * 32 + 4 * tzi));
        const int t = txi + 8;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (!m[r]) continue;
            if (MODE == FWD) {
                mem[r] = tb.x[1][t] * mem[r] + tb.x[0][t] * dx[r];
                dx[r] += mem[r];
            } else {
                mem[r] = tb.x[1][t] * (mem[r] + pold[r]);
            }
        }
        st4(nxt.psiv[1] + o, mem);
    }
    if (yslab(g, y)) {
        const long long yo = yslab_off(g, c.s, oz, ox, y);
        float mem[4];
        ld4(mem, cur.psiv[2] + yo);
        const float A = g.cpa[2][y], B = g.cpb[2][y];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (!m[r]) continue;
            if (MODE == FWD) {
                mem[r] = B * mem[r] + A * dy[r];
                dy[r] += mem[r];
            } else {
                mem[r] = B * (mem[r] + pold[r]);
            }
        }
        st4(nxt.psiv[2] + yo, mem);
    }
    float np[4];
#pragma unroll
    for (int r = 0; r < 4; r++) np[r] = m[r] ? pold[r] - g.dt * K[r] * (dz[r] + dx[r] + dy[r]) : pold[r];
    st4(nxt.p + o, np);
}

// ===========================================================================
// The fused step.  MODE FWD: the forward scheme with the forward CPML (box
// of the source); MODE ADJ: the adjoint in lambda form with the transposed
// CPML (box of the receivers after `step` reverse steps).
template <int N, int MODE, bool BAND>
__global__ void __launch_bounds__(NTHR, SMI_FMINB)
k3_fused(const __grid_constant__ CUtensorMap tm_pA, const __grid_constant__ CUtensorMap tm_pB,
         const __grid_constant__ CUtensorMap tm_vzA, const __grid_constant__ CUtensorMap tm_vxB,
         const __grid_constant__ CUtensorMap tm_vy, const __grid_constant__ CUtensorMap tm_pc,
         const __grid_constant__ CUtensorMap tm_rA, const __grid_constant__ CUtensorMap tm_rB,
         const __grid_constant__ CUtensorMap tm_rc, const __grid_constant__ CUtensorMap tm_Kc,
         const __grid_constant__ CUtensorMap tm_mzA, const __grid_constant__ CUtensorMap tm_mxB,
         const __grid_constant__ CUtensorMap tm_mzV, const __grid_constant__ CUtensorMap tm_mxV, Grid g, Batch b,
         Fields cur, Fields nxt, int step, unsigned *err)
{
    using Lay = FLay<N, BAND>;
    constexpr int Q = 2 * N;
    extern __shared__ __align__(128) float sm[];
    float *vzn = sm + FD1 * Lay::SLOT;
    float *vxn = vzn + Lay::VZN;
    __shared__ __align__(8) uint64_t bar[FD1];
    __shared__ FTabs tb;
    const int tid = threadIdx.x, tzi = tid & 7, txi = tid >> 3;
    if (tid == 0) {
        for (int k = 0; k < FD1; k++) mbar_init(&bar[k], 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned parity = 0;

    Item it;
    for (long long w = blockIdx.x; get_citem(g, b, MODE, step, BAND, w, it); w += gridDim.x) {
        FCtx c;
        c.s = it.s;
        c.z0 = it.z0;
        c.x0 = it.x0;
        for (int a = 0; a < 3; a++) {
            c.lo[a] = it.lo[a];
            c.hi[a] = it.hi[a];
        }
        c.sh = (long long)it.s * g.ntot;
        c.zb = BAND && band_z(g, c.z0);
        c.xb = BAND && band_x(g, c.x0);
        const int ya = it.ya, yb = it.yb;
        const int oz = c.z0 + 4 * tzi, ox = c.x0 + txi;
        const bool memq = oz < g.ne[0] && ox < g.ne[1];
        const int own = txi * TZ + 4 * tzi;        // own quad in the core tiles
        const long long plane = (long long)g.px * g.ne[1];
        // box masks of the quads this thread updates (z, x parts; y per plane)
        bool mzo[4], mzh[4], mzv[4];
        const bool mxo = in_range(ox, c.lo[1], c.hi[1]);
        const bool hvz = tid >= NTHR - 32;         // warp 3: the z halo of v_z
        const bool hvx = tid < 8 * (2 * N - 1);    // warps 0, 1: the x halo of v_x
        const int hzt = tid - (NTHR - 32);
        const int hz_x = hzt & (TX - 1), hz_z = (hzt >= TX) ? c.z0 + TZ : c.z0 - 4;
        const int hx_zq = tid & 7, hx_col = tid >> 3;
        const int hx_x = hx_col < N ? c.x0 - N + hx_col : c.x0 + TX + hx_col - N;
        const bool mxh = in_range(c.x0 + hz_x, c.lo[1], c.hi[1]);
        const bool mxv = in_range(hx_x, c.lo[1], c.hi[1]);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            mzo[r] = in_range(oz + r, c.lo[0], c.hi[0]);
            mzh[r] = in_range(hz_z + r, c.lo[0], c.hi[0]);
            mzv[r] = in_range(c.z0 + 4 * hx_zq + r, c.lo[0], c.hi[0]);
        }
        // own-node offset at plane 0 (v_z, v_x, p and the full-size memory variables share it)
        const long long o0 = c.sh + foff(g, oz, ox, 0);

        // CPML coefficient tables of a band tile (published by the barrier below)
        if (BAND) load_tabs(g, c.z0, c.x0, tb);

        auto issue = [&](int y) {
            const int k = (y - ya) % FD1;
            float *sl = sm + k * Lay::SLOT;
            mbar_expect(&bar[k], Lay::BYTES + (BAND && c.zb ? Lay::ZBYTES : 0u) + (BAND && c.xb ? Lay::XBYTES : 0u));
            tma4(sl + Lay::PA, &tm_pA, c.z0 - 8, c.x0, y, c.s, &bar[k]);
            tma4(sl + Lay::PB, &tm_pB, c.z0, c.x0 - 2 * N + 1, y, c.s, &bar[k]);
            tma4(sl + Lay::VZ, &tm_vzA, c.z0 - 4, c.x0, y, c.s, &bar[k]);
            tma4(sl + Lay::VX, &tm_vxB, c.z0, c.x0 - N, y, c.s, &bar[k]);
            tma4(sl + Lay::RA, &tm_rA, c.z0 - 4, c.x0, y, 0, &bar[k]);
            tma4(sl + Lay::RB, &tm_rB, c.z0, c.x0 - N, y, 0, &bar[k]);
            tma4(sl + Lay::KC, &tm_Kc, c.z0, c.x0, y, 0, &bar[k]);
            tma4(sl + Lay::P0, &tm_pc, c.z0, c.x0, y, c.s, &bar[k]);
            tma4(sl + Lay::VY, &tm_vy, c.z0, c.x0, y + N - 1, c.s, &bar[k]);
            tma4(sl + Lay::RY, &tm_rc, c.z0, c.x0, y + N, 0, &bar[k]);
            tma4(sl + Lay::PQ, &tm_pc, c.z0, c.x0, y + 2 * N - 1, c.s, &bar[k]);
            if (BAND) {
                if (c.zb) {
                    tma4(sl + Lay::ZA, &tm_mzA, c.z0 - 8, c.x0, y, c.s, &bar[k]);
                    tma4(sl + Lay::ZV, &tm_mzV, c.z0 - 4, c.x0, y, c.s, &bar[k]);
                }
                if (c.xb) {
                    tma4(sl + Lay::XB, &tm_mxB, c.z0, c.x0 - 2 * N + 1, y, c.s, &bar[k]);
                    tma4(sl + Lay::XV, &tm_mxV, c.z0, c.x0 - N, y, c.s, &bar[k]);
                }
            }
        };
        Ring rr{ya, min(yb, ya + FD1 - 1)};
        if (tid == 0)
            for (int y = ya; y <= rr.issued; y++) issue(y);

        // ---- prologue (plain loads, while the first copies fly) ----
        // p queue: logical entry l = plane y + l; v_y queue: l = plane y - N + l
        float pq[Q][4], vq[Q][4], ry0[4];
        {
            constexpr int NP = 4 * N - 2;
            const int base = ya - 2 * N + 1;
            float pre[NP][4];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const int yy = base + j;
                const bool in = memq && yy >= 0 && yy < g.ne[2];
                float t[4] = {0.f, 0.f, 0.f, 0.f};
                if (in) ld4(t, cur.p + c.sh + foff(g, oz, ox, yy));
                if (MODE == ADJ && in && yslab(g, yy)) {
                    float ph[4];
                    ld4(ph, cur.psiv[2] + yslab_off(g, c.s, oz, ox, yy));
                    const float A = g.cpa[2][yy];
#pragma unroll
                    for (int r = 0; r < 4; r++) t[r] += A * (t[r] + ph[r]);
                }
#pragma unroll
                for (int r = 0; r < 4; r++) pre[j][r] = t[r];
            }
#pragma unroll
            for (int j = 0; j < Q - 1; j++) {
                const int yv = ya - N + j;
                const bool in = memq && yv >= 0 && yv < g.ne[2];
                float D[4], v[4] = {0.f, 0.f, 0.f, 0.f}, r0[4] = {1.f, 1.f, 1.f, 1.f}, r1[4] = {1.f, 1.f, 1.f, 1.f};
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[2][l - 1] * (pre[j + N - 1 + l][r] - pre[j + N - l][r]);
                    D[r] = d;
                }
                if (in) {
                    ld4(v, cur.v[2] + c.sh + foff(g, oz, ox, yv));
                    ld4(r0, g.rho + foff(g, oz, ox, yv));
                    if (yv + 1 < g.ne[2]) ld4(r1, g.rho + foff(g, oz, ox, yv + 1));
                }
                vy_update<MODE>(g, c, oz, ox, yv, memq, yv >= ya && yv <= yb, D, r0, r1, v, cur, nxt, vq[j]);
            }
#pragma unroll
            for (int l = 0; l < Q - 1; l++)
#pragma unroll
                for (int r = 0; r < 4; r++) pq[l][r] = pre[Q - 1 + l][r];
            const int yr = ya + N - 1;
#pragma unroll
            for (int r = 0; r < 4; r++) ry0[r] = 1.f;
            if (memq && yr < g.ne[2]) ld4(ry0, g.rho + foff(g, oz, ox, yr));
        }
        bool ok = true;
        if (__syncthreads_or(!ok)) goto timeout;      // publishes the coefficient tables

        {
        bool stop = false;
        int y = ya;
        auto body = [&](auto kc) {
            constexpr int kq = decltype(kc)::value;
            ok = ring_wait(bar, FD1, 0, parity, rr, y, ya);
            const float *slot = sm + ((y - ya) % FD1) * Lay::SLOT;
            // the p plane y+2N-1 enters the queue (adjoint: transposed operand on y-slab planes)
            {
                float e[4];
                put(e, lds4(slot + Lay::PQ + own));
                const int ye = y + 2 * N - 1;
                if (MODE == ADJ && memq && ye < g.ne[2] && yslab(g, ye)) {
                    float ph[4];
                    ld4(ph, cur.psiv[2] + yslab_off(g, c.s, oz, ox, ye));
                    const float A = g.cpa[2][ye];
#pragma unroll
                    for (int r = 0; r < 4; r++) e[r] += A * (e[r] + ph[r]);
                }
#pragma unroll
                for (int r = 0; r < 4; r++) pq[(Q - 1 + kq) % Q][r] = e[r];
            }
            float t4[4];
            const bool my = in_range(y, c.lo[2], c.hi[2]);
            const long long oy = o0 + (long long)y * plane;
            bool m[4];
            // ---- v_z at plane y: own quad, then the z halo (warp 3) ----
#pragma unroll
            for (int r = 0; r < 4; r++) m[r] = mzo[r] && mxo && my;
            vz_quad<N, MODE, BAND>(g, c, tb, slot, oz, txi, m, memq && mxo && my, oy, nxt, t4);
            sts4(vzn + txi * 40 + 4 * tzi + 4, t4);
            if (hvz) {
                bool mh[4];
#pragma unroll
                for (int r = 0; r < 4; r++) mh[r] = mzh[r] && mxh && my;
                vz_quad<N, MODE, BAND>(g, c, tb, slot, hz_z, hz_x, mh, false, 0, nxt, t4);
                sts4(vzn + hz_x * 40 + (hz_z - c.z0 + 4), t4);
            }
            // ---- v_x at plane y: own quad, then the x halo (warps 0, 1) ----
            vx_quad<N, MODE, BAND>(g, c, tb, slot, 4 * tzi, ox, m, memq && mxo && my, oy, nxt, t4);
            sts4(vxn + (txi + N) * 32 + 4 * tzi, t4);
            if (hvx) {
                bool mh[4];
#pragma unroll
                for (int r = 0; r < 4; r++) mh[r] = mzv[r] && mxv && my;
                vx_quad<N, MODE, BAND>(g, c, tb, slot, 4 * hx_zq, hx_x, mh, false, 0, nxt, t4);
                sts4(vxn + (hx_x - c.x0 + N) * 32 + 4 * hx_zq, t4);
            }
            // ---- v_y at plane y+N-1 (own quad) ----
            {
                const int yv = y + N - 1;
                float D[4], r1[4], v[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++)
                        d += g.c[2][l - 1] * (pq[(N - 1 + l + kq) % Q][r] - pq[(N - l + kq) % Q][r]);
                    D[r] = d;
                }
                put(r1, lds4(slot + Lay::RY + own));
                put(v, lds4(slot + Lay::VY + own));
                if (yv + 1 >= g.ne[2]) {
#pragma unroll
                    for (int r = 0; r < 4; r++) r1[r] = 1.f;
                }
                vy_update<MODE>(g, c, oz, ox, yv, memq, yv <= yb, D, ry0, r1, v, cur, nxt, vq[(Q - 1 + kq) % Q]);
#pragma unroll
                for (int r = 0; r < 4; r++) ry0[r] = r1[r];
            }
            __syncthreads();                               // new v_z / v_x tiles complete
            // ---- p at plane y ----
            {
                float dz[4], dx[4], dy[4], K[4], p0[4];
                {
                    const float *row = vzn + txi * 40 + 4 * tzi;
                    float W[12];
                    float4 a0 = lds4(row), a1 = lds4(row + 4), a2 = lds4(row + 8);
                    W[0] = a0.x; W[1] = a0.y; W[2] = a0.z; W[3] = a0.w;
                    W[4] = a1.x; W[5] = a1.y; W[6] = a1.z; W[7] = a1.w;
                    W[8] = a2.x; W[9] = a2.y; W[10] = a2.z; W[11] = a2.w;
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        float d = 0.f;
#pragma unroll
                        for (int l = 1; l <= N; l++) d += g.c[0][l - 1] * (W[4 + r + l - 1] - W[4 + r - l]);
                        dz[r] = d;
                    }
                }
                {
                    float Xr[2 * N][4];
#pragma unroll
                    for (int l = 1; l <= N; l++) {
                        put(Xr[N + l - 1], lds4(vxn + (txi + N + l - 1) * 32 + 4 * tzi));
                        put(Xr[N - l], lds4(vxn + (txi + N - l) * 32 + 4 * tzi));
                    }
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        float d = 0.f;
#pragma unroll
                        for (int l = 1; l <= N; l++) d += g.c[1][l - 1] * (Xr[N + l - 1][r] - Xr[N - l][r]);
                        dx[r] = d;
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++)
                        d += g.c[2][l - 1] * (vq[(N + l - 1 + kq) % Q][r] - vq[(N - l + kq) % Q][r]);
                    dy[r] = d;
                }
                put(K, lds4(slot + Lay::KC + own));
                put(p0, lds4(slot + Lay::P0 + own));
                bool mp[4];
#pragma unroll
                for (int r = 0; r < 4; r++) mp[r] = memq && m[r];
                p_update<N, MODE, BAND>(g, c, tb, slot, oz, ox, y, txi, tzi, mp, oy, dz, dx, dy, p0, K, cur, nxt);
            }
            // all reads of plane y's slot and of the new v tiles are done
            if (__syncthreads_or(!ok)) {
                stop = true;
                return;
            }
            if (tid == 0 && rr.issued < yb) issue(rr.issued + 1);
            if (rr.issued < yb) rr.issued++;
        };
        constexpr int G = Q % SMI_FUNROLL == 0 ? SMI_FUNROLL : Q;
        while (y <= yb && !stop) {
            Unroll<0, G>::run(body, y, yb, stop);
            rotate_queue<G>(pq);
            rotate_queue<G>(vq);
        }
        if (stop) goto timeout;
        }
        continue;
    timeout:
        if (tid == 0) atomicOr(err, 1u);
        ring_drain(bar, FD1, 0, parity, rr, ya);
        return;
    }
}

}  // namespace s3

// ---------------------------------------------------------------------------
// Host side.
namespace {

template <int N, int MODE, bool BAND>
void run_class(const LaunchCtx &lc, const MapsF &mc, const MapsM &mm, const Grid &g, const Batch &b, Fields cur,
               Fields nxt, int step, unsigned *err)
{
    constexpr int smem = s3::FLay<N, BAND>::SMEM;
    static const int grid = [] {
        cudaFuncSetAttribute(s3::k3_fused<N, MODE, BAND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(s3::k3_fused<N, MODE, BAND>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int per = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, s3::k3_fused<N, MODE, BAND>, s3::NTHR, smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, per) * std::max(1, sms);
    }();
    s3::k3_fused<N, MODE, BAND><<<grid, s3::NTHR, smem, static_cast<cudaStream_t>(lc.stream)>>>(
        mc.pA, mc.pB, mc.vzA, mc.vxB, mc.vy, mc.pc, mm.rA, mm.rB, mm.rc, mm.Kc, mc.mzA, mc.mxB, mc.mzV, mc.mxV, g, b,
        cur, nxt, step, err);
    ++*lc.launches;
}

// The two classes write disjoint nodes and read only `cur`: no ordering
// between them is needed.
template <int N, int MODE>
void run_fused(const LaunchCtx &lc, const MapsF &mc, const MapsM &mm, const Grid &g, const Batch &b, Fields cur,
               Fields nxt, int step, unsigned *err)
{
    run_class<N, MODE, true>(lc, mc, mm, g, b, cur, nxt, step, err);
    run_class<N, MODE, false>(lc, mc, mm, g, b, cur, nxt, step, err);
}

}  // namespace

bool fused3d_supported(const Grid &g) { return stencil3d_supported(g) && !g.freesurf; }

bool make_maps_fused(MapsF &m, const Grid &g, const Fields &f, int nshot)
{
    const int N = g.N, TX = s3::TX;
    return make_tile_map(&m.pA, g, f.p, nshot, 48, TX) && make_tile_map(&m.pB, g, f.p, nshot, 32, TX + 4 * N - 2) &&
           make_tile_map(&m.vzA, g, f.v[0], nshot, 40, TX) &&
           make_tile_map(&m.vxB, g, f.v[1], nshot, 32, TX + 2 * N - 1) &&
           make_tile_map(&m.vy, g, f.v[2], nshot, 32, TX) && make_tile_map(&m.pc, g, f.p, nshot, 32, TX) &&
           make_tile_map(&m.mzA, g, f.psiv[0], nshot, 48, TX) &&
           make_tile_map(&m.mxB, g, f.psiv[1], nshot, 32, TX + 4 * N - 2) &&
           make_tile_map(&m.mzV, g, f.psip[0], nshot, 40, TX) &&
           make_tile_map(&m.mxV, g, f.psip[1], nshot, 32, TX + 2 * N - 1);
}

bool make_maps_model(MapsM &m, const Grid &g)
{
    const int N = g.N, TX = s3::TX;
    return make_tile_map(&m.rA, g, g.rho, 1, 44, TX) && make_tile_map(&m.rB, g, g.rho, 1, 32, TX + 2 * N) &&
           make_tile_map(&m.rc, g, g.rho, 1, 32, TX) && make_tile_map(&m.Kc, g, g.K, 1, 32, TX);
}

void launch3_fused(const LaunchCtx &lc, const MapsF &mc, const MapsM &mm, const Grid &g, const Batch &b, Fields cur,
                   Fields nxt, int step, int mode, unsigned *err)
{
    if (g.N == 2) {
        if (mode == 0) run_fused<2, s3::FWD>(lc, mc, mm, g, b, cur, nxt, step, err);
        else run_fused<2, s3::ADJ>(lc, mc, mm, g, b, cur, nxt, step, err);
    } else {
        if (mode == 0) run_fused<4, s3::FWD>(lc, mc, mm, g, b, cur, nxt, step, err);
        else run_fused<4, s3::ADJ>(lc, mc, mm, g, b, cur, nxt, step, err);
    }
}

}  // namespace smi
