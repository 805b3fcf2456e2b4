// smi_stencil3d.cu -- 3D staggered-grid stencil kernels for sm_103a.
//
// Two kernels advance one half of a leap-frog step each (Sec. 2.1 update
// equations): k3_v updates the three velocity components from p, k3_p
// updates p from the velocities.  They run in two modes:
//   FWD  the branch-free interior update, applied to every node of the box
//        for both the forward scheme and the adjoint in "same solver" form;
//        the CPML terms (forward, and transposed for the adjoint) are added
//        by slab-only correction kernels (smi_kernels.cu);
//   REC  source-field reconstruction backwards in time (Sec. 4.2) on the
//        physical domain, with the imaging / gradient accumulation fused
//        into the pressure kernel.
//
// Work decomposition: persistent CTAs (a fixed multiple of the SM count)
// walk the work items of the computing box (Sec. 4.1, evaluated on the
// device from the step counter): 32 (z) x 16 (x) column tiles times chunks
// of y planes.  A CTA streams its chunk along y.  Plane tiles with their z/x
// halos arrive by TMA (cp.async.bulk.tensor) into a ring of shared-memory
// slots guarded by mbarriers; out-of-grid parts of a tile are filled with
// zeros by the TMA unit, which is exactly the scheme's zero value outside
// the extended grid.  y-neighbours are kept in a register queue.  Each
// thread owns 4 consecutive z nodes of one x column: z-derivatives read a
// 12-float window with three 128-bit shared loads, x-derivatives one 128-bit
// load per tap.  Every mbarrier wait is bounded; a CTA that gives up sets
// bit 0 of the error word, drains its own copies (bounded) and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "smi_box.h"
#include "smi_internal.h"
#include "smi_stencil3d.h"
#include "smi_tile3d.h"

namespace smi {
namespace s3 {


// --- shared-memory slot layouts (floats) ---------------------------------
// Haloed ring: slots resident while their plane feeds a derivative (N+1
// planes for the velocity kernel, N for the pressure kernel) plus PFP planes
// of lead.  Core ring: the pointwise 32 x 16 tiles of one plane, SC slots.
#ifndef SMI_SC
#define SMI_SC 3            // core-tile ring depth of the interior kernels
#endif
constexpr int PFP = SMI_PFP, SC = SMI_SC, CORE = TZ * TX;

// Tile classes of a launch (template CLS): ALLT every tile column of the box
// (z / x CPML terms then come from the band kernels), INT the interior
// columns only, BND the CPML-band columns only, with the z / x CPML terms
// applied inline from memory-variable tiles that arrive in the core ring
// (BND core slots: two deep).
enum { ALLT = 0, INT = 1, BND = 2 };

// Band extras of the velocity kernel's core slot: the p-grid memory
// variables (adjoint phi_z, phi_x) over the p tile's geometry, and the
// v-grid ones (forward psi / adjoint chi, z and x) over the core tile.
template <int N, int CLS = ALLT> struct VLay {
    static constexpr int PR = TX + 2 * N - 1;            // p tile rows: x0-N+1 .. x0+TX-1+N
    static constexpr int P_OFF = 0, P_SZ = rup32(ZW * PR);
    static constexpr int R_OFF = P_SZ, R_SZ = rup32(36 * (TX + 1));   // rho: z0..z0+35, x0..x0+TX
    static constexpr int SLOT = P_SZ + R_SZ;
    static constexpr int S = N + 1 + PFP;
    static constexpr unsigned BYTES = (unsigned)(ZW * PR + 36 * (TX + 1)) * 4u;
    static constexpr int E_PZ = 3 * CORE, E_PX = E_PZ + P_SZ, E_CZ = E_PX + P_SZ, E_CX = E_CZ + CORE;
    static constexpr int CSLOT = CLS == BND ? E_CX + CORE : 3 * CORE;   // vz, vx, vy (+ band extras)
    static constexpr unsigned CBYTES = 3u * CORE * 4u;
    static constexpr unsigned PBYTES = (unsigned)(ZW * PR) * 4u;        // one p-geometry memory tile
    static constexpr int NC = CLS == BND ? 2 : SC;
    static constexpr int SMEM = (S * SLOT + NC * CSLOT) * 4;
};
// Band extras of the pressure kernel's core slot: the v-grid memory
// variables (adjoint chi_z, chi_x) over the v_z / v_x tile geometries, and
// the p-grid ones (forward psi / adjoint phi, z and x) over the core tile.
template <int N, int CLS = ALLT> struct PLay {
    static constexpr int XR = TX + 2 * N - 1;            // vx tile rows: x0-N .. x0+TX-2+N
    static constexpr int Z_OFF = 0, Z_SZ = rup32(ZW * TX);            // vz: z0-4.., x core
    static constexpr int X_OFF = Z_SZ, X_SZ = rup32(TZ * XR);         // vx: z core
    static constexpr int Y_OFF = Z_SZ + X_SZ, Y_SZ = CORE;            // vy: core
    static constexpr int SLOT = Z_SZ + X_SZ + Y_SZ;
    static constexpr int S = N + PFP;
    static constexpr unsigned BYTES = (unsigned)(ZW * TX + TZ * XR + CORE) * 4u;
    static constexpr int E_HZ = 3 * CORE, E_HX = E_HZ + Z_SZ, E_CZ = E_HX + X_SZ, E_CX = E_CZ + CORE;
    static constexpr int CSLOT = CLS == BND ? E_CX + CORE : 3 * CORE;   // p, kappa, lambda_p (+ band extras)
    static constexpr int NC = CLS == BND ? 2 : SC;
    static constexpr int SMEM = (S * SLOT + NC * CSLOT) * 4;
};


// ===========================================================================
// Velocity kernel.  FWD/ADJ: v_a -= dt b_a D_a p (+ CPML terms); REC:
// v_a += dt b_a D_a p on L_a+N-1..H_a-N, zero outside the previous box.
template <int N, int MODE, int CLS>
__global__ void __launch_bounds__(NTHR, CLS == BND ? 3 : SMI_MINB)
k3_v(const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_rho,
     const __grid_constant__ CUtensorMap tm_vz, const __grid_constant__ CUtensorMap tm_vx,
     const __grid_constant__ CUtensorMap tm_vy, const __grid_constant__ CUtensorMap tm_pzh,
     const __grid_constant__ CUtensorMap tm_pxh, const __grid_constant__ CUtensorMap tm_cz,
     const __grid_constant__ CUtensorMap tm_cx, Grid g, Batch b, Fields f, int step, unsigned *err)
{
    using Lay = VLay<N, CLS>;
    constexpr int S = Lay::S;
    constexpr int SC = Lay::NC;
    extern __shared__ __align__(128) float sm[];
    float *cbase = sm + S * Lay::SLOT;
    __shared__ __align__(8) uint64_t bar[S], cbar[SC];
    __shared__ FTabs tb;
    const int tid = threadIdx.x, tzi = tid & 7, txi = tid >> 3;
    if (tid == 0) {
        for (int k = 0; k < S; k++) mbar_init(&bar[k], 1);
        for (int k = 0; k < SC; k++) mbar_init(&cbar[k], 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned parity = 0;
    const float dt = g.dt;
#ifdef SMI_TIMING
    long long t_wait = 0, t_sync = 0, t_all = clock64(), n_planes = 0;
#endif

    Item it;
    for (long long w = blockIdx.x;
         CLS == ALLT ? get_item(g, b, MODE, step, w, it) : get_citem(g, b, MODE, step, CLS == BND, w, it);
         w += gridDim.x) {
        const int s = it.s, z0 = it.z0, x0 = it.x0, ya = it.ya, yb = it.yb;
        const int ylast = yb + N;                 // last haloed plane needed
        const bool zb = CLS == BND && band_z(g, z0), xb = CLS == BND && band_x(g, x0);
        if (CLS == BND) load_tabs(g, z0, x0, tb);   // published by the barrier after the first waits
        // band extras of a core slot: bytes and copies (adjoint: p-geometry phi tiles too)
        const unsigned cbytes = Lay::CBYTES + (zb ? CORE * 4u + (MODE == ADJ ? Lay::PBYTES : 0u) : 0u) +
                                (xb ? CORE * 4u + (MODE == ADJ ? Lay::PBYTES : 0u) : 0u);
        auto issue_core = [&](int yy) {
            const int k = (yy - ya) % SC;
            float *cs = cbase + k * Lay::CSLOT;
            mbar_expect(&cbar[k], cbytes);
            tma4(cs, &tm_vz, z0, x0, yy, s, &cbar[k]);
            tma4(cs + CORE, &tm_vx, z0, x0, yy, s, &cbar[k]);
            tma4(cs + 2 * CORE, &tm_vy, z0, x0, yy, s, &cbar[k]);
            if (CLS == BND) {
                if (zb) {
                    if (MODE == ADJ) tma4(cs + Lay::E_PZ, &tm_pzh, z0 - 4, x0 - N + 1, yy, s, &cbar[k]);
                    tma4(cs + Lay::E_CZ, &tm_cz, z0, x0, yy, s, &cbar[k]);
                }
                if (xb) {
                    if (MODE == ADJ) tma4(cs + Lay::E_PX, &tm_pxh, z0 - 4, x0 - N + 1, yy, s, &cbar[k]);
                    tma4(cs + Lay::E_CX, &tm_cx, z0, x0, yy, s, &cbar[k]);
                }
            }
        };
        const int oz = z0 + 4 * tzi, ox = x0 + txi;
        const bool mem = oz < g.ne[0] && ox < g.ne[1];
        const long long sh = (long long)s * g.ntot;
        bool mz[4];
#pragma unroll
        for (int r = 0; r < 4; r++) mz[r] = in_range(oz + r, it.lo[0], it.hi[0]);
        const bool mx = in_range(ox, it.lo[1], it.hi[1]);
        const int own = (txi + N - 1) * ZW + 4 * tzi + 4;   // own nodes in a p tile

        // y queue of own p: entry l = plane y-N+1+l; planes before ya by plain loads
        float q[2 * N][4];
#pragma unroll
        for (int l = 0; l < N - 1; l++) {
            const int y = ya - N + 1 + l;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mem && y >= 0 && y < g.ne[2]) v = *reinterpret_cast<const float4 *>(f.p + sh + gidx(g, oz, ox, y));
            put(q[l], v);
        }
        Ring hr{ya, min(ylast, ya + S - 1)}, cr{ya, min(yb, ya + SC - 1)};
        if (tid == 0) {
            for (int y = ya; y <= hr.issued; y++) {
                const int k = (y - ya) % S;
                float *slot = sm + k * Lay::SLOT;
                mbar_expect(&bar[k], Lay::BYTES);
                tma4(slot + Lay::P_OFF, &tm_p, z0 - 4, x0 - N + 1, y, s, &bar[k]);
                tma4(slot + Lay::R_OFF, &tm_rho, z0, x0, y, 0, &bar[k]);
            }
            for (int y = ya; y <= cr.issued; y++) issue_core(y);
        }
        bool ok = true;
#pragma unroll
        for (int l = 0; l < N; l++) {
            ok &= ring_wait(bar, S, 0, parity, hr, ya + l, ya);
            put(q[N - 1 + l], lds4(sm + ((l) % S) * Lay::SLOT + Lay::P_OFF + own));
        }
        if (MODE == ADJ && mem && mx) {
            // transposed y CPML: the queue holds lp + Ap_y (lp + phi_y) on y-slab planes
#pragma unroll
            for (int l = 0; l < 2 * N - 1; l++) {
                const int yq = ya - N + 1 + l;
                if (yq < 0 || yq >= g.ne[2] || !yslab(g, yq)) continue;
                float ph[4];
                put(ph, ldg4(f.psiv[2] + yslab_off(g, s, oz, ox, yq)));
                const float A = g.cpa[2][yq];
#pragma unroll
                for (int r = 0; r < 4; r++) q[l][r] += A * (q[l][r] + ph[r]);
            }
        }
        if (__syncthreads_or(!ok)) goto timeout;

        {
        bool stop = false;
        int y = ya;
        auto body = [&](auto kc) {
            constexpr int kq = decltype(kc)::value;
#ifdef SMI_TIMING
            const long long tw0 = clock64();
#endif
            // y CPML operands, loaded before the waits: FWD psi_y, ADJ chi_y
            // of plane y; ADJ phi_y of the plane entering the queue
            const bool my = in_range(y, it.lo[2], it.hi[2]);
            const bool ysl = MODE != REC && mem && mx && my && yslab(g, y);
            const int ye = y + N;
            const bool yent = MODE == ADJ && mem && mx && ye < g.ne[2] && yslab(g, ye);
            float ym[4] = {0.f, 0.f, 0.f, 0.f}, yp[4] = {0.f, 0.f, 0.f, 0.f};
            if (ysl) put(ym, ldg4(f.psip[2] + yslab_off(g, s, oz, ox, y)));
            if (yent) put(yp, ldg4(f.psiv[2] + yslab_off(g, s, oz, ox, ye)));
            ok = ring_wait(bar, S, 0, parity, hr, y + N, ya);
            ok &= ring_wait(cbar, SC, 16, parity, cr, y, ya);
#ifdef SMI_TIMING
            t_wait += clock64() - tw0;
#endif
            const float *pt = sm + ((y - ya) % S) * Lay::SLOT;
            const float *rt = pt + Lay::R_OFF;
            const float *rt1 = sm + ((y + 1 - ya) % S) * Lay::SLOT + Lay::R_OFF;
            put(q[((2 * N - 1) + kq) % (2 * N)], lds4(sm + ((y + N - ya) % S) * Lay::SLOT + Lay::P_OFF + own));
            const float *cslot = cbase + ((y - ya) % SC) * Lay::CSLOT;   // this plane's core slot
            const float *cs = cslot + txi * TZ + 4 * tzi;
            bool keep[4];
            if (MODE == REC) {
                const bool kxy = in_range(ox, it.plo[1], it.phi[1]) && in_range(y, it.plo[2], it.phi[2]);
#pragma unroll
                for (int r = 0; r < 4; r++) keep[r] = kxy && in_range(oz + r, it.plo[0], it.phi[0]);
            }
            const bool act = mem && mx && my;
            float rho0[4];
            put(rho0, lds4(rt + txi * 36 + 4 * tzi));
            float4 nzv, nxv, nyv;

            // ---- z component ----
            {
                float W[12];
                {
                    const float *row = pt + Lay::P_OFF + (txi + N - 1) * ZW + 4 * tzi;
                    float4 a0 = lds4(row), a1 = lds4(row + 4), a2 = lds4(row + 8);
                    W[0] = a0.x; W[1] = a0.y; W[2] = a0.z; W[3] = a0.w;
                    W[4] = a1.x; W[5] = a1.y; W[6] = a1.z; W[7] = a1.w;
                    W[8] = a2.x; W[9] = a2.y; W[10] = a2.z; W[11] = a2.w;
                }
                if (MODE == ADJ && CLS == BND && zb && (oz - 4 < g.nb || oz + 7 >= g.ne[0] - g.nb - 1)) {
                    // transposed CPML operand over the window: lp + Ap (lp + phi) (Ap = 0 off the slab)
                    const float *ph = cslot + Lay::E_PZ + (txi + N - 1) * ZW + 4 * tzi;
#pragma unroll
                    for (int i = 0; i < 12; i++) W[i] += tb.z[0][oz - z0 + 4 + i] * (W[i] + ph[i]);
                }
                const float r4 = rt[txi * 36 + 4 * tzi + 4];
                const float rz[5] = {rho0[0], rho0[1], rho0[2], rho0[3], r4};
                float v[4];
                put(v, lds4(cs));
                float D[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[0][l - 1] * (W[4 + r + l] - W[4 + r - l + 1]);
                    D[r] = d;
                }
                if (CLS == BND && zb && zquad_slab(g, oz) && act) {
                    // z memory variable at the quad's slab nodes: forward psi <- Bv psi + Av D (added to D);
                    // adjoint chi <- Bv (chi + lv before this step)
                    float mz4[4];
                    put(mz4, lds4(cs + Lay::E_CZ));
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const int t = oz - z0 + 8 + r;
                        if (!(mz[r] && slab_at(g, 0, oz + r))) continue;
                        if (MODE == FWD) {
                            mz4[r] = tb.z[3][t] * mz4[r] + tb.z[2][t] * D[r];
                            D[r] += mz4[r];
                        } else {
                            mz4[r] = tb.z[3][t] * (mz4[r] + v[r]);
                        }
                    }
                    stg4(f.psip[0] + sh + gidx(g, oz, ox, y), mz4);
                }
                float nv[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float bz = buoy(rz[r], rz[r + 1], oz + r + 1 >= g.ne[0]);
                    if (MODE == REC) {
                        const bool rr = mz[r] && in_range(oz + r, g.L[0] + N - 1, g.H[0] - N);
                        nv[r] = rr ? (keep[r] ? v[r] + dt * bz * D[r] : 0.f) : v[r];
                    } else {
                        nv[r] = mz[r] ? v[r] - dt * bz * D[r] : v[r];
                    }
                }
                nzv = make_float4(nv[0], nv[1], nv[2], nv[3]);
            }
            // ---- x component ----
            {
                float Xr[2 * N][4];
#pragma unroll
                for (int l = 1; l <= N; l++) {
                    put(Xr[N - 1 + l], lds4(pt + Lay::P_OFF + (txi + N - 1 + l) * ZW + 4 * tzi + 4));
                    put(Xr[N - l], lds4(pt + Lay::P_OFF + (txi + N - l) * ZW + 4 * tzi + 4));
                }
                if (MODE == ADJ && CLS == BND && xb) {
                    // transposed CPML operand at the taps x - N + 1 + t (Ap = 0 off the slab)
#pragma unroll
                    for (int t = 0; t < 2 * N; t++) {
                        const float A = tb.x[0][txi + t - N + 1 + 8];
                        if (A != 0.f) {
                            float ph[4];
                            put(ph, lds4(cslot + Lay::E_PX + (txi + t) * ZW + 4 * tzi + 4));
#pragma unroll
                            for (int r = 0; r < 4; r++) Xr[t][r] += A * (Xr[t][r] + ph[r]);
                        }
                    }
                }
                float rx[4], v[4];
                put(rx, lds4(rt + (txi + 1) * 36 + 4 * tzi));
                put(v, lds4(cs + CORE));
                float D[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[1][l - 1] * (Xr[N - 1 + l][r] - Xr[N - l][r]);
                    D[r] = d;
                }
                if (CLS == BND && xb && ox < g.ne[1] && slab_at(g, 1, ox) && act) {
                    float mx4[4];
                    put(mx4, lds4(cs + Lay::E_CX));
                    const int t = txi + 8;
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        if (!mz[r]) continue;
                        if (MODE == FWD) {
                            mx4[r] = tb.x[3][t] * mx4[r] + tb.x[2][t] * D[r];
                            D[r] += mx4[r];
                        } else {
                            mx4[r] = tb.x[3][t] * (mx4[r] + v[r]);
                        }
                    }
                    stg4(f.psip[1] + sh + gidx(g, oz, ox, y), mx4);
                }
                const bool lastx = ox + 1 >= g.ne[1];
                const bool rxm = MODE == REC && in_range(ox, g.L[1] + N - 1, g.H[1] - N);
                float nv[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float bx = buoy(rho0[r], rx[r], lastx);
                    if (MODE == REC) nv[r] = (mz[r] && rxm) ? (keep[r] ? v[r] + dt * bx * D[r] : 0.f) : v[r];
                    else nv[r] = mz[r] ? v[r] - dt * bx * D[r] : v[r];
                }
                nxv = make_float4(nv[0], nv[1], nv[2], nv[3]);
            }
            // ---- y component ----
            {
                if (yent) {                       // entering plane: lp + Ap_y (lp + phi_y)
                    const float A = g.cpa[2][ye];
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        float &e = q[((2 * N - 1) + kq) % (2 * N)][r];
                        e += A * (e + yp[r]);
                    }
                }
                float ry[4], v[4];
                put(ry, lds4(rt1 + txi * 36 + 4 * tzi));
                put(v, lds4(cs + 2 * CORE));
                float D[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[2][l - 1] * (q[((N - 1 + l) + kq) % (2 * N)][r] - q[((N - l) + kq) % (2 * N)][r]);
                    D[r] = d;
                }
                if (ysl) {
                    const long long yo = yslab_off(g, s, oz, ox, y);
                    if (MODE == FWD) {            // psi_y <- Bv psi_y + Av D_y p;  v_y -= dt b (D_y p + psi_y)
                        const float B = g.cvb[2][y], A = g.cva[2][y];
#pragma unroll
                        for (int r = 0; r < 4; r++) {
                            const float ps = B * ym[r] + A * D[r];
                            if (mz[r]) {
                                ym[r] = ps;
                                D[r] += ps;
                            }
                        }
                    } else {                      // deferred chi_y <- Bv (chi_y + lv_y), lv_y before this step
                        const float B = g.cvb[2][y];
#pragma unroll
                        for (int r = 0; r < 4; r++)
                            if (mz[r]) ym[r] = B * (ym[r] + v[r]);
                    }
                    stg4(f.psip[2] + yo, ym);
                }
                const bool lasty = y + 1 >= g.ne[2];
                const bool rym = MODE == REC && in_range(y, g.L[2] + N - 1, g.H[2] - N);
                float nv[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float by = buoy(rho0[r], ry[r], lasty);
                    if (MODE == REC) nv[r] = (mz[r] && rym) ? (keep[r] ? v[r] + dt * by * D[r] : 0.f) : v[r];
                    else nv[r] = mz[r] ? v[r] - dt * by * D[r] : v[r];
                }
                nyv = make_float4(nv[0], nv[1], nv[2], nv[3]);
            }
            if (act) {
                const long long base = sh + gidx(g, oz, ox, y);
                *reinterpret_cast<float4 *>(f.v[0] + base) = nzv;
                *reinterpret_cast<float4 *>(f.v[1] + base) = nxv;
                *reinterpret_cast<float4 *>(f.v[2] + base) = nyv;
            }
            // all reads of plane y's slots are done; refill them
#ifdef SMI_TIMING
            const long long ts0 = clock64();
            n_planes++;
#endif
            if (__syncthreads_or(!ok)) {
                stop = true;
                return;
            }
#ifdef SMI_TIMING
            t_sync += clock64() - ts0;
#endif
            if (tid == 0) {
                if (hr.issued < ylast) {
                    const int yn = hr.issued + 1;
                    const int k = (yn - ya) % S;
                    float *slot = sm + k * Lay::SLOT;
                    mbar_expect(&bar[k], Lay::BYTES);
                    tma4(slot + Lay::P_OFF, &tm_p, z0 - 4, x0 - N + 1, yn, s, &bar[k]);
                    tma4(slot + Lay::R_OFF, &tm_rho, z0, x0, yn, 0, &bar[k]);
                }
                if (cr.issued < yb) issue_core(cr.issued + 1);
            }
            if (hr.issued < ylast) hr.issued++;
            if (cr.issued < yb) cr.issued++;
        };
        constexpr int G = (2 * N) % SMI_YUNROLL == 0 ? SMI_YUNROLL : 2 * N;
        while (y <= yb && !stop) {
            Unroll<0, G>::run(body, y, yb, stop);
            rotate_queue<G>(q);
        }
        if (stop) goto timeout;
        }
        continue;
    timeout:
        if (tid == 0) atomicOr(err, 1u);
        ring_drain(bar, S, 0, parity, hr, ya);
        ring_drain(cbar, SC, 16, parity, cr, ya);
        return;
    }
#ifdef SMI_TIMING
    if (threadIdx.x == 0 && (blockIdx.x % 97) == 0 && n_planes > 0)
        printf("T%d blk %d planes %lld all %lld wait %lld (%.0f%%) sync %lld (%.0f%%)\n", MODE, blockIdx.x, n_planes,
               clock64() - t_all, t_wait, 100.0 * t_wait / (clock64() - t_all), t_sync, 100.0 * t_sync / (clock64() - t_all));
#endif
}

// ===========================================================================
// Pressure kernel.  FWD/ADJ: p -= dt kappa sum_a D_a v_a (+ CPML terms);
// REC: acc += lp * (div v | p), p += dt kappa div v - source, zero outside the
// previous box, on the physical domain.
template <int N, int MODE, int CLS>
__global__ void __launch_bounds__(NTHR, CLS == BND ? 3 : SMI_MINB)
k3_p(const __grid_constant__ CUtensorMap tm_vz, const __grid_constant__ CUtensorMap tm_vx,
     const __grid_constant__ CUtensorMap tm_vy, const __grid_constant__ CUtensorMap tm_pc,
     const __grid_constant__ CUtensorMap tm_K, const __grid_constant__ CUtensorMap tm_lp,
     const __grid_constant__ CUtensorMap tm_czh, const __grid_constant__ CUtensorMap tm_cxh,
     const __grid_constant__ CUtensorMap tm_pzc, const __grid_constant__ CUtensorMap tm_pxc, Grid g, Batch b,
     Fields f, int step, unsigned *err, float *acc, int img_mode, const float *stf, float src_scale)
{
    using Lay = PLay<N, CLS>;
    constexpr int S = Lay::S;
    constexpr int SC = Lay::NC;
    constexpr unsigned CBYTES = (MODE == REC ? 3u : 2u) * CORE * 4u;
    extern __shared__ __align__(128) float sm[];
    float *cbase = sm + S * Lay::SLOT;
    __shared__ __align__(8) uint64_t bar[S], cbar[SC];
    __shared__ FTabs tb;
    const int tid = threadIdx.x, tzi = tid & 7, txi = tid >> 3;
    if (tid == 0) {
        for (int k = 0; k < S; k++) mbar_init(&bar[k], 1);
        for (int k = 0; k < SC; k++) mbar_init(&cbar[k], 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned parity = 0;
    const float dt = g.dt;
#ifdef SMI_TIMING
    long long t_wait = 0, t_sync = 0, t_all = clock64(), n_planes = 0;
#endif

    Item it;
    for (long long w = blockIdx.x;
         CLS == ALLT ? get_item(g, b, MODE, step, w, it) : get_citem(g, b, MODE, step, CLS == BND, w, it);
         w += gridDim.x) {
        const int s = it.s, z0 = it.z0, x0 = it.x0, ya = it.ya, yb = it.yb;
        const int ylast = yb + N - 1;
        const bool zb = CLS == BND && band_z(g, z0), xb = CLS == BND && band_x(g, x0);
        if (CLS == BND) load_tabs(g, z0, x0, tb);   // published by the barrier after the first waits
        // band extras of a core slot (adjoint: the chi tiles in the v_z / v_x geometries too)
        const unsigned cbytes = CBYTES + (zb ? CORE * 4u + (MODE == ADJ ? ZW * TX * 4u : 0u) : 0u) +
                                (xb ? CORE * 4u + (MODE == ADJ ? TZ * Lay::XR * 4u : 0u) : 0u);
        auto issue_core = [&](int yy) {
            const int k = (yy - ya) % SC;
            float *cs = cbase + k * Lay::CSLOT;
            mbar_expect(&cbar[k], cbytes);
            tma4(cs, &tm_pc, z0, x0, yy, s, &cbar[k]);
            tma4(cs + CORE, &tm_K, z0, x0, yy, 0, &cbar[k]);
            if (MODE == REC) tma4(cs + 2 * CORE, &tm_lp, z0, x0, yy, s, &cbar[k]);
            if (CLS == BND) {
                if (zb) {
                    if (MODE == ADJ) tma4(cs + Lay::E_HZ, &tm_czh, z0 - 4, x0, yy, s, &cbar[k]);
                    tma4(cs + Lay::E_CZ, &tm_pzc, z0, x0, yy, s, &cbar[k]);
                }
                if (xb) {
                    if (MODE == ADJ) tma4(cs + Lay::E_HX, &tm_cxh, z0, x0 - N, yy, s, &cbar[k]);
                    tma4(cs + Lay::E_CX, &tm_pxc, z0, x0, yy, s, &cbar[k]);
                }
            }
        };
        const int oz = z0 + 4 * tzi, ox = x0 + txi;
        const bool mem = oz < g.ne[0] && ox < g.ne[1];
        const long long sh = (long long)s * g.ntot;
        bool mz[4];
#pragma unroll
        for (int r = 0; r < 4; r++) mz[r] = in_range(oz + r, it.lo[0], it.hi[0]);
        const bool mx = in_range(ox, it.lo[1], it.hi[1]);
        const int own = txi * TZ + 4 * tzi;           // own nodes in a core tile
        // REC: whether the source stencil reaches this item's tile column and
        // y range (the per-node test runs only then)
        bool src_col = false;
        if (MODE == REC) {
            const Stencil &st = b.src[s];
            src_col = st.first[0] <= z0 + TZ - 1 && st.first[0] + st.cnt[0] - 1 >= z0 && st.first[1] <= x0 + TX - 1 &&
                      st.first[1] + st.cnt[1] - 1 >= x0 && st.first[2] <= yb && st.first[2] + st.cnt[2] - 1 >= ya;
        }

        // y queue of own vy: entry l = plane y-N+l; planes before ya by plain loads
        float q[2 * N][4];
#pragma unroll
        for (int l = 0; l < N; l++) {
            const int y = ya - N + l;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mem && y >= 0 && y < g.ne[2]) v = *reinterpret_cast<const float4 *>(f.v[2] + sh + gidx(g, oz, ox, y));
            put(q[l], v);
        }
        Ring hr{ya, min(ylast, ya + S - 1)}, cr{ya, min(yb, ya + SC - 1)};
        if (tid == 0) {
            for (int y = ya; y <= hr.issued; y++) {
                const int k = (y - ya) % S;
                float *slot = sm + k * Lay::SLOT;
                mbar_expect(&bar[k], Lay::BYTES);
                tma4(slot + Lay::Z_OFF, &tm_vz, z0 - 4, x0, y, s, &bar[k]);
                tma4(slot + Lay::X_OFF, &tm_vx, z0, x0 - N, y, s, &bar[k]);
                tma4(slot + Lay::Y_OFF, &tm_vy, z0, x0, y, s, &bar[k]);
            }
            for (int y = ya; y <= cr.issued; y++) issue_core(y);
        }
        bool ok = true;
#pragma unroll
        for (int l = 0; l < N - 1; l++) {
            ok &= ring_wait(bar, S, 0, parity, hr, ya + l, ya);
            put(q[N + l], lds4(sm + (l % S) * Lay::SLOT + Lay::Y_OFF + own));
        }
        if (MODE == ADJ && mem && mx) {
            // transposed y CPML: the queue holds lv_y + Av_y (lv_y + chi_y) on y-slab planes
#pragma unroll
            for (int l = 0; l < 2 * N - 1; l++) {
                const int yq = ya - N + l;
                if (yq < 0 || yq >= g.ne[2] || !yslab(g, yq)) continue;
                float ch[4];
                put(ch, ldg4(f.psip[2] + yslab_off(g, s, oz, ox, yq)));
                const float A = g.cva[2][yq];
#pragma unroll
                for (int r = 0; r < 4; r++) q[l][r] += A * (q[l][r] + ch[r]);
            }
        }
        // ADJ: nodes whose phi_y update the z / x CPML kernel makes (it reads
        // lp before that kernel changes it): the adjoint z and x bands
        bool zxb[4];
#pragma unroll
        for (int r = 0; r < 4; r++)
            zxb[r] = CLS == ALLT && (oz + r < g.nb + N || oz + r >= g.ne[0] - g.nb - N - 1 || ox < g.nb + N ||
                                     ox >= g.ne[1] - g.nb - N - 1);
        if (__syncthreads_or(!ok)) goto timeout;

        {
        bool stop = false;
        int y = ya;
        auto body = [&](auto kc) {
            constexpr int kq = decltype(kc)::value;
            // accumulator of this plane (REC), loaded before the waits
            float accv[4] = {0.f, 0.f, 0.f, 0.f};
            long long accb = 0;
            bool acc4 = false;                   // the quad as one aligned 16-byte access
            if (MODE == REC && mem && mx && in_range(y, it.lo[2], it.hi[2])) {
                const long long n0 = g.H[0] - g.L[0] + 1, n1 = g.H[1] - g.L[1] + 1;
                accb = (long long)s * g.nphys + (long long)(oz - g.L[0]) +
                       n0 * ((long long)(ox - g.L[1]) + n1 * (long long)(y - g.L[2]));
                acc4 = mz[0] && mz[1] && mz[2] && mz[3] && (accb & 3) == 0;
                if (acc4) {
                    put(accv, *reinterpret_cast<const float4 *>(acc + accb));
                } else {
#pragma unroll
                    for (int r = 0; r < 4; r++)
                        if (mz[r]) accv[r] = acc[accb + r];
                }
            }
#ifdef SMI_TIMING
            const long long tw0 = clock64();
#endif
            // y CPML operands, loaded before the waits: FWD psi_vy, ADJ phi_y
            // of plane y; ADJ chi_y of the plane entering the queue
            const bool my = in_range(y, it.lo[2], it.hi[2]);
            const bool ysl = MODE != REC && mem && mx && my && yslab(g, y);
            const int ye = y + N - 1;
            const bool yent = MODE == ADJ && mem && mx && ye < g.ne[2] && yslab(g, ye);
            float ym[4] = {0.f, 0.f, 0.f, 0.f}, yc[4] = {0.f, 0.f, 0.f, 0.f};
            if (ysl) put(ym, ldg4(f.psiv[2] + yslab_off(g, s, oz, ox, y)));
            if (yent) put(yc, ldg4(f.psip[2] + yslab_off(g, s, oz, ox, ye)));
            ok = ring_wait(bar, S, 0, parity, hr, y + N - 1, ya);
            ok &= ring_wait(cbar, SC, 16, parity, cr, y, ya);
#ifdef SMI_TIMING
            t_wait += clock64() - tw0;
#endif
            put(q[((2 * N - 1) + kq) % (2 * N)], lds4(sm + ((y + N - 1 - ya) % S) * Lay::SLOT + Lay::Y_OFF + own));
            const float *slot = sm + ((y - ya) % S) * Lay::SLOT;
            const float *cslot = cbase + ((y - ya) % SC) * Lay::CSLOT;   // this plane's core slot
            const float *cs = cslot + own;
            const bool act = mem && mx && my;
            float pv[4], Kv[4];
            put(pv, lds4(cs));
            put(Kv, lds4(cs + CORE));
            float div[4];
            const bool bact = CLS == BND && act;     // band tile, quad column inside the box
            // ---- z ----
            {
                float W[12];
                {
                    const float *row = slot + Lay::Z_OFF + txi * ZW + 4 * tzi;
                    float4 a0 = lds4(row), a1 = lds4(row + 4), a2 = lds4(row + 8);
                    W[0] = a0.x; W[1] = a0.y; W[2] = a0.z; W[3] = a0.w;
                    W[4] = a1.x; W[5] = a1.y; W[6] = a1.z; W[7] = a1.w;
                    W[8] = a2.x; W[9] = a2.y; W[10] = a2.z; W[11] = a2.w;
                }
                if (MODE == ADJ && CLS == BND && zb && (oz - 4 < g.nb || oz + 7 >= g.ne[0] - g.nb - 1)) {
                    // transposed CPML operand over the v_z window: lv + Av (lv + chi) (Av = 0 off the slab)
                    const float *ch = cslot + Lay::E_HZ + txi * ZW + 4 * tzi;
#pragma unroll
                    for (int i = 0; i < 12; i++) W[i] += tb.z[2][oz - z0 + 4 + i] * (W[i] + ch[i]);
                }
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[0][l - 1] * (W[4 + r + l - 1] - W[4 + r - l]);
                    div[r] = d;
                }
                if (bact && zb && zquad_slab(g, oz)) {
                    // z memory variable at the quad's slab nodes: forward psi <- Bp psi + Ap D (added);
                    // adjoint phi <- Bp (phi + lp before this step)
                    float mz4[4];
                    put(mz4, lds4(cslot + Lay::E_CZ + own));
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const int t = oz - z0 + 8 + r;
                        if (!(mz[r] && slab_at(g, 0, oz + r))) continue;
                        if (MODE == FWD) {
                            mz4[r] = tb.z[1][t] * mz4[r] + tb.z[0][t] * div[r];
                            div[r] += mz4[r];
                        } else {
                            mz4[r] = tb.z[1][t] * (mz4[r] + pv[r]);
                        }
                    }
                    stg4(f.psiv[0] + sh + gidx(g, oz, ox, y), mz4);
                }
            }
            // ---- x ----
            {
                float Xr[2 * N][4];
#pragma unroll
                for (int l = 1; l <= N; l++) {
                    put(Xr[N + l - 1], lds4(slot + Lay::X_OFF + (txi + N + l - 1) * TZ + 4 * tzi));
                    put(Xr[N - l], lds4(slot + Lay::X_OFF + (txi + N - l) * TZ + 4 * tzi));
                }
                if (MODE == ADJ && CLS == BND && xb) {
                    // transposed CPML operand at the taps x - N + t (Av = 0 off the slab)
#pragma unroll
                    for (int t = 0; t < 2 * N; t++) {
                        const float A = tb.x[2][txi + t - N + 8];
                        if (A != 0.f) {
                            float ch[4];
                            put(ch, lds4(cslot + Lay::E_HX + (txi + t) * TZ + 4 * tzi));
#pragma unroll
                            for (int r = 0; r < 4; r++) Xr[t][r] += A * (Xr[t][r] + ch[r]);
                        }
                    }
                }
                float D[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[1][l - 1] * (Xr[N + l - 1][r] - Xr[N - l][r]);
                    D[r] = d;
                }
                if (bact && xb && ox < g.ne[1] && slab_at(g, 1, ox)) {
                    float mx4[4];
                    put(mx4, lds4(cslot + Lay::E_CX + own));
                    const int t = txi + 8;
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        if (!mz[r]) continue;
                        if (MODE == FWD) {
                            mx4[r] = tb.x[1][t] * mx4[r] + tb.x[0][t] * D[r];
                            D[r] += mx4[r];
                        } else {
                            mx4[r] = tb.x[1][t] * (mx4[r] + pv[r]);
                        }
                    }
                    stg4(f.psiv[1] + sh + gidx(g, oz, ox, y), mx4);
                }
#pragma unroll
                for (int r = 0; r < 4; r++) div[r] += D[r];
            }
            // ---- y ----
            {
                if (yent) {                       // entering plane: lv_y + Av_y (lv_y + chi_y)
                    const float A = g.cva[2][ye];
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        float &e = q[((2 * N - 1) + kq) % (2 * N)][r];
                        e += A * (e + yc[r]);
                    }
                }
                float D[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float d = 0.f;
#pragma unroll
                    for (int l = 1; l <= N; l++) d += g.c[2][l - 1] * (q[((N + l - 1) + kq) % (2 * N)][r] - q[((N - l) + kq) % (2 * N)][r]);
                    D[r] = d;
                }
                if (ysl) {
                    if (MODE == FWD) {            // psi_vy <- Bp psi_vy + Ap D_y v_y, added to div v
                        const float B = g.cpb[2][y], A = g.cpa[2][y];
#pragma unroll
                        for (int r = 0; r < 4; r++) {
                            const float ps = B * ym[r] + A * D[r];
                            if (mz[r]) {
                                ym[r] = ps;
                                D[r] += ps;
                            }
                        }
                    } else {                      // phi_y <- Bp (phi_y + lp), lp before this step
                        const float B = g.cpb[2][y];
#pragma unroll
                        for (int r = 0; r < 4; r++)
                            if (mz[r] && !zxb[r]) ym[r] = B * (ym[r] + pv[r]);
                    }
                    stg4(f.psiv[2] + yslab_off(g, s, oz, ox, y), ym);
                }
#pragma unroll
                for (int r = 0; r < 4; r++) div[r] += D[r];
            }
            if (act) {
                float np[4];
                if (MODE == REC) {
                    const Stencil &st = b.src[s];
                    float lpv[4];
                    put(lpv, lds4(cs + 2 * CORE));
                    const bool kxy = in_range(ox, it.plo[1], it.phi[1]) && in_range(y, it.plo[2], it.phi[2]);
                    float na[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) na[r] = accv[r] + lpv[r] * (img_mode == 0 ? div[r] : pv[r]);
                    if (acc4) *reinterpret_cast<float4 *>(acc + accb) = make_float4(na[0], na[1], na[2], na[3]);
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const int z = oz + r;
                        np[r] = pv[r];
                        if (!mz[r]) continue;
                        if (!acc4) acc[accb + r] = na[r];
                        if (img_mode == 2) acc[(long long)b.nshot * g.nphys + accb + r] += pv[r] * pv[r];   // illumination
                        float pn = pv[r] + dt * Kv[r] * div[r];
                        if (src_col) {           // the source stencil reaches this tile column
                            const int t0 = z - st.first[0], t1 = ox - st.first[1], t2 = y - st.first[2];
                            if (t0 >= 0 && t0 < st.cnt[0] && t1 >= 0 && t1 < st.cnt[1] && t2 >= 0 && t2 < st.cnt[2])
                                pn -= src_scale * stf[step] * st.w[0][t0] * st.w[1][t1] * st.w[2][t2];
                        }
                        np[r] = (kxy && in_range(z, it.plo[0], it.phi[0])) ? pn : 0.f;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 4; r++) np[r] = mz[r] ? pv[r] - dt * Kv[r] * div[r] : pv[r];
                }
                *reinterpret_cast<float4 *>(f.p + sh + gidx(g, oz, ox, y)) = make_float4(np[0], np[1], np[2], np[3]);
            }
#ifdef SMI_TIMING
            const long long ts0 = clock64();
            n_planes++;
#endif
            if (__syncthreads_or(!ok)) {
                stop = true;
                return;
            }
#ifdef SMI_TIMING
            t_sync += clock64() - ts0;
#endif
            if (tid == 0) {
                if (hr.issued < ylast) {
                    const int yn = hr.issued + 1;
                    const int k = (yn - ya) % S;
                    float *sl = sm + k * Lay::SLOT;
                    mbar_expect(&bar[k], Lay::BYTES);
                    tma4(sl + Lay::Z_OFF, &tm_vz, z0 - 4, x0, yn, s, &bar[k]);
                    tma4(sl + Lay::X_OFF, &tm_vx, z0, x0 - N, yn, s, &bar[k]);
                    tma4(sl + Lay::Y_OFF, &tm_vy, z0, x0, yn, s, &bar[k]);
                }
                if (cr.issued < yb) issue_core(cr.issued + 1);
            }
            if (hr.issued < ylast) hr.issued++;
            if (cr.issued < yb) cr.issued++;
        };
        constexpr int G = (2 * N) % SMI_YUNROLL == 0 ? SMI_YUNROLL : 2 * N;
        while (y <= yb && !stop) {
            Unroll<0, G>::run(body, y, yb, stop);
            rotate_queue<G>(q);
        }
        if (stop) goto timeout;
        }
        continue;
    timeout:
        if (tid == 0) atomicOr(err, 1u);
        ring_drain(bar, S, 0, parity, hr, ya);
        ring_drain(cbar, SC, 16, parity, cr, ya);
        return;
    }
#ifdef SMI_TIMING
    if (threadIdx.x == 0 && (blockIdx.x % 97) == 0 && n_planes > 0)
        printf("T%d blk %d planes %lld all %lld wait %lld (%.0f%%) sync %lld (%.0f%%)\n", MODE, blockIdx.x, n_planes,
               clock64() - t_all, t_wait, 100.0 * t_wait / (clock64() - t_all), t_sync, 100.0 * t_sync / (clock64() - t_all));
#endif
}

// Give-up path of the bounded waits: one warp waits, with the tile kernels'
// own wait helper, on an mbarrier that nothing completes; when the polls run
// out it records the give-up in err like a tile kernel does, and returns.
__global__ void k_wait_check(unsigned *err, long long polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, polls);
    if (!ok && threadIdx.x == 0) atomicOr(err, 1u);
}

}  // namespace s3


// ---------------------------------------------------------------------------
// Host side: tensor maps and launches.

namespace {

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder()
{
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 4D map (z, x, y, shot) over a padded field array with a box of bz x bx x 1 x 1.
bool make_map(CUtensorMap *tm, const Grid &g, const float *base, int nshot, int bz, int bx)
{
    EncodeFn fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g.ne[0], (cuuint64_t)g.ne[1], (cuuint64_t)g.ne[2], (cuuint64_t)nshot};
    cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.px * g.ne[1] * 4,
                             (cuuint64_t)g.px * g.ne[1] * g.ne[2] * 4};
    cuuint32_t box[4] = {(cuuint32_t)bz, (cuuint32_t)bx, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <class K> int grid_for(K kernel, int smem)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int per = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, s3::NTHR, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, per) * std::max(1, sms);
}

template <int N, int MODE, int CLS>
void run_v(const LaunchCtx &lc, const Maps3 &m, const Grid &g, const Batch &b, Fields f, int step, unsigned *err)
{
    constexpr int smem = s3::VLay<N, CLS>::SMEM;
    static const int grid = grid_for(s3::k3_v<N, MODE, CLS>, smem);
    s3::k3_v<N, MODE, CLS><<<grid, s3::NTHR, smem, static_cast<cudaStream_t>(lc.stream)>>>(
        m.p_halo, m.rho_v, m.vz_core, m.vx_core, m.vy_core, m.pz_halo, m.px_halo, m.cz_core, m.cx_core, g, b, f,
        step, err);
    ++*lc.launches;
}

template <int N, int MODE, int CLS>
void run_p(const LaunchCtx &lc, const Maps3 &m, const Maps3 *lpm, const Grid &g, const Batch &b, Fields f, int step,
           unsigned *err, float *acc, int img_mode, const float *stf, float src_scale)
{
    constexpr int smem = s3::PLay<N, CLS>::SMEM;
    static const int grid = grid_for(s3::k3_p<N, MODE, CLS>, smem);
    s3::k3_p<N, MODE, CLS><<<grid, s3::NTHR, smem, static_cast<cudaStream_t>(lc.stream)>>>(
        m.vz_halo, m.vx_halo, m.vy_core, m.p_core, m.K_core, lpm ? lpm->p_core : m.p_core, m.cz_vhalo, m.cx_vhalo,
        m.pz_core, m.px_core, g, b, f, step, err, acc, img_mode, stf, src_scale);
    ++*lc.launches;
}

// One forward / adjoint stencil half-step: every tile column in one launch
// (inl = false: the z / x CPML terms come from the band kernels), or the
// interior columns and then the CPML-band columns with the terms inline.
// The two classes update disjoint nodes and, within a half-step, read only
// what the other does not write.
template <int N, int MODE>
void run_v_cls(const LaunchCtx &lc, const Maps3 &m, const Grid &g, const Batch &b, Fields f, int step,
               unsigned *err, bool inl)
{
    if (!inl) {
        run_v<N, MODE, s3::ALLT>(lc, m, g, b, f, step, err);
        return;
    }
    run_v<N, MODE, s3::BND>(lc, m, g, b, f, step, err);
    run_v<N, MODE, s3::INT>(lc, m, g, b, f, step, err);
}

template <int N, int MODE>
void run_p_cls(const LaunchCtx &lc, const Maps3 &m, const Maps3 *lpm, const Grid &g, const Batch &b, Fields f,
               int step, unsigned *err, float *acc, int img_mode, const float *stf, float src_scale, bool inl)
{
    if (!inl) {
        run_p<N, MODE, s3::ALLT>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale);
        return;
    }
    run_p<N, MODE, s3::BND>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale);
    run_p<N, MODE, s3::INT>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale);
}

}  // namespace

bool make_tile_map(CUtensorMap *tm, const Grid &g, const float *base, int nshot, int bz, int bx)
{
    return make_map(tm, g, base, nshot, bz, bx);
}

// The 3D path indexes one shot's arrays with 32-bit offsets.
void launch_wait_check(const LaunchCtx &lc, unsigned *err, long long polls)
{
    s3::k_wait_check<<<1, 32, 0, static_cast<cudaStream_t>(lc.stream)>>>(err, polls);
    ++*lc.launches;
}

long long wait_polls_default() { return s3::kSpin; }

bool stencil3d_supported(const Grid &g)
{
    return g.ndim == 3 && (g.N == 2 || g.N == 4) && g.ntot < (1LL << 31) && encoder() != nullptr;
}

bool make_maps3(Maps3 &m, const Grid &g, const Fields &f, int nshot, bool fullmem)
{
    const int R = s3::TX + 2 * g.N - 1;
    bool ok = make_map(&m.p_halo, g, f.p, nshot, s3::ZW, R) && make_map(&m.p_core, g, f.p, nshot, s3::TZ, s3::TX) &&
              make_map(&m.vz_core, g, f.v[0], nshot, s3::TZ, s3::TX) &&
              make_map(&m.vx_core, g, f.v[1], nshot, s3::TZ, s3::TX) &&
              make_map(&m.vy_core, g, f.v[2], nshot, s3::TZ, s3::TX) &&
              make_map(&m.vz_halo, g, f.v[0], nshot, s3::ZW, s3::TX) &&
              make_map(&m.vx_halo, g, f.v[1], nshot, s3::TZ, R) &&
              make_map(&m.rho_v, g, g.rho, 1, 36, s3::TX + 1) && make_map(&m.K_core, g, g.K, 1, s3::TZ, s3::TX);
    if (!ok) return false;
    if (!fullmem) {
        // compressed CPML slabs: the band maps are never read (the band kernels apply the terms)
        m.pz_halo = m.px_halo = m.p_halo;
        m.cz_core = m.cx_core = m.pz_core = m.px_core = m.p_core;
        m.cz_vhalo = m.vz_halo;
        m.cx_vhalo = m.vx_halo;
        return true;
    }
    return make_map(&m.pz_halo, g, f.psiv[0], nshot, s3::ZW, R) && make_map(&m.px_halo, g, f.psiv[1], nshot, s3::ZW, R) &&
           make_map(&m.cz_core, g, f.psip[0], nshot, s3::TZ, s3::TX) &&
           make_map(&m.cx_core, g, f.psip[1], nshot, s3::TZ, s3::TX) &&
           make_map(&m.cz_vhalo, g, f.psip[0], nshot, s3::ZW, s3::TX) &&
           make_map(&m.cx_vhalo, g, f.psip[1], nshot, s3::TZ, R) &&
           make_map(&m.pz_core, g, f.psiv[0], nshot, s3::TZ, s3::TX) &&
           make_map(&m.px_core, g, f.psiv[1], nshot, s3::TZ, s3::TX);
}

void launch3_v(const LaunchCtx &lc, const Maps3 &m, const Grid &g, const Batch &b, Fields f, int step, int mode,
               unsigned *err, bool inl)
{
    // the adjoint's interior update is the forward scheme; only its box differs
    if (g.N == 2) {
        if (mode == 0) run_v_cls<2, 0>(lc, m, g, b, f, step, err, inl);
        else if (mode == 1) run_v_cls<2, 1>(lc, m, g, b, f, step, err, inl);
        else run_v<2, 2, s3::ALLT>(lc, m, g, b, f, step, err);
    } else {
        if (mode == 0) run_v_cls<4, 0>(lc, m, g, b, f, step, err, inl);
        else if (mode == 1) run_v_cls<4, 1>(lc, m, g, b, f, step, err, inl);
        else run_v<4, 2, s3::ALLT>(lc, m, g, b, f, step, err);
    }
}

void launch3_p(const LaunchCtx &lc, const Maps3 &m, const Maps3 *lpm, const Grid &g, const Batch &b, Fields f,
               int step, int mode, unsigned *err, float *acc, int img_mode, const float *stf, float src_scale, bool inl)
{
    if (g.N == 2) {
        if (mode == 0) run_p_cls<2, 0>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale, inl);
        else if (mode == 1) run_p_cls<2, 1>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale, inl);
        else run_p<2, 2, s3::ALLT>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale);
    } else {
        if (mode == 0) run_p_cls<4, 0>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale, inl);
        else if (mode == 1) run_p_cls<4, 1>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale, inl);
        else run_p<4, 2, s3::ALLT>(lc, m, lpm, g, b, f, step, err, acc, img_mode, stf, src_scale);
    }
}

}  // namespace smi
