// smi_tile3d.h -- device helpers shared by the TMA-streamed 3D stencil
// kernels (smi_stencil3d.cu: the two-pass velocity / pressure kernels;
// smi_fused3d.cu: the single-pass kernel): mbarrier and TMA wrappers in
// inline PTX, the work decomposition of a computing box into 32 x 16 tile
// columns times y-chunks walked by persistent CTAs, the bounded ring waits
// and the register-queue rotation.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#ifdef SMI_TIMING
#include <cstdio>
#endif

#include "smi_box.h"
#include "smi_internal.h"

namespace smi {
namespace s3 {

#ifndef SMI_TX
#define SMI_TX 16
#endif
#ifndef SMI_PFP
#define SMI_PFP 1
#endif
#ifndef SMI_MINB
#define SMI_MINB 4
#endif
#ifndef SMI_YUNROLL
#define SMI_YUNROLL 2        // y planes per unrolled group (divides 2N)
#endif
constexpr int TZ = 32, TX = SMI_TX, NTHR = 8 * TX;
constexpr int ZW = 40;                 // z extent of haloed tiles: [z0-4, z0+36)
constexpr long long kSpin = 1LL << 18; // bounded mbarrier polls: about 1 s on GB300 (a poll suspends ~3.8 us)

enum { FWD = 0, ADJ = 1, REC = 2 };

__host__ __device__ constexpr int rup32(int n) { return (n + 31) / 32 * 32; }

// --- PTX helpers ------------------------------------------------------------
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(sptr(b)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, long long polls = kSpin)
{
    for (long long i = 0; i < polls; i++)
        if (mbar_test(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma4(float *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(sptr(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(sptr(bar))
        : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void put(float (&a)[4], float4 v) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }

__device__ __forceinline__ long long gidx(const Grid &g, int i1, int i2, int i3)
{
    return (long long)i1 + (long long)g.px * ((long long)i2 + (long long)g.ne[1] * i3);
}
// y slab (Sec. 2.1 CPML): membership of plane y, and the offset of node
// (oz, ox, y) in the y-slab arrays (row pitch px, so 4 consecutive z nodes
// from a multiple of 4 form an aligned float4).
__device__ __forceinline__ bool yslab(const Grid &g, int y) { return y < g.nb || y >= g.ne[2] - g.nb - 1; }
__device__ __forceinline__ long long yslab_off(const Grid &g, int s, int oz, int ox, int y)
{
    const int js = y < g.nb ? y : y - (g.ne[2] - 2 * g.nb - 1);
    return (long long)s * g.slab_n[2] + oz + (long long)g.px * (ox + (long long)g.ne[1] * js);
}
__device__ __forceinline__ float4 ldg4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void stg4(float *p, const float (&a)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
}

// --- work decomposition ---------------------------------------------------
struct Item {
    int s, z0, x0, ya, yb;
    int lo[3], hi[3];     // update region (box, clipped per mode)
    int plo[3], phi[3];   // REC: previous-step box
};

// Box of shot s for this launch, clipped to the physical domain in REC.
__device__ __forceinline__ void item_box(const Grid &g, const Batch &b, int mode, int s, int step, int lo[3],
                                         int hi[3], int plo[3], int phi[3])
{
    if (mode == ADJ) {
        box_at(b.tab_rec, b.nt1, s, step, lo, hi);
    } else {
        box_at(b.tab_src, b.nt1, s, step, lo, hi);
    }
    if (mode == REC) {
        box_at(b.tab_src, b.nt1, s, step - 1, plo, phi);
        for (int a = 0; a < 3; a++) {
            lo[a] = max(lo[a], g.L[a]);
            hi[a] = min(hi[a], g.H[a]);
        }
    }
}

struct Decomp {
    int nzt, nxt, nyc, cy, zb;
};

// Column tiles x y-chunks of a box.  Long chunks: each chunk pays a
// pipeline start-up of about 2N planes, so a box is split into
// min(ylen / 16, grid / columns) chunks a column, one wave of the persistent
// grid.  When that wave leaves more than a tenth of the CTAs idle (the
// 340^3 box makes 242 columns for a 608-CTA grid: 2 chunks fill 80 %), the
// chunk count grows to the smallest that fills the waves to 90 % (5 there:
// 99.5 %).
__device__ __forceinline__ Decomp decomp(const int lo[3], const int hi[3], int grid)
{
    Decomp d;
    d.zb = lo[0] & ~31;
    d.nzt = hi[0] >= lo[0] ? (hi[0] - d.zb) / TZ + 1 : 0;
    d.nxt = hi[1] >= lo[1] ? (hi[1] - lo[1]) / TX + 1 : 0;
    const int ylen = hi[2] - lo[2] + 1;
    if (d.nzt == 0 || d.nxt == 0 || ylen <= 0) {
        d.nzt = d.nxt = d.nyc = 0;
        d.cy = 1;
        return d;
    }
    const long long cols = (long long)d.nzt * d.nxt;
    const int cmax = max(1, ylen / 16);
    auto fill = [&](int c) {
        const long long items = cols * c;
        return (float)items / (float)(((items + grid - 1) / grid) * grid);
    };
    int chunks = max(1, min(cmax, (int)(grid / cols)));
    if (fill(chunks) < 0.9f) {
        for (int c = chunks + 1; c <= min(cmax, 4 * chunks + 4); c++) {
            if (fill(c) >= 0.9f) {
                chunks = c;
                break;
            }
        }
    }
    d.cy = (ylen + chunks - 1) / chunks;
    d.nyc = (ylen + d.cy - 1) / d.cy;
    return d;
}

// Item w of the launch (shots in order), false past the end.
__device__ __forceinline__ bool get_item(const Grid &g, const Batch &b, int mode, int step, long long w, Item &it)
{
    const int target = (int)gridDim.x;
    for (int s = 0; s < b.nshot; s++) {
        int lo[3], hi[3], plo[3] = {0, 0, 0}, phi[3] = {-1, -1, -1};
        item_box(g, b, mode, s, step, lo, hi, plo, phi);
        const Decomp d = decomp(lo, hi, target);
        const long long n = (long long)d.nzt * d.nxt * d.nyc;
        if (w < n) {
            const int zi = (int)(w % d.nzt);
            const int xi = (int)((w / d.nzt) % d.nxt);
            const int ci = (int)(w / ((long long)d.nzt * d.nxt));
            it.s = s;
            it.z0 = d.zb + TZ * zi;
            it.x0 = lo[1] + TX * xi;
            it.ya = lo[2] + ci * d.cy;
            it.yb = min(hi[2], it.ya + d.cy - 1);
            for (int a = 0; a < 3; a++) {
                it.lo[a] = lo[a];
                it.hi[a] = hi[a];
                it.plo[a] = plo[a];
                it.phi[a] = phi[a];
            }
            return true;
        }
        w -= n;
    }
    return false;
}

__device__ __forceinline__ bool in_range(int v, int lo, int hi) { return v >= lo && v <= hi; }

// ===========================================================================
// Ring bookkeeping shared by both kernels.  All threads wait on a slot's
// mbarrier themselves (bounded); `parity` holds the phase parity of the next
// completion of every slot (bit k for haloed slot k, bit 16+k for core slot k).
struct Ring {
    int next_wait;     // next plane to wait for
    int issued;        // last plane whose copies were issued
};

__device__ __forceinline__ bool ring_wait(uint64_t *bars, int nslots, int bitbase, unsigned &parity, Ring &r,
                                          int plane, int base)
{
    const int k = (plane - base) % nslots;
    const bool ok = mbar_wait(&bars[k], (parity >> (bitbase + k)) & 1u);
    if (ok) {
        parity ^= 1u << (bitbase + k);
        r.next_wait = plane + 1;
    }
    return ok;
}

__device__ __forceinline__ void ring_drain(uint64_t *bars, int nslots, int bitbase, unsigned &parity, Ring &r,
                                           int base)
{
    for (int y = r.next_wait; y <= r.issued; y++) {
        const int k = (y - base) % nslots;
        if (mbar_wait(&bars[k], (parity >> (bitbase + k)) & 1u)) parity ^= 1u << (bitbase + k);
    }
}

// Buoyancy on a half node: 2 / (rho_i + rho_{i+1}), 1/rho at the last node
// (fast reciprocal-based division: a few ulp, far below the FP32 scheme error).
// y-loop unrolled in groups of G planes: step K of a group sees logical
// queue entry l at physical index (l + K) % 2N, so inside a group the queue
// rotates by renaming registers; rotate_queue moves it back between groups.
template <int K, int M> struct Unroll {
    template <class F> __device__ __forceinline__ static void run(F &f, int &y, int yb, const bool &stop)
    {
        if (y > yb || stop) return;
        f(std::integral_constant<int, K>{});
        ++y;
        Unroll<K + 1, M>::run(f, y, yb, stop);
    }
};
template <int M> struct Unroll<M, M> {
    template <class F> __device__ __forceinline__ static void run(F &, int &, int, const bool &) {}
};

// After a group of G planes the logical entry l sits at (l + G) % L: move
// it back to l so the next group starts at step 0 (fewer unrolled copies of
// the loop body keep the code inside the instruction cache).
template <int G, int L>
__device__ __forceinline__ void rotate_queue(float (&q)[L][4])
{
    if (G % L == 0) return;
    float t[L][4];
#pragma unroll
    for (int l = 0; l < L; l++)
#pragma unroll
        for (int r = 0; r < 4; r++) t[l][r] = q[(l + G) % L][r];
#pragma unroll
    for (int l = 0; l < L; l++)
#pragma unroll
        for (int r = 0; r < 4; r++) q[l][r] = t[l][r];
}

__device__ __forceinline__ float buoy(float r0, float r1, bool last)
{
    return last ? __fdividef(1.0f, r0) : __fdividef(2.0f, r0 + r1);
}

// CPML coefficient tables of one tile (band tiles only): [0] Ap, [1] Bp,
// [2] Av, [3] Bv along z for z0-8 .. z0+39 and along x for x0-8 .. x0+TX+7,
// zero outside the grid.
struct FTabs {
    float z[4][48];
    float x[4][TX + 16];
};

__device__ __forceinline__ bool slab_at(const Grid &g, int a, int j)
{
    return j < g.nb || j >= g.ne[a] - g.nb - 1;
}
// Quad of z nodes z..z+3 touches the z slab.
__device__ __forceinline__ bool zquad_slab(const Grid &g, int z)
{
    return z < g.nb || z + 3 >= g.ne[0] - g.nb - 1;
}

// Loads the CPML coefficient tables of the tile at (z0, x0) (all threads of
// the CTA; published by the caller's next barrier).
__device__ __forceinline__ void load_tabs(const Grid &g, int z0, int x0, FTabs &tb)
{
    for (int i = threadIdx.x; i < 4 * 48; i += blockDim.x) {
        const int k = i / 48, j = i % 48, zz = z0 - 8 + j;
        const float *src = k == 0 ? g.cpa[0] : k == 1 ? g.cpb[0] : k == 2 ? g.cva[0] : g.cvb[0];
        tb.z[k][j] = (zz >= 0 && zz < g.ne[0]) ? src[zz] : 0.f;
    }
    for (int i = threadIdx.x; i < 4 * (TX + 16); i += blockDim.x) {
        const int k = i / (TX + 16), j = i % (TX + 16), xx = x0 - 8 + j;
        const float *src = k == 0 ? g.cpa[1] : k == 1 ? g.cpb[1] : k == 2 ? g.cva[1] : g.cvb[1];
        tb.x[k][j] = (xx >= 0 && xx < g.ne[1]) ? src[xx] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Work of one launch: the tile columns of one class (interior: no stencil of
// the tile reaches a z or x slab; band: the others) times y-chunks of the
// box.  A column is a band column when its z window [z0-8, z0+39] or x
// window [x0-8, x0+TX+7] meets a slab; interior z tiles (and x tiles) form
// one contiguous range, so the interior columns are a rectangle.
__device__ __forceinline__ bool band_z(const Grid &g, int z0) { return z0 - 8 < g.nb || z0 + 39 >= g.ne[0] - g.nb - 1; }
__device__ __forceinline__ bool band_x(const Grid &g, int x0)
{
    return x0 - 8 < g.nb || x0 + TX + 7 >= g.ne[1] - g.nb - 1;
}

struct CDecomp {
    int zbase, nzt, nxt, iz0, iz1, ix0, ix1, ncol, nyc, cy;
};

__device__ __forceinline__ CDecomp cdecomp(const Grid &g, const int lo[3], const int hi[3], int grid, bool band)
{
    CDecomp d;
    d.zbase = lo[0] & ~31;
    const int ylen = hi[2] - lo[2] + 1;
    d.nzt = hi[0] >= lo[0] ? (hi[0] - d.zbase) / TZ + 1 : 0;
    d.nxt = hi[1] >= lo[1] ? (hi[1] - lo[1]) / TX + 1 : 0;
    d.iz0 = d.iz1 = d.ix0 = d.ix1 = 0;
    d.ncol = 0;
    d.nyc = 0;
    d.cy = 1;
    if (d.nzt == 0 || d.nxt == 0 || ylen <= 0) return d;
    d.iz0 = d.nzt;
    for (int i = 0; i < d.nzt; i++)
        if (!band_z(g, d.zbase + TZ * i)) {
            if (d.iz0 == d.nzt) d.iz0 = i;
            d.iz1 = i + 1;
        }
    if (d.iz0 == d.nzt) d.iz0 = d.iz1 = 0;
    d.ix0 = d.nxt;
    for (int i = 0; i < d.nxt; i++)
        if (!band_x(g, lo[1] + TX * i)) {
            if (d.ix0 == d.nxt) d.ix0 = i;
            d.ix1 = i + 1;
        }
    if (d.ix0 == d.nxt) d.ix0 = d.ix1 = 0;
    const int nint = (d.iz1 - d.iz0) * (d.ix1 - d.ix0);
    d.ncol = band ? d.nzt * d.nxt - nint : nint;
    if (d.ncol == 0) return d;
    // chunks along y: as many as fill the persistent grid's waves to 90 %
    const long long cols = d.ncol;
    const int cmax = max(1, ylen / 16);
    auto fill = [&](int c) {
        const long long items = cols * c;
        return (float)items / (float)(((items + grid - 1) / grid) * grid);
    };
    int chunks = max(1, min(cmax, (int)(grid / cols)));
    if (fill(chunks) < 0.9f) {
        for (int c = chunks + 1; c <= min(cmax, 4 * chunks + 4); c++) {
            if (fill(c) >= 0.9f) {
                chunks = c;
                break;
            }
        }
    }
    d.cy = (ylen + chunks - 1) / chunks;
    d.nyc = (ylen + d.cy - 1) / d.cy;
    return d;
}

// Column k (0 .. ncol-1) of the class -> tile indices (zi, xi).
__device__ __forceinline__ void class_column(const CDecomp &d, bool band, int k, int &zi, int &xi)
{
    const int nix = d.ix1 - d.ix0;
    if (!band) {
        zi = d.iz0 + k / nix;
        xi = d.ix0 + k % nix;
        return;
    }
    for (zi = 0; zi < d.nzt; zi++) {
        const bool zint = zi >= d.iz0 && zi < d.iz1;
        const int cnt = zint ? d.nxt - nix : d.nxt;
        if (k < cnt) {
            xi = (zint && k >= d.ix0) ? k - d.ix0 + d.ix1 : k;
            return;
        }
        k -= cnt;
    }
    xi = 0;
}

// Item w of a class's launch (shots in order), false past the end.
__device__ __forceinline__ bool get_citem(const Grid &g, const Batch &b, int mode, int step, bool band, long long w,
                                          Item &it)
{
    const int target = (int)gridDim.x;
    for (int s = 0; s < b.nshot; s++) {
        int lo[3], hi[3], plo[3] = {0, 0, 0}, phi[3] = {-1, -1, -1};
        item_box(g, b, mode, s, step, lo, hi, plo, phi);
        const CDecomp d = cdecomp(g, lo, hi, target, band);
        const long long n = (long long)d.ncol * d.nyc;
        if (w < n) {
            const int k = (int)(w % d.ncol), ci = (int)(w / d.ncol);
            int zi, xi;
            class_column(d, band, k, zi, xi);
            it.s = s;
            it.z0 = d.zbase + TZ * zi;
            it.x0 = lo[1] + TX * xi;
            it.ya = lo[2] + ci * d.cy;
            it.yb = min(hi[2], it.ya + d.cy - 1);
            for (int a = 0; a < 3; a++) {
                it.lo[a] = lo[a];
                it.hi[a] = hi[a];
                it.plo[a] = plo[a];
                it.phi[a] = phi[a];
            }
            return true;
        }
        w -= n;
    }
    return false;
}

}  // namespace s3
}  // namespace smi
