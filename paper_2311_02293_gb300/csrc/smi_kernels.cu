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
#ifndef SMI_CPML_U
#define SMI_CPML_U 4
#endif
#ifndef SMI_CPML_UZ
#define SMI_CPML_UZ 2        // adjoint kinds; the forward kinds take twice as many
#endif
constexpr int kCpmlChunk = SMI_CPML_U;     // nodes per thread along x, CPML kernel of the x piece
constexpr int kCpmlChunkZ = SMI_CPML_UZ;   // x lines a unit of the z-piece kernel k_cpml_zp (adjoint kinds)
constexpr int kMaxBlocksX = 152 * 16;
#ifndef SMI_CPML_ZP_MINB
#define SMI_CPML_ZP_MINB 4   // resident 256-thread blocks of k_cpml_zp (its warps loop: fewer are needed)
#endif
#ifndef SMI_CPML_XW_U
#define SMI_CPML_XW_U 4      // nodes a chunk of the walk
#endif
#ifndef SMI_CPML_XW_PARTS
#define SMI_CPML_XW_PARTS 2  // runs a band of k_cpml_xw is cut into (more lines walk at once)
#endif
#ifndef SMI_CPML_XW_MINB
#define SMI_CPML_XW_MINB 4   // resident 256-thread blocks of k_cpml_xw
#endif
#ifndef SMI_CPML_MINB_F
#define SMI_CPML_MINB_F 4
#endif

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
    return (long long)i1 + (long long)g.px * ((long long)i2 + (long long)g.ne[1] * js);
}

__device__ __forceinline__ float buoyancy(const Grid &g, int a, int ia, long long k, float rho0)
{
    // fast reciprocal-based division: a few ulp, far below the FP32 scheme error
    return (ia + 1 < g.ne[a]) ? __fdividef(2.0f, rho0 + g.rho[k + gstride(g, a)]) : __fdividef(1.0f, rho0);
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
        if (vol < (1LL << 31)) {          // 32-bit division (uniform branch)
            const int qq = (int)q, r = qq / w0;
            i[0] = lo[0] + (qq - r * w0);
            i[1] = lo[1] + r % w1;
            i[2] = lo[2] + r / w1;
            return;
        }
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
// ---------------------------------------------------------------------------
// CPML terms over the slabs only (Sec. 2.1), added to the interior update of
// the main 3D kernels, which apply the plain scheme everywhere.
//
// Forward (the CPML of Komatitsch & Martin):
//   FV: psi_a <- Bv_a psi_a + Av_a D_a p;    v_a -= dt b_a psi_a
//   FP: psi_a <- Bp_a psi_a + Ap_a D_a v_a;  p -= dt kappa sum_a psi_a
// Adjoint (transpose of one forward step; runs before the interior adjoint
// kernels; chi / phi are the adjoint memory variables, kept in the psip /
// psiv slabs):
//   AV: chi_a <- Bv_a (chi_a + lv_a);  lv_a -= dt b_a D_a[Ap_a (lp + phi_a)]
//   AP: phi_a <- Bp_a (phi_a + lp);    lp -= dt kappa sum_a D_a[Av_a (lv_a + chi_a)]
//
// Every D_a above is sum_l c_l (h(j + o + l) - h(j + o + 1 - l)) over a
// field h along axis a (o = 0 for the V kinds, -1 for the P kinds), with
// h = p, v_a, Ap_a (lp + phi_a) or Av_a (lv_a + chi_a), zero outside the
// grid (and, for the adjoint kinds, outside the slab).
//
// The main 3D kernels apply the y terms themselves (their register queue
// along y holds the operand of D_y; see smi_stencil3d.cu).  The kernels here
// cover the z and x terms over the union of the z and x bands (nodes within
// w_lo of the low end or w_hi of the high end of the axis; forward: the
// slabs; adjoint: every node whose stencil reaches a slab node), cut into
// two disjoint pieces clipped to the union of the batch's computing boxes
// (see Pieces).  Each node belongs to one thread, which applies the terms of
// both axes where both bands hold it, so the kinds that update p / lp (read
// at the node only) need no ordering between axes.  A thread takes a chunk
// of consecutive nodes along x and issues all the chunk's loads before its
// first store (these kernels are bound by memory latency, not bytes).  The
// adjoint phi_y update needs lp before the step, so the AP kernel makes it
// at its own nodes of the y slab and the main pressure kernel at the rest.
enum CpmlKind { kFV = 0, kFP = 1, kAV = 2, kAP = 3 };

__device__ __forceinline__ bool in_band(const Grid &g, const Pieces &P, int a, int j)
{
    return j < P.w_lo || j >= g.ne[a] - P.w_hi;
}

// Offsets inside one shot's arrays are 32-bit: the 3D path requires a
// field of one shot to hold fewer than 2^31 points.
__device__ __forceinline__ int gidx32(const Grid &g, int i0, int i1, int i2) { return i0 + g.px * (i1 + g.ne[1] * i2); }
__device__ __forceinline__ int gstride32(const Grid &g, int a) { return a == 0 ? 1 : (a == 1 ? g.px : g.px * g.ne[1]); }

// Offset and stride of axis a's slab index at node i with i[a] replaced.
__device__ __forceinline__ void slab_base(const Grid &g, int a, const int i[3], int &base, int &stride)
{
    if (a == 0) { base = g.S * (i[1] + g.ne[1] * i[2]); stride = 1; }
    else if (a == 1) { base = i[0] + g.ne[0] * g.S * i[2]; stride = g.ne[0]; }
    else { base = i[0] + g.px * i[1]; stride = g.px * g.ne[1]; }
}

// Arrays of kind KIND along axis A for one shot.
template <int KIND, int A>
struct CpmlAxis {
    static constexpr bool VK = KIND == kFV || KIND == kAV;
    const float *src;      // h's field: p (FV, AV) or v_a (FP, AP)
    const float *hmem;     // adjoint kinds: phi_a (AV) or chi_a (AP), the memory variable in h
    float *mem;            // memory variable updated at the node: psi / chi (V kinds), psi / phi (P kinds)
    float *fld;            // V kinds: v_a / lv_a
    int st, ne, sb, ss;    // flat stride, axis length; slab base of the line and slab stride
    __device__ __forceinline__ CpmlAxis(const Grid &g, const Fields &f, int s, const int i[3])
    {
        const long long so = (long long)s * g.ntot, ms = (long long)s * g.slab_n[A];
        src = VK ? f.p + so : f.v[A] + so;
        hmem = (KIND == kAV ? f.psiv[A] : f.psip[A]) + ms;
        mem = (VK ? f.psip[A] : f.psiv[A]) + ms;
        fld = f.v[A] + so;
        st = gstride32(g, A);
        ne = g.ne[A];
        slab_base(g, A, i, sb, ss);
    }
    __device__ __forceinline__ bool slab(const Grid &g, int j) const { return j < g.nb || j >= ne - g.nb - 1; }
    __device__ __forceinline__ int msi(const Grid &g, int j) const   // slab index of node j (j in the slab)
    {
        return sb + (j < g.nb ? j : j - (ne - 2 * g.nb - 1)) * ss;
    }
    // h at index j of the line through node k (index ia); zero where the
    // scheme has none.  Loads depend only on index arithmetic.
    __device__ __forceinline__ float h(const Grid &g, int k, int ia, int j) const
    {
        bool valid = (unsigned)j < (unsigned)ne;
        if (KIND == kAV || KIND == kAP) valid = valid && slab(g, j);
        float x = 0.0f;
        if (valid) {
            const int kk = k + (j - ia) * st;
            if (KIND == kFV || KIND == kFP) x = src[kk];
            else x = __ldg((KIND == kAV ? g.cpa[A] : g.cva[A]) + j) * (src[kk] + hmem[msi(g, j)]);
        }
        return x;
    }
};

// D_a at a node from its 2N values of h: w[t] = h(ia + o - N + 1 + t).
template <int N>
__device__ __forceinline__ float cpml_d(const Grid &g, int a, const float *w)
{
    float D = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; l++) D += g.c[a][l - 1] * (w[N - 1 + l] - w[N - l]);
    return D;
}

// Values of one axis at one node, loaded before any store of the chunk:
// mem = memory variable (if the node is in the slab), fld = v_a / lv_a (V
// kinds), rho1 = rho one node up the axis (buoyancy).
struct CpmlOwn {
    float mem, fld, rho1;
};

template <int KIND, int A>
__device__ __forceinline__ CpmlOwn cpml_own(const Grid &g, const CpmlAxis<KIND, A> &x, int ia, int k, bool sl)
{
    CpmlOwn o{0.0f, 0.0f, 0.0f};
    if (sl) o.mem = x.mem[x.msi(g, ia)];
    if (CpmlAxis<KIND, A>::VK) {
        o.fld = x.fld[k];
        if (ia + 1 < x.ne) o.rho1 = g.rho[k + x.st];
    }
    return o;
}

// Applies the axis-A terms of one node from its preloaded values; the P
// kinds add their term to acc (p / lp is written once per node).
template <int KIND, int A>
__device__ __forceinline__ void cpml_apply(const Grid &g, const CpmlAxis<KIND, A> &x, int ia, int k, bool sl,
                                           const CpmlOwn &o, float rho0, float lp0, float D, float &acc)
{
    if (KIND == kFV || KIND == kAV) {
        const float b = (ia + 1 < x.ne) ? __fdividef(2.0f, rho0 + o.rho1) : __fdividef(1.0f, rho0);
        if (KIND == kFV) {
            const float psi = g.cvb[A][ia] * o.mem + g.cva[A][ia] * D;
            x.mem[x.msi(g, ia)] = psi;
            x.fld[k] = o.fld - g.dt * b * psi;
        } else {
            if (sl) x.mem[x.msi(g, ia)] = g.cvb[A][ia] * (o.mem + o.fld);   // deferred chi update, lv before this step
            if (D != 0.0f) x.fld[k] = o.fld - g.dt * b * D;
        }
    } else if (KIND == kFP) {
        const float psi = g.cpb[A][ia] * o.mem + g.cpa[A][ia] * D;
        x.mem[x.msi(g, ia)] = psi;
        acc += psi;
    } else {
        if (sl) x.mem[x.msi(g, ia)] = g.cpb[A][ia] * (o.mem + lp0);         // phi update, lp before this step
        acc += D;
    }
}

// Band membership of index j on axis a for kind KIND (forward: the slab).
template <int KIND>
__device__ __forceinline__ bool cpml_in(const Grid &g, const Pieces &P, int a, int j)
{
    return (KIND == kFV || KIND == kFP) ? in_slab(g, a, j) : in_band(g, P, a, j);
}

__device__ __forceinline__ int iv_map(const int *iv, int c) { return c < iv[1] ? iv[0] + c : iv[2] + c - iv[1]; }

// AP only: phi_y <- Bp_y (phi_y + lp) at nodes of the y slab, with lp
// before this step (these kernels run before the main pressure kernel,
// which makes the update at the y-slab nodes outside the z and x bands).
struct CpmlPhiY {
    float *ph;             // shot's phi_y slab array at node 0 of the chunk, or null
    float B;
    int step;              // offset between consecutive nodes of the chunk
    __device__ __forceinline__ CpmlPhiY(const Grid &g, const Fields &f, int s, const int i[3], int step_)
    {
        ph = nullptr;
        B = 0.0f;
        step = step_;
        const int y = i[2];
        if (g.ndim == 3 && (y < g.nb || y >= g.ne[2] - g.nb - 1)) {
            const int js = y < g.nb ? y : y - (g.ne[2] - 2 * g.nb - 1);
            ph = f.psiv[2] + (long long)s * g.slab_n[2] + i[0] + g.px * (i[1] + g.ne[1] * js);
            B = g.cpb[2][y];
        }
    }
};

// x piece: a thread takes up to U consecutive nodes along x of one line
// (fixed z index i0 and y index i2); z is inner there, so the nodes have x
// terms only.  Phase 1 issues every load of the chunk: the window of h
// along x shared by the U nodes (U + 2N - 1 values instead of 2N per node)
// and the nodes' own values.  Phase 2 computes and stores.
template <int N, int KIND, int U>
__device__ __forceinline__ void cpml_chunk(const Grid &g, const Fields &f, const Piece &p, int s, int c0, int cr,
                                           int ch, const int lo[3], const int hi[3])
{
    constexpr int W = 1;
    constexpr bool VK = KIND == kFV || KIND == kAV;
    constexpr int O = VK ? 0 : -1;
    int i[3];
    i[0] = iv_map(p.iv[0], c0);
    i[2] = iv_map(p.iv[2], cr);
    if (i[0] < lo[0] || i[0] > hi[0] || i[2] < lo[2] || i[2] > hi[2]) return;
    const int nc0 = (p.iv[W][1] + U - 1) / U;
    const int seg = ch < nc0 ? 0 : 1;
    ch -= seg ? nc0 : 0;
    const int j0 = p.iv[W][2 * seg] + ch * U;
    const int jend = min(p.iv[W][2 * seg] + p.iv[W][2 * seg + 1] - 1, hi[W]);
    i[W] = j0;
    const int k0 = gidx32(g, i[0], i[1], i[2]);
    const CpmlAxis<KIND, W> x(g, f, s, i);
    float *ps = f.p + (long long)s * g.ntot;
    const CpmlPhiY py(g, f, s, i, g.px);

    // ---- phase 1: loads ----
    float win[U + 2 * N - 1];
#pragma unroll
    for (int q = 0; q < U + 2 * N - 1; q++) win[q] = x.h(g, k0, j0, j0 + O - N + 1 + q);
    CpmlOwn oW[U];
    float rho0[U], own_p[U], kap[U], phy[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = j0 + u, k = k0 + u * x.st;
        const bool ok = j <= jend && j >= lo[W];
        rho0[u] = (VK && ok) ? g.rho[k] : 1.0f;
        own_p[u] = (!VK && ok) ? ps[k] : 0.0f;
        kap[u] = (!VK && ok) ? g.K[k] : 0.0f;
        phy[u] = (KIND == kAP && ok && py.ph) ? py.ph[u * py.step] : 0.0f;
        oW[u] = CpmlOwn{0.0f, 0.0f, 0.0f};
        if (ok) oW[u] = cpml_own(g, x, j, k, x.slab(g, j));
    }

    // ---- phase 2: compute and store ----
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = j0 + u, k = k0 + u * x.st;
        if (!(j <= jend && j >= lo[W])) continue;
        float acc = 0.0f;
        cpml_apply(g, x, j, k, x.slab(g, j), oW[u], rho0[u], own_p[u], cpml_d<N>(g, W, win + u), acc);
        if (KIND == kFP) ps[k] = own_p[u] - g.dt * kap[u] * acc;
        if (KIND == kAP) {
            if (py.ph) py.ph[u * py.step] = py.B * (phy[u] + own_p[u]);
            if (acc != 0.0f) ps[k] = own_p[u] - g.dt * kap[u] * acc;
        }
    }
}

// x piece, walking: a thread takes one line along x (fixed z index i0 and y
// index i2) and walks run `part` of one band of it (seg: the low or the high
// band, cut into nparts runs of whole chunks) in chunks of U nodes.  The
// window of h along x rolls from chunk to chunk: the last 2N - 1 values of
// one chunk's window open the next, so each h value is loaded once per run
// (cpml_chunk loads U + 2N - 1 values for every U nodes).  Same arithmetic as
// cpml_chunk.
template <int N, int KIND, int U>
__device__ __forceinline__ void cpml_xwalk(const Grid &g, const Fields &f, const Piece &p, int s, int c0, int cr,
                                           int seg, int part, int nparts, const int lo[3], const int hi[3])
{
    constexpr int W = 1;
    constexpr bool VK = KIND == kFV || KIND == kAV;
    constexpr int O = VK ? 0 : -1;
    constexpr int NW = U + 2 * N - 1;
    int i[3];
    i[0] = iv_map(p.iv[0], c0);
    i[2] = iv_map(p.iv[2], cr);
    if (i[0] < lo[0] || i[0] > hi[0] || i[2] < lo[2] || i[2] > hi[2]) return;
    // the band's chunks, cut into nparts runs of whole chunks; this thread walks run `part`
    const int jb = max(p.iv[W][2 * seg], lo[W]);
    const int jl = min(p.iv[W][2 * seg] + p.iv[W][2 * seg + 1] - 1, hi[W]);
    const int per = ((jl - jb + U) / U + nparts - 1) / nparts * U;
    const int js = jb + part * per;
    const int jend = min(jl, js + per - 1);
    if (js > jend) return;
    i[W] = js;
    const int k0 = gidx32(g, i[0], i[1], i[2]);
    const CpmlAxis<KIND, W> x(g, f, s, i);
    float *ps = f.p + (long long)s * g.ntot;
    const CpmlPhiY py(g, f, s, i, g.px);

    float win[NW];
#pragma unroll
    for (int q = 0; q < 2 * N - 1; q++) win[q] = x.h(g, k0, js, js + O - N + 1 + q);
    for (int j0 = js; j0 <= jend; j0 += U) {
        // ---- loads: the window's U new values and the chunk's own values ----
#pragma unroll
        for (int q = 2 * N - 1; q < NW; q++) win[q] = x.h(g, k0, js, j0 + O - N + 1 + q);
        CpmlOwn oW[U];
        float rho0[U], own_p[U], kap[U], phy[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int j = j0 + u, k = k0 + (j - js) * x.st;
            const bool ok = j <= jend;
            rho0[u] = (VK && ok) ? g.rho[k] : 1.0f;
            own_p[u] = (!VK && ok) ? ps[k] : 0.0f;
            kap[u] = (!VK && ok) ? g.K[k] : 0.0f;
            phy[u] = (KIND == kAP && ok && py.ph) ? py.ph[(j - js) * py.step] : 0.0f;
            oW[u] = CpmlOwn{0.0f, 0.0f, 0.0f};
            if (ok) oW[u] = cpml_own(g, x, j, k, x.slab(g, j));
        }
        // ---- compute and store ----
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int j = j0 + u, k = k0 + (j - js) * x.st;
            if (j > jend) continue;
            float acc = 0.0f;
            cpml_apply(g, x, j, k, x.slab(g, j), oW[u], rho0[u], own_p[u], cpml_d<N>(g, W, win + u), acc);
            if (KIND == kFP) ps[k] = own_p[u] - g.dt * kap[u] * acc;
            if (KIND == kAP) {
                if (py.ph) py.ph[(j - js) * py.step] = py.B * (phy[u] + own_p[u]);
                if (acc != 0.0f) ps[k] = own_p[u] - g.dt * kap[u] * acc;
            }
        }
#pragma unroll
        for (int q = 0; q < 2 * N - 1; q++) win[q] = win[q + U];
    }
}

// z piece: a warp takes one line segment along z (32 lanes = BW owned nodes
// plus the 2N - 1 halo nodes of their stencils) times up to U consecutive
// nodes along x.  Each lane loads h along z at its own position and the z
// derivatives come from warp shuffles; chunks that reach the x band also
// load a per-lane window of h along x for the x terms.  Control flow is
// warp-uniform up to the shuffles.
template <int N, int KIND, int U>
__device__ __forceinline__ void cpml_zwarp(const Grid &g, const Fields &f, const Pieces &P, const Piece &p, int s,
                                           int lane, int zw, int cr, int ch, const int lo[3], const int hi[3])
{
    constexpr int W = 1;
    constexpr bool VK = KIND == kFV || KIND == kAV;
    constexpr int O = VK ? 0 : -1;
    constexpr int HL = N - 1 - O, HR = N + O, BW = 32 - HL - HR;
    const int nz0 = (p.iv[0][1] + BW - 1) / BW;
    const int cw0 = (p.iv[W][1] + U - 1) / U;
    int i[3];                                                      // warp-uniform from here to the shuffles
    i[2] = iv_map(p.iv[2], cr);
    if (i[2] < lo[2] || i[2] > hi[2]) return;
    const int zseg = zw < nz0 ? 0 : 1;
    zw -= zseg ? nz0 : 0;
    const int zs = p.iv[0][2 * zseg], ze = min(zs + p.iv[0][2 * zseg + 1] - 1, hi[0]);
    const int z = zs + zw * BW + lane - HL;
    const bool zown = lane >= HL && lane < 32 - HR && z <= ze && z >= lo[0];
    const int wseg = ch < cw0 ? 0 : 1;
    ch -= wseg ? cw0 : 0;
    const int j0 = p.iv[W][2 * wseg] + ch * U;
    const int jend = min(p.iv[W][2 * wseg] + p.iv[W][2 * wseg + 1] - 1, hi[W]);
    const int zc = min(max(z, 0), g.ne[0] - 1);
    i[0] = zc;
    i[W] = j0;
    const int k0 = gidx32(g, i[0], i[1], i[2]);
    const CpmlAxis<KIND, W> xw(g, f, s, i);
    float *ps = f.p + (long long)s * g.ntot;
    // axis-0 arrays: the slab base moves by S per node along x
    const CpmlAxis<KIND, 0> xz(g, f, s, i);
    const bool s0 = xz.slab(g, zc);
    const bool wband = cpml_in<KIND>(g, P, W, j0) || cpml_in<KIND>(g, P, W, j0 + U - 1);   // warp-uniform
    const CpmlPhiY py(g, f, s, i, g.px);

    // ---- phase 1: loads ----
    float hz[U], win[U + 2 * N - 1];
#pragma unroll
    for (int u = 0; u < U; u++) {
        CpmlAxis<KIND, 0> xu = xz;
        xu.sb += u * g.S;
        hz[u] = j0 + u <= jend ? xu.h(g, k0 + u * xw.st, zc, z) : 0.0f;   // no line past the chunk's end
    }
#pragma unroll
    for (int q = 0; q < U + 2 * N - 1; q++) win[q] = (zown && wband) ? xw.h(g, k0, j0, j0 + O - N + 1 + q) : 0.0f;
    CpmlOwn o0[U], oW[U];
    float rho0[U], own_p[U], kap[U], phy[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = j0 + u, k = k0 + u * xw.st;
        const bool ok = zown && j <= jend && j >= lo[W];
        rho0[u] = (VK && ok) ? g.rho[k] : 1.0f;
        own_p[u] = (!VK && ok) ? ps[k] : 0.0f;
        kap[u] = (!VK && ok) ? g.K[k] : 0.0f;
        phy[u] = (KIND == kAP && ok && py.ph) ? py.ph[u * py.step] : 0.0f;
        o0[u] = CpmlOwn{0.0f, 0.0f, 0.0f};
        oW[u] = CpmlOwn{0.0f, 0.0f, 0.0f};
        CpmlAxis<KIND, 0> xu = xz;
        xu.sb += u * g.S;
        if (ok) o0[u] = cpml_own(g, xu, zc, k, s0);
        if (ok && wband && cpml_in<KIND>(g, P, W, j)) oW[u] = cpml_own(g, xw, j, k, xw.slab(g, j));
    }

    // ---- phase 2: compute and store ----
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = j0 + u, k = k0 + u * xw.st;
        if (!(j <= jend && j >= lo[W])) continue;                 // warp-uniform
        float Dz = 0.0f;
#pragma unroll
        for (int l = 1; l <= N; l++)
            Dz += g.c[0][l - 1] * (__shfl_sync(0xffffffffu, hz[u], lane + O + l) -
                                   __shfl_sync(0xffffffffu, hz[u], lane + O + 1 - l));
        if (!zown) continue;
        float acc = 0.0f;
        CpmlAxis<KIND, 0> xu = xz;
        xu.sb += u * g.S;
        cpml_apply(g, xu, zc, k, s0, o0[u], rho0[u], own_p[u], Dz, acc);
        if (wband && cpml_in<KIND>(g, P, W, j))
            cpml_apply(g, xw, j, k, xw.slab(g, j), oW[u], rho0[u], own_p[u], cpml_d<N>(g, W, win + u), acc);
        if (KIND == kFP) ps[k] = own_p[u] - g.dt * kap[u] * acc;
        if (KIND == kAP) {
            if (py.ph) py.ph[u * py.step] = py.B * (phy[u] + own_p[u]);
            if (acc != 0.0f) ps[k] = own_p[u] - g.dt * kap[u] * acc;
        }
    }
}

// Resident 256-thread blocks per SM that k_cpml_x's register budget must
// allow (the forward kinds' x piece is load-latency bound: more warps hide
// more latency).  Measured on the 340^3 RTM step, box off, 30 steps: without
// a bound (62-95 registers) forward 18.3 ms, with 4 blocks (64 registers)
// 17.8 ms.

// x piece: block = ZB z indices x 256/ZB y indices (ZB = 64 in 3D, 256 in 2D
// where y has one index); blockIdx.y = chunk along x, blockIdx.z = shot.
template <int N, int KIND>
__global__ void __launch_bounds__(256, SMI_CPML_MINB_F) k_cpml_x(Grid g, Batch b, Fields f, Pieces P, int m)
{
    const Piece &p = P.q[1];
    const int zb = g.ndim == 3 ? 64 : 256;
    const int nbz = (p.cnt[0] + zb - 1) / zb;
    const int bz = blockIdx.x % nbz, br = blockIdx.x / nbz;
    const int c0 = bz * zb + (int)threadIdx.x % zb, cr = br * (256 / zb) + (int)threadIdx.x / zb;
    if (c0 >= p.cnt[0] || cr >= p.cnt[2]) return;
    const int s = blockIdx.z;
    int lo[3], hi[3];
    box_at((KIND == kFV || KIND == kFP) ? b.tab_src : b.tab_rec, b.nt1, s, m, lo, hi);
    cpml_chunk<N, KIND, kCpmlChunk>(g, f, p, s, c0, cr, blockIdx.y, lo, hi);
}

// x piece, walking (cpml_xwalk): block = ZB z indices x 256/ZB y indices
// as in k_cpml_x; blockIdx.y = band (low, high) x run of the band
// (SMI_CPML_XW_PARTS runs a band, so that enough lines walk at once),
// blockIdx.z = shot.
template <int N, int KIND>
__global__ void __launch_bounds__(256, SMI_CPML_XW_MINB) k_cpml_xw(Grid g, Batch b, Fields f, Pieces P, int m)
{
    const Piece &p = P.q[1];
    const int zb = g.ndim == 3 ? 64 : 256;
    const int nbz = (p.cnt[0] + zb - 1) / zb;
    const int bz = blockIdx.x % nbz, br = blockIdx.x / nbz;
    const int c0 = bz * zb + (int)threadIdx.x % zb, cr = br * (256 / zb) + (int)threadIdx.x / zb;
    const int side = blockIdx.y / SMI_CPML_XW_PARTS, part = blockIdx.y % SMI_CPML_XW_PARTS;
    if (c0 >= p.cnt[0] || cr >= p.cnt[2] || p.iv[1][2 * side + 1] == 0) return;
    const int s = blockIdx.z;
    int lo[3], hi[3];
    box_at((KIND == kFV || KIND == kFP) ? b.tab_src : b.tab_rec, b.nt1, s, m, lo, hi);
    cpml_xwalk<N, KIND, SMI_CPML_XW_U>(g, f, p, s, c0, cr, side, part, SMI_CPML_XW_PARTS, lo, hi);
}

// z piece, persistent: blockIdx.y = z warp segment (those of the low band,
// then those of the high band), blockIdx.z = shot; the warps of a segment
// walk its units (UZ consecutive x lines at one y, the chunks cpml_zwarp
// takes) in a strided loop.  What depends on z alone -- the lane's node, its
// CPML coefficients, slab offsets and box test -- is computed once per warp
// instead of once per unit.  Units whose x range reaches the x band take
// cpml_zwarp, which adds the x terms there; the others run the z terms
// below, the same arithmetic as cpml_apply.
template <int N, int KIND>
__global__ void __launch_bounds__(256, SMI_CPML_ZP_MINB) k_cpml_zp(Grid g, Batch b, Fields f, Pieces P, int m)
{
    constexpr bool VK = KIND == kFV || KIND == kAV;
    constexpr bool ADJ = KIND == kAV || KIND == kAP;
    constexpr int O = VK ? 0 : -1;
    constexpr int HL = N - 1 - O, HR = N + O, BW = 32 - HL - HR;
    constexpr int U = ADJ ? kCpmlChunkZ : 2 * kCpmlChunkZ;
    const Piece &p = P.q[0];
    const int s = blockIdx.z, lane = threadIdx.x & 31;
    int lo[3], hi[3];
    box_at(ADJ ? b.tab_rec : b.tab_src, b.nt1, s, m, lo, hi);

    // ---- per warp: the segment and the lane's node along z ----
    const int zw = blockIdx.y;
    const int nz0 = (p.iv[0][1] + BW - 1) / BW;
    const int zseg = zw < nz0 ? 0 : 1;
    const int zs = p.iv[0][2 * zseg], ze = min(zs + p.iv[0][2 * zseg + 1] - 1, hi[0]);
    const int ne = g.ne[0], hib = ne - 2 * g.nb - 1;           // slab index = j, or j - hib in the high slab
    const int z = zs + (zw - (zseg ? nz0 : 0)) * BW + lane - HL;
    const bool zown = lane >= HL && lane < 32 - HR && z <= ze && z >= lo[0];
    const int zc = min(max(z, 0), ne - 1);
    bool hv = (unsigned)z < (unsigned)ne;                          // h exists at z
    if (ADJ) hv = hv && (z < g.nb || z >= ne - g.nb - 1);
    const int hms = z < g.nb ? z : z - hib;
    const float hca = (ADJ && hv) ? __ldg((KIND == kAV ? g.cpa[0] : g.cva[0]) + z) : 0.0f;
    const bool sl = zc < g.nb || zc >= ne - g.nb - 1;              // own node in the slab
    const int oms = zc < g.nb ? zc : zc - hib;
    const bool up = zc + 1 < ne;
    const float cb = sl ? (VK ? g.cvb[0][zc] : g.cpb[0][zc]) : 0.0f;
    const float ca = (!ADJ && sl) ? (VK ? g.cva[0][zc] : g.cpa[0][zc]) : 0.0f;

    const long long so = (long long)s * g.ntot, ms = (long long)s * g.slab_n[0];
    const float *src = (VK ? f.p : f.v[0]) + so;
    const float *hmem = (KIND == kAV ? f.psiv[0] : f.psip[0]) + ms;
    float *mem = (VK ? f.psip[0] : f.psiv[0]) + ms;
    float *fld = f.v[0] + so;
    float *ps = f.p + so;

    const int nch = (p.iv[1][1] + U - 1) / U;
    const int nunit = p.cnt[2] * nch;
    const int xend = min(p.iv[1][0] + p.iv[1][1] - 1, hi[1]);
    for (int t = blockIdx.x * 8 + (int)(threadIdx.x >> 5); t < nunit; t += gridDim.x * 8) {   // warp-uniform
        const int cr = t / nch, ch = t - cr * nch;
        const int y = iv_map(p.iv[2], cr);
        if (y < lo[2] || y > hi[2]) continue;
        const int x0 = p.iv[1][0] + ch * U;
        if (cpml_in<KIND>(g, P, 1, x0) || cpml_in<KIND>(g, P, 1, x0 + U - 1)) {
            cpml_zwarp<N, KIND, U>(g, f, P, p, s, lane, zw, cr, ch, lo, hi);
            continue;
        }
        const int kl = gidx32(g, 0, x0, y), sL = g.S * (x0 + g.ne[1] * y);
        int iz[3] = {zc, x0, y};
        const CpmlPhiY py(g, f, s, iz, g.px);

        // ---- loads ----
        float hz[U], rho0[U], rho1[U], fo[U], mo[U], pk[U], kp[U], phy[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = kl + u * g.px + zc, mi = sL + u * g.S;
            const bool ok = zown && x0 + u <= xend && x0 + u >= lo[1];
            hz[u] = 0.0f;
            if (hv && x0 + u <= xend) {
                const int kk = kl + u * g.px + z;
                hz[u] = ADJ ? hca * (src[kk] + hmem[mi + hms]) : src[kk];
            }
            rho0[u] = (VK && ok) ? g.rho[k] : 1.0f;
            rho1[u] = (VK && ok && up) ? g.rho[k + 1] : 0.0f;
            fo[u] = (VK && ok) ? fld[k] : 0.0f;
            mo[u] = (ok && sl) ? mem[mi + oms] : 0.0f;
            pk[u] = (!VK && ok) ? ps[k] : 0.0f;
            kp[u] = (!VK && ok) ? g.K[k] : 0.0f;
            phy[u] = (KIND == kAP && ok && py.ph) ? py.ph[u * py.step] : 0.0f;
        }

        // ---- compute and store ----
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (!(x0 + u <= xend && x0 + u >= lo[1])) continue;    // warp-uniform
            float Dz = 0.0f;
#pragma unroll
            for (int l = 1; l <= N; l++)
                Dz += g.c[0][l - 1] * (__shfl_sync(0xffffffffu, hz[u], lane + O + l) -
                                       __shfl_sync(0xffffffffu, hz[u], lane + O + 1 - l));
            if (!zown) continue;
            const int k = kl + u * g.px + zc, mi = sL + u * g.S + oms;
            if (VK) {
                const float bb = up ? __fdividef(2.0f, rho0[u] + rho1[u]) : __fdividef(1.0f, rho0[u]);
                if (KIND == kFV) {
                    const float psi = cb * mo[u] + ca * Dz;
                    mem[mi] = psi;
                    fld[k] = fo[u] - g.dt * bb * psi;
                } else {
                    if (sl) mem[mi] = cb * (mo[u] + fo[u]);                // deferred chi update
                    if (Dz != 0.0f) fld[k] = fo[u] - g.dt * bb * Dz;
                }
            } else if (KIND == kFP) {
                const float psi = cb * mo[u] + ca * Dz;
                mem[mi] = psi;
                ps[k] = pk[u] - g.dt * kp[u] * psi;
            } else {
                if (sl) mem[mi] = cb * (mo[u] + pk[u]);                    // phi update, lp before this step
                if (py.ph) py.ph[u * py.step] = py.B * (phy[u] + pk[u]);
                if (Dz != 0.0f) ps[k] = pk[u] - g.dt * kp[u] * Dz;
            }
        }
    }
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
        if (mode == 2) acc[(long long)(b.nshot + s) * g.nphys + kp] += pk * pk;   // illumination
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

// Adjoint of the wavelet samples (the transpose of k_inject_source): the
// source of step it enters p^{it+1} as dt stf[it] w / dV, so its adjoint is
// dt / dV sum_w w pbar over the source stencil, with pbar = lambda_p / kappa
// (the library's adjoint pressure is kappa times the plain adjoint).  One
// block per shot; part[s][it] = the shot's sample, summed in FP64.
__global__ void k_src_adjoint(Grid g, Batch b, const float *lp, double *part, int nt, int it, double scale)
{
    __shared__ double red[kThreads];
    const int s = blockIdx.x;
    const Stencil &st = b.src[s];
    const int n = st.cnt[0] * st.cnt[1] * st.cnt[2];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int a0 = t % st.cnt[0], r = t / st.cnt[0];
        const int a1 = r % st.cnt[1], a2 = r / st.cnt[1];
        const long long k = gidx(g, st.first[0] + a0, st.first[1] + a1, st.first[2] + a2);
        const double w = (double)st.w[0][a0] * (double)st.w[1][a1] * (double)st.w[2][a2];
        acc += w * (double)lp[s * g.ntot + k] / (double)g.K[k];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)s * nt + it] = scale * red[0];
}

// out[it] (+)= sum_s part[s][it], shots in order.
__global__ void k_sum_series(const double *part, int nshot, int nt, double *out, int accumulate)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nt) return;
    double v = accumulate ? out[it] : 0.0;
    for (int s = 0; s < nshot; s++) v += part[(long long)s * nt + it];
    out[it] = v;
}

__global__ void k_to_float(const double *a, int n, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// FP64 partial sums of a[i] * b[i], one per block (grid-stride; the
// partials are summed in block order afterwards, so the result does not
// depend on scheduling).
__global__ void k_dot(const float *a, const float *b, long long n, double *partials)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        acc += (double)a[t] * (double)b[t];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// Boundary bands.  blockIdx.y = region r = 2 axis + side, blockIdx.z =
// shot; a thread moves kBandVals values of the region (stride 256, all
// loads issued before the stores).  One step of one shot holds fewer than
// 2^31 values (checked at set-up), so offsets are 32-bit.
constexpr int kBandVals = 4;

struct BandRegion {
    int a, sd, w0, w1, n, off;
    const int *lo;
    unsigned m0, m1;                  // u / w0 and q / w1 by multiply-high (band_divisor)
    int l0, l1;
    __device__ __forceinline__ BandRegion(const Bands &bd, int r)
    {
        a = r >> 1;
        sd = r & 1;
        lo = bd.lo[a][sd];
        const int *hi = bd.hi[a][sd];
        w0 = hi[0] - lo[0] + 1;
        w1 = hi[1] - lo[1] + 1;
        n = w0 * w1 * (hi[2] - lo[2] + 1);
        off = (int)bd.off[a][sd];
        m0 = bd.dm[a][sd][0];
        l0 = bd.dl[a][sd][0];
        m1 = bd.dm[a][sd][1];
        l1 = bd.dl[a][sd][1];
    }
    // flat field index of value u of the region
    __device__ __forceinline__ int node(const Grid &g, int u) const
    {
        const unsigned uu = (unsigned)u;
        const unsigned q = (__umulhi(m0, uu) + uu) >> l0;
        const unsigned q1 = (__umulhi(m1, q) + q) >> l1;
        return (lo[0] + u - (int)q * w0) + g.px * ((lo[1] + (int)q - (int)q1 * w1) + g.ne[1] * (lo[2] + (int)q1));
    }
};

__global__ void k_band_absmax(Grid g, Fields f, Bands bd, unsigned *amax)
{
    const BandRegion R(bd, blockIdx.y);
    if (R.a >= g.ndim || R.n <= 0) return;
    const int s = blockIdx.z;
    const float *v = f.v[R.a] + (long long)s * g.ntot;
    float m = 0.0f;
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        if (u < R.n) m = fmaxf(m, fabsf(v[R.node(g, u)]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(amax + s * 6 + blockIdx.y, __float_as_uint(m));
}

__global__ void k_band_save(Grid g, Fields f, Bands bd, int it, const unsigned *amax)
{
    const BandRegion R(bd, blockIdx.y);
    if (R.a >= g.ndim || R.n <= 0) return;
    const int s = blockIdx.z;
    const float *v = f.v[R.a] + (long long)s * g.ntot;
    const long long o0 = ((long long)s * bd.nt + it) * bd.count + R.off;
    float x[kBandVals];
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        x[q] = u < R.n ? v[R.node(g, u)] : 0.0f;
    }
    // 16-bit storage scaled per (step, axis, side): the largest magnitude
    // maps to 2^14 (FP16) or 1 (BF16).
    float inv = 1.0f;
    if (bd.prec != SMI_PREC_F32) {
        const float m = __uint_as_float(amax[s * 6 + blockIdx.y]);
        const float scale = m > 0.0f ? m / (bd.prec == SMI_PREC_F16 ? 16384.0f : 1.0f) : 0.0f;
        if (blockIdx.x == 0 && threadIdx.x == 0) bd.scale[((long long)s * bd.nt + it) * 6 + blockIdx.y] = scale;
        inv = scale;
    }
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        if (u >= R.n) continue;
        if (bd.prec == SMI_PREC_F32) {
            static_cast<float *>(bd.data)[o0 + u] = x[q];
        } else {
            const float y = inv > 0.0f ? x[q] / inv : 0.0f;
            if (bd.prec == SMI_PREC_F16) static_cast<__half *>(bd.data)[o0 + u] = __float2half_rn(y);
            else static_cast<__nv_bfloat16 *>(bd.data)[o0 + u] = __float2bfloat16_rn(y);
        }
    }
}

__global__ void k_band_restore(Grid g, Fields f, Bands bd, int it)
{
    const BandRegion R(bd, blockIdx.y);
    if (R.a >= g.ndim || R.n <= 0) return;
    const int s = blockIdx.z;
    float *v = f.v[R.a] + (long long)s * g.ntot;
    const long long o0 = ((long long)s * bd.nt + it) * bd.count + R.off;
    const float scale = bd.prec == SMI_PREC_F32 ? 1.0f : bd.scale[((long long)s * bd.nt + it) * 6 + blockIdx.y];
    float x[kBandVals];
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        x[q] = 0.0f;
        if (u < R.n) {
            if (bd.prec == SMI_PREC_F32) x[q] = static_cast<const float *>(bd.data)[o0 + u];
            else if (bd.prec == SMI_PREC_F16) x[q] = __half2float(static_cast<const __half *>(bd.data)[o0 + u]) * scale;
            else x[q] = __bfloat162float(static_cast<const __nv_bfloat16 *>(bd.data)[o0 + u]) * scale;
        }
    }
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        if (u < R.n) v[R.node(g, u)] = x[q];
    }
}

// Band of a step between stored samples: sum_q w_q sample[first+q] over the
// samples that exist (before sample 0 the field is zero).
__global__ void k_band_restore_interp(Grid g, Fields f, Bands bd, TimeWeights tw)
{
    const BandRegion R(bd, blockIdx.y);
    if (R.a >= g.ndim || R.n <= 0) return;
    const int s = blockIdx.z;
    float *v = f.v[R.a] + (long long)s * g.ntot;
    float x[kBandVals];
#pragma unroll
    for (int q = 0; q < kBandVals; q++) x[q] = 0.0f;
#pragma unroll
    for (int t = 0; t < 2 * kTimeR; t++) {
        const int k = tw.first + t;
        if (k < 0 || k >= tw.nsamp || tw.w[t] == 0.0f) continue;
        const long long o0 = ((long long)s * bd.nt + k) * bd.count + R.off;
        const float wt = bd.prec == SMI_PREC_F32 ? tw.w[t] : tw.w[t] * bd.scale[((long long)s * bd.nt + k) * 6 + blockIdx.y];
#pragma unroll
        for (int q = 0; q < kBandVals; q++) {
            const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
            if (u >= R.n) continue;
            float y;
            if (bd.prec == SMI_PREC_F32) y = static_cast<const float *>(bd.data)[o0 + u];
            else if (bd.prec == SMI_PREC_F16) y = __half2float(static_cast<const __half *>(bd.data)[o0 + u]);
            else y = __bfloat162float(static_cast<const __nv_bfloat16 *>(bd.data)[o0 + u]);
            x[q] += wt * y;
        }
    }
#pragma unroll
    for (int q = 0; q < kBandVals; q++) {
        const int u = (blockIdx.x * kBandVals + q) * blockDim.x + threadIdx.x;
        if (u < R.n) v[R.node(g, u)] = x[q];
    }
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

// Normalised image (Sec. 2.3): per shot s the largest illumination ill_s,
// then out (+)= sum_s acc_s / (ill_s + 1e-3 max ill_s), shots in order.
// Illuminations are non-negative, so their bit patterns order as unsigned.
__global__ void k_shot_max(const float *ill, long long n, unsigned *mx)
{
    const int s = blockIdx.y;
    float m = 0.0f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, ill[s * n + t]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(mx + s, __float_as_uint(m));
}

__global__ void k_reduce_norm(const float *acc, const float *ill, long long n, int nshot, const unsigned *mx,
                              float *out, int accumulate)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        float s = accumulate ? out[t] : 0.0f;
        for (int k = 0; k < nshot; k++) s += acc[k * n + t] / (ill[k * n + t] + 1e-3f * __uint_as_float(mx[k]));
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

// Density gradient (Eq. gradrhokappa, rho varied at fixed Vp).  Step it sets
// v^{it+1/2} = v^{it-1/2} - dt b (D p + psi) and nothing else of the step
// depends on b; with lambda_v = -b vbar and b = 2 / (rho_i + rho_{i+1}),
// each half node gives half of G = sum_it lambda_v (v^{it+1/2} - v^{it-1/2})
// to dJ/drho of both of its nodes (the b^2 of db/drho cancels the 1/b^2 of
// vbar dv/db).  k_rho_acc runs at the end of reverse step it, when vprev
// holds v^{it+1/2}, the source field v^{it-1/2} and the adjoint lambda_v of
// v^{it+1/2}: G_a += sum_s lambda_v (vprev - v), then vprev <- v.
// Four z-consecutive nodes per thread (float4): box.lo[0] is a multiple of
// 4 and the box's z width a multiple of 4 (the host widens the box; G is
// read only on the half nodes next to the physical domain, which the
// widened box always covers).
template <int NDIM>
__global__ void __launch_bounds__(kThreads) k_rho_acc(Grid g, int nshot, Fields F, Fields A, RhoAcc r, IBox box)
{
    const int wq = (box.hi[0] - box.lo[0] + 1) >> 2;
    const int w1 = box.hi[1] - box.lo[1] + 1;
    const long long vol = (long long)wq * w1 * (box.hi[2] - box.lo[2] + 1);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < vol;
         q += (long long)gridDim.x * blockDim.x) {
        int iq, i1, i2;
        if (vol < (1LL << 31)) {          // 32-bit division (uniform branch)
            const int qq = (int)q, rr = qq / wq;
            iq = qq - rr * wq;
            i1 = rr % w1;
            i2 = rr / w1;
        } else {
            const long long rr = q / wq;
            iq = (int)(q - rr * wq);
            i1 = (int)(rr % w1);
            i2 = (int)(rr / w1);
        }
        const long long k = gidx(g, box.lo[0] + 4 * iq, box.lo[1] + i1, box.lo[2] + i2);
        float4 c[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; a++) c[a] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int s = 0; s < nshot; s++) {
            const long long kk = s * g.ntot + k;
            float4 v[NDIM], l[NDIM], pv[NDIM];
#pragma unroll
            for (int a = 0; a < NDIM; a++) {
                v[a] = *reinterpret_cast<const float4 *>(F.v[a] + kk);
                l[a] = *reinterpret_cast<const float4 *>(A.v[a] + kk);
                pv[a] = *reinterpret_cast<const float4 *>(r.vprev[a] + kk);
            }
#pragma unroll
            for (int a = 0; a < NDIM; a++) {
                c[a].x += l[a].x * (pv[a].x - v[a].x);
                c[a].y += l[a].y * (pv[a].y - v[a].y);
                c[a].z += l[a].z * (pv[a].z - v[a].z);
                c[a].w += l[a].w * (pv[a].w - v[a].w);
                *reinterpret_cast<float4 *>(r.vprev[a] + kk) = v[a];
            }
        }
#pragma unroll
        for (int a = 0; a < NDIM; a++) {
            float4 *G = reinterpret_cast<float4 *>(r.G[a] + k);
            float4 t = *G;
            t.x += c[a].x;
            t.y += c[a].y;
            t.z += c[a].z;
            t.w += c[a].w;
            *G = t;
        }
    }
}

// Outputs of a gradient with a parametrisation family (Sec. 2.2).  acc =
// sum over shots and steps of lambda_p div v on the physical grid, so that
// dJ/dkappa = -dt acc / kappa; then
//   dJ/dVp|rho = 2 rho Vp dJ/dkappa,  dJ/drho|Vp = Vp^2 dJ/dkappa + buoyancy part,
// family 1 (Vp, rho): those two; family 2 (Vp, Ip = rho Vp):
//   dJ/dVp|Ip = dJ/dVp|rho - dJ/drho|Vp rho / Vp,  dJ/dIp|Vp = dJ/drho|Vp / Vp;
// logp: with respect to the logarithms (each times its parameter).
// g1 may alias acc.
__global__ void k_finalize_family(Grid g, const float *vp, const float *rho, const float *acc, RhoAcc r,
                                  int family, int logp, float *g1, float *g2)
{
    const int n0 = g.H[0] - g.L[0] + 1, n1 = g.H[1] - g.L[1] + 1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < g.nphys;
         t += (long long)gridDim.x * blockDim.x) {
        const int i0 = (int)(t % n0);
        const int i1 = (int)((t / n0) % n1);
        const int i2 = (int)(t / ((long long)n0 * n1));
        const long long k = gidx(g, i0 + g.L[0], i1 + g.L[1], i2 + g.L[2]);
        const float v = vp[t], d = rho[t], A0 = acc[t];
        float gb = 0.0f;
        for (int a = 0; a < g.ndim; a++) gb += r.G[a][k] + r.G[a][k - gstride(g, a)];
        float gv = -2.0f * g.dt * A0 / v;
        float gr = -g.dt * A0 / d + 0.5f * gb;
        if (family == 2) {
            gv -= gr * d / v;
            gr /= v;
        }
        if (logp) {
            gv *= v;
            gr *= family == 2 ? d * v : d;
        }
        g1[t] = gv;
        g2[t] = gr;
    }
}

// Free-surface mirrors and their transposes; thread (j, row, shot), j in
// 0..N fastest.
__global__ void k_free_surface(Grid g, float *f, int nshot, int op)
{
    const int N = g.N;
    const long long rows = (long long)g.ne[1] * g.ne[2];
    const long long n = rows * nshot * (N + 1);
    const int L = g.L[0];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % (N + 1));
        const long long r = t / (N + 1);                 // shot * rows + row
        const long long s = r / rows, row = r - s * rows;
        float *c = f + s * g.ntot + row * g.px;          // the z column of this (x, y)
        if (op == kFsMirrorV) {
            if (j < N) c[L - 1 - j] = c[L + j];
        } else if (op == kFsMirrorP) {
            if (j == 0) c[L] = 0.0f;
            else c[L - j] = -c[L + j];
        } else if (op == kFsFoldV) {
            if (j < N) {
                c[L + j] += c[L - 1 - j];
                c[L - 1 - j] = 0.0f;
            }
        } else {
            if (j == 0) {
                c[L] = 0.0f;
            } else {
                c[L + j] -= c[L - j];
                c[L - j] = 0.0f;
            }
        }
    }
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
        // free surface: the top layer mirrors the model about the surface node,
        // so that the transposed mirrors of the adjoint take no model ratio
        const int j1 = (g.freesurf && i1 < g.L[0]) ? min(g.L[0] - i1, n1 - 1) : min(max(i1 - g.L[0], 0), n1 - 1);
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

void launch_fwd_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_fwd_v, grid, g, b, f, it);
}

void launch_fwd_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_fwd_p, grid, g, b, f, it);
}

void launch_adj_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_adj_v, grid, g, b, f, m);
}

void launch_adj_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_adj_p, grid, g, b, f, m);
}

void launch_recon_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, const float *lp,
                    float *acc, int mode, const float *stf, int it, float src_scale, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_recon_p, grid, g, b, f, lp, acc, mode, stf, it, src_scale);
}

void launch_recon_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work)
{
    dim3 grid(blocks_for(work), b.nshot);
    SMI_DISPATCH(k_recon_v, grid, g, b, f, it);
}

// Pieces of the union of the bands (Sec. 2.1 CPML terms), clipped to the
// box [lo, hi].  Axis a: band = [0, w_lo) u [ne - w_hi, ne), the rest is
// "inner"; piece a = band of a x inner of every lower axis x box of every
// higher axis.  Inactive axes hold the single node 0.
Pieces make_pieces(const Grid &g, const int lo[3], const int hi[3], int w_lo, int w_hi, int uz)
{
    Pieces P{};
    P.w_lo = w_lo;
    P.w_hi = w_hi;
    int band[3][4], inner[3][4], full[3][4];
    auto clip = [](int x0, int x1, int l, int h, int *out) {
        const int s = std::max(x0, l), e = std::min(x1, h);
        out[0] = s;
        out[1] = e >= s ? e - s + 1 : 0;
    };
    for (int a = 0; a < 3; a++) {
        for (int k = 0; k < 4; k++) band[a][k] = inner[a][k] = full[a][k] = 0;
        const int ne = g.ne[a];
        clip(0, ne - 1, lo[a], hi[a], full[a]);
        if (ne - w_hi <= w_lo) {              // the two bands meet: the whole axis
            clip(0, ne - 1, lo[a], hi[a], band[a]);
        } else {
            clip(0, w_lo - 1, lo[a], hi[a], band[a]);
            clip(ne - w_hi, ne - 1, lo[a], hi[a], band[a] + 2);
            clip(w_lo, ne - w_hi - 1, lo[a], hi[a], inner[a]);
        }
    }
    // piece 0: z band x all x x all y; piece 1: x band x inner z x all y
    for (int a = 0; a < 2; a++) {
        Piece &p = P.q[a];
        p.axis = a;
        long long cnt = 1;
        for (int b = 0; b < 3; b++) {
            const int *src = b == a ? band[b] : (b < a ? inner[b] : full[b]);
            for (int k = 0; k < 4; k++) p.iv[b][k] = src[k];
            p.cnt[b] = src[1] + src[3];
            cnt *= p.cnt[b];
        }
        if (cnt == 0) continue;
        P.n++;
        // x piece: blocks of 64 z x 4 y lines (k_cpml_x: y = chunks along x;
        // k_cpml_xw: y = band).  z piece: nonzero counts mark the piece as
        // present (k_cpml_zp sizes its own persistent launch).
        const int u = a == 0 ? uz : kCpmlChunk;
        p.chunks = (p.iv[1][1] + u - 1) / u + (p.iv[1][3] + u - 1) / u;
        if (a == 0) {
            const int bw = 32 - (2 * g.N - 1);
            const long long zw = (p.iv[0][1] + bw - 1) / bw + (p.iv[0][3] + bw - 1) / bw;
            p.blocks = (int)((zw * p.cnt[2] + 7) / 8);
        } else {
            const int zb = g.ndim == 3 ? 64 : 256;
            p.blocks = ((p.cnt[0] + zb - 1) / zb) * ((p.cnt[2] + 256 / zb - 1) / (256 / zb));
        }
    }
    return P;
}

namespace {

// Persistent z-piece launch: one block column per z warp segment and shot,
// as many blocks along x as fill the GPU once (at least one unit a warp).
template <int N, int KIND>
void zp_launch(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, const Pieces &P, int m)
{
    static const int fill = [] {
        int per = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cpml_zp<N, KIND>, 256, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, per) * std::max(1, sms);
    }();
    constexpr int BW = 32 - (2 * N - 1);
    constexpr int U = KIND >= kAV ? kCpmlChunkZ : 2 * kCpmlChunkZ;
    const Piece &p = P.q[0];
    const int nseg = (p.iv[0][1] + BW - 1) / BW + (p.iv[0][3] + BW - 1) / BW;
    const long long nunit = (long long)p.cnt[2] * ((p.iv[1][1] + U - 1) / U);
    if (nseg == 0 || nunit == 0) return;
    const long long per_col = (long long)nseg * b.nshot;
    const long long nblk = std::max(1LL, std::min((fill + per_col - 1) / per_col, (nunit + 7) / 8));
    k_cpml_zp<N, KIND><<<dim3((unsigned)nblk, nseg, b.nshot), 256, 0, S(lc)>>>(g, b, f, P, m);
    ++*lc.launches;
}

template <int N>
void corr_launch(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, int kind,
                 const int lo[3], const int hi[3])
{
    // adjoint bands: nodes whose stencil reaches a slab node; forward: the slabs
    const Pieces P = kind >= kAV ? make_pieces(g, lo, hi, g.nb + N, g.nb + N + 1, kCpmlChunkZ)
                                 : make_pieces(g, lo, hi, g.nb, g.nb + 1, 2 * kCpmlChunkZ);
    // the two pieces hold disjoint nodes: launches in any order
    for (int a = 0; a < 2; a++) {
        const Piece &p = P.q[a];
        if (p.blocks == 0 || p.chunks == 0) continue;
        const dim3 grid(p.blocks, p.chunks, b.nshot);
        if (a == 0) {
            if (kind == kFV) zp_launch<N, kFV>(lc, g, b, f, P, m);
            else if (kind == kFP) zp_launch<N, kFP>(lc, g, b, f, P, m);
            else if (kind == kAV) zp_launch<N, kAV>(lc, g, b, f, P, m);
            else zp_launch<N, kAP>(lc, g, b, f, P, m);
            continue;                                     // counts its own launch
        } else if (kind >= kAV) {                          // measured: the walk pays in the adjoint kinds only
            const dim3 gw(p.blocks, 2 * SMI_CPML_XW_PARTS, b.nshot);
            if (kind == kAV) k_cpml_xw<N, kAV><<<gw, 256, 0, S(lc)>>>(g, b, f, P, m);
            else k_cpml_xw<N, kAP><<<gw, 256, 0, S(lc)>>>(g, b, f, P, m);
        } else {
            if (kind == kFV) k_cpml_x<N, kFV><<<grid, 256, 0, S(lc)>>>(g, b, f, P, m);
            else k_cpml_x<N, kFP><<<grid, 256, 0, S(lc)>>>(g, b, f, P, m);
        }
        ++*lc.launches;
    }
}

void corr_dispatch(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, int kind,
                   const int lo[3], const int hi[3])
{
    if (g.N == 2) corr_launch<2>(lc, g, b, f, m, kind, lo, hi);
    else corr_launch<4>(lc, g, b, f, m, kind, lo, hi);
}

}  // namespace

void launch_adj_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, bool vel,
                            const int lo[3], const int hi[3])
{
    corr_dispatch(lc, g, b, f, m, vel ? kAV : kAP, lo, hi);
}

void launch_fwd_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, bool vel,
                            const int lo[3], const int hi[3])
{
    corr_dispatch(lc, g, b, f, it, vel ? kFV : kFP, lo, hi);
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

// Band kernels: x = chunks of the largest region, y = region, z = shot.
static dim3 band_grid(const Bands &bd, int nshot)
{
    long long nmax = 0;
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            long long n = 1;
            for (int b = 0; b < 3; b++) n *= std::max(0, bd.hi[a][sd][b] - bd.lo[a][sd][b] + 1);
            nmax = std::max(nmax, n);
        }
    return dim3((unsigned)std::max<long long>(1, (nmax + kThreads * kBandVals - 1) / (kThreads * kBandVals)), 6, nshot);
}

void launch_save_bands(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, Bands bd, int it,
                       unsigned *absmax_tmp)
{
    const dim3 grid = band_grid(bd, b.nshot);
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
    const dim3 grid = band_grid(bd, b.nshot);
    k_band_restore<<<grid, kThreads, 0, S(lc)>>>(g, f, bd, it);
    ++*lc.launches;
}

void launch_restore_bands_interp(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, Bands bd,
                                 const TimeWeights &tw)
{
    const dim3 grid = band_grid(bd, b.nshot);
    k_band_restore_interp<<<grid, kThreads, 0, S(lc)>>>(g, f, bd, tw);
    ++*lc.launches;
}

void launch_residual(const LaunchCtx &lc, const float *seis, const float *dobs, long long n, int mode,
                     float *res, double *partials, int npart)
{
    k_residual<<<npart, kThreads, 0, S(lc)>>>(seis, dobs, n, mode, res, partials);
    ++*lc.launches;
}

void launch_src_adjoint(const LaunchCtx &lc, const Grid &g, const Batch &b, const float *lp, double *part, int nt,
                        int it, double scale)
{
    k_src_adjoint<<<b.nshot, kThreads, 0, S(lc)>>>(g, b, lp, part, nt, it, scale);
    ++*lc.launches;
}

void launch_sum_series(const LaunchCtx &lc, const double *part, int nshot, int nt, double *out, int accumulate)
{
    k_sum_series<<<(nt + kThreads - 1) / kThreads, kThreads, 0, S(lc)>>>(part, nshot, nt, out, accumulate);
    ++*lc.launches;
}

void launch_to_float(const LaunchCtx &lc, const double *a, int n, float *out)
{
    k_to_float<<<(n + kThreads - 1) / kThreads, kThreads, 0, S(lc)>>>(a, n, out);
    ++*lc.launches;
}

void launch_dot(const LaunchCtx &lc, const float *a, const float *b, long long n, double *partials, int npart)
{
    k_dot<<<npart, kThreads, 0, S(lc)>>>(a, b, n, partials);
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

void launch_reduce_norm(const LaunchCtx &lc, const Grid &g, const float *acc, int nshot, unsigned *mx, float *out,
                        int accumulate)
{
    const float *ill = acc + (long long)nshot * g.nphys;
    cudaMemsetAsync(mx, 0, sizeof(unsigned) * nshot, S(lc));
    k_shot_max<<<dim3(blocks_for(g.nphys), nshot), kThreads, 0, S(lc)>>>(ill, g.nphys, mx);
    k_reduce_norm<<<blocks_for(g.nphys), kThreads, 0, S(lc)>>>(acc, ill, g.nphys, nshot, mx, out, accumulate);
    *lc.launches += 2;
}

void launch_finalize_grad(const LaunchCtx &lc, long long n, const float *vp, float dt, float *gr)
{
    k_finalize_grad<<<blocks_for(n), kThreads, 0, S(lc)>>>(n, vp, dt, gr);
    ++*lc.launches;
}

void launch_rho_acc(const LaunchCtx &lc, const Grid &g, int nshot, Fields F, Fields A, RhoAcc r, IBox box)
{
    long long vol = 1;
    for (int a = 0; a < 3; a++) vol *= std::max(0, box.hi[a] - box.lo[a] + 1);
    if (vol == 0) return;
    box.lo[0] &= ~3;                       // whole float4 quads; px is a multiple of 8
    box.hi[0] |= 3;
    const long long quads = (long long)((box.hi[0] - box.lo[0] + 1) >> 2) * (box.hi[1] - box.lo[1] + 1) *
                            (box.hi[2] - box.lo[2] + 1);
    if (g.ndim == 3) k_rho_acc<3><<<blocks_for(quads), kThreads, 0, S(lc)>>>(g, nshot, F, A, r, box);
    else k_rho_acc<2><<<blocks_for(quads), kThreads, 0, S(lc)>>>(g, nshot, F, A, r, box);
    ++*lc.launches;
}

void launch_finalize_family(const LaunchCtx &lc, const Grid &g, const float *vp, const float *rho, const float *acc,
                            RhoAcc r, int family, int logp, float *g1, float *g2)
{
    k_finalize_family<<<blocks_for(g.nphys), kThreads, 0, S(lc)>>>(g, vp, rho, acc, r, family, logp, g1, g2);
    ++*lc.launches;
}

void launch_free_surface(const LaunchCtx &lc, const Grid &g, float *f, int nshot, int op)
{
    if (!g.freesurf) return;
    const long long n = (long long)g.ne[1] * g.ne[2] * nshot * (g.N + 1);
    k_free_surface<<<blocks_for(n), kThreads, 0, S(lc)>>>(g, f, nshot, op);
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
