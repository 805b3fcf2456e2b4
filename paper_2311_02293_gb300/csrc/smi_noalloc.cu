// smi_noalloc.cu -- smi_forward_noalloc: forward modelling that allocates no
// device memory.  Its working state (extended model, CPML tables, stencils,
// wavefields and CPML memory variables) lives in one file-scope device array
// of fixed size, so callers that are not allowed to allocate device memory
// can still model seismograms.  Shots are propagated one after another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "smi_box.h"
#include "smi_internal.h"

namespace smi {
void record_error(const char *msg);     // smi_api.cu
}

namespace {

using namespace smi;

// 64 MiB of working memory, resident on every GPU that loads the library
// until the process exits.  All calls share it.
constexpr size_t kScratchBytes = 64ull << 20;
constexpr int kMaxAxis = 8192;          // extended nodes per axis (host CPML staging)
constexpr int kStencilChunk = 64;       // receiver stencils staged per copy

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_ptr[256] = {nullptr};           // device address of g_scratch per device ordinal

int err(int code, const char *fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    record_error(buf);
    return code;
}

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as an address).
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(SMI_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return err(SMI_ERR_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return err(SMI_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                       cudaGetErrorString(e));
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return SMI_OK;
}

// Device (or managed) memory that the current device, which owns the
// scratch array and runs the kernels, may use: device memory of another
// device is refused.
bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && a.device == dev;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
    size_t off = 0;
    unsigned char *base = nullptr;     // nullptr: only count bytes
    template <class T> T *take(size_t n)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += std::max<size_t>(n, 1) * sizeof(T);
        return p;
    }
};

struct Plan {
    unsigned *mm_tmp;
    float *mm;
    unsigned *flag;
    float *cpml[3];
    float *K, *rho;
    Stencil *src, *rec;
    int *box_src, *box_rec, *rec_off;
    int *tab;                 // [nt+1][6] source box of every step
    long long *seis_off;
    float *p, *v[3], *psip[3], *psiv[3];
};

void lay_out(Carve &c, Plan &pl, const Grid &g, int max_rec, int nt)
{
    pl.mm_tmp = c.take<unsigned>(4);
    pl.mm = c.take<float>(4);
    pl.flag = c.take<unsigned>(1);
    for (int a = 0; a < 3; a++) pl.cpml[a] = a < g.ndim ? c.take<float>(4 * (size_t)g.ne[a]) : nullptr;
    pl.K = c.take<float>((size_t)g.ntot);
    pl.rho = c.take<float>((size_t)g.ntot);
    pl.src = c.take<Stencil>(1);
    pl.rec = c.take<Stencil>((size_t)max_rec);
    pl.box_src = c.take<int>(6);
    pl.box_rec = c.take<int>(6);
    pl.rec_off = c.take<int>(2);
    pl.tab = c.take<int>(6 * ((size_t)nt + 1));
    pl.seis_off = c.take<long long>(1);
    pl.p = c.take<float>((size_t)g.ntot);
    for (int a = 0; a < 3; a++) {
        const bool act = a < g.ndim;
        pl.v[a] = act ? c.take<float>((size_t)g.ntot) : nullptr;
        pl.psip[a] = act ? c.take<float>((size_t)g.slab_n[a]) : nullptr;
        pl.psiv[a] = act ? c.take<float>((size_t)g.slab_n[a]) : nullptr;
    }
}

void extent_of(const Grid &g, const Stencil &s, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) {
        if (a >= g.ndim) { lo[a] = hi[a] = 0; continue; }
        lo[a] = s.cnt[a] == 1 ? s.first[a] - g.ri + 1 : s.first[a];
        hi[a] = s.cnt[a] == 1 ? s.first[a] + g.ri : s.first[a] + s.cnt[a] - 1;
    }
}

int sync(cudaStream_t st)
{
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? SMI_OK : err(SMI_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(e));
}

int forward_noalloc(const smi_model *m, const smi_geometry *geo, const smi_wavelet *w,
                    const smi_opts *o, float *seis)
{
    record_error("");
    if (!m || !geo || !w || !o || !seis) return err(SMI_ERR_ARG, "null argument");
    if (m->ndim != 2 && m->ndim != 3) return err(SMI_ERR_ARG, "ndim must be 2 or 3");
    if (o->order != 4 && o->order != 8) return err(SMI_ERR_ARG, "order must be 4 or 8");
    if (o->freesurf != 0 && o->freesurf != 1) return err(SMI_ERR_ARG, "freesurf must be 0 or 1");
    if (o->dr < 1) return err(SMI_ERR_ARG, "dr must be >= 1");
    if (o->shell_prec < SMI_PREC_F32 || o->shell_prec > SMI_PREC_BF16)
        return err(SMI_ERR_ARG, "shell_prec must be SMI_PREC_F32, F16 or BF16");
    const int N = o->order / 2;
    if (o->nb < N) return err(SMI_ERR_ARG, "nb must be >= order/2");
    if (!m->vp || !m->rho || !w->stf) return err(SMI_ERR_ARG, "model or wavelet array is null");
    if (w->nt < 1 || !(w->dt > 0.0) || !(w->fm >= 0.0)) return err(SMI_ERR_ARG, "bad nt, dt or fm");
    if (geo->nshot < 1 || !geo->src || !geo->rec_offset || geo->rec_offset[0] != 0)
        return err(SMI_ERR_ARG, "bad geometry");
    if (m->ndim == 2 && m->n3 != 1 && m->n3 != 0) return err(SMI_ERR_ARG, "n3 must be 1 in 2D");

    Grid g{};
    const int n[3] = {m->n1, m->n2, m->ndim == 3 ? m->n3 : 1};
    const double hh[3] = {m->d1, m->d2, m->ndim == 3 ? m->d3 : 1.0};
    g.ndim = m->ndim;
    g.N = N;
    g.ri = N;
    g.nb = o->nb;
    g.ntot = 1;
    g.nphys = 1;
    for (int a = 0; a < 3; a++) {
        const bool act = a < m->ndim;
        if (act && (n[a] < 2 * N || !(hh[a] > 0.0))) return err(SMI_ERR_ARG, "bad size or spacing on axis %d", a);
        g.ne[a] = act ? n[a] + 2 * o->nb : 1;
        if (g.ne[a] > kMaxAxis) return err(SMI_ERR_ARG, "axis %d has %d extended nodes; at most %d here", a, g.ne[a], kMaxAxis);
        g.L[a] = act ? o->nb : 0;
        g.H[a] = act ? o->nb + n[a] - 1 : 0;
        g.h[a] = hh[a];
        g.ntot *= g.ne[a];
        g.nphys *= n[a];
    }
    set_layout(g, n);
    g.dt = (float)w->dt;
    g.use_box = o->use_box ? 1 : 0;
    g.freesurf = o->freesurf;
    double coef[kMaxHalf] = {0};
    fd_coefficients(N, coef);
    for (int a = 0; a < 3; a++)
        for (int l = 0; l < kMaxHalf; l++) g.c[a][l] = (a < m->ndim && l < N) ? (float)(coef[l] / hh[a]) : 0.0f;

    int max_rec = 0;
    for (int s = 0; s < geo->nshot; s++) {
        const int nr = geo->rec_offset[s + 1] - geo->rec_offset[s];
        if (nr < 0) return err(SMI_ERR_ARG, "rec_offset must be nondecreasing");
        max_rec = std::max(max_rec, nr);
    }
    if (max_rec > 0 && !geo->rec) return err(SMI_ERR_ARG, "receiver array is null");

    // size check before touching the device
    Carve count;
    Plan pl{};
    lay_out(count, pl, g, max_rec, w->nt);
    if (count.off > kScratchBytes)
        return err(SMI_ERR_ARG,
                   "problem needs %zu bytes of working memory; smi_forward_noalloc holds at most %zu "
                   "(use smi_forward)", count.off, kScratchBytes);

    if (!on_device(m->vp) || !on_device(m->rho) || !on_device(w->stf) || !on_device(seis))
        return err(SMI_ERR_ARG, "smi_forward_noalloc needs device pointers of the current device for vp, rho, "
                                "stf and seis");

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    Carve c;
    c.base = static_cast<unsigned char *>(base);
    lay_out(c, pl, g, max_rec, w->nt);

    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    long long launches = 0;
    LaunchCtx lc{st, &launches};

    // vmin / vmax and rho positivity
    float hm[4];
    launch_minmax(lc, m->vp, g.nphys, pl.mm, pl.mm_tmp);
    launch_minmax(lc, m->rho, g.nphys, pl.mm + 2, pl.mm_tmp + 2);
    cudaMemcpyAsync(hm, pl.mm, sizeof hm, cudaMemcpyDeviceToHost, st);
    if ((rc = sync(st))) return rc;
    if (!(hm[0] > 0.0f) || !(hm[2] > 0.0f) || !std::isfinite(hm[1]) || !std::isfinite(hm[3]))
        return err(SMI_ERR_ARG, "vp and rho must be positive and finite");
    g.vdt = (double)hm[1] * w->dt;
    // the same admission as smi_forward (Sec. 4.2 dr rule, although forward
    // modelling stores no boundaries)
    if (o->dr > 1 && (double)o->dr > 5.0 * (double)hm[1] / (double)hm[0])
        return err(SMI_ERR_ARG, "dr = %d exceeds 5 vmax / vmin = %.2f (Sec. 4.2)", o->dr,
                   5.0 * (double)hm[1] / (double)hm[0]);
    const double cfl = cfl_number(m->ndim, hh, w->dt, hm[1], N);
    if (cfl > 1.0) return err(SMI_ERR_CFL, "CFL number %.4f exceeds 1 (Eq. cfl)", cfl);
    if (w->fm > 0.0) {
        const double ppw = points_per_wavelength(m->ndim, hh, hm[0], w->fm);
        const double need = N >= 4 ? 4.0 : 5.0;
        if (ppw < need)
            return err(SMI_ERR_DISPERSION, "%.2f points per shortest wavelength, order %d needs %.0f",
                       ppw, o->order, need);
    }

    // CPML tables (staged through a host stack buffer)
    const double R = o->cpml_R > 0.0 ? o->cpml_R : 1e-3;
    const double kb = o->kaiser_b > 0.0 ? o->kaiser_b : 4.0;
    for (int a = 0; a < m->ndim; a++) {
        float tab[4 * kMaxAxis];
        const int ne = g.ne[a];
        cpml_tables(ne, o->nb, hh[a], hm[1], w->fm, R, w->dt, false, tab, tab + ne);
        cpml_tables(ne, o->nb, hh[a], hm[1], w->fm, R, w->dt, true, tab + 2 * ne, tab + 3 * ne);
        if (a == 0 && g.freesurf)              // the top layer is the image zone: no absorption
            for (int q = 0; q < 4; q++)
                for (int i = 0; i < g.L[0]; i++) tab[q * ne + i] = 0.0f;
        cudaMemcpyAsync(pl.cpml[a], tab, sizeof(float) * 4 * ne, cudaMemcpyHostToDevice, st);
        if ((rc = sync(st))) return rc;
        g.cpa[a] = pl.cpml[a];
        g.cpb[a] = pl.cpml[a] + ne;
        g.cva[a] = pl.cpml[a] + 2 * ne;
        g.cvb[a] = pl.cpml[a] + 3 * ne;
    }
    g.K = pl.K;
    g.rho = pl.rho;
    launch_extend_model(lc, g, m->vp, m->rho, n[0], n[1], n[2], pl.K, pl.rho);
    cudaMemsetAsync(pl.flag, 0, sizeof(unsigned), st);

    double dV = 1.0;
    for (int a = 0; a < m->ndim; a++) dV *= hh[a];
    const float src_scale = (float)(w->dt / dV);

    for (int s = 0; s < geo->nshot; s++) {
        const int r0 = geo->rec_offset[s], nr = geo->rec_offset[s + 1] - r0;
        Stencil sst;
        if (!make_stencil(g, geo->src + 3 * s, kb, &sst))
            return err(SMI_ERR_ARG, "source %d lies outside the model or its stencil leaves the grid", s);
        int box[12], lo[3], hi[3];
        extent_of(g, sst, lo, hi);
        for (int a = 0; a < 3; a++) {
            box[a] = lo[a];
            box[3 + a] = hi[a];
            box[6 + a] = lo[a];
            box[9 + a] = hi[a];
        }
        bool first = true;
        for (int r = 0; r < nr; r += kStencilChunk) {
            Stencil chunk[kStencilChunk];
            const int k = std::min(kStencilChunk, nr - r);
            for (int j = 0; j < k; j++) {
                if (!make_stencil(g, geo->rec + 3 * (size_t)(r0 + r + j), kb, &chunk[j]))
                    return err(SMI_ERR_ARG, "receiver %d lies outside the model or its stencil leaves the grid", r0 + r + j);
                extent_of(g, chunk[j], lo, hi);
                for (int a = 0; a < 3; a++) {
                    box[6 + a] = first ? lo[a] : std::min(box[6 + a], lo[a]);
                    box[9 + a] = first ? hi[a] : std::max(box[9 + a], hi[a]);
                }
                first = false;
            }
            cudaMemcpyAsync(pl.rec + r, chunk, sizeof(Stencil) * k, cudaMemcpyHostToDevice, st);
            if ((rc = sync(st))) return rc;
        }
        const int roff[2] = {0, nr};
        const long long soff = 0;
        cudaMemcpyAsync(pl.src, &sst, sizeof sst, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(pl.box_src, box, sizeof(int) * 6, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(pl.box_rec, box + 6, sizeof(int) * 6, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(pl.rec_off, roff, sizeof roff, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(pl.seis_off, &soff, sizeof soff, cudaMemcpyHostToDevice, st);
        // the scratch keeps the previous call's contents: start every shot from rest
        cudaMemsetAsync(pl.p, 0, sizeof(float) * g.ntot, st);
        for (int a = 0; a < m->ndim; a++) {
            cudaMemsetAsync(pl.v[a], 0, sizeof(float) * g.ntot, st);
            cudaMemsetAsync(pl.psip[a], 0, sizeof(float) * g.slab_n[a], st);
            cudaMemsetAsync(pl.psiv[a], 0, sizeof(float) * g.slab_n[a], st);
        }
        Batch b{};
        b.nshot = 1;
        b.box_src = pl.box_src;
        b.box_rec = pl.box_rec;
        b.src = pl.src;
        b.rec = pl.rec;
        b.rec_off = pl.rec_off;
        b.max_rec = nr;
        launch_box_fill(lc, g, pl.box_src, 1, w->nt, pl.tab);
        b.tab_src = pl.tab;
        b.tab_rec = pl.tab;
        b.nt1 = w->nt + 1;
        Fields F{};
        F.p = pl.p;
        for (int a = 0; a < 3; a++) {
            F.v[a] = pl.v[a];
            F.psip[a] = pl.psip[a];
            F.psiv[a] = pl.psiv[a];
        }
        float *out = seis + (size_t)w->nt * r0;
        for (int it = 0; it < w->nt; it++) {
            int lo[3], hi[3];
            box_bounds(g, box, it, lo, hi);
            launch_fwd_v(lc, g, b, F, it, box_points(lo, hi));
            launch_free_surface(lc, g, F.v[0], 1, kFsMirrorV);
            launch_fwd_p(lc, g, b, F, it, box_points(lo, hi));
            launch_inject_source(lc, g, b, F.p, w->stf, it, src_scale);
            launch_free_surface(lc, g, F.p, 1, kFsMirrorP);
            if (nr > 0) launch_gather(lc, g, b, F.p, out, pl.seis_off, w->nt, it);
        }
        if (nr > 0) launch_nonfinite(lc, out, (long long)w->nt * nr, pl.flag);
        launch_nonfinite(lc, F.p, g.ntot, pl.flag);
        // the host staging above is synchronous, so the next shot may reuse it
        if ((rc = sync(st))) return rc;
    }
    unsigned flag = 0;
    cudaMemcpyAsync(&flag, pl.flag, sizeof flag, cudaMemcpyDeviceToHost, st);
    if ((rc = sync(st))) return rc;
    if (flag) return err(SMI_ERR_UNSTABLE, "non-finite values in the wavefield or seismograms");
    return SMI_OK;
}

}  // namespace

extern "C" int smi_forward_noalloc(const smi_model *model, const smi_geometry *geom,
                                   const smi_wavelet *wav, const smi_opts *opts, float *seis)
{
    return forward_noalloc(model, geom, wav, opts, seis);
}
