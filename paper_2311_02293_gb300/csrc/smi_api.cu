// smi_api.cu -- the C ABI of libsmi (include/smi.h) and the per-call driver:
// validation, set-up, shot batching and the forward / reverse time loops of
// Algorithm 2 (SMIwiz, arXiv 2311.02293).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "smi_box.h"
#include "smi_fused3d.h"
#include "smi_internal.h"
#include "smi_stencil3d.h"

namespace smi {
namespace {

thread_local std::string t_err;
thread_local smi_stats t_stats;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// SMI_OK if p is null, host memory, managed memory or device memory of the
// current device (the one that runs the call's kernels); SMI_ERR_ARG for
// device memory of another device, which the kernels must not read.
int check_same_device(const void *p, const char *name)
{
    if (!p) return SMI_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return SMI_OK;                          // plain host memory
    }
    if (a.type != cudaMemoryTypeDevice) return SMI_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SMI_ERR_CUDA, "cudaGetDevice failed");
    if (a.device != dev)
        return fail(SMI_ERR_ARG, "%s is memory of device %d but the current device is %d", name, a.device, dev);
    return SMI_OK;
}

// Stream-ordered device allocations of one call, released in the destructor.
struct Arena {
    cudaStream_t st;
    std::vector<std::pair<void *, size_t>> ptrs;
    size_t cur = 0, peak = 0;
    bool ok = true;
    explicit Arena(cudaStream_t s) : st(s) {}
    void *raw(size_t bytes)
    {
        bytes = std::max<size_t>(bytes, 256);
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return nullptr;
        }
        ptrs.emplace_back(p, bytes);
        cur += bytes;
        peak = std::max(peak, cur);
        return p;
    }
    template <class T> T *get(size_t n) { return static_cast<T *>(raw(n * sizeof(T))); }
    // Hands the allocations over to dst (a tape); the arena frees nothing then.
    void release_to(std::vector<std::pair<void *, size_t>> &dst)
    {
        dst.insert(dst.end(), ptrs.begin(), ptrs.end());
        ptrs.clear();
    }
    ~Arena()
    {
        for (auto &pr : ptrs) cudaFreeAsync(pr.first, st);
    }
};

struct Setup {
    Grid g{};
    int ndim = 0, n[3] = {1, 1, 1};
    int nshot = 0, nt = 0;
    int dr = 1, nsamp = 0, nt_fwd = 0;     // boundary decimation: stored samples, forward steps
    int img_norm = 0;                      // normalised RTM image
    bool rho_grad = false;                 // gradient with the density part (parametrisation families)
    bool fused = false;                    // 3D forward / adjoint steps by the single-pass kernel
    bool inline3 = false;                  // 3D two-pass tile kernels with the z / x CPML terms inline
    bool fullmem = false;                  // z / x CPML memory variables as full-size arrays (either of the above)
    long long nrec_total = 0;
    size_t setup_bytes = 0;                // sizes-only set-up: estimated bytes of the set-up arena
    std::vector<int> rec_offset;
    std::vector<Stencil> src_st, rec_st;
    std::vector<int> box_src, box_rec;      // [nshot][6]
    float vmin = 0, vmax = 0;
    double src_scale = 0;                   // dt / dV
    const float *vp = nullptr, *rho = nullptr, *stf = nullptr;   // device
    // device tables
    Stencil *d_src = nullptr, *d_rec = nullptr;
    int *d_box_src = nullptr, *d_box_rec = nullptr;
    int *d_tab_src = nullptr, *d_tab_rec = nullptr;   // [nshot][nt_fwd+1][6] box tables
    Bands bands{};
};

// What a forward call with a tape (smi_forward_tape) keeps on the device for
// a later reverse-only call (smi_tape_vjp): the set-up (extended model,
// tables), the saved boundaries and the state after the last forward step
// of one batch holding every shot, and the reverse loop's buffers.
struct TapeState {
    Setup S;
    smi_opts o{};
    std::vector<std::pair<void *, size_t>> mem;   // owned device allocations
    Fields F{}, F2{}, A{}, A2{};
    Bands bd{};
    float *res = nullptr, *acc = nullptr;
    double *partials = nullptr;
    int *d_roff = nullptr;
    long long *d_soff = nullptr;
    std::vector<int> roff;
    std::vector<long long> soff;
    int max_rec = 0;
    long long batch_seis = 0;
    bool done = false;                            // the reverse pass ran (a tape serves one)
};

int classify_and_upload(Arena &ar, const float *p, size_t n, const float **dev, cudaStream_t st)
{
    if (is_device_ptr(p)) {
        *dev = p;
        return SMI_OK;
    }
    float *d = ar.get<float>(n);
    if (!d) return fail(SMI_ERR_NOMEM, "device allocation of %zu bytes failed", n * sizeof(float));
    if (cudaMemcpyAsync(d, p, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(SMI_ERR_CUDA, "host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
    *dev = d;
    return SMI_OK;
}

// Nominal stencil extent along each axis (the box is grown around it).
void stencil_extent(const Grid &g, const Stencil &s, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) {
        if (a >= g.ndim) { lo[a] = hi[a] = 0; continue; }
        if (s.cnt[a] == 1) {
            lo[a] = s.first[a] - g.ri + 1;
            hi[a] = s.first[a] + g.ri;
        } else {
            lo[a] = s.first[a];
            hi[a] = s.first[a] + s.cnt[a] - 1;
        }
    }
}

int validate_and_setup(const smi_model *m, const smi_geometry *geo, const smi_wavelet *w,
                       const smi_opts *o, Arena &ar, cudaStream_t st, long long *launches, Setup &S,
                       bool sizes_only = false)
{
    if (!m || !geo || !w || !o) return fail(SMI_ERR_ARG, "null argument");
    if (m->ndim != 2 && m->ndim != 3) return fail(SMI_ERR_ARG, "ndim must be 2 or 3");
    if (o->order != 4 && o->order != 8) return fail(SMI_ERR_ARG, "order must be 4 or 8");
    if (o->freesurf != 0 && o->freesurf != 1) return fail(SMI_ERR_ARG, "freesurf must be 0 or 1");
    if (o->dr < 1) return fail(SMI_ERR_ARG, "dr must be >= 1");
    if (o->shell_prec < SMI_PREC_F32 || o->shell_prec > SMI_PREC_BF16)
        return fail(SMI_ERR_ARG, "shell_prec must be SMI_PREC_F32, F16 or BF16");
    if (o->kernels < SMI_KERNELS_AUTO || o->kernels > SMI_KERNELS_INLINE)
        return fail(SMI_ERR_ARG, "kernels must be SMI_KERNELS_AUTO, _GENERIC, _TWOPASS, _FUSED or _INLINE");
    const int N = o->order / 2;
    if (o->nb < N) return fail(SMI_ERR_ARG, "nb must be >= order/2");
    if (!m->vp || !m->rho) return fail(SMI_ERR_ARG, "model arrays are null");
    if (!w->stf) return fail(SMI_ERR_ARG, "wavelet is null");
    if (int rc = check_same_device(m->vp, "vp")) return rc;
    if (int rc = check_same_device(m->rho, "rho")) return rc;
    if (int rc = check_same_device(w->stf, "stf")) return rc;
    if (w->nt < 1 || !(w->dt > 0.0) || !(w->fm >= 0.0)) return fail(SMI_ERR_ARG, "bad nt, dt or fm");
    if (geo->nshot < 1 || !geo->src || !geo->rec_offset) return fail(SMI_ERR_ARG, "bad geometry");
    S.ndim = m->ndim;
    S.n[0] = m->n1;
    S.n[1] = m->n2;
    S.n[2] = m->ndim == 3 ? m->n3 : 1;
    if (m->ndim == 2 && m->n3 != 1 && m->n3 != 0) return fail(SMI_ERR_ARG, "n3 must be 1 in 2D");
    const double hh[3] = {m->d1, m->d2, m->ndim == 3 ? m->d3 : 1.0};
    for (int a = 0; a < m->ndim; a++) {
        if (S.n[a] < 2 * N) return fail(SMI_ERR_ARG, "axis %d has fewer than order nodes", a);
        if (!(hh[a] > 0.0)) return fail(SMI_ERR_ARG, "grid spacing must be positive");
    }
    S.nshot = geo->nshot;
    S.nt = w->nt;
    S.dr = o->dr;
    S.img_norm = o->img_norm ? 1 : 0;
    S.nsamp = band_samples(S.nt, S.dr);
    S.nt_fwd = forward_steps(S.nt, S.dr);
    S.rec_offset.assign(geo->rec_offset, geo->rec_offset + geo->nshot + 1);
    if (S.rec_offset[0] != 0) return fail(SMI_ERR_ARG, "rec_offset[0] must be 0");
    for (int s = 0; s < S.nshot; s++)
        if (S.rec_offset[s + 1] < S.rec_offset[s]) return fail(SMI_ERR_ARG, "rec_offset must be nondecreasing");
    S.nrec_total = S.rec_offset[S.nshot];
    if (S.nrec_total > 0 && !geo->rec) return fail(SMI_ERR_ARG, "receiver array is null");

    Grid &g = S.g;
    g.ndim = m->ndim;
    g.N = N;
    g.ri = N;
    g.nb = o->nb;
    g.ntot = 1;
    g.nphys = 1;
    for (int a = 0; a < 3; a++) {
        const bool act = a < m->ndim;
        g.ne[a] = act ? S.n[a] + 2 * o->nb : 1;
        g.L[a] = act ? o->nb : 0;
        g.H[a] = act ? o->nb + S.n[a] - 1 : 0;
        g.h[a] = hh[a];
        g.ntot *= g.ne[a];
        g.nphys *= S.n[a];
    }
    set_layout(g, S.n);
    g.dt = (float)w->dt;
    g.use_box = o->use_box ? 1 : 0;
    g.freesurf = o->freesurf;
    double coef[kMaxHalf] = {0};
    fd_coefficients(N, coef);
    for (int a = 0; a < 3; a++)
        for (int l = 0; l < kMaxHalf; l++) g.c[a][l] = (a < m->ndim && l < N) ? (float)(coef[l] / hh[a]) : 0.0f;
    S.fused = o->kernels == SMI_KERNELS_FUSED && fused3d_supported(g);
    S.inline3 = o->kernels == SMI_KERNELS_INLINE && stencil3d_supported(g);
    S.fullmem = S.fused || S.inline3;

    // boundary bands: v_a on the 2N-1 half nodes straddling each face of the
    // physical domain, over the physical cross-section, stored every dr-th
    // step (Sec. 4.2)
    Bands &bd = S.bands;
    bd.count = 0;
    bd.prec = o->shell_prec;
    bd.nt = S.nsamp;
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            bd.off[a][sd] = bd.count;
            for (int b = 0; b < 3; b++) {
                bd.lo[a][sd][b] = g.L[b];
                bd.hi[a][sd][b] = g.H[b];
            }
            if (a >= m->ndim) {
                bd.hi[a][sd][0] = bd.lo[a][sd][0] - 1;   // empty
                continue;
            }
            if (sd == 0) {
                bd.lo[a][sd][a] = g.L[a] - N;
                bd.hi[a][sd][a] = g.L[a] + N - 2;
            } else {
                bd.lo[a][sd][a] = g.H[a] - N + 1;
                bd.hi[a][sd][a] = g.H[a] + N - 1;
            }
            long long c = 1;
            for (int b = 0; b < 3; b++) c *= bd.hi[a][sd][b] - bd.lo[a][sd][b] + 1;
            bd.count += c;
            for (int b = 0; b < 2; b++)
                band_divisor((unsigned)(bd.hi[a][sd][b] - bd.lo[a][sd][b] + 1), bd.dm[a][sd][b], bd.dl[a][sd][b]);
        }
    if (bd.count >= (1LL << 31)) return fail(SMI_ERR_UNSUPPORTED, "boundary bands of one step exceed 2^31 values");
    if (sizes_only) {
        // the set-up arena of a call: host inputs copied to the device, the
        // extended model, CPML tables, stencils and the box tables
        size_t b = 2 * (size_t)g.ntot * 4 + 64;
        b += (is_device_ptr(m->vp) ? 0 : (size_t)g.nphys * 4) + (is_device_ptr(m->rho) ? 0 : (size_t)g.nphys * 4);
        b += is_device_ptr(w->stf) ? 0 : (size_t)w->nt * 4;
        for (int a = 0; a < m->ndim; a++) b += 16 * (size_t)g.ne[a];
        b += sizeof(Stencil) * (size_t)(S.nshot + std::max<long long>(1, S.nrec_total));
        b += 2 * 6 * 4 * (size_t)S.nshot * (S.nt_fwd + 2);
        S.setup_bytes = b;
        return SMI_OK;
    }


    // inputs on the device
    const size_t nphys = (size_t)g.nphys;
    int rc = classify_and_upload(ar, m->vp, nphys, &S.vp, st);
    if (!rc) rc = classify_and_upload(ar, m->rho, nphys, &S.rho, st);
    if (!rc) rc = classify_and_upload(ar, w->stf, (size_t)w->nt, &S.stf, st);
    if (rc) return rc;

    // vmin / vmax (and rho positivity) on the device
    float *mm = ar.get<float>(4);
    unsigned *tmp = ar.get<unsigned>(4);
    if (!mm || !tmp) return fail(SMI_ERR_NOMEM, "device allocation failed");
    LaunchCtx lc{st, launches};
    launch_minmax(lc, S.vp, g.nphys, mm, tmp);
    launch_minmax(lc, S.rho, g.nphys, mm + 2, tmp + 2);
    float hm[4];
    if (cudaMemcpyAsync(hm, mm, sizeof hm, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(SMI_ERR_CUDA, "model reduction failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (!(hm[0] > 0.0f) || !(hm[2] > 0.0f) || !std::isfinite(hm[1]) || !std::isfinite(hm[3]))
        return fail(SMI_ERR_ARG, "vp and rho must be positive and finite");
    S.vmin = hm[0];
    S.vmax = hm[1];
    g.vdt = (double)S.vmax * w->dt;
    // Sec. 4.2: dr = 5 vmax / vmin, read as the largest ratio that keeps the
    // stored boundary above its Nyquist rate
    if (S.dr > 1 && (double)S.dr > 5.0 * (double)S.vmax / (double)S.vmin)
        return fail(SMI_ERR_ARG, "dr = %d exceeds 5 vmax / vmin = %.2f (Sec. 4.2)", S.dr,
                    5.0 * (double)S.vmax / (double)S.vmin);
    const double cfl = cfl_number(m->ndim, hh, w->dt, S.vmax, N);
    if (cfl > 1.0) return fail(SMI_ERR_CFL, "CFL number %.4f exceeds 1 (Eq. cfl)", cfl);
    if (w->fm > 0.0) {
        const double ppw = points_per_wavelength(m->ndim, hh, S.vmin, w->fm);
        const double need = N >= 4 ? 4.0 : 5.0;
        if (ppw < need)
            return fail(SMI_ERR_DISPERSION, "%.2f points per shortest wavelength, order %d needs %.0f",
                        ppw, o->order, need);
    }

    // CPML tables
    const double R = o->cpml_R > 0.0 ? o->cpml_R : 1e-3;
    const double kb = o->kaiser_b > 0.0 ? o->kaiser_b : 4.0;
    for (int a = 0; a < m->ndim; a++) {
        std::vector<float> tab(4 * (size_t)g.ne[a]);
        cpml_tables(g.ne[a], o->nb, hh[a], S.vmax, w->fm, R, w->dt, false, tab.data(), tab.data() + g.ne[a]);
        cpml_tables(g.ne[a], o->nb, hh[a], S.vmax, w->fm, R, w->dt, true, tab.data() + 2 * g.ne[a],
                    tab.data() + 3 * g.ne[a]);
        if (a == 0 && g.freesurf)              // the top layer is the image zone: no absorption
            for (int q = 0; q < 4; q++)
                for (int i = 0; i < g.L[0]; i++) tab[(size_t)q * g.ne[0] + i] = 0.0f;
        float *d = ar.get<float>(tab.size());
        if (!d) return fail(SMI_ERR_NOMEM, "device allocation failed");
        cudaMemcpyAsync(d, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        g.cpa[a] = d;
        g.cpb[a] = d + g.ne[a];
        g.cva[a] = d + 2 * g.ne[a];
        g.cvb[a] = d + 3 * g.ne[a];
    }
    for (int a = m->ndim; a < 3; a++) g.cpa[a] = g.cpb[a] = g.cva[a] = g.cvb[a] = nullptr;

    // extended model
    float *K = ar.get<float>((size_t)g.ntot), *rho_e = ar.get<float>((size_t)g.ntot);
    if (!K || !rho_e) return fail(SMI_ERR_NOMEM, "device allocation of the extended model failed");
    g.K = K;
    g.rho = rho_e;
    launch_extend_model(lc, g, S.vp, S.rho, S.n[0], S.n[1], S.n[2], K, rho_e);

    // stencils and box extents
    S.src_st.resize(S.nshot);
    S.rec_st.resize((size_t)S.nrec_total);
    S.box_src.resize(6 * (size_t)S.nshot);
    S.box_rec.resize(6 * (size_t)S.nshot);
    for (int s = 0; s < S.nshot; s++) {
        if (!make_stencil(g, geo->src + 3 * s, kb, &S.src_st[s]))
            return fail(SMI_ERR_ARG, "source %d lies outside the model or its stencil leaves the grid", s);
        int lo[3], hi[3];
        stencil_extent(g, S.src_st[s], lo, hi);
        for (int a = 0; a < 3; a++) {
            S.box_src[6 * s + a] = lo[a];
            S.box_src[6 * s + 3 + a] = hi[a];
        }
        int rlo[3] = {1 << 30, 1 << 30, 1 << 30}, rhi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
        for (int r = S.rec_offset[s]; r < S.rec_offset[s + 1]; r++) {
            if (!make_stencil(g, geo->rec + 3 * (size_t)r, kb, &S.rec_st[r]))
                return fail(SMI_ERR_ARG, "receiver %d lies outside the model or its stencil leaves the grid", r);
            stencil_extent(g, S.rec_st[r], lo, hi);
            for (int a = 0; a < 3; a++) {
                rlo[a] = std::min(rlo[a], lo[a]);
                rhi[a] = std::max(rhi[a], hi[a]);
            }
        }
        if (S.rec_offset[s + 1] == S.rec_offset[s])   // no receivers: empty adjoint box seed
            for (int a = 0; a < 3; a++) { rlo[a] = lo[a]; rhi[a] = hi[a]; }
        for (int a = 0; a < 3; a++) {
            S.box_rec[6 * s + a] = rlo[a];
            S.box_rec[6 * s + 3 + a] = rhi[a];
        }
    }
    S.d_src = ar.get<Stencil>(S.nshot);
    S.d_rec = ar.get<Stencil>(std::max<size_t>(1, (size_t)S.nrec_total));
    S.d_box_src = ar.get<int>(6 * (size_t)S.nshot);
    S.d_box_rec = ar.get<int>(6 * (size_t)S.nshot);
    if (!ar.ok) return fail(SMI_ERR_NOMEM, "device allocation failed");
    cudaMemcpyAsync(S.d_src, S.src_st.data(), sizeof(Stencil) * S.nshot, cudaMemcpyHostToDevice, st);
    if (S.nrec_total)
        cudaMemcpyAsync(S.d_rec, S.rec_st.data(), sizeof(Stencil) * S.nrec_total, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(S.d_box_src, S.box_src.data(), sizeof(int) * 6 * S.nshot, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(S.d_box_rec, S.box_rec.data(), sizeof(int) * 6 * S.nshot, cudaMemcpyHostToDevice, st);
    // the computing box of every step, evaluated once on the device
    S.d_tab_src = ar.get<int>((size_t)S.nshot * (S.nt_fwd + 1) * 6);
    S.d_tab_rec = ar.get<int>((size_t)S.nshot * (S.nt_fwd + 1) * 6);
    if (!ar.ok) return fail(SMI_ERR_NOMEM, "device allocation failed");
    launch_box_fill(lc, g, S.d_box_src, S.nshot, S.nt_fwd, S.d_tab_src);
    launch_box_fill(lc, g, S.d_box_rec, S.nshot, S.nt_fwd, S.d_tab_rec);
    double dV = 1.0;
    for (int a = 0; a < m->ndim; a++) dV *= hh[a];
    S.src_scale = w->dt / dV;

    return SMI_OK;
}

size_t band_bytes(int prec) { return prec == SMI_PREC_F32 ? 4 : 2; }

// Device bytes of one shot in a batch.
size_t per_shot_bytes(const Setup &S, int kind)
{
    const Grid &g = S.g;
    const size_t fields = (size_t)(1 + g.ndim) * g.ntot * 4;
    const int nbuf = S.fused ? 2 : 1;          // the single-pass step reads one state buffer, writes the other
    size_t slabs = 0;
    for (int a = 0; a < g.ndim; a++) slabs += 2 * (size_t)(S.fullmem && a < 2 ? g.ntot : g.slab_n[a]) * 4;
    long long maxrec = 0;                      // receivers of the largest shot
    for (int k = 0; k < S.nshot; k++) maxrec = std::max<long long>(maxrec, S.rec_offset[k + 1] - S.rec_offset[k]);
    size_t b = nbuf * (fields + slabs) + (size_t)S.nt * maxrec * 4;
    if (kind != 0) {
        b += nbuf * fields;                                            // adjoint fields
        if (kind != 5) {
            b += (size_t)S.nsamp * S.bands.count * band_bytes(S.bands.prec);   // saved bands
            b += (size_t)S.nsamp * 6 * 4;                                  // band scales
        }
        if (S.dr > 1) b += fields;                                     // state kept during the continuation
        b += (size_t)g.nphys * 4 * (kind == 1 && S.img_norm ? 2 : 1);  // accumulator (+ illumination)
        if (S.rho_grad) b += (size_t)g.ndim * g.ntot * 4;              // velocities of the previous step
        b += (size_t)S.nt * maxrec * 4 * 2;                            // seis + residual
    }
    return b;
}

struct Timer {
    bool on = false;
    cudaStream_t st{};
    std::vector<cudaEvent_t> ev;   // pairs
    std::vector<int> cls;
    size_t used = 0;
    void begin(int c)
    {
        if (!on) return;
        if (used + 2 > ev.size()) {
            for (int k = 0; k < 2; k++) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ev.push_back(e);
            }
        }
        cudaEventRecord(ev[used], st);
        cls.push_back(c);
    }
    void end()
    {
        if (!on) return;
        cudaEventRecord(ev[used + 1], st);
        used += 2;
    }
    void collect(smi_stats &s)
    {
        for (size_t i = 0; i + 1 < used; i += 2) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            s.ms[cls[i / 2]] += ms;
        }
    }
    ~Timer()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// Algorithmic bytes and point updates of one stencil step of one shot.
void account(const Grid &g, const int lo[3], const int hi[3], int cls, smi_stats &s)
{
    long long w[3];
    for (int a = 0; a < 3; a++) w[a] = std::max(0, hi[a] - lo[a] + 1);
    const double vol = (double)w[0] * w[1] * w[2];
    if (vol <= 0) return;
    double bytes;
    if (cls == 2) {
        bytes = vol * (g.ndim == 3 ? 52.0 : 44.0);
    } else {
        bytes = vol * (g.ndim == 3 ? 40.0 : 32.0);
        for (int a = 0; a < g.ndim; a++) {
            // slab nodes of axis a inside the box: two memory variables r/w
            long long in = 0;
            for (int j = lo[a]; j <= hi[a]; j++) in += (j < g.nb || j >= g.ne[a] - g.nb - 1);
            bytes += 16.0 * (double)in * vol / (double)w[a];
        }
    }
    s.bytes[cls] += bytes;
    s.point_updates += vol;
    s.steps[cls] += 1;
}

int finish_stream(cudaStream_t st)
{
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SMI_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(e));
    return SMI_OK;
}

// kind: 0 forward, 1 rtm, 2 gradient, 3 vector-Jacobian product of the
// forward map with respect to vp (adjoint source given), 5 adjoint of the
// forward map with respect to the wavelet (adjoint source given; img_out
// receives nt floats; no forward run, no reconstruction).  family > 0 (kind
// 2): the gradient of parametrisation family 1 (Vp, rho) or 2 (Vp, Ip), of
// the logarithms when logp, into img_out and img2_out.
// kind 6: forward modelling with boundary saving that writes the seismograms
// and keeps its state in *tape_out (one batch of all shots); kind 7: the
// reverse pass of kind 3 (vector-Jacobian product) from tape_in, no forward
// run.
int run(int kind, const smi_model *m, const smi_geometry *geo, const smi_wavelet *w, const smi_opts *o,
        const float *dobs, float *seis_out, float *img_out, double *misfit_out, float *img2_out = nullptr,
        int family = 0, int logp = 0, TapeState *tape_out = nullptr, TapeState *tape_in = nullptr)
{
    t_err.clear();
    memset(&t_stats, 0, sizeof t_stats);
    if (!o) return fail(SMI_ERR_ARG, "null options");
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    long long launches = 0;
    Setup S;
    int rc = SMI_OK;
    {
        Arena ar(st);
        if (kind == 7) S = tape_in->S;        // set-up kept by the tape
        else rc = validate_and_setup(m, geo, w, o, ar, st, &launches, S);
        if (rc) {
            cudaStreamSynchronize(st);
            return rc;
        }
        const Grid &g = S.g;
        LaunchCtx lc{st, &launches};
        const bool out_seis = kind == 0 || kind == 6;   // the call writes seismograms
        const size_t nseis = (size_t)S.nt * S.nrec_total;
        S.rho_grad = kind == 2 && family > 0;
        // per-shot results: images / gradients [nshot][nphys], misfits [nshot]
        const bool per_shot = o->per_shot != 0 && (kind == 1 || kind == 2);
        if (o->per_shot && kind != 0 && (!per_shot || S.rho_grad || (kind == 1 && S.img_norm)))
            return fail(SMI_ERR_ARG, "per_shot: smi_rtm without img_norm and smi_fwi_gradient only");
        const size_t nimg = kind == 5 ? (size_t)S.nt : (size_t)g.nphys * (per_shot ? S.nshot : 1);   // floats of img_out
        const int nmis = per_shot ? S.nshot : 1;       // misfit values
        if (out_seis && !seis_out) return fail(SMI_ERR_ARG, "seis is null");
        if (!out_seis && !dobs)
            return fail(SMI_ERR_ARG, kind == 3 || kind == 5 || kind == 7 ? "adj_src is null" : "dobs is null");
        if ((rc = check_same_device(seis_out, "seis")) || (rc = check_same_device(dobs, "dobs")) ||
            (rc = check_same_device(img_out, "image / gradient")) || (rc = check_same_device(img2_out, "grad2")) ||
            (rc = check_same_device(misfit_out, "misfit")))
            return rc;

        // outputs and observed data on the device
        float *d_seis_out = nullptr, *d_img = nullptr;
        const float *d_dobs = nullptr;
        double *d_misfit = ar.get<double>((size_t)nmis);
        if (!d_misfit) return fail(SMI_ERR_NOMEM, "device allocation failed");
        launch_zero(lc, d_misfit, sizeof(double) * nmis);
        if (out_seis) {
            d_seis_out = is_device_ptr(seis_out) ? seis_out : ar.get<float>(nseis);
        } else {
            rc = classify_and_upload(ar, dobs, nseis, &d_dobs, st);
            if (rc) return rc;
            if (img_out) d_img = is_device_ptr(img_out) ? img_out : ar.get<float>(nimg);
            else d_img = ar.get<float>(nimg);
        }
        double *d_series = kind == 5 ? ar.get<double>((size_t)S.nt) : nullptr;   // wavelet adjoint (FP64)
        float *d_img2 = nullptr;
        RhoAcc R{};
        if (S.rho_grad) {
            d_img2 = is_device_ptr(img2_out) ? img2_out : ar.get<float>((size_t)g.nphys);
            for (int a = 0; a < g.ndim; a++) {
                R.G[a] = ar.get<float>((size_t)g.ntot);
                if (R.G[a]) launch_zero(lc, R.G[a], sizeof(float) * g.ntot);
            }
        }
        if (!ar.ok) return fail(SMI_ERR_NOMEM, "device allocation of outputs failed");

        // batch size by device memory
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t per = std::max<size_t>(per_shot_bytes(S, kind), 1);
        int B = (int)std::max<size_t>(1, (size_t)(0.8 * (double)free_b) / per);
        B = std::min(B, S.nshot);
        if (o->max_batch > 0) B = std::min(B, o->max_batch);
        if (kind == 6 && B < S.nshot)
            return fail(SMI_ERR_NOMEM, "a tape keeps every shot's state on the device: %d of %d shots fit", B, S.nshot);
        if (kind == 7) B = S.nshot;

        Timer tm;
        tm.on = o->profile != 0;
        tm.st = st;
        unsigned *d_flag = ar.get<unsigned>(1);
        unsigned *d_wait = ar.get<unsigned>(1);
        unsigned *d_absmax = ar.get<unsigned>(6 * (size_t)B);
        if (!ar.ok) return fail(SMI_ERR_NOMEM, "device allocation failed");
        launch_zero(lc, d_flag, sizeof(unsigned));
        launch_zero(lc, d_wait, sizeof(unsigned));
        const bool fast3 = o->kernels != SMI_KERNELS_GENERIC && stencil3d_supported(g);
        const bool fast2 = o->kernels != SMI_KERNELS_GENERIC && stencil2d_supported(g);
        const bool fused = S.fused;
        const bool inl = S.inline3;            // two-pass 3D kernels with the z / x CPML terms inline
        const bool norm = kind == 1 && S.img_norm;       // normalised RTM image

        size_t batch_peak = 0;                   // largest batch arena (fields, bands, accumulators)
        for (int s0 = 0; s0 < S.nshot; s0 += B) {
            const int nb_shot = std::min(B, S.nshot - s0);
            // per-batch tables
            std::vector<int> roff(nb_shot + 1);
            std::vector<long long> soff(nb_shot);
            int max_rec = 0;
            for (int s = 0; s <= nb_shot; s++) roff[s] = S.rec_offset[s0 + s] - S.rec_offset[s0];
            for (int s = 0; s < nb_shot; s++) {
                soff[s] = (long long)S.nt * roff[s];
                max_rec = std::max(max_rec, roff[s + 1] - roff[s]);
            }
            const long long batch_seis = (long long)S.nt * roff[nb_shot];
            if (kind == 7) {
                roff = tape_in->roff;
                soff = tape_in->soff;
                max_rec = tape_in->max_rec;
            }
            Arena ba(st);
            int *d_roff = ba.get<int>(roff.size());
            long long *d_soff = ba.get<long long>(soff.size());
            // F, A: the current source-field and adjoint states; with the
            // single-pass step, F2 and A2 are the buffers it writes (swapped
            // after every step).  Memory variables of the single-pass step:
            // z and x full-size, y in the y-slab layout.
            Fields F{}, A{}, F2{}, A2{};
            auto mem_n = [&](int a) { return (size_t)(S.fullmem && a < 2 ? g.ntot : g.slab_n[a]) * nb_shot; };
            for (Fields *f : {&F, &F2}) {
                if ((f == &F2 && !fused) || kind == 7) break;
                f->p = ba.get<float>((size_t)g.ntot * nb_shot);
                for (int a = 0; a < g.ndim; a++) {
                    f->v[a] = ba.get<float>((size_t)g.ntot * nb_shot);
                    f->psip[a] = ba.get<float>(mem_n(a));
                    f->psiv[a] = ba.get<float>(mem_n(a));
                }
            }
            float *seis = out_seis ? d_seis_out + (size_t)S.nt * S.rec_offset[s0]
                                   : ba.get<float>(std::max<long long>(1, batch_seis));
            Bands bd = S.bands;
            float *res = nullptr, *acc = nullptr, *keep = nullptr;
            unsigned *norm_mx = nullptr;
            double *partials = nullptr, *part = nullptr;
            const int npart = 256;
            if (kind == 7) {                                 // the state the forward call kept
                const TapeState &T = *tape_in;
                F = T.F; F2 = T.F2; A = T.A; A2 = T.A2;
                bd = T.bd;
                res = T.res;
                acc = T.acc;
                partials = T.partials;
            } else if (kind != 0) {
                for (int k = 0; k < (fused ? 2 : 1); k++) {   // the adjoint reuses the forward's memory variables
                    Fields &a_ = k ? A2 : A;
                    const Fields &f_ = k ? F2 : F;
                    a_.p = ba.get<float>((size_t)g.ntot * nb_shot);
                    for (int a = 0; a < g.ndim; a++) {
                        a_.v[a] = ba.get<float>((size_t)g.ntot * nb_shot);
                        a_.psip[a] = f_.psip[a];
                        a_.psiv[a] = f_.psiv[a];
                    }
                }
                if (kind != 5) {
                    bd.data = ba.raw((size_t)nb_shot * S.nsamp * bd.count * band_bytes(bd.prec));
                    bd.scale = ba.get<float>((size_t)nb_shot * S.nsamp * 6);
                    if (S.dr > 1) keep = ba.get<float>((size_t)(1 + g.ndim) * g.ntot * nb_shot);
                    acc = ba.get<float>((size_t)g.nphys * nb_shot * (norm ? 2 : 1));   // [images | illuminations]
                } else {
                    part = ba.get<double>((size_t)nb_shot * S.nt);
                }
                res = ba.get<float>(std::max<long long>(1, batch_seis));
                if (norm) norm_mx = ba.get<unsigned>(nb_shot);
                partials = ba.get<double>(npart);
                if (S.rho_grad)
                    for (int a = 0; a < g.ndim; a++) R.vprev[a] = ba.get<float>((size_t)g.ntot * nb_shot);
            }
            if (!ba.ok) return fail(SMI_ERR_NOMEM, "device allocation for a batch of %d shots failed", nb_shot);
            batch_peak = std::max(batch_peak, ba.peak);
            if (kind == 7) {
                d_roff = tape_in->d_roff;
                d_soff = tape_in->d_soff;
            } else {
                cudaMemcpyAsync(d_roff, roff.data(), sizeof(int) * roff.size(), cudaMemcpyHostToDevice, st);
                cudaMemcpyAsync(d_soff, soff.data(), sizeof(long long) * soff.size(), cudaMemcpyHostToDevice, st);
            }
            Maps3 mF{}, mA{}, mF2{}, mA2{};
            if (fast3 && (!make_maps3(mF, g, F, nb_shot, S.fullmem) ||
                          (kind != 0 && !make_maps3(mA, g, A, nb_shot, S.fullmem))))
                return fail(SMI_ERR_CUDA, "tensor map encoding failed");
            MapsF fF{}, fF2{}, fA{}, fA2{};
            MapsM fM{};
            if (fused && (!make_maps3(mF2, g, F2, nb_shot, true) || !make_maps_fused(fF, g, F, nb_shot) ||
                          !make_maps_fused(fF2, g, F2, nb_shot) || !make_maps_model(fM, g) ||
                          (kind != 0 && (!make_maps3(mA2, g, A2, nb_shot, true) || !make_maps_fused(fA, g, A, nb_shot) ||
                                         !make_maps_fused(fA2, g, A2, nb_shot)))))
                return fail(SMI_ERR_CUDA, "tensor map encoding failed");
            // after a single-pass step the written buffers become the current ones
            auto swap_F = [&] {
                std::swap(F, F2);
                std::swap(mF, mF2);
                std::swap(fF, fF2);
            };
            auto swap_A = [&] {
                std::swap(A, A2);
                std::swap(mA, mA2);
                std::swap(fA, fA2);
            };
            Batch b{};
            b.nshot = nb_shot;
            b.box_src = S.d_box_src + 6 * s0;
            b.box_rec = S.d_box_rec + 6 * s0;
            b.src = S.d_src + s0;
            b.rec = S.d_rec + S.rec_offset[s0];
            b.rec_off = d_roff;
            b.max_rec = max_rec;
            b.tab_src = S.d_tab_src + (size_t)s0 * (S.nt + 1) * 6;
            b.tab_rec = S.d_tab_rec + (size_t)s0 * (S.nt + 1) * 6;
            b.nt1 = S.nt_fwd + 1;
            // union of the batch's boxes after n steps (bounds the CPML launches)
            auto batch_box = [&](const std::vector<int> &ext, int n, int lo[3], int hi[3]) {
                for (int a = 0; a < 3; a++) {
                    lo[a] = INT_MAX;
                    hi[a] = INT_MIN;
                }
                for (int s = 0; s < nb_shot; s++) {
                    int l[3], h[3];
                    box_bounds(g, ext.data() + 6 * (s0 + s), n, l, h);
                    for (int a = 0; a < 3; a++) {
                        lo[a] = std::min(lo[a], l[a]);
                        hi[a] = std::max(hi[a], h[a]);
                    }
                }
            };
            for (const Fields *f : {&F, &F2}) {
                if ((f == &F2 && !fused) || kind == 7) break;
                launch_zero(lc, f->p, sizeof(float) * g.ntot * nb_shot);
                for (int a = 0; a < g.ndim; a++) {
                    launch_zero(lc, f->v[a], sizeof(float) * g.ntot * nb_shot);
                    launch_zero(lc, f->psip[a], sizeof(float) * mem_n(a));
                    launch_zero(lc, f->psiv[a], sizeof(float) * mem_n(a));
                }
            }

            // ---- forward loop (Algorithm 2) ----
            // With dr > 1 the loop continues past nt-1 without a source until
            // the last stored sample (every time-interpolation window of the
            // reverse loop complete); the state after step nt-1 is kept.
            const size_t fbytes = sizeof(float) * g.ntot * nb_shot;
            const int nsteps = kind == 5 || kind == 7 ? 0 : kind != 0 ? S.nt_fwd : S.nt;
            for (int it = 0; it < nsteps; it++) {
                if (kind != 0 && it % S.dr == 0) launch_save_bands(lc, g, b, F, bd, it / S.dr, d_absmax);
                tm.begin(0);
                int blo[3], bhi[3];
                batch_box(S.box_src, it, blo, bhi);
                // free surface (no-ops without): the v_z mirror after the velocity
                // update, the p mirror after the pressure update and the source
                if (fused) {
                    launch3_fused(lc, fF, fM, g, b, F, F2, it, 0, d_wait);
                    swap_F();
                } else if (fast3) {
                    launch3_v(lc, mF, g, b, F, it, 0, d_wait, inl);
                    if (!inl) launch_fwd_corrections(lc, g, b, F, it, true, blo, bhi);
                    launch_free_surface(lc, g, F.v[0], nb_shot, kFsMirrorV);
                    launch3_p(lc, mF, nullptr, g, b, F, it, 0, d_wait, nullptr, 0, nullptr, 0.0f, inl);
                    if (!inl) launch_fwd_corrections(lc, g, b, F, it, false, blo, bhi);
                } else if (fast2) {                    // CPML and (it < nt) the source inline
                    launch2_v(lc, g, b, F, it, 0, blo, bhi);
                    launch_free_surface(lc, g, F.v[0], nb_shot, kFsMirrorV);
                    launch2_p(lc, g, b, F, it, 0, blo, bhi, nullptr, nullptr, 0, it < S.nt ? S.stf : nullptr,
                              (float)S.src_scale);
                } else {
                    const long long work = box_points(blo, bhi);
                    launch_fwd_v(lc, g, b, F, it, work);
                    launch_free_surface(lc, g, F.v[0], nb_shot, kFsMirrorV);
                    launch_fwd_p(lc, g, b, F, it, work);
                }
                tm.end();
                if (it < S.nt && !fast2) launch_inject_source(lc, g, b, F.p, S.stf, it, (float)S.src_scale);
                launch_free_surface(lc, g, F.p, nb_shot, kFsMirrorP);
                if (it < S.nt && max_rec > 0) launch_gather(lc, g, b, F.p, seis, d_soff, S.nt, it);
                for (int s = 0; s < nb_shot; s++) {
                    int lo[3], hi[3];
                    box_bounds(g, S.box_src.data() + 6 * (s0 + s), it, lo, hi);
                    account(g, lo, hi, 0, t_stats);
                }
                if (keep && it == S.nt - 1) {
                    cudaMemcpyAsync(keep, F.p, fbytes, cudaMemcpyDeviceToDevice, st);
                    for (int a = 0; a < g.ndim; a++)
                        cudaMemcpyAsync(keep + (size_t)(1 + a) * g.ntot * nb_shot, F.v[a], fbytes,
                                        cudaMemcpyDeviceToDevice, st);
                }
            }
            if (keep) {
                cudaMemcpyAsync(F.p, keep, fbytes, cudaMemcpyDeviceToDevice, st);
                for (int a = 0; a < g.ndim; a++)
                    cudaMemcpyAsync(F.v[a], keep + (size_t)(1 + a) * g.ntot * nb_shot, fbytes,
                                    cudaMemcpyDeviceToDevice, st);
            }
            if (batch_seis > 0 && kind != 5 && kind != 7) launch_nonfinite(lc, seis, batch_seis, d_flag);
            launch_nonfinite(lc, F.p, g.ntot * nb_shot, d_flag);
            if (kind == 0) continue;
            if (kind == 6) {                       // keep the state for the reverse pass
                TapeState &T = *tape_out;
                T.F = F; T.F2 = F2; T.A = A; T.A2 = A2;
                T.bd = bd;
                T.res = res;
                T.acc = acc;
                T.partials = partials;
                T.d_roff = d_roff;
                T.d_soff = d_soff;
                T.roff = roff;
                T.soff = soff;
                T.max_rec = max_rec;
                T.batch_seis = batch_seis;
                batch_peak = std::max(batch_peak, ba.peak);
                ba.release_to(T.mem);
                continue;
            }

            // ---- residual, misfit ----
            if (batch_seis > 0 && per_shot && kind == 2) {
                // one residual and FP64 sum per shot: the same launches as the shot alone
                const float *dob = d_dobs + (size_t)S.nt * S.rec_offset[s0];
                for (int s = 0; s < nb_shot; s++) {
                    const long long ns = (long long)S.nt * (roff[s + 1] - roff[s]);
                    if (ns <= 0) continue;
                    launch_residual(lc, seis + soff[s], dob + soff[s], ns, 0, res + soff[s], partials, npart);
                    launch_sum_partials(lc, partials, npart, d_misfit + s0 + s);
                }
            } else if (batch_seis > 0) {
                const float *dob = d_dobs + (size_t)S.nt * S.rec_offset[s0];
                launch_residual(lc, kind == 5 || kind == 7 ? dob : seis, dob, batch_seis, kind == 2 ? 0 : 1, res,
                                partials, npart);
                if (kind == 2) launch_sum_partials(lc, partials, npart, d_misfit);
            }
            // ---- reverse loop ----
            for (const Fields *f : {&A, &A2}) {
                if (f == &A2 && !fused) break;
                launch_zero(lc, f->p, sizeof(float) * g.ntot * nb_shot);
                for (int a = 0; a < g.ndim; a++) {
                    launch_zero(lc, f->v[a], sizeof(float) * g.ntot * nb_shot);
                    launch_zero(lc, f->psip[a], sizeof(float) * mem_n(a));
                    launch_zero(lc, f->psiv[a], sizeof(float) * mem_n(a));
                }
            }
            if (acc) launch_zero(lc, acc, sizeof(float) * g.nphys * nb_shot * (norm ? 2 : 1));
            if (S.rho_grad)
                for (int a = 0; a < g.ndim; a++)
                    cudaMemcpyAsync(R.vprev[a], F.v[a], fbytes, cudaMemcpyDeviceToDevice, st);
            // 0: gradient, 1: image, 2: image and source illumination
            const int mode = (kind == 2 || kind == 3 || kind == 7) ? 0 : (norm ? 2 : 1);
            // one reverse step of the source field (reconstruction with the fused
            // imaging / gradient accumulation), then its boundary re-imposed
            auto reconstruct = [&](int it) {
                tm.begin(2);
                if (fast3) {
                    launch3_p(lc, mF, &mA, g, b, F, it, 2, d_wait, acc, mode, S.stf, (float)S.src_scale, false);
                    launch_free_surface(lc, g, F.p, nb_shot, kFsMirrorP);
                    launch3_v(lc, mF, g, b, F, it, 2, d_wait, false);
                } else {
                    int blo[3], bhi[3];
                    batch_box(S.box_src, it, blo, bhi);
                    for (int a = 0; a < 3; a++) {        // reconstruction: box within the physical domain
                        blo[a] = std::max(blo[a], g.L[a]);
                        bhi[a] = std::min(bhi[a], g.H[a]);
                    }
                    if (fast2) {
                        launch2_p(lc, g, b, F, it, 2, blo, bhi, A.p, acc, mode, S.stf, (float)S.src_scale);
                        launch_free_surface(lc, g, F.p, nb_shot, kFsMirrorP);
                        launch2_v(lc, g, b, F, it, 2, blo, bhi);
                    } else {
                        const long long work = box_points(blo, bhi);
                        launch_recon_p(lc, g, b, F, A.p, acc, mode, S.stf, it, (float)S.src_scale, work);
                        launch_free_surface(lc, g, F.p, nb_shot, kFsMirrorP);
                        launch_recon_v(lc, g, b, F, it, work);
                    }
                }
                tm.end();
                if (S.dr == 1) launch_restore_bands(lc, g, b, F, bd, it);
                else launch_restore_bands_interp(lc, g, b, F, bd, time_weights(it, S.dr, S.nsamp));
            };
            for (int it = S.nt - 1; it >= 0; it--) {
                const int mrev = S.nt - 1 - it;
                if (max_rec > 0) launch_adj_inject(lc, g, b, A.p, res, d_soff, S.nt, it);
                // free surface (no-ops without): the transposed p mirror on the
                // adjoint before anything reads it; p = 0 again at the surface node
                // of the reversed source field; the transposed v_z mirror between
                // the two adjoint stages
                launch_free_surface(lc, g, A.p, nb_shot, kFsFoldP);
                if (kind == 5) launch_src_adjoint(lc, g, b, A.p, part, S.nt, it, S.src_scale);   // wavelet adjoint
                else reconstruct(it);
                tm.begin(1);
                int blo[3], bhi[3];
                batch_box(S.box_rec, mrev, blo, bhi);
                if (fused) {
                    launch3_fused(lc, fA, fM, g, b, A, A2, mrev, 1, d_wait);
                    swap_A();
                } else if (fast3) {
                    if (!inl) launch_adj_corrections(lc, g, b, A, mrev, true, blo, bhi);
                    launch3_v(lc, mA, g, b, A, mrev, 1, d_wait, inl);
                    launch_free_surface(lc, g, A.v[0], nb_shot, kFsFoldV);
                    if (!inl) launch_adj_corrections(lc, g, b, A, mrev, false, blo, bhi);
                    launch3_p(lc, mA, nullptr, g, b, A, mrev, 1, d_wait, nullptr, 0, nullptr, 0.0f, inl);
                } else if (fast2) {                    // transposed CPML inline in the 2D kernels
                    launch2_v(lc, g, b, A, mrev, 1, blo, bhi);
                    launch_free_surface(lc, g, A.v[0], nb_shot, kFsFoldV);
                    launch2_p(lc, g, b, A, mrev, 1, blo, bhi, nullptr, nullptr, 0, nullptr, 0.0f);
                } else {
                    const long long work = box_points(blo, bhi);
                    launch_adj_v(lc, g, b, A, mrev, work);
                    launch_free_surface(lc, g, A.v[0], nb_shot, kFsFoldV);
                    launch_adj_p(lc, g, b, A, mrev, work);
                }
                tm.end();
                if (S.rho_grad) {                      // half nodes touching the physical domain
                    IBox rb;
                    batch_box(S.box_src, it, rb.lo, rb.hi);
                    for (int a = 0; a < 3; a++) {
                        rb.lo[a] = std::max(rb.lo[a], a < g.ndim ? g.L[a] - 1 : 0);
                        rb.hi[a] = std::min(rb.hi[a], g.H[a]);
                    }
                    launch_rho_acc(lc, g, nb_shot, F, A, R, rb);
                }
                for (int s = 0; s < nb_shot; s++) {
                    int lo[3], hi[3];
                    box_bounds(g, S.box_rec.data() + 6 * (s0 + s), mrev, lo, hi);
                    account(g, lo, hi, 1, t_stats);
                    if (kind == 5) continue;
                    box_bounds(g, S.box_src.data() + 6 * (s0 + s), it, lo, hi);
                    for (int a = 0; a < 3; a++) {
                        lo[a] = std::max(lo[a], g.L[a]);
                        hi[a] = std::min(hi[a], g.H[a]);
                    }
                    account(g, lo, hi, 2, t_stats);
                }
            }
            if (kind == 5) {
                launch_sum_series(lc, part, nb_shot, S.nt, d_series, s0 > 0);
                continue;
            }
            launch_nonfinite(lc, acc, g.nphys * nb_shot, d_flag);
            if (per_shot)
                cudaMemcpyAsync(d_img + (size_t)s0 * g.nphys, acc, sizeof(float) * g.nphys * nb_shot,
                                cudaMemcpyDeviceToDevice, st);
            else if (norm) launch_reduce_norm(lc, g, acc, nb_shot, norm_mx, d_img, s0 > 0);
            else launch_reduce_shots(lc, g, acc, nb_shot, d_img, s0 > 0);
            // batch buffers are released (stream-ordered) when `ba` goes out of scope
        }
        if (S.rho_grad) launch_finalize_family(lc, g, S.vp, S.rho, d_img, R, family, logp, d_img, d_img2);
        else if (kind == 2 || kind == 3 || kind == 7)
            for (int s = 0; s < (per_shot ? S.nshot : 1); s++)
                launch_finalize_grad(lc, g.nphys, S.vp, g.dt, d_img + (size_t)s * g.nphys);
        else if (kind == 5) {
            launch_to_float(lc, d_series, S.nt, d_img);
            launch_nonfinite(lc, d_img, S.nt, d_flag);
        }

        // outputs back to the host where needed
        if (out_seis && d_seis_out != seis_out)
            cudaMemcpyAsync(seis_out, d_seis_out, nseis * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (!out_seis && img_out && d_img != img_out)
            cudaMemcpyAsync(img_out, d_img, nimg * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (d_img2 && d_img2 != img2_out)
            cudaMemcpyAsync(img2_out, d_img2, (size_t)g.nphys * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (kind == 2 && misfit_out) {
            cudaMemcpyAsync(misfit_out, d_misfit, sizeof(double) * nmis,
                            is_device_ptr(misfit_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        }
        unsigned flag = 0, waitflag = 0;
        cudaMemcpyAsync(&flag, d_flag, sizeof flag, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&waitflag, d_wait, sizeof waitflag, cudaMemcpyDeviceToHost, st);
        rc = finish_stream(st);
        if (!rc && waitflag) rc = fail(SMI_ERR_TIMEOUT, "a bounded wait for a tile copy gave up");
        if (!rc && flag) rc = fail(SMI_ERR_UNSTABLE, "non-finite values in the wavefield or outputs");
        tm.collect(t_stats);
        t_stats.kernel_launches = launches;
        t_stats.device_bytes = (double)(ar.peak + batch_peak);
        t_stats.band_values = kind == 0 || kind == 5 ? 0 : S.bands.count;
        if (kind == 6) {
            if (!rc) {
                tape_out->S = S;
                ar.release_to(tape_out->mem);      // the set-up tables stay with the tape
            } else {
                // the batch allocations were handed over: give them back to be freed
                for (auto &pr : tape_out->mem) cudaFreeAsync(pr.first, st);
                tape_out->mem.clear();
            }
        }
    }
    // the arena's frees are stream ordered; make them complete before return
    if (!rc) rc = finish_stream(st);
    return rc;
}

}  // namespace

// Error message of the calling thread, for entry points in other files.
void record_error(const char *msg) { t_err = msg; }

}  // namespace smi

using namespace smi;

struct smi_tape {
    TapeState st;
};

extern "C" {

void smi_opts_default(smi_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->order = 4;
    o->nb = 20;
    o->freesurf = 0;
    o->dr = 1;
    o->use_box = 1;
    o->shell_prec = SMI_PREC_F32;
    o->kaiser_b = 4.0;
    o->cpml_R = 1e-3;
    o->stream = nullptr;
    o->max_batch = 0;
    o->profile = 0;
    o->img_norm = 0;
    o->kernels = SMI_KERNELS_AUTO;
}

int smi_forward(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                const smi_opts *opts, float *seis)
{
    return run(0, model, geom, wav, opts, nullptr, seis, nullptr, nullptr);
}

int smi_rtm(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
            const smi_opts *opts, const float *dobs, float *image)
{
    if (!image) return fail(SMI_ERR_ARG, "image is null");
    return run(1, model, geom, wav, opts, dobs, nullptr, image, nullptr);
}

int smi_fwi_gradient(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                     const smi_opts *opts, const float *dobs, double *misfit, float *grad_vp)
{
    return run(2, model, geom, wav, opts, dobs, nullptr, grad_vp, misfit);
}

int smi_fwi_gradient_family(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                            const smi_opts *opts, const float *dobs, int family, int log_param, double *misfit,
                            float *grad1, float *grad2)
{
    if (family != 1 && family != 2) return fail(SMI_ERR_ARG, "family must be 1 (Vp, rho) or 2 (Vp, Ip)");
    if (log_param != 0 && log_param != 1) return fail(SMI_ERR_ARG, "log_param must be 0 or 1");
    if (!grad1 || !grad2) return fail(SMI_ERR_ARG, "gradient outputs are null");
    return run(2, model, geom, wav, opts, dobs, nullptr, grad1, misfit, grad2, family, log_param);
}

int smi_forward_vjp(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                    const smi_opts *opts, const float *adj_src, float *grad_vp)
{
    if (!grad_vp) return fail(SMI_ERR_ARG, "grad_vp is null");
    return run(3, model, geom, wav, opts, adj_src, nullptr, grad_vp, nullptr);
}

int smi_forward_tape(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                     const smi_opts *opts, float *seis, smi_tape **tape)
{
    if (!tape) return fail(SMI_ERR_ARG, "tape is null");
    *tape = nullptr;
    if (!opts) return fail(SMI_ERR_ARG, "null options");
    auto *t = new smi_tape();
    const int rc = run(6, model, geom, wav, opts, nullptr, seis, nullptr, nullptr, nullptr, 0, 0, &t->st, nullptr);
    if (rc) {
        delete t;
        return rc;
    }
    t->st.o = *opts;
    *tape = t;
    return SMI_OK;
}

int smi_tape_vjp(smi_tape *tape, const float *adj_src, float *grad_vp, void *stream)
{
    if (!tape || !grad_vp) return fail(SMI_ERR_ARG, "null argument");
    if (tape->st.done) return fail(SMI_ERR_ARG, "this tape's reverse pass has already run (a tape serves one)");
    smi_opts o = tape->st.o;
    o.stream = stream;
    const int rc = run(7, nullptr, nullptr, nullptr, &o, adj_src, nullptr, grad_vp, nullptr, nullptr, 0, 0, nullptr,
                       &tape->st);
    tape->st.done = true;                  // the reverse pass consumed the kept source field
    return rc;
}

void smi_tape_free(smi_tape *tape)
{
    if (!tape) return;
    for (auto &pr : tape->st.mem) cudaFree(pr.first);
    delete tape;
}

int smi_forward_adjoint(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                        const smi_opts *opts, const float *adj_src, float *stf_adj)
{
    if (!stf_adj) return fail(SMI_ERR_ARG, "stf_adj is null");
    return run(5, model, geom, wav, opts, adj_src, nullptr, stf_adj, nullptr);
}

int smi_dot(const float *a, const float *b, size_t n, double *out, void *stream)
{
    t_err.clear();
    if (!out || (n > 0 && (!a || !b))) return fail(SMI_ERR_ARG, "null argument");
    if (n > 0 && (!is_device_ptr(a) || !is_device_ptr(b)))
        return fail(SMI_ERR_ARG, "smi_dot needs device arrays");
    int rc;
    if ((rc = check_same_device(a, "a")) || (rc = check_same_device(b, "b")) || (rc = check_same_device(out, "out")))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long launches = 0;
    LaunchCtx lc{st, &launches};
    {
        Arena ar(st);
        const int npart = 512;
        double *partials = ar.get<double>(npart), *d_out = ar.get<double>(1);
        if (!ar.ok) return fail(SMI_ERR_NOMEM, "device allocation failed");
        launch_zero(lc, d_out, sizeof(double));
        if (n > 0) {
            launch_dot(lc, a, b, (long long)n, partials, npart);
            launch_sum_partials(lc, partials, npart, d_out);
        }
        cudaMemcpyAsync(out, d_out, sizeof(double), is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st);
        rc = finish_stream(st);
    }
    int rc2 = finish_stream(st);
    return rc ? rc : rc2;
}

int smi_query(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
              const smi_opts *opts, int kind, size_t *seis_elems, size_t *image_elems,
              size_t *device_bytes)
{
    t_err.clear();
    if (!opts) return fail(SMI_ERR_ARG, "null options");
    if (kind < 0 || kind > 4) return fail(SMI_ERR_ARG, "kind must be 0 .. 4");
    cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
    long long launches = 0;
    Setup S;
    int rc;
    {
        Arena ar(st);
        rc = validate_and_setup(model, geom, wav, opts, ar, st, &launches, S);
        if (!rc) {
            if (seis_elems) *seis_elems = (size_t)S.nt * S.nrec_total;
            if (image_elems)
                *image_elems = (size_t)S.g.nphys * (opts->per_shot && (kind == 1 || kind == 2) ? S.nshot : 1);
            if (device_bytes) {
                int B = S.nshot;
                if (opts->max_batch > 0) B = std::min(B, opts->max_batch);
                S.rho_grad = kind == 4;
                size_t extra = kind == 4 ? (size_t)S.g.ndim * S.g.ntot * 4 + (size_t)S.g.nphys * 4 : 0;
                *device_bytes = ar.peak + extra + (size_t)B * per_shot_bytes(S, kind == 4 ? 2 : kind);
            }
        }
    }
    int rc2 = finish_stream(st);
    return rc ? rc : rc2;
}

int smi_footprint(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                  const smi_opts *opts, int kind, size_t *device_bytes)
{
    t_err.clear();
    if (!opts || !device_bytes) return fail(SMI_ERR_ARG, "null argument");
    if (kind < 0 || kind > 4) return fail(SMI_ERR_ARG, "kind must be 0 .. 4");
    Setup S;
    Arena ar(nullptr);                     // not used: the sizes-only set-up allocates nothing
    long long launches = 0;
    const int rc = validate_and_setup(model, geom, wav, opts, ar, nullptr, &launches, S, true);
    if (rc) return rc;
    int B = S.nshot;
    if (opts->max_batch > 0) B = std::min(B, opts->max_batch);
    S.rho_grad = kind == 4;
    const size_t extra = kind == 4 ? (size_t)S.g.ndim * S.g.ntot * 4 + (size_t)S.g.nphys * 4 : 0;
    *device_bytes = S.setup_bytes + extra + (size_t)B * per_shot_bytes(S, kind == 4 ? 2 : kind);
    return SMI_OK;
}

int smi_box_table(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                  const smi_opts *opts, int shot, int which, int n0, int count, int *lo, int *hi)
{
    t_err.clear();
    if (!opts || !lo || !hi || count < 0) return fail(SMI_ERR_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
    long long launches = 0;
    Setup S;
    int rc;
    {
        Arena ar(st);
        rc = validate_and_setup(model, geom, wav, opts, ar, st, &launches, S);
        if (!rc && (shot < 0 || shot >= S.nshot || (which != 0 && which != 1)))
            rc = fail(SMI_ERR_ARG, "bad shot or which");
        if (!rc && count > 0) {
            int *d = ar.get<int>(6 * (size_t)count);
            if (!d) {
                rc = fail(SMI_ERR_NOMEM, "device allocation failed");
            } else {
                LaunchCtx lc{st, &launches};
                const int *ext = (which == 0 ? S.d_box_src : S.d_box_rec) + 6 * shot;
                launch_box_table(lc, S.g, ext, n0, count, d, d + 3 * (size_t)count);
                cudaMemcpyAsync(lo, d, sizeof(int) * 3 * count, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(hi, d + 3 * (size_t)count, sizeof(int) * 3 * count, cudaMemcpyDeviceToHost, st);
                rc = finish_stream(st);
            }
        }
    }
    int rc2 = finish_stream(st);
    return rc ? rc : rc2;
}

int smi_wait_check(void *stream, long long polls, double *ms)
{
    t_err.clear();
    if (polls < 0) polls = wait_polls_default();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long launches = 0;
    LaunchCtx lc{st, &launches};
    int rc;
    {
        Arena ar(st);
        unsigned *d_err = ar.get<unsigned>(1);
        if (!d_err) return fail(SMI_ERR_NOMEM, "device allocation failed");
        launch_zero(lc, d_err, sizeof(unsigned));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        launch_wait_check(lc, d_err, polls);
        cudaEventRecord(e1, st);
        unsigned h_err = 0;
        cudaMemcpyAsync(&h_err, d_err, sizeof h_err, cudaMemcpyDeviceToHost, st);
        rc = finish_stream(st);
        float t = 0.0f;
        if (!rc) cudaEventElapsedTime(&t, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (ms) *ms = t;
        if (!rc && h_err) rc = fail(SMI_ERR_TIMEOUT, "the bounded wait gave up after %lld polls (as designed)", polls);
    }
    int rc2 = finish_stream(st);
    return rc ? rc : rc2;
}

int smi_last_stats(smi_stats *st)
{
    if (!st) return fail(SMI_ERR_ARG, "null stats");
    *st = t_stats;
    return SMI_OK;
}

const char *smi_last_error(void) { return t_err.c_str(); }

const char *smi_version(void) { return "smi 0.1 sm_103a"; }

}  // extern "C"
