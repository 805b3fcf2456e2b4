// smi_internal.h -- data shared by the host driver (smi_api.cu, smi_setup.cpp)
// and the CUDA kernels (smi_kernels.cu) of libsmi.  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/smi.h"

namespace smi {

constexpr int kMaxHalf = 4;        // N = order/2 <= 4
constexpr int kMaxTaps = 8;        // 2 * ri, ri = order/2 <= 4

// Grid, scheme constants and read-only model arrays, passed by value to
// every kernel.  Axis 0 = z (fastest), 1 = x, 2 = y.
struct Grid {
    int ndim, N, ri, nb;
    int ne[3];             // extended sizes (1 for an inactive axis)
    int px;                // allocated row length along z: ne[0] rounded up to 8 (16-byte rows)
    int L[3], H[3];        // first/last physical node along each axis (extended index)
    long long ntot;        // allocated points of one extended field: px * ne[1] * ne[2]
    long long nphys;       // points of the physical grid
    int S;                 // slab length along its axis: 2*nb + 1
    long long slab_n[3];   // points of the slab array of axis a
    float dt;
    float c[3][kMaxHalf];  // a_l / h_a
    double vdt;            // vmax * dt (FP64, for the computing box)
    double h[3];           // spacings (FP64, for the computing box)
    int use_box;
    int freesurf;          // free surface on the top face (image method): the top layer is the image zone
    const float *K;        // bulk modulus rho*vp^2 on the extended grid
    const float *rho;      // density on the extended grid
    const float *cpa[3], *cpb[3];   // CPML a, b on the p grid of axis a (length ne[a])
    const float *cva[3], *cvb[3];   // CPML a, b on the v grid of axis a
};

// Interpolation stencil of one point: per axis a first node, a node count
// (1 on a node, 2*ri otherwise) and the 1D weights.
struct Stencil {
    int first[3];
    int cnt[3];
    float w[3][kMaxTaps];
};

// Shots propagated together in one launch (blockIdx.y / grid.z = shot).
struct Batch {
    int nshot;
    const int *box_src;     // [nshot][6] source stencil extent lo0,lo1,lo2,hi0,hi1,hi2
    const int *box_rec;     // [nshot][6] receiver stencil extent
    const Stencil *src;     // [nshot]
    const Stencil *rec;     // [nrec_total of the batch]
    const int *rec_off;     // [nshot+1] batch-local receiver offsets
    int max_rec;            // largest receiver count of a shot in the batch
    // Computing-box tables, evaluated once per call on the device:
    // [nshot][nt+1][6] (lo0,lo1,lo2,hi0,hi1,hi2) after n = -1 .. nt-1 steps.
    const int *tab_src;     // around the source
    const int *tab_rec;     // around the receivers
    int nt1;                // nt + 1
};

// Wavefields of a batch; shot s of field f is at f + s * ntot, node
// (i1, i2, i3) at i1 + px * (i2 + ne1 * i3); z nodes px > i1 >= ne0 are padding
// that no kernel reads as grid data.
struct Fields {
    float *p;
    float *v[3];
    float *psip[3];        // slab memory variables on the v grid of axis a (stride slab_n[a])
    float *psiv[3];        // slab memory variables on the p grid of axis a
};

// Boundary bands (saved source-field velocities, Sec. 4.2).
struct Bands {
    long long count;             // values per shot per step
    long long off[3][2];         // start of (axis, side) within one step
    int lo[3][2][3], hi[3][2][3];  // region of (axis, side): inclusive bounds per axis
    int prec;                    // SMI_PREC_*
    void *data;                  // [nshot][nt][count] of float / half / bf16
    float *scale;                // [nshot][nt][3][2] (16-bit storage only)
    int nt;                      // stored samples per shot (steps 0, dr, 2dr, ...)
    // division of a region's value index by its z extent and by its x extent:
    // multiplier and shift per (axis, side, divisor), see band_divisor()
    unsigned dm[3][2][2];
    int dl[3][2][2];
};
// Multiplier m and shift l with u / d = (mulhi(m, u) + u) >> l for every
// u < 2^31 (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994: l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1).
inline void band_divisor(unsigned d, unsigned &m, int &l)
{
    l = 0;
    while ((1ull << l) < d) l++;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
}

// ---------------------------------------------------------------------------
// Host set-up (smi_setup.cpp): exact FP64 arithmetic, rounded to FP32 tables.

// Staggered FD coefficients a_1..a_N (Sec. 2.1) from the closed-form product
// a_m = (-1)^{m+1}/(2m-1) prod_{n != m} (2n-1)^2 / |(2m-1)^2 - (2n-1)^2|.
void fd_coefficients(int N, double *a);

// CFL number of Eq. cfl; the call fails if it exceeds 1.
double cfl_number(int ndim, const double *h, double dt, double vmax, int N);

// Points per shortest wavelength vmin / (2.5 fm) / max(h).
double points_per_wavelength(int ndim, const double *h, double vmin, double fm);

// CPML a/b tables along one axis (length ne) on the p grid or the v grid.
void cpml_tables(int ne, int nb, double h, double vmax, double fm, double R, double dt,
                 bool vgrid, float *a, float *b);

// Kaiser-windowed sinc stencil of a position (metres) on the extended grid;
// false if it leaves the physical domain or its stencil leaves the grid.
bool make_stencil(const Grid &g, const double pos[3], double kaiser_b, Stencil *st);

// Decimated boundaries (Sec. 4.2): the band of step k*dr is stored for
// k = 0..nsamp-1, and the band of step it is a Kaiser-windowed sinc (radius
// kTimeR samples, shape kTimeB) of the stored samples first..first+2kTimeR-1
// at the fractional sample it/dr; a step on a stored sample takes that
// sample alone.  Samples before 0 are zero (the field before the first
// step); the forward run continues past nt-1 without a source so that the
// window of every step it < nt is complete.
constexpr int kTimeR = 8;
constexpr double kTimeB = 8.0;
struct TimeWeights {
    int first;             // first stored sample of the window
    int nsamp;             // stored samples per shot
    float w[2 * kTimeR];
};
TimeWeights time_weights(int it, int dr, int nsamp);
// Samples stored per shot, and forward steps including the continuation.
inline int band_samples(int nt, int dr) { return dr == 1 ? nt : (nt - 1) / dr + kTimeR + 1; }
inline int forward_steps(int nt, int dr) { return dr == 1 ? nt : (band_samples(nt, dr) - 1) * dr + 1; }

// ---------------------------------------------------------------------------
// Kernel launchers (smi_kernels.cu).  All run on `stream`.

struct LaunchCtx {
    void *stream;           // cudaStream_t
    long long *launches;    // incremented per kernel launch
};

void launch_extend_model(const LaunchCtx &lc, const Grid &g, const float *vp, const float *rho,
                         int n1, int n2, int n3, float *K, float *rho_e);
void launch_minmax(const LaunchCtx &lc, const float *vp, long long n, float *out2, unsigned *tmp);
void launch_zero(const LaunchCtx &lc, void *ptr, size_t bytes);

// Generic kernels (2D, and 3D without the TMA path): `work` = the largest
// number of points a shot of the batch updates in this launch (its box), which
// sizes the grid.
void launch_fwd_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work);
void launch_fwd_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work);
void launch_inject_source(const LaunchCtx &lc, const Grid &g, const Batch &b, float *p,
                          const float *stf, int it, float scale);
void launch_gather(const LaunchCtx &lc, const Grid &g, const Batch &b, const float *p,
                   float *seis, const long long *seis_off, int nt, int it);
void launch_save_bands(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f,
                       Bands bd, int it, unsigned *absmax_tmp);
void launch_restore_bands(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f,
                          Bands bd, int it);
// Band of a step between stored samples (decimated boundaries).
void launch_restore_bands_interp(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, Bands bd,
                                 const TimeWeights &tw);
void launch_residual(const LaunchCtx &lc, const float *seis, const float *dobs, long long n,
                     int mode, float *res, double *partials, int npart);
void launch_sum_partials(const LaunchCtx &lc, const double *partials, int npart, double *out);
// Wavelet adjoint: part[s][it] = scale * sum over shot s's source stencil of
// w * lp / kappa (FP64), the transpose of the source injection.
void launch_src_adjoint(const LaunchCtx &lc, const Grid &g, const Batch &b, const float *lp, double *part, int nt,
                        int it, double scale);
// out[it] (+)= sum_s part[s][it] in shot order (FP64).
void launch_sum_series(const LaunchCtx &lc, const double *part, int nshot, int nt, double *out, int accumulate);
void launch_to_float(const LaunchCtx &lc, const double *a, int n, float *out);
// FP64 partial dot products of a and b, npart of them (blocks), summed by
// launch_sum_partials in block order.
void launch_dot(const LaunchCtx &lc, const float *a, const float *b, long long n, double *partials, int npart);
void launch_adj_inject(const LaunchCtx &lc, const Grid &g, const Batch &b, float *lp,
                       const float *res, const long long *seis_off, int nt, int it);
void launch_adj_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, long long work);
void launch_adj_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, long long work);
// One piece of the union of the CPML bands: per axis up to two index
// intervals {start0, len0, start1, len1}; nodes = product of the counts.
struct Piece {
    int iv[3][4];
    int cnt[3];
    int axis;              // the axis whose band defines the piece
    int blocks;            // 256-thread blocks of this piece per chunk and shot; 0: empty
    int chunks;            // chunks along the piece's walk axis
};
// Disjoint pieces covering the nodes within w_lo of the low end or w_hi of
// the high end of axis z or x, clipped to a box (make_pieces); q[a] is the
// piece of axis a (q[2] unused).
struct Pieces {
    int n;                 // non-empty pieces
    int w_lo, w_hi;
    Piece q[3];
};
// uz: nodes per lane along x in the z piece's kernel.
Pieces make_pieces(const Grid &g, const int lo[3], const int hi[3], int w_lo, int w_hi, int uz);
// Transposed z and x CPML terms of the adjoint (vel: velocity part, else
// pressure part, which in 3D also updates phi_y at its own nodes) over the
// union of the z and x bands within the box [lo, hi] (union of the batch's
// receiver boxes after m reverse steps); run before the main kernels (in 3D
// those apply the y terms).
void launch_adj_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int m, bool vel,
                            const int lo[3], const int hi[3]);
// Forward z and x CPML memory-variable updates over the slabs (vel:
// velocity part, else pressure part) within the box [lo, hi] (union of the
// batch's source boxes at step it); added to the update of the main kernels
// (in 3D those apply the y terms).
void launch_fwd_corrections(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, bool vel,
                            const int lo[3], const int hi[3]);
void launch_recon_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f,
                    const float *lp, float *acc, int mode, const float *stf, int it,
                    float src_scale, long long work);
void launch_recon_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int it, long long work);

// 2D kernels (smi_stencil2d.cu): mode 0 forward, 1 adjoint (both with the
// CPML terms inline), 2 reconstruction + imaging; [lo, hi] = the batch's box
// union (for mode 2 within the physical domain).
bool stencil2d_supported(const Grid &g);
void launch2_v(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int step, int mode, const int lo[3],
               const int hi[3]);
void launch2_p(const LaunchCtx &lc, const Grid &g, const Batch &b, Fields f, int step, int mode, const int lo[3],
               const int hi[3], const float *lp, float *acc, int img_mode, const float *stf, float src_scale);
void launch_reduce_shots(const LaunchCtx &lc, const Grid &g, const float *acc, int nshot,
                         float *out, int accumulate);
// Normalised image: acc holds [nshot][nphys] images then [nshot][nphys]
// illuminations; mx = nshot unsigned scratch.
void launch_reduce_norm(const LaunchCtx &lc, const Grid &g, const float *acc, int nshot, unsigned *mx, float *out,
                        int accumulate);
void launch_finalize_grad(const LaunchCtx &lc, long long n, const float *vp, float dt,
                          float *g);
// Density gradient (Eq. gradrhokappa): per axis, vprev = [nshot][ntot] source
// velocities of the previous reverse step, G = [ntot] half-node sums of
// lambda_v (v^{it+1/2} - v^{it-1/2}) over shots and steps.
struct RhoAcc {
    float *vprev[3];
    float *G[3];
};
struct IBox {
    int lo[3], hi[3];
};
// G += sum_s lambda_v (vprev - v) and vprev <- v over the nodes of box.
void launch_rho_acc(const LaunchCtx &lc, const Grid &g, int nshot, Fields F, Fields A, RhoAcc r, IBox box);
// (dJ/dm1, dJ/dm2) of parametrisation family 1 (Vp, rho) or 2 (Vp, Ip), of
// the logarithms when logp; acc = summed lambda_p div v (physical grid); vp,
// rho physical; g1 may alias acc.
void launch_finalize_family(const LaunchCtx &lc, const Grid &g, const float *vp, const float *rho, const float *acc,
                            RhoAcc r, int family, int logp, float *g1, float *g2);
// Free surface on the top face (image method, Sec. 2.1), on every x, y of
// nshot fields f (z component for the velocity ops):
//   kFsMirrorV: v_z on the N half nodes above the surface node L = g.L[0]
//               mirrors v_z below it (half node L-1-j takes L+j);
//   kFsMirrorP: p = 0 at L, p at L-j takes -p at L+j (j = 1..N);
//   kFsFoldV, kFsFoldP: the transposes (adjoint fields): the image node's
//               value goes to its mirror node (negated for p) and is cleared,
//               and for p the surface node is cleared.
enum { kFsMirrorV = 0, kFsMirrorP = 1, kFsFoldV = 2, kFsFoldP = 3 };
void launch_free_surface(const LaunchCtx &lc, const Grid &g, float *f, int nshot, int op);
void launch_nonfinite(const LaunchCtx &lc, const float *x, long long n, unsigned *flag);
// Sets the padded layout: px, ntot, nphys and the slab sizes (ne, nb, ndim set).
void set_layout(Grid &g, const int n[3]);

void launch_box_table(const LaunchCtx &lc, const Grid &g, const int *ext, int n0, int count,
                      int *lo, int *hi);
// Fills tab[nshot][nt+1][6] with the boxes of n = -1 .. nt-1 around ext[nshot][6].
void launch_box_fill(const LaunchCtx &lc, const Grid &g, const int *ext, int nshot, int nt, int *tab);

}  // namespace smi
