/*
 * smi_oracle.c -- plain, slow, FP64 CPU oracle for staggered-grid acoustic
 * modelling, RTM imaging and FWI gradients (SMIwiz, arXiv 2311.02293).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table with the
 * CUDA library; the two are written independently from the paper.
 *
 * What it computes, in the paper's order (Algorithm 2):
 *   check_cfl (Eq. cfl, Sec. 2.1; accuracy control, Sec. 3.8)
 *   cpml_init (Sec. 2.1: 20 PML layers after Komatitsch & Martin 2007)
 *   extend_model (Algorithm 2)
 *   computing_box_init (Sec. 4.1)
 *   forward loop: save boundary -> update v (-> free-surface mirror) ->
 *                 update p -> inject source (-> free-surface mirror) ->
 *                 extract wavefield (Sec. 2.1 update equations)
 *   residual + misfit (Eq. objfwi, Sec. 2.2)
 *   reverse loop: adjoint source -> adjoint v/p -> remove source ->
 *                 reconstruct p, v -> re-impose boundary -> image/gradient
 *                 (Eqs. gradrhokappa, adj, rtmimage; Sec. 4.2), with the
 *                 density part of the gradient on request (Sec. 2.2)
 *
 * Readings of the paper (where it is silent) are listed at each function
 * and collected in the design notes: zero-valued reads outside the grid,
 * edge-replicated model extension, arithmetic-mean buoyancy, the CPML
 * profile constants, Kaiser window b, the box radius margin, the boundary
 * band layout, the discrete misfit without a dt factor, the exact
 * discrete adjoint (scatter-form transpose of every forward operation), the
 * free surface's image zone and folded interpolation weights, and the CPML
 * cells' model held fixed in the gradients.  Every function is pinned by a
 * CPU test against something other than itself (no function is parity
 * unpinned).
 *
 * Layout: n1 = z fastest, then x (n2), then y (n3); axis 0 = z, 1 = x,
 * 2 = y.  p lives on integer nodes; v_a lives half a cell up axis a and is
 * stored at the index of its lower p neighbour (Sec. 2.1, staggered grid).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Wall-clock seconds (phase timing of the CPU baseline; no effect on results). */
static double wall_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
#endif
}

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_CFL (-2)
#define ORC_ERR_DISPERSION (-3)
#define ORC_ERR_NOMEM (-4)

/* Problem parameters (mirrored field by field by the ctypes wrapper). */
typedef struct {
    int ndim;             /* 2 or 3 */
    int n1, n2, n3;       /* physical sizes z, x, y (n3 ignored in 2D) */
    double d1, d2, d3;    /* grid spacings in metres */
    int order;            /* 2 (tests only), 4 or 8 */
    int nb;               /* CPML layers on every face */
    int nt;               /* time steps */
    double dt;            /* time step in seconds */
    double fm;            /* wavelet centre frequency (CPML alpha, dispersion) */
    double kaiser_b;      /* Kaiser window shape */
    double cpml_R;        /* target reflection coefficient (1 = no absorption) */
    int use_box;          /* dynamic computing box on/off (Sec. 4.1) */
    int periodic;         /* tests only: periodic wrap instead of zero reads */
    int nthreads;         /* OpenMP threads, 0 = library default */
    int dr;               /* boundary decimation ratio (Sec. 4.2); 1 = every step */
    int freesurf;         /* 1: free surface on the top face (image method, Sec. 2.1) */
} orc_par;

#define MAXN 8
#define MAXW 16

typedef struct {
    int ndim, N, ri;
    int ne[3];            /* extended sizes */
    int L[3], H[3];       /* first/last physical node per axis (extended index) */
    long ntot;
    double d[3], dt, dV;
    double a[MAXN];       /* FD coefficients a_1..a_N stored at a[0..N-1] */
    int periodic, use_box, nt, dr, freesurf;
    double vmax, vmin;
    double *K;            /* bulk modulus at p nodes */
    double *bu[3];        /* buoyancy at v_a nodes */
    double *cpa[3], *cpb[3];  /* CPML a, b along axis a on the p grid */
    double *cva[3], *cvb[3];  /* CPML a, b along axis a on the v grid */
} grid_t;

typedef struct {
    double *p, *v[3];
    double *psip[3];      /* memory variable of D_a p, on the v_a grid */
    double *psiv[3];      /* memory variable of D_a v_a, on the p grid */
} state_t;

/* Interpolation stencil of one point (Kaiser-windowed sinc, Sec. 2.1). */
typedef struct {
    int first[3];         /* first node per axis */
    int cnt[3];           /* nodes per axis */
    double w[3][MAXW];    /* 1D weights per axis */
} stencil_t;

static long IDX(const grid_t *g, int i1, int i2, int i3)
{
    return (long)i1 + (long)g->ne[0] * ((long)i2 + (long)g->ne[1] * (long)i3);
}

/* ---------------------------------------------------------------------- */
/* FD coefficients: the staggered derivative sum_l a_l (f(x+(2l-1)h/2) -
 * f(x-(2l-1)h/2))/h is exact for polynomials up to degree 2N-1 iff
 * sum_l a_l (2l-1)^(2k-1) = delta_k1 for k = 1..N (Taylor expansion; the
 * paper refers to Fornberg for these values, Sec. 2.1).  Solved by Gaussian
 * elimination with partial pivoting. */
int orc_fd_coeffs(int N, double *a)
{
    double M[MAXN][MAXN + 1];
    if (N < 1 || N > MAXN) return ORC_ERR_ARG;
    for (int k = 0; k < N; k++) {
        for (int l = 0; l < N; l++) M[k][l] = pow(2.0 * l + 1.0, 2.0 * k + 1.0);
        M[k][N] = (k == 0) ? 1.0 : 0.0;
    }
    for (int c = 0; c < N; c++) {
        int piv = c;
        for (int r = c + 1; r < N; r++)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        for (int j = 0; j <= N; j++) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
        for (int r = 0; r < N; r++) {
            if (r == c) continue;
            double f = M[r][c] / M[c][c];
            for (int j = c; j <= N; j++) M[r][j] -= f * M[c][j];
        }
    }
    for (int l = 0; l < N; l++) a[l] = M[l][N] / M[l][l];
    return ORC_OK;
}

/* Modified Bessel function I0 from its power series sum_k ((x/2)^k / k!)^2. */
double orc_bessel_i0(double x)
{
    double s = 1.0, t = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 1000; k++) {
        t *= q / ((double)k * (double)k);
        s += t;
        if (t < 1e-17 * s) break;
    }
    return s;
}

/* 1D Kaiser-windowed sinc weights (Hicks 2002, cited in Sec. 2.1) for a
 * point at fractional grid coordinate x0, radius ri (ri = order/2, Sec. 3.8).
 * A point within 1e-6 cells of a node is snapped onto it and gets a unit
 * weight there (sinc vanishes on every other node, so this is the limit of
 * the formula).  Nodes first..first+2ri-1; returns the first node. */
int orc_kaiser_1d(double x0, int ri, double b, int *first, double *w)
{
    double r = nearbyint(x0);
    int snapped = fabs(x0 - r) <= 1e-6;
    int base = snapped ? (int)r : (int)floor(x0);
    double i0b = orc_bessel_i0(b);
    *first = base - ri + 1;
    for (int j = 0; j < 2 * ri; j++) {
        int node = base - ri + 1 + j;
        if (snapped) {
            w[j] = (node == base) ? 1.0 : 0.0;
            continue;
        }
        double x = (double)node - x0;
        double sinc = (x == 0.0) ? 1.0 : sin(M_PI * x) / (M_PI * x);
        double u = x / (double)ri;
        double arg = 1.0 - u * u;
        w[j] = (arg <= 0.0) ? 0.0 : sinc * orc_bessel_i0(b * sqrt(arg)) / i0b;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* CPML profile along one axis (Komatitsch & Martin 2007, cited in Sec. 2.1).
 * Readings: damping d(x) = d0 (x/Lp)^2 with d0 = -3 vmax ln(R) / (2 Lp),
 * Lp = nb*h; alpha(x) = pi fm (1 - x/Lp); kappa = 1; b = exp(-(d+alpha) dt),
 * a = d (b-1)/(d+alpha).  x is the distance into the layer from the outermost
 * physical node, clamped to Lp (the last half-node lies half a cell beyond).
 * a = b = 0 where d = 0 (physical interior), so memory variables stay zero. */
static void cpml_axis(int ne, int L, int H, int nb, double h, double vmax,
                      double fm, double R, double dt, int vgrid,
                      double *pa, double *pb)
{
    double Lp = nb * h;
    double d0 = (nb > 0) ? -3.0 * vmax * log(R) / (2.0 * Lp) : 0.0;
    for (int j = 0; j < ne; j++) {
        double pos = vgrid ? j + 0.5 : (double)j;
        double dist = 0.0;
        if (pos < L) dist = (L - pos) * h;
        else if (pos > H) dist = (pos - H) * h;
        pa[j] = 0.0;
        pb[j] = 0.0;
        if (dist <= 0.0 || nb == 0) continue;
        if (dist > Lp) dist = Lp;
        double x = dist / Lp;
        double dd = d0 * x * x;
        double al = M_PI * fm * (1.0 - x);
        if (dd <= 0.0) continue;
        double bb = exp(-(dd + al) * dt);
        pb[j] = bb;
        pa[j] = dd * (bb - 1.0) / (dd + al);
    }
}

/* ---------------------------------------------------------------------- */
static void grid_free(grid_t *g)
{
    free(g->K);
    for (int a = 0; a < 3; a++) {
        free(g->bu[a]); free(g->cpa[a]); free(g->cpb[a]); free(g->cva[a]); free(g->cvb[a]);
    }
    memset(g, 0, sizeof *g);
}

#ifdef _OPENMP
/* The OpenMP thread count the process started with (OMP_NUM_THREADS or the
 * core count), taken before any call sets one: nthreads = 0 restores it, so
 * a one-thread call does not leave later calls on one thread. */
static int default_threads(void)
{
    static int n = 0;
    if (n == 0) n = omp_get_max_threads();
    return n;
}
#endif

/* check_cfl + cpml_init + extend_model (Algorithm 2).  Reading: the model is
 * extended into the layers by copying the nearest physical value. */
static int grid_init(grid_t *g, const orc_par *par, const double *vp, const double *rho)
{
    memset(g, 0, sizeof *g);
    if (par->ndim != 2 && par->ndim != 3) return ORC_ERR_ARG;
    if (par->order != 2 && par->order != 4 && par->order != 8) return ORC_ERR_ARG;
    if (par->nt < 1 || !(par->dt > 0.0) || par->nb < 0) return ORC_ERR_ARG;
    if (par->periodic && par->nb != 0) return ORC_ERR_ARG;
    if (par->freesurf && (par->periodic || par->nb < par->order / 2)) return ORC_ERR_ARG;
#ifdef _OPENMP
    omp_set_num_threads(par->nthreads > 0 ? par->nthreads : default_threads());
#endif
    g->ndim = par->ndim;
    g->N = par->order / 2;
    g->ri = g->N;
    g->periodic = par->periodic;
    g->freesurf = par->freesurf != 0;
    g->use_box = par->use_box;
    g->nt = par->nt;
    g->dt = par->dt;
    if (par->dr < 0) return ORC_ERR_ARG;
    g->dr = par->dr > 1 ? par->dr : 1;
    int n[3] = {par->n1, par->n2, par->ndim == 3 ? par->n3 : 1};
    double d[3] = {par->d1, par->d2, par->ndim == 3 ? par->d3 : 1.0};
    g->dV = 1.0;
    for (int a = 0; a < 3; a++) {
        int act = a < g->ndim;
        if (act && (n[a] < 2 * g->N || !(d[a] > 0.0))) return ORC_ERR_ARG;
        g->ne[a] = act ? n[a] + 2 * par->nb : 1;
        g->L[a] = act ? par->nb : 0;
        g->H[a] = act ? par->nb + n[a] - 1 : 0;
        g->d[a] = d[a];
        if (act) g->dV *= d[a];
    }
    g->ntot = (long)g->ne[0] * g->ne[1] * g->ne[2];
    orc_fd_coeffs(g->N, g->a);

    long nphys = (long)n[0] * n[1] * n[2];
    g->vmax = 0.0;
    g->vmin = INFINITY;
    for (long k = 0; k < nphys; k++) {
        if (!(vp[k] > 0.0) || !(rho[k] > 0.0)) return ORC_ERR_ARG;
        if (vp[k] > g->vmax) g->vmax = vp[k];
        if (vp[k] < g->vmin) g->vmin = vp[k];
    }
    /* Eq. cfl: dt vmax sqrt(sum 1/h^2) sum |a_l| <= 1 */
    double s2 = 0.0, sa = 0.0;
    for (int a = 0; a < g->ndim; a++) s2 += 1.0 / (d[a] * d[a]);
    for (int l = 0; l < g->N; l++) sa += fabs(g->a[l]);
    if (g->dt * g->vmax * sqrt(s2) * sa > 1.0) return ORC_ERR_CFL;
    /* Boundary decimation (Sec. 4.2): the paper's dr = 5 vmax / vmin, read
     * as the largest ratio that keeps the stored boundary above its Nyquist
     * rate. */
    if (g->dr > 1 && (double)g->dr > 5.0 * g->vmax / g->vmin) return ORC_ERR_ARG;
    /* Dispersion (Sec. 3.8; threshold is a reading): shortest wavelength
     * vmin / (2.5 fm) must span >= 5 cells at order 4, >= 4 cells at order 8. */
    if (par->fm > 0.0 && g->N >= 2) {
        double hmax = 0.0;
        for (int a = 0; a < g->ndim; a++) if (d[a] > hmax) hmax = d[a];
        double ppw = g->vmin / (2.5 * par->fm) / hmax;
        double need = (g->N >= 4) ? 4.0 : 5.0;
        if (ppw < need) return ORC_ERR_DISPERSION;
    }

    g->K = malloc(sizeof(double) * g->ntot);
    double *rhoe = malloc(sizeof(double) * g->ntot);
    if (!g->K || !rhoe) { free(rhoe); grid_free(g); return ORC_ERR_NOMEM; }
    for (int i3 = 0; i3 < g->ne[2]; i3++)
    for (int i2 = 0; i2 < g->ne[1]; i2++)
    for (int i1 = 0; i1 < g->ne[0]; i1++) {
        int i[3] = {i1, i2, i3}, j[3];
        for (int a = 0; a < 3; a++) {
            j[a] = i[a] - g->L[a];
            if (j[a] < 0) j[a] = 0;
            if (j[a] > n[a] - 1) j[a] = n[a] - 1;
        }
        long kp = (long)j[0] + (long)n[0] * ((long)j[1] + (long)n[1] * j[2]);
        long k = IDX(g, i1, i2, i3);
        rhoe[k] = rho[kp];
        g->K[k] = rho[kp] * vp[kp] * vp[kp];      /* kappa = rho Vp^2 (Sec. 2.1) */
    }
    /* Buoyancy on the half nodes (reading): b = 2/(rho_i + rho_{i+1}), and
     * 1/rho at the last node of an axis (periodic: wrap). */
    for (int a = 0; a < g->ndim; a++) {
        g->bu[a] = malloc(sizeof(double) * g->ntot);
        if (!g->bu[a]) { free(rhoe); grid_free(g); return ORC_ERR_NOMEM; }
        for (int i3 = 0; i3 < g->ne[2]; i3++)
        for (int i2 = 0; i2 < g->ne[1]; i2++)
        for (int i1 = 0; i1 < g->ne[0]; i1++) {
            int i[3] = {i1, i2, i3};
            long k = IDX(g, i1, i2, i3);
            if (i[a] + 1 < g->ne[a] || g->periodic) {
                i[a] = (i[a] + 1) % g->ne[a];
                long k2 = IDX(g, i[0], i[1], i[2]);
                g->bu[a][k] = 2.0 / (rhoe[k] + rhoe[k2]);
            } else {
                g->bu[a][k] = 1.0 / rhoe[k];
            }
        }
    }
    free(rhoe);
    for (int a = 0; a < g->ndim; a++) {
        g->cpa[a] = calloc(g->ne[a], sizeof(double));
        g->cpb[a] = calloc(g->ne[a], sizeof(double));
        g->cva[a] = calloc(g->ne[a], sizeof(double));
        g->cvb[a] = calloc(g->ne[a], sizeof(double));
        if (!g->cpa[a] || !g->cpb[a] || !g->cva[a] || !g->cvb[a]) { grid_free(g); return ORC_ERR_NOMEM; }
        cpml_axis(g->ne[a], g->L[a], g->H[a], par->nb, d[a], g->vmax, par->fm,
                  par->cpml_R, g->dt, 0, g->cpa[a], g->cpb[a]);
        cpml_axis(g->ne[a], g->L[a], g->H[a], par->nb, d[a], g->vmax, par->fm,
                  par->cpml_R, g->dt, 1, g->cva[a], g->cvb[a]);
    }
    /* Free surface: the top layer holds the image of the field, not an
     * absorbing layer (its memory variables stay zero). */
    for (int i = 0; g->freesurf && i < g->L[0]; i++)
        g->cpa[0][i] = g->cpb[0][i] = g->cva[0][i] = g->cvb[0][i] = 0.0;
    return ORC_OK;
}

static int state_alloc(const grid_t *g, state_t *s)
{
    memset(s, 0, sizeof *s);
    s->p = calloc(g->ntot, sizeof(double));
    if (!s->p) return ORC_ERR_NOMEM;
    for (int a = 0; a < g->ndim; a++) {
        s->v[a] = calloc(g->ntot, sizeof(double));
        s->psip[a] = calloc(g->ntot, sizeof(double));
        s->psiv[a] = calloc(g->ntot, sizeof(double));
        if (!s->v[a] || !s->psip[a] || !s->psiv[a]) return ORC_ERR_NOMEM;
    }
    return ORC_OK;
}

static void state_free(state_t *s)
{
    free(s->p);
    for (int a = 0; a < 3; a++) { free(s->v[a]); free(s->psip[a]); free(s->psiv[a]); }
    memset(s, 0, sizeof *s);
}

/* ---------------------------------------------------------------------- */
/* Field value at a node; reads outside the grid are zero (reading), or wrap
 * around in the periodic test mode. */
static double fget(const grid_t *g, const double *f, const int i[3])
{
    int j[3];
    for (int a = 0; a < 3; a++) {
        j[a] = i[a];
        if (j[a] < 0 || j[a] >= g->ne[a]) {
            if (!g->periodic) return 0.0;
            j[a] = ((j[a] % g->ne[a]) + g->ne[a]) % g->ne[a];
        }
    }
    return f[IDX(g, j[0], j[1], j[2])];
}

/* Scatter-add into a node (transpose of fget): dropped outside the grid. */
static void fadd(const grid_t *g, double *f, const int i[3], double val)
{
    int j[3];
    for (int a = 0; a < 3; a++) {
        j[a] = i[a];
        if (j[a] < 0 || j[a] >= g->ne[a]) {
            if (!g->periodic) return;
            j[a] = ((j[a] % g->ne[a]) + g->ne[a]) % g->ne[a];
        }
    }
    f[IDX(g, j[0], j[1], j[2])] += val;
}

/* d_a p at the v_a node i (position i+1/2): sum_l a_l (p_{i+l} - p_{i-l+1}) / h
 * (Sec. 2.1, staggered FD operator). */
static double deriv_p(const grid_t *g, const double *p, int a, const int i[3])
{
    double s = 0.0;
    for (int l = 1; l <= g->N; l++) {
        int ip[3] = {i[0], i[1], i[2]}, im[3] = {i[0], i[1], i[2]};
        ip[a] += l;
        im[a] += 1 - l;
        s += g->a[l - 1] * (fget(g, p, ip) - fget(g, p, im));
    }
    return s / g->d[a];
}

/* d_a v_a at the p node i: sum_l a_l (v_{i+(2l-1)/2} - v_{i-(2l-1)/2}) / h,
 * i.e. stored indices i+l-1 and i-l (Sec. 2.1). */
static double deriv_v(const grid_t *g, const double *v, int a, const int i[3])
{
    double s = 0.0;
    for (int l = 1; l <= g->N; l++) {
        int ip[3] = {i[0], i[1], i[2]}, im[3] = {i[0], i[1], i[2]};
        ip[a] += l - 1;
        im[a] -= l;
        s += g->a[l - 1] * (fget(g, v, ip) - fget(g, v, im));
    }
    return s / g->d[a];
}

/* ---------------------------------------------------------------------- */
/* fdtd_update_v (Sec. 2.1): v_a <- v_a - dt b_a (d_a p + psi_a), with the
 * CPML memory variable psi_a <- b psi_a + a d_a p updated first. */
static void update_v(const grid_t *g, state_t *s, const int lo[3], const int hi[3])
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int i3 = lo[2]; i3 <= hi[2]; i3++)
    for (int i2 = lo[1]; i2 <= hi[1]; i2++)
    for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
        int i[3] = {i1, i2, i3};
        long k = IDX(g, i1, i2, i3);
        for (int a = 0; a < g->ndim; a++) {
            double D = deriv_p(g, s->p, a, i);
            s->psip[a][k] = g->cvb[a][i[a]] * s->psip[a][k] + g->cva[a][i[a]] * D;
            s->v[a][k] -= g->dt * g->bu[a][k] * (D + s->psip[a][k]);
        }
    }
}

/* fdtd_update_p (Sec. 2.1): p <- p - dt kappa sum_a (d_a v_a + psi_a). */
static void update_p(const grid_t *g, state_t *s, const int lo[3], const int hi[3])
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int i3 = lo[2]; i3 <= hi[2]; i3++)
    for (int i2 = lo[1]; i2 <= hi[1]; i2++)
    for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
        int i[3] = {i1, i2, i3};
        long k = IDX(g, i1, i2, i3);
        double div = 0.0;
        for (int a = 0; a < g->ndim; a++) {
            double D = deriv_v(g, s->v[a], a, i);
            s->psiv[a][k] = g->cpb[a][i[a]] * s->psiv[a][k] + g->cpa[a][i[a]] * D;
            div += D + s->psiv[a][k];
        }
        s->p[k] -= g->dt * g->K[k] * div;
    }
}

/* Transpose of update_p at one node (exact discrete adjoint, written as the
 * scatter-form transpose of each assignment).  Adjoint variables: pb (of p),
 * vb (of v), psivb (of psi_v).  Reads only the node's own pb and psivb and
 * scatters into vb within N nodes of it along each axis. */
static void adjoint_node_p(const grid_t *g, state_t *ad, int i1, int i2, int i3)
{
    int i[3] = {i1, i2, i3};
    long k = IDX(g, i1, i2, i3);
    double q = -g->dt * g->K[k] * ad->p[k];         /* adjoint of div at i */
    for (int a = 0; a < g->ndim; a++) {
        double e = ad->psiv[a][k] + q;                /* adjoint of new psi_v */
        ad->psiv[a][k] = g->cpb[a][i[a]] * e;
        double y = (q + g->cpa[a][i[a]] * e) / g->d[a];  /* adjoint of d_a v_a */
        for (int l = 1; l <= g->N; l++) {
            int ip[3] = {i[0], i[1], i[2]}, im[3] = {i[0], i[1], i[2]};
            ip[a] += l - 1;
            im[a] -= l;
            fadd(g, ad->v[a], ip, g->a[l - 1] * y);
            fadd(g, ad->v[a], im, -g->a[l - 1] * y);
        }
    }
}

/* Transpose of update_v at one node: reads the node's own vb and psipb and
 * scatters into pb within N nodes of it along each axis. */
static void adjoint_node_v(const grid_t *g, state_t *ad, int i1, int i2, int i3)
{
    int i[3] = {i1, i2, i3};
    long k = IDX(g, i1, i2, i3);
    for (int a = 0; a < g->ndim; a++) {
        double y = -g->dt * g->bu[a][k] * ad->v[a][k];  /* adjoint of (d_a p + psi) */
        double e = ad->psip[a][k] + y;                    /* adjoint of new psi_p */
        ad->psip[a][k] = g->cvb[a][i[a]] * e;
        double z = (y + g->cva[a][i[a]] * e) / g->d[a];   /* adjoint of d_a p */
        for (int l = 1; l <= g->N; l++) {
            int ip[3] = {i[0], i[1], i[2]}, im[3] = {i[0], i[1], i[2]};
            ip[a] += l;
            im[a] += 1 - l;
            fadd(g, ad->p, ip, g->a[l - 1] * z);
            fadd(g, ad->p, im, -g->a[l - 1] * z);
        }
    }
}

/* Visits every node of the box [lo, hi] with fn, threads sharing the work
 * without two of them ever scattering into the same node: the outermost
 * active axis c is cut into chunks of at least 2N nodes, and chunks 0, 2,
 * 4, ... run in parallel, then chunks 1, 3, 5, ...  A node of chunk k
 * scatters only within N nodes of it along c, and two chunks of one colour
 * are separated by a whole chunk of the other colour (2N nodes or more), so
 * their scatter targets are disjoint.  Within a chunk the nodes are visited
 * in the plain loop order; only the order in which contributions from
 * different chunks add up at a node differs from one sequential sweep (an
 * FP64 rounding-order difference). */
static void adjoint_sweep(const grid_t *g, state_t *ad, const int lo[3], const int hi[3],
                          void (*fn)(const grid_t *, state_t *, int, int, int))
{
    const int c = g->ndim - 1;
    const int len = hi[c] - lo[c] + 1;
    if (len <= 0 || hi[0] < lo[0] || hi[1] < lo[1]) return;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    int C = (len + 2 * nth - 1) / (2 * nth);
    if (C < 2 * g->N) C = 2 * g->N;
    if (g->periodic) C = len;         /* scatters wrap around: one sequential sweep */
    const int nchunk = (len + C - 1) / C;
    for (int colour = 0; colour < 2; colour++) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int ch = colour; ch < nchunk; ch += 2) {
            int a[3] = {lo[0], lo[1], lo[2]}, b[3] = {hi[0], hi[1], hi[2]};
            a[c] = lo[c] + ch * C;
            b[c] = a[c] + C - 1 < hi[c] ? a[c] + C - 1 : hi[c];
            for (int i3 = a[2]; i3 <= b[2]; i3++)
            for (int i2 = a[1]; i2 <= b[1]; i2++)
            for (int i1 = a[0]; i1 <= b[0]; i1++)
                fn(g, ad, i1, i2, i3);
        }
    }
}

/* Transpose of update_p restricted to a box. */
static void adjoint_update_p(const grid_t *g, state_t *ad, const int lo[3], const int hi[3])
{
    adjoint_sweep(g, ad, lo, hi, adjoint_node_p);
}

/* Transpose of update_v restricted to a box. */
static void adjoint_update_v(const grid_t *g, state_t *ad, const int lo[3], const int hi[3])
{
    adjoint_sweep(g, ad, lo, hi, adjoint_node_v);
}

/* ---------------------------------------------------------------------- */
/* Free surface on the top face by the image method (Sec. 2.1, after
 * Levander 1988).  The surface is the first physical node row L = L[0].
 * After the velocity update, v_z on the N half nodes above it mirrors v_z
 * below it (symmetric: half node L-1-j takes L+j); after the pressure
 * update and the source, p = 0 at L and p on the N nodes above it is minus
 * its mirror (antisymmetric: node L-j takes -p at L+j).  Every x and y. */
static void fs_mirror_v(const grid_t *g, double *vz)
{
    if (!g->freesurf) return;
    for (int i3 = 0; i3 < g->ne[2]; i3++)
    for (int i2 = 0; i2 < g->ne[1]; i2++)
    for (int j = 0; j < g->N; j++)
        vz[IDX(g, g->L[0] - 1 - j, i2, i3)] = vz[IDX(g, g->L[0] + j, i2, i3)];
}

static void fs_mirror_p(const grid_t *g, double *p)
{
    if (!g->freesurf) return;
    for (int i3 = 0; i3 < g->ne[2]; i3++)
    for (int i2 = 0; i2 < g->ne[1]; i2++) {
        p[IDX(g, g->L[0], i2, i3)] = 0.0;
        for (int j = 1; j <= g->N; j++)
            p[IDX(g, g->L[0] - j, i2, i3)] = -p[IDX(g, g->L[0] + j, i2, i3)];
    }
}

/* Transposes of the two mirrors, applied to the adjoint fields: an image
 * node's adjoint goes (negated for p) to its mirror node and is cleared; the
 * adjoint of p at the surface node is cleared. */
static void fs_fold_v(const grid_t *g, double *vzb)
{
    if (!g->freesurf) return;
    for (int i3 = 0; i3 < g->ne[2]; i3++)
    for (int i2 = 0; i2 < g->ne[1]; i2++)
    for (int j = 0; j < g->N; j++) {
        long ki = IDX(g, g->L[0] - 1 - j, i2, i3);
        vzb[IDX(g, g->L[0] + j, i2, i3)] += vzb[ki];
        vzb[ki] = 0.0;
    }
}

static void fs_fold_p(const grid_t *g, double *pb)
{
    if (!g->freesurf) return;
    for (int i3 = 0; i3 < g->ne[2]; i3++)
    for (int i2 = 0; i2 < g->ne[1]; i2++) {
        for (int j = 1; j <= g->N; j++) {
            long ki = IDX(g, g->L[0] - j, i2, i3);
            pb[IDX(g, g->L[0] + j, i2, i3)] -= pb[ki];
            pb[ki] = 0.0;
        }
        pb[IDX(g, g->L[0], i2, i3)] = 0.0;
    }
}

static void stencil_add(const grid_t *g, double *f, const stencil_t *st, double scale);

/* One forward step (Algorithm 2, Sec. 2.1) on the box [lo, hi]: velocity
 * update, velocity mirror, pressure update, the source (src may be NULL:
 * none), pressure mirror. */
static void forward_step(const grid_t *g, state_t *s, const int lo[3], const int hi[3], const stencil_t *src,
                         double scale)
{
    update_v(g, s, lo, hi);
    fs_mirror_v(g, s->v[0]);
    update_p(g, s, lo, hi);
    if (src) stencil_add(g, s->p, src, scale);
    fs_mirror_p(g, s->p);
}

/* Transpose of forward_step's propagation, after the step's adjoint sources
 * are in ad->p and whatever reads the adjoint of the updated pressure has run
 * (fs_fold_p goes before that). */
static void adjoint_step(const grid_t *g, state_t *ad, const int lo[3], const int hi[3])
{
    adjoint_update_p(g, ad, lo, hi);
    fs_fold_v(g, ad->v[0]);
    adjoint_update_v(g, ad, lo, hi);
}

/* ---------------------------------------------------------------------- */
/* Stencil of a point given in metres (z, x, y) from the first physical node.
 * The point must lie inside the physical domain and its 2ri-node stencil
 * inside the extended grid. */
static int point_stencil(const grid_t *g, const double pos[3], double kb, stencil_t *st)
{
    for (int a = 0; a < 3; a++) {
        if (a >= g->ndim) {
            st->first[a] = 0;
            st->cnt[a] = 1;
            st->w[a][0] = 1.0;
            continue;
        }
        double x0 = pos[a] / g->d[a];
        int nphys = g->H[a] - g->L[a] + 1;
        if (!(x0 >= -1e-6 && x0 <= nphys - 1 + 1e-6)) return ORC_ERR_ARG;
        orc_kaiser_1d(x0 + g->L[a], g->ri, kb, &st->first[a], st->w[a]);
        st->cnt[a] = 2 * g->ri;
        if (st->first[a] < 0 || st->first[a] + st->cnt[a] - 1 > g->ne[a] - 1) return ORC_ERR_ARG;
        if (a == 0 && g->freesurf) {
            /* Free surface (reading, the image-source form of Hicks 2002): a
             * weight above the surface node L goes, negated, to its mirror
             * node 2L - i; the weight at L is dropped (p = 0 there). */
            for (int q = 0; q < st->cnt[0]; q++) {
                int node = st->first[0] + q;
                if (node >= g->L[0]) continue;
                int qm = 2 * g->L[0] - node - st->first[0];
                if (qm >= st->cnt[0]) return ORC_ERR_ARG;
                st->w[0][qm] -= st->w[0][q];
                st->w[0][q] = 0.0;
            }
            int q0 = g->L[0] - st->first[0];
            if (q0 >= 0 && q0 < st->cnt[0]) st->w[0][q0] = 0.0;
        }
    }
    return ORC_OK;
}

/* inject_source: p += scale * w at the stencil nodes. */
static void stencil_add(const grid_t *g, double *f, const stencil_t *st, double scale)
{
    for (int c = 0; c < st->cnt[2]; c++)
    for (int b = 0; b < st->cnt[1]; b++)
    for (int a = 0; a < st->cnt[0]; a++) {
        double w = st->w[0][a] * st->w[1][b] * st->w[2][c];
        if (w == 0.0) continue;
        f[IDX(g, st->first[0] + a, st->first[1] + b, st->first[2] + c)] += scale * w;
    }
}

/* extract_wavefield: sum_nodes w * f. */
static double stencil_get(const grid_t *g, const double *f, const stencil_t *st)
{
    double s = 0.0;
    for (int c = 0; c < st->cnt[2]; c++)
    for (int b = 0; b < st->cnt[1]; b++)
    for (int a = 0; a < st->cnt[0]; a++) {
        double w = st->w[0][a] * st->w[1][b] * st->w[2][c];
        if (w == 0.0) continue;
        s += w * f[IDX(g, st->first[0] + a, st->first[1] + b, st->first[2] + c)];
    }
    return s;
}

/* Subtract the source only at nodes of the physical domain (reconstruction). */
static void stencil_sub_interior(const grid_t *g, double *f, const stencil_t *st, double scale)
{
    for (int c = 0; c < st->cnt[2]; c++)
    for (int b = 0; b < st->cnt[1]; b++)
    for (int a = 0; a < st->cnt[0]; a++) {
        int i[3] = {st->first[0] + a, st->first[1] + b, st->first[2] + c};
        int in = 1;
        for (int x = 0; x < g->ndim; x++) in &= (i[x] >= g->L[x] && i[x] <= g->H[x]);
        double w = st->w[0][a] * st->w[1][b] * st->w[2][c];
        if (!in || w == 0.0) continue;
        f[IDX(g, i[0], i[1], i[2])] -= scale * w;
    }
}

/* ---------------------------------------------------------------------- */
/* Computing box (Sec. 4.1).  Reading: after n steps have elapsed the wave
 * has travelled at most vmax (n+1) dt; the box is the extent [slo, shi] of
 * the emitting stencil(s) grown by r_n = ceil(vmax (n+1) dt / h) + 2N + ri
 * cells on each side (2N covers the two half-step stencils, ri the
 * injection width), clipped to the extended grid.  n < 0 gives an empty
 * box.  The FP64 expression is evaluated as ((vmax * dt) * (n+1)) / h. */
static void box_at(const grid_t *g, const int slo[3], const int shi[3], int n,
                   int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) {
        if (a >= g->ndim) { lo[a] = 0; hi[a] = (n < 0) ? -1 : 0; continue; }
        if (n < 0) { lo[a] = 0; hi[a] = -1; continue; }
        if (!g->use_box) { lo[a] = 0; hi[a] = g->ne[a] - 1; continue; }
        double r = g->vmax * g->dt;
        r = r * (double)(n + 1);
        r = r / g->d[a];
        int rn = (int)ceil(r) + 2 * g->N + g->ri;
        lo[a] = slo[a] - rn;
        hi[a] = shi[a] + rn;
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > g->ne[a] - 1) hi[a] = g->ne[a] - 1;
    }
    if (n >= 0 && g->freesurf && lo[0] < g->L[0] - g->N) lo[0] = g->L[0] - g->N;
}

/* With the free surface, the nodes above the image zone (more than N above
 * the surface) are never updated and stay zero. */
static void full_box(const grid_t *g, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) { lo[a] = 0; hi[a] = g->ne[a] - 1; }
    if (g->freesurf) lo[0] = g->L[0] - g->N;
}

static int in_box(const int i[3], const int lo[3], const int hi[3])
{
    return i[0] >= lo[0] && i[0] <= hi[0] && i[1] >= lo[1] && i[1] <= hi[1] &&
           i[2] >= lo[2] && i[2] <= hi[2];
}

static void stencil_extent(const stencil_t *st, int n, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; a++) {
        int l = st[0].first[a], h = st[0].first[a] + st[0].cnt[a] - 1;
        for (int k = 1; k < n; k++) {
            if (st[k].first[a] < l) l = st[k].first[a];
            if (st[k].first[a] + st[k].cnt[a] - 1 > h) h = st[k].first[a] + st[k].cnt[a] - 1;
        }
        lo[a] = l;
        hi[a] = h;
    }
}

/* ---------------------------------------------------------------------- */
/* Boundary bands for source-field reconstruction (Sec. 4.2).
 * Reading of the band layout: for each axis a, the face-normal velocity v_a
 * on the 2N-1 half nodes straddling each face of the physical domain,
 * [L-N, L+N-2] and [H-N+1, H+N-1] along a, over the physical cross-section.
 * With these, p can be reversed on the whole physical domain and v_a on
 * [L+N-1, H-N] along a, and div v stays available on every physical node. */
static long band_count(const grid_t *g)
{
    long c = 0;
    for (int a = 0; a < g->ndim; a++) {
        long cross = 1;
        for (int b = 0; b < g->ndim; b++) if (b != a) cross *= (g->H[b] - g->L[b] + 1);
        c += 2L * (2 * g->N - 1) * cross;
    }
    return c;
}

static void band_copy(const grid_t *g, double *const v[3], double *buf, int restore)
{
    long c = 0;
    for (int a = 0; a < g->ndim; a++) {
        for (int side = 0; side < 2; side++) {
            int lo[3], hi[3];
            for (int b = 0; b < 3; b++) { lo[b] = g->L[b]; hi[b] = g->H[b]; }
            if (side == 0) { lo[a] = g->L[a] - g->N; hi[a] = g->L[a] + g->N - 2; }
            else { lo[a] = g->H[a] - g->N + 1; hi[a] = g->H[a] + g->N - 1; }
            for (int i3 = lo[2]; i3 <= hi[2]; i3++)
            for (int i2 = lo[1]; i2 <= hi[1]; i2++)
            for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
                long k = IDX(g, i1, i2, i3);
                if (restore) v[a][k] = buf[c++];
                else buf[c++] = v[a][k];
            }
        }
    }
}

/* Decimated boundary saving (Sec. 4.2).  The band of step k*dr is stored
 * for k = 0..nsamp-1 and the band of any step is interpolated from the
 * stored samples in time with a Kaiser-windowed sinc (the window family the
 * paper uses for sources and receivers, Hicks 2002) of radius TIME_R = 8
 * samples and shape TIME_B = 8.  Readings: the interpolator (the paper
 * names none; this one keeps the error of a sinusoid at or below 1.5e-4 up to
 * 0.3 cycles a sample, the band that the dr rule below admits), and a
 * forward run that continues past nt-1 without a source up to step
 * (nsamp-1)*dr, so that every step it < nt has all 2 TIME_R samples of its
 * window.  A step on a stored sample gets it exactly (sinc vanishes at the
 * other samples), so dr = 1 stores every step and needs no continuation. */
#define TIME_R 8
#define TIME_B 8.0
static int band_samples(const grid_t *g)
{
    return g->dr == 1 ? g->nt : (g->nt - 1) / g->dr + TIME_R + 1;
}

/* Band of step it from the stored samples into out[nband]. */
static void band_at(const grid_t *g, const double *bands, long nband, int nsamp, int it, double *out)
{
    if (g->dr == 1) {
        memcpy(out, bands + nband * (long)it, sizeof(double) * nband);
        return;
    }
    int first;
    double w[2 * TIME_R];
    orc_kaiser_1d((double)it / (double)g->dr, TIME_R, TIME_B, &first, w);
    for (long c = 0; c < nband; c++) out[c] = 0.0;
    for (int q = 0; q < 2 * TIME_R; q++) {
        int k = first + q;
        if (k < 0 || k >= nsamp || w[q] == 0.0) continue;   /* before step 0 the field is zero */
        const double *b = bands + nband * (long)k;
        for (long c = 0; c < nband; c++) out[c] += w[q] * b[c];
    }
}

/* dr > 1: continue the forward run (no source) from step nt to step
 * (nsamp-1)*dr, storing the bands of the multiples of dr, then put p and v
 * back to their state after step nt-1. */
static int forward_continue(const grid_t *g, state_t *s, const int slo[3], const int shi[3], double *bands,
                            long nband, int nsamp)
{
    if (g->dr == 1) return ORC_OK;
    double *keep = malloc(sizeof(double) * g->ntot * (1 + g->ndim));
    if (!keep) return ORC_ERR_NOMEM;
    memcpy(keep, s->p, sizeof(double) * g->ntot);
    for (int a = 0; a < g->ndim; a++) memcpy(keep + g->ntot * (1 + a), s->v[a], sizeof(double) * g->ntot);
    for (int it = g->nt; it <= (nsamp - 1) * g->dr; it++) {
        if (it % g->dr == 0) band_copy(g, s->v, bands + nband * (long)(it / g->dr), 0);
        int lo[3], hi[3];
        box_at(g, slo, shi, it, lo, hi);
        forward_step(g, s, lo, hi, NULL, 0.0);
    }
    memcpy(s->p, keep, sizeof(double) * g->ntot);
    for (int a = 0; a < g->ndim; a++) memcpy(s->v[a], keep + g->ntot * (1 + a), sizeof(double) * g->ntot);
    free(keep);
    return ORC_OK;
}

/* One reverse step of the source field (Algorithm 2: remove source,
 * reconstruct p, reconstruct v, re-impose boundary).  box = forward box of
 * step it, prev = forward box of step it-1; nodes of box not in prev are set
 * to zero (they were zero before step it ran). */
static void reconstruct_step(const grid_t *g, state_t *s, const stencil_t *src,
                             double src_scale, const int box[2][3], const int prev[2][3],
                             const double *band)
{
    stencil_sub_interior(g, s->p, src, src_scale);
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = g->L[a] > box[0][a] ? g->L[a] : box[0][a];
        hi[a] = g->H[a] < box[1][a] ? g->H[a] : box[1][a];
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int i3 = lo[2]; i3 <= hi[2]; i3++)
    for (int i2 = lo[1]; i2 <= hi[1]; i2++)
    for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
        int i[3] = {i1, i2, i3};
        long k = IDX(g, i1, i2, i3);
        double div = 0.0;
        for (int a = 0; a < g->ndim; a++) div += deriv_v(g, s->v[a], a, i);
        s->p[k] += g->dt * g->K[k] * div;
        if (!in_box(i, prev[0], prev[1]) || (g->freesurf && i1 == g->L[0])) s->p[k] = 0.0;
    }
    for (int a = 0; a < g->ndim; a++) {
        int vlo[3], vhi[3];
        for (int b = 0; b < 3; b++) { vlo[b] = lo[b]; vhi[b] = hi[b]; }
        int rl = g->L[a] + g->N - 1, rh = g->H[a] - g->N;
        if (vlo[a] < rl) vlo[a] = rl;
        if (vhi[a] > rh) vhi[a] = rh;
#pragma omp parallel for collapse(2) schedule(static)
        for (int i3 = vlo[2]; i3 <= vhi[2]; i3++)
        for (int i2 = vlo[1]; i2 <= vhi[1]; i2++)
        for (int i1 = vlo[0]; i1 <= vhi[0]; i1++) {
            int i[3] = {i1, i2, i3};
            long k = IDX(g, i1, i2, i3);
            s->v[a][k] += g->dt * g->bu[a][k] * deriv_p(g, s->p, a, i);
            if (!in_box(i, prev[0], prev[1])) s->v[a][k] = 0.0;
        }
    }
    band_copy(g, s->v, (double *)band, 1);
}

/* ---------------------------------------------------------------------- */
/* Forward modelling of one shot (Algorithm 2 forward loop, mode 0).
 * seis: [nt][nrec] samples of p^{it+1} at the receivers.  psnap (optional):
 * [nt][n1*n2*n3] p^{it+1} on the physical grid. */
int orc_forward(const orc_par *par, const double *vp, const double *rho, const double *stf,
                const double *src, int nrec, const double *rec, double *seis, double *psnap)
{
    grid_t g;
    state_t s;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    stencil_t sst, *rst = calloc(nrec > 0 ? nrec : 1, sizeof(stencil_t));
    if (!rst) { grid_free(&g); return ORC_ERR_NOMEM; }
    rc = point_stencil(&g, src, par->kaiser_b, &sst);
    for (int r = 0; r < nrec && !rc; r++) rc = point_stencil(&g, rec + 3 * r, par->kaiser_b, &rst[r]);
    if (!rc) rc = state_alloc(&g, &s);
    if (rc) { free(rst); grid_free(&g); return rc; }
    int slo[3], shi[3];
    stencil_extent(&sst, 1, slo, shi);
    for (int it = 0; it < g.nt; it++) {
        int lo[3], hi[3];
        box_at(&g, slo, shi, it, lo, hi);
        forward_step(&g, &s, lo, hi, &sst, g.dt * stf[it] / g.dV);
        for (int r = 0; r < nrec; r++) seis[(long)it * nrec + r] = stencil_get(&g, s.p, &rst[r]);
        if (psnap) {
            long c = 0, nphys = (long)(g.H[0] - g.L[0] + 1) * (g.H[1] - g.L[1] + 1) * (g.H[2] - g.L[2] + 1);
            for (int i3 = g.L[2]; i3 <= g.H[2]; i3++)
            for (int i2 = g.L[1]; i2 <= g.H[1]; i2++)
            for (int i1 = g.L[0]; i1 <= g.H[0]; i1++)
                psnap[(long)it * nphys + c++] = s.p[IDX(&g, i1, i2, i3)];
        }
    }
    state_free(&s);
    free(rst);
    grid_free(&g);
    return ORC_OK;
}

/* Advance a given state nsteps steps with no source over the full grid
 * (tests: plane waves, impulse responses).  Arrays are full extended size;
 * v/psi arrays of inactive axes may be NULL.  seis (optional) gets
 * [nsteps][nrec] receiver samples after each step. */
int orc_propagate(const orc_par *par, const double *vp, const double *rho,
                  double *p, double *vz, double *vx, double *vy,
                  double *psip_z, double *psip_x, double *psip_y,
                  double *psiv_z, double *psiv_x, double *psiv_y,
                  int nsteps, int nrec, const double *rec, double *seis)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    stencil_t *rst = calloc(nrec > 0 ? nrec : 1, sizeof(stencil_t));
    if (!rst) { grid_free(&g); return ORC_ERR_NOMEM; }
    for (int r = 0; r < nrec && !rc; r++) rc = point_stencil(&g, rec + 3 * r, par->kaiser_b, &rst[r]);
    if (rc) { free(rst); grid_free(&g); return rc; }
    state_t s;
    memset(&s, 0, sizeof s);
    double *vv[3] = {vz, vx, vy}, *pp[3] = {psip_z, psip_x, psip_y}, *pv[3] = {psiv_z, psiv_x, psiv_y};
    double *tmp[6] = {0};
    s.p = p;
    for (int a = 0; a < g.ndim; a++) {
        s.v[a] = vv[a];
        s.psip[a] = pp[a] ? pp[a] : (tmp[a] = calloc(g.ntot, sizeof(double)));
        s.psiv[a] = pv[a] ? pv[a] : (tmp[3 + a] = calloc(g.ntot, sizeof(double)));
    }
    int lo[3], hi[3];
    full_box(&g, lo, hi);
    for (int it = 0; it < nsteps; it++) {
        forward_step(&g, &s, lo, hi, NULL, 0.0);
        for (int r = 0; r < nrec; r++) seis[(long)it * nrec + r] = stencil_get(&g, s.p, &rst[r]);
    }
    for (int k = 0; k < 6; k++) free(tmp[k]);
    free(rst);
    grid_free(&g);
    return ORC_OK;
}

/* Adjoint run for the dot-product identity <L f, d> = <f, L^T d>, with L the
 * map from the source wavelet to the seismograms.  res: [nt][nrec].
 * box_mode: 0 full grid, 1 the forward (source) box sequence -- the exact
 * transpose of the boxed forward run --, 2 the receiver box (Sec. 4.1).
 * sbar: [nt] adjoint of the wavelet samples. */
int orc_adjoint(const orc_par *par, const double *vp, const double *rho, const double *src,
                int nrec, const double *rec, const double *res, int box_mode, double *sbar)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    stencil_t sst, *rst = calloc(nrec > 0 ? nrec : 1, sizeof(stencil_t));
    if (!rst) { grid_free(&g); return ORC_ERR_NOMEM; }
    rc = point_stencil(&g, src, par->kaiser_b, &sst);
    for (int r = 0; r < nrec && !rc; r++) rc = point_stencil(&g, rec + 3 * r, par->kaiser_b, &rst[r]);
    state_t ad;
    if (!rc) rc = state_alloc(&g, &ad);
    if (rc) { free(rst); grid_free(&g); return rc; }
    int slo[3], shi[3], rlo[3], rhi[3];
    stencil_extent(&sst, 1, slo, shi);
    stencil_extent(rst, nrec, rlo, rhi);
    for (int it = g.nt - 1; it >= 0; it--) {
        for (int r = 0; r < nrec; r++) stencil_add(&g, ad.p, &rst[r], res[(long)it * nrec + r]);
        fs_fold_p(&g, ad.p);
        sbar[it] = g.dt / g.dV * stencil_get(&g, ad.p, &sst);
        int lo[3], hi[3];
        if (box_mode == 1) box_at(&g, slo, shi, it, lo, hi);
        else if (box_mode == 2) box_at(&g, rlo, rhi, g.nt - 1 - it, lo, hi);
        else full_box(&g, lo, hi);
        adjoint_step(&g, &ad, lo, hi);
    }
    state_free(&ad);
    free(rst);
    grid_free(&g);
    return ORC_OK;
}

/* Density part of the gradient (Eq. gradrhokappa with rho varied at fixed
 * Vp).  Step it sets v_a^{it+1/2} = v_a^{it-1/2} - dt b_a (d_a p + psi_a), and
 * nothing else of the step depends on b_a, so
 *   dJ/db_a = sum_it vbar_a^{it+1/2} (v_a^{it+1/2} - v_a^{it-1/2}) / b_a,
 * with vbar_a^{it+1/2} the complete adjoint of v_a^{it+1/2} (what the adjoint
 * velocity holds once the transposed pressure update of step it has run).
 * Accumulated on the half nodes that touch a physical node: i_a in
 * [L_a-1, H_a] along a, the other coordinates physical.  vold NULL: zero. */
static void accumulate_gb(const grid_t *g, const state_t *ad, double *const vnew[3], double *const vold[3],
                          double *gb[3])
{
    for (int a = 0; a < g->ndim; a++) {
        int lo[3], hi[3];
        for (int b = 0; b < 3; b++) { lo[b] = g->L[b]; hi[b] = g->H[b]; }
        if (lo[a] > 0) lo[a]--;
#pragma omp parallel for collapse(2) schedule(static)
        for (int i3 = lo[2]; i3 <= hi[2]; i3++)
        for (int i2 = lo[1]; i2 <= hi[1]; i2++)
        for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
            long k = IDX(g, i1, i2, i3);
            double dv = vnew[a][k] - (vold ? vold[a][k] : 0.0);
            gb[a][k] += ad->v[a][k] * dv / g->bu[a][k];
        }
    }
}

/* dJ/drho at fixed Vp on the physical nodes: kappa = rho Vp^2 gives
 * Vp^2 dJ/dkappa; each half-node buoyancy b = 2 / (rho_i + rho_{i+1}) gives
 * -b^2/2 dJ/db to both of its nodes (b = 1/rho at the last node of an axis:
 * -b^2 dJ/db).  The CPML cells' rho is held fixed, like their kappa in the
 * Vp gradient. */
static int finish_rho(const grid_t *g, const double *vp, const double *acc, double *const gb[3], double *out_rho)
{
    double *gr = calloc(g->ntot, sizeof(double));
    if (!gr) return ORC_ERR_NOMEM;
    for (int a = 0; a < g->ndim; a++) {
        int lo[3], hi[3];
        for (int b = 0; b < 3; b++) { lo[b] = g->L[b]; hi[b] = g->H[b]; }
        if (lo[a] > 0) lo[a]--;
        for (int i3 = lo[2]; i3 <= hi[2]; i3++)
        for (int i2 = lo[1]; i2 <= hi[1]; i2++)
        for (int i1 = lo[0]; i1 <= hi[0]; i1++) {
            int i[3] = {i1, i2, i3};
            long k = IDX(g, i1, i2, i3);
            double b = g->bu[a][k];
            if (i[a] + 1 < g->ne[a] || g->periodic) {
                i[a] = (i[a] + 1) % g->ne[a];
                gr[k] += -0.5 * b * b * gb[a][k];
                gr[IDX(g, i[0], i[1], i[2])] += -0.5 * b * b * gb[a][k];
            } else {
                gr[k] += -b * b * gb[a][k];
            }
        }
    }
    long c = 0;
    for (int i3 = g->L[2]; i3 <= g->H[2]; i3++)
    for (int i2 = g->L[1]; i2 <= g->H[1]; i2++)
    for (int i1 = g->L[0]; i1 <= g->H[0]; i1++, c++) {
        long k = IDX(g, i1, i2, i3);
        out_rho[c] = vp[c] * vp[c] * acc[k] + gr[k];
    }
    free(gr);
    return ORC_OK;
}

/* FWI misfit + gradient (mode 0) or RTM image (mode 1) of one shot
 * (Algorithm 2).
 *   mode 0: residual r = u - d, misfit J = 1/2 sum r^2 (Eq. objfwi, read with
 *           the time integral as a plain sum over samples); out = dJ/dVp on
 *           the physical grid = 2 rho Vp dJ/dkappa, where dJ/dkappa =
 *           -dt sum_it pbar(it) (div v^{it+1/2}) is the exact gradient of the
 *           discrete J (Eq. gradrhokappa), with the layer model held fixed.
 *   mode 1: the adjoint source is the observed data (Sec. 2.3); out =
 *           sum_it kappa pbar(it) p^{it+1}, the zero-lag cross-correlation of
 *           the receiver field kappa*pbar (which obeys the forward equations,
 *           Eq. adj) with the source field at the same time level
 *           (Eq. rtmimage).
 *   mode 2: the image of mode 1 divided by the shot's source illumination
 *           sum_it (p^{it+1})^2 + eps, eps = 1e-3 max_x of the illumination
 *           (the normalised imaging condition of Sec. 2.3; eps is a
 *           reading).
 * pbar(it) is the adjoint of p^{it+1} after the receivers of step it have
 * been injected.  recon = 1 rebuilds the source field backwards from the
 * saved boundary bands (Sec. 4.2, every dr-th step, interpolated in time
 * when dr > 1); recon = 0 keeps every forward
 * state in memory (small grids only; tests).  The adjoint field uses the
 * receiver box when use_box is set (Sec. 4.1).
 * seis (optional): the forward seismograms [nt][nrec].
 * out_rho (optional, mode 0): dJ/drho at fixed Vp on the physical grid (see
 * accumulate_gb).
 * phase_s (optional, [4]): wall-clock seconds of the forward time loop after
 * its first step, of the reverse time loop after its first step, of the
 * forward loop's first step and of the reverse loop's first step (the first
 * steps touch the freshly allocated fields); set-up and the final output pass
 * are excluded. */
int orc_gradient(const orc_par *par, const double *vp, const double *rho, const double *stf,
                 const double *src, int nrec, const double *rec, const double *dobs,
                 int mode, int recon, double *misfit, double *out, double *seis_out, double *out_rho,
                 double *phase_s)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    if (recon && par->nb < g.N) { grid_free(&g); return ORC_ERR_ARG; }
    stencil_t sst, *rst = calloc(nrec > 0 ? nrec : 1, sizeof(stencil_t));
    double *seis = malloc(sizeof(double) * ((long)g.nt * nrec + 1));
    double *acc = calloc(g.ntot, sizeof(double));
    double *ill = mode == 2 ? calloc(g.ntot, sizeof(double)) : NULL;
    const int want_rho = out_rho && mode == 0;
    double *gb[3] = {0}, *vsave[3] = {0};
    int nomem = !rst || !seis || !acc || (mode == 2 && !ill);
    for (int a = 0; a < g.ndim && want_rho; a++) {
        gb[a] = calloc(g.ntot, sizeof(double));
        vsave[a] = malloc(sizeof(double) * g.ntot);
        nomem |= !gb[a] || !vsave[a];
    }
    if (nomem) {
        free(rst); free(seis); free(acc); free(ill);
        for (int a = 0; a < 3; a++) { free(gb[a]); free(vsave[a]); }
        grid_free(&g);
        return ORC_ERR_NOMEM;
    }
    rc = point_stencil(&g, src, par->kaiser_b, &sst);
    for (int r = 0; r < nrec && !rc; r++) rc = point_stencil(&g, rec + 3 * r, par->kaiser_b, &rst[r]);
    state_t s, ad;
    memset(&s, 0, sizeof s);
    memset(&ad, 0, sizeof ad);
    if (!rc) rc = state_alloc(&g, &s);
    if (!rc) rc = state_alloc(&g, &ad);
    long nband = band_count(&g);
    const int nsamp = band_samples(&g);
    double *bands = NULL, *bandt = NULL, *store_p = NULL, *store_v[3] = {0};
    if (!rc && recon) {
        bands = malloc(sizeof(double) * (nband * (long)nsamp + 1));
        bandt = malloc(sizeof(double) * (nband + 1));
        if (!bands || !bandt) rc = ORC_ERR_NOMEM;
    }
    if (!rc && !recon) {
        store_p = malloc(sizeof(double) * g.ntot * (long)g.nt);
        if (!store_p) rc = ORC_ERR_NOMEM;
        for (int a = 0; a < g.ndim && !rc; a++) {
            store_v[a] = malloc(sizeof(double) * g.ntot * (long)g.nt);
            if (!store_v[a]) rc = ORC_ERR_NOMEM;
        }
    }
    if (rc) goto done;

    int slo[3], shi[3], rlo[3], rhi[3];
    stencil_extent(&sst, 1, slo, shi);
    stencil_extent(rst, nrec, rlo, rhi);
    /* forward loop */
    double t_fwd0 = wall_seconds(), t_fwd1 = t_fwd0;
    for (int it = 0; it < g.nt; it++) {
        if (it == 1) t_fwd1 = wall_seconds();
        if (recon && it % g.dr == 0) band_copy(&g, s.v, bands + nband * (long)(it / g.dr), 0);
        int lo[3], hi[3];
        box_at(&g, slo, shi, it, lo, hi);
        forward_step(&g, &s, lo, hi, &sst, g.dt * stf[it] / g.dV);
        for (int r = 0; r < nrec; r++) seis[(long)it * nrec + r] = stencil_get(&g, s.p, &rst[r]);
        if (!recon) {
            memcpy(store_p + g.ntot * (long)it, s.p, sizeof(double) * g.ntot);
            for (int a = 0; a < g.ndim; a++)
                memcpy(store_v[a] + g.ntot * (long)it, s.v[a], sizeof(double) * g.ntot);
        }
    }
    if (recon && (rc = forward_continue(&g, &s, slo, shi, bands, nband, nsamp))) goto done;
    if (phase_s) {
        double t = wall_seconds();
        phase_s[0] = g.nt > 1 ? t - t_fwd1 : 0.0;
        phase_s[2] = (g.nt > 1 ? t_fwd1 : t) - t_fwd0;
    }
    /* residual and misfit */
    double J = 0.0;
    for (long k = 0; k < (long)g.nt * nrec; k++) {
        double r = seis[k] - dobs[k];
        if (mode == 0) J += 0.5 * r * r;
    }
    if (misfit) *misfit = J;
    if (seis_out) memcpy(seis_out, seis, sizeof(double) * (long)g.nt * nrec);

    /* reverse loop */
    double t_rev0 = wall_seconds(), t_rev1 = t_rev0;
    for (int it = g.nt - 1; it >= 0; it--) {
        if (it == g.nt - 2) t_rev1 = wall_seconds();
        if (!recon) {
            memcpy(s.p, store_p + g.ntot * (long)it, sizeof(double) * g.ntot);
            for (int a = 0; a < g.ndim; a++)
                memcpy(s.v[a], store_v[a] + g.ntot * (long)it, sizeof(double) * g.ntot);
        }
        for (int r = 0; r < nrec; r++) {
            long k = (long)it * nrec + r;
            double src_r = (mode == 0) ? seis[k] - dobs[k] : dobs[k];
            stencil_add(&g, ad.p, &rst[r], src_r);
        }
        fs_fold_p(&g, ad.p);
        int box[2][3], prev[2][3];
        box_at(&g, slo, shi, it, box[0], box[1]);
        box_at(&g, slo, shi, it - 1, prev[0], prev[1]);
        /* imaging / gradient at the physical nodes of the forward box (each node
         * writes only its own accumulators) */
#pragma omp parallel for collapse(2) schedule(static)
        for (int i3 = g.L[2]; i3 <= g.H[2]; i3++)
        for (int i2 = g.L[1]; i2 <= g.H[1]; i2++)
        for (int i1 = g.L[0]; i1 <= g.H[0]; i1++) {
            int i[3] = {i1, i2, i3};
            if (!in_box(i, box[0], box[1])) continue;
            long k = IDX(&g, i1, i2, i3);
            if (mode == 0) {
                double div = 0.0;
                for (int a = 0; a < g.ndim; a++) div += deriv_v(&g, s.v[a], a, i);
                acc[k] += -g.dt * ad.p[k] * div;
            } else {
                acc[k] += g.K[k] * ad.p[k] * s.p[k];
                if (mode == 2) ill[k] += s.p[k] * s.p[k];
            }
        }
        int lo[3], hi[3];
        if (g.use_box) box_at(&g, rlo, rhi, g.nt - 1 - it, lo, hi);
        else full_box(&g, lo, hi);
        adjoint_step(&g, &ad, lo, hi);
        if (want_rho)
            for (int a = 0; a < g.ndim; a++) memcpy(vsave[a], s.v[a], sizeof(double) * g.ntot);
        if (recon) {
            band_at(&g, bands, nband, nsamp, it, bandt);
            reconstruct_step(&g, &s, &sst, g.dt * stf[it] / g.dV, box, prev, bandt);
            if (want_rho) accumulate_gb(&g, &ad, vsave, s.v, gb);
        } else if (want_rho) {
            double *vold[3] = {0};
            for (int a = 0; a < g.ndim; a++) vold[a] = it > 0 ? store_v[a] + g.ntot * (long)(it - 1) : NULL;
            accumulate_gb(&g, &ad, vsave, it > 0 ? vold : NULL, gb);
        }
    }
    if (phase_s) {
        double t = wall_seconds();
        phase_s[1] = g.nt > 1 ? t - t_rev1 : 0.0;
        phase_s[3] = (g.nt > 1 ? t_rev1 : t) - t_rev0;
    }
    if (want_rho && (rc = finish_rho(&g, vp, acc, gb, out_rho))) goto done;
    {
        double eps = 0.0;
        if (mode == 2) {
            for (long k = 0; k < g.ntot; k++) if (ill[k] > eps) eps = ill[k];
            eps *= 1e-3;
        }
        long c = 0;
        for (int i3 = g.L[2]; i3 <= g.H[2]; i3++)
        for (int i2 = g.L[1]; i2 <= g.H[1]; i2++)
        for (int i1 = g.L[0]; i1 <= g.H[0]; i1++, c++) {
            long k = IDX(&g, i1, i2, i3);
            if (mode == 2) {
                out[c] = acc[k] / (ill[k] + eps);
            } else if (mode == 0) {
                /* dJ/dVp = dJ/dkappa * dkappa/dVp = dJ/dkappa * 2 rho Vp */
                out[c] = acc[k] * 2.0 * rho[c] * vp[c];
            } else {
                out[c] = acc[k];
            }
        }
    }
done:
    state_free(&s);
    state_free(&ad);
    free(bands);
    free(bandt);
    free(store_p);
    for (int a = 0; a < 3; a++) { free(store_v[a]); free(gb[a]); free(vsave[a]); }
    free(acc);
    free(ill);
    free(seis);
    free(rst);
    grid_free(&g);
    return rc;
}

/* Source-field reconstruction alone (tests): forward run saving the bands,
 * then the reverse loop of Algorithm 2 restricted to the source field.
 * prec: [nt][nphys], prec[it] = reconstructed p^{it} on the physical grid. */
int orc_reconstruct(const orc_par *par, const double *vp, const double *rho, const double *stf,
                    const double *src, double *prec)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    if (par->nb < g.N) { grid_free(&g); return ORC_ERR_ARG; }
    stencil_t sst;
    rc = point_stencil(&g, src, par->kaiser_b, &sst);
    state_t s;
    memset(&s, 0, sizeof s);
    if (!rc) rc = state_alloc(&g, &s);
    long nband = band_count(&g);
    const int nsamp = band_samples(&g);
    double *bands = rc ? NULL : malloc(sizeof(double) * (nband * (long)nsamp + 1));
    double *bandt = rc ? NULL : malloc(sizeof(double) * (nband + 1));
    if (!rc && (!bands || !bandt)) rc = ORC_ERR_NOMEM;
    int slo[3], shi[3];
    stencil_extent(&sst, 1, slo, shi);
    for (int it = 0; it < g.nt && !rc; it++) {
        if (it % g.dr == 0) band_copy(&g, s.v, bands + nband * (long)(it / g.dr), 0);
        int lo[3], hi[3];
        box_at(&g, slo, shi, it, lo, hi);
        forward_step(&g, &s, lo, hi, &sst, g.dt * stf[it] / g.dV);
    }
    if (!rc) rc = forward_continue(&g, &s, slo, shi, bands, nband, nsamp);
    if (rc) { free(bands); free(bandt); state_free(&s); grid_free(&g); return rc; }
    long nphys = (long)(g.H[0] - g.L[0] + 1) * (g.H[1] - g.L[1] + 1) * (g.H[2] - g.L[2] + 1);
    for (int it = g.nt - 1; it >= 0; it--) {
        int box[2][3], prev[2][3];
        box_at(&g, slo, shi, it, box[0], box[1]);
        box_at(&g, slo, shi, it - 1, prev[0], prev[1]);
        band_at(&g, bands, nband, nsamp, it, bandt);
        reconstruct_step(&g, &s, &sst, g.dt * stf[it] / g.dV, box, prev, bandt);
        long c = 0;
        for (int i3 = g.L[2]; i3 <= g.H[2]; i3++)
        for (int i2 = g.L[1]; i2 <= g.H[1]; i2++)
        for (int i1 = g.L[0]; i1 <= g.H[0]; i1++)
            prec[(long)it * nphys + c++] = s.p[IDX(&g, i1, i2, i3)];
    }
    free(bands);
    free(bandt);
    state_free(&s);
    grid_free(&g);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Small accessors for tests. */

/* Validation only: 0 or the error grid_init reports (CFL, dispersion, ...). */
int orc_check(const orc_par *par, const double *vp, const double *rho)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (!rc) grid_free(&g);
    return rc;
}

/* CPML a/b along one axis on the p grid (vgrid = 0) or v grid (vgrid = 1). */
int orc_cpml_profile(const orc_par *par, const double *vp, const double *rho, int axis,
                     int vgrid, double *pa, double *pb)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    if (axis < 0 || axis >= g.ndim) { grid_free(&g); return ORC_ERR_ARG; }
    memcpy(pa, vgrid ? g.cva[axis] : g.cpa[axis], sizeof(double) * g.ne[axis]);
    memcpy(pb, vgrid ? g.cvb[axis] : g.cpb[axis], sizeof(double) * g.ne[axis]);
    grid_free(&g);
    return ORC_OK;
}

/* Box bounds for steps n = n0..n0+count-1 around the stencils of npts points
 * (source: 1 point; adjoint: all receivers).  lo/hi: [count][3]. */
int orc_box_table(const orc_par *par, const double *vp, const double *rho, int npts,
                  const double *pts, int n0, int count, int *lo, int *hi)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    stencil_t *st = calloc(npts > 0 ? npts : 1, sizeof(stencil_t));
    if (!st || npts < 1) { free(st); grid_free(&g); return ORC_ERR_ARG; }
    for (int k = 0; k < npts && !rc; k++) rc = point_stencil(&g, pts + 3 * k, par->kaiser_b, &st[k]);
    if (!rc) {
        int slo[3], shi[3];
        stencil_extent(st, npts, slo, shi);
        for (int c = 0; c < count; c++) box_at(&g, slo, shi, n0 + c, lo + 3 * c, hi + 3 * c);
    }
    free(st);
    grid_free(&g);
    return rc;
}

/* Number of values saved per step by the boundary bands. */
long orc_band_count(const orc_par *par, const double *vp, const double *rho)
{
    grid_t g;
    int rc = grid_init(&g, par, vp, rho);
    if (rc) return rc;
    long c = band_count(&g);
    grid_free(&g);
    return c;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return default_threads();
#else
    return 1;
#endif
}
