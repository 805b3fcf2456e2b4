// smi_setup.cpp -- host-side set-up of libsmi in FP64: FD coefficients,
// stability and dispersion checks, CPML tables and Kaiser-sinc stencils.
// Results are rounded to FP32 tables for the kernels.
#include <cmath>
#include <algorithm>

#include "smi_internal.h"

namespace smi {

// Staggered-grid coefficients (Sec. 2.1; the paper refers to Fornberg).  The
// derivative sum_m a_m (f(x+(2m-1)h/2) - f(x-(2m-1)h/2))/h is the derivative
// at x of the polynomial interpolating f at the 2N half nodes; writing that
// interpolant in Lagrange form gives the closed product
//   a_m = (-1)^{m+1} / (2m-1) * prod_{n != m} (2n-1)^2 / |(2m-1)^2 - (2n-1)^2|.
void fd_coefficients(int N, double *a)
{
    for (int m = 1; m <= N; m++) {
        double om = 2.0 * m - 1.0;
        double prod = 1.0;
        for (int n = 1; n <= N; n++) {
            if (n == m) continue;
            double on = 2.0 * n - 1.0;
            prod *= (on * on) / std::fabs(om * om - on * on);
        }
        a[m - 1] = ((m % 2) ? 1.0 : -1.0) / om * prod;
    }
}

// Eq. cfl: dt vmax sqrt(sum_a 1/h_a^2) sum_l |a_l|.
double cfl_number(int ndim, const double *h, double dt, double vmax, int N)
{
    double a[kMaxHalf];
    fd_coefficients(N, a);
    double sum_a = 0.0, inv2 = 0.0;
    for (int l = 0; l < N; l++) sum_a += std::fabs(a[l]);
    for (int k = 0; k < ndim; k++) inv2 += 1.0 / (h[k] * h[k]);
    return dt * vmax * std::sqrt(inv2) * sum_a;
}

// Sec. 3.8 asks for "sufficient points per wavelength"; the shortest
// wavelength is taken as vmin / (2.5 fm) (a Ricker wavelet's band ends near
// 2.5 fm) over the coarsest spacing.
double points_per_wavelength(int ndim, const double *h, double vmin, double fm)
{
    double hmax = 0.0;
    for (int k = 0; k < ndim; k++) hmax = std::max(hmax, h[k]);
    return vmin / (2.5 * fm) / hmax;
}

// CPML after Komatitsch & Martin (2007) with kappa = 1: along a layer of
// thickness Lp = nb*h, at distance x (clamped to Lp) from the outermost
// physical node, d = d0 (x/Lp)^2 with d0 = -3 vmax ln(R) / (2 Lp) and
// alpha = pi fm (1 - x/Lp); b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha).
// Nodes of the physical domain (and any node with d = 0) get a = b = 0.
void cpml_tables(int ne, int nb, double h, double vmax, double fm, double R, double dt,
                 bool vgrid, float *a, float *b)
{
    const int first = nb, last = ne - nb - 1;       // physical nodes
    const double Lp = nb * h;
    const double d0 = (nb > 0 && R < 1.0) ? -3.0 * vmax * std::log(R) / (2.0 * Lp) : 0.0;
    for (int j = 0; j < ne; j++) {
        const double x = vgrid ? j + 0.5 : (double)j;
        double depth = 0.0;                          // cells into the layer
        if (x < first) depth = first - x;
        if (x > last) depth = x - last;
        a[j] = 0.0f;
        b[j] = 0.0f;
        if (depth <= 0.0 || d0 <= 0.0) continue;
        const double xr = std::min(depth * h, Lp) / Lp;
        const double damp = d0 * xr * xr;
        const double alpha = M_PI * fm * (1.0 - xr);
        const double bb = std::exp(-(damp + alpha) * dt);
        b[j] = (float)bb;
        a[j] = (float)(damp * (bb - 1.0) / (damp + alpha));
    }
}

// Kaiser-windowed sinc (Hicks 2002, cited in Sec. 2.1) of radius ri = order/2
// (Sec. 3.8).  Window I0(b sqrt(1 - (x/ri)^2)) / I0(b), sinc(x) =
// sin(pi x)/(pi x).  A position within 1e-6 cells of a node is that node
// (weight 1; sinc vanishes on every other node).  The nominal extent of a
// stencil, used by the computing box, is base-ri+1 .. base+ri with base the
// node (on a node) or floor(x) (off the nodes).
bool make_stencil(const Grid &g, const double pos[3], double kaiser_b, Stencil *st)
{
    const double i0b = std::cyl_bessel_i(0.0, kaiser_b);
    for (int ax = 0; ax < 3; ax++) {
        for (int k = 0; k < kMaxTaps; k++) st->w[ax][k] = 0.0f;
        if (ax >= g.ndim) {
            st->first[ax] = 0;
            st->cnt[ax] = 1;
            st->w[ax][0] = 1.0f;
            continue;
        }
        const double rel = pos[ax] / g.h[ax];        // physical grid units
        const int nphys = g.H[ax] - g.L[ax] + 1;
        if (!(rel >= -1e-6 && rel <= nphys - 1 + 1e-6)) return false;
        const double x = rel + g.nb;
        const double nearest = std::nearbyint(x);
        const bool on_node = std::fabs(x - nearest) <= 1e-6;
        const int base = on_node ? (int)nearest : (int)std::floor(x);
        // the nominal 2*ri-node stencil must fit in the extended grid
        if (base - g.ri + 1 < 0 || base + g.ri > g.ne[ax] - 1) return false;
        // free surface on the top face (image-source form of Hicks 2002): a
        // weight above the surface node L folds, negated, onto its mirror
        // node 2L - i, and the weight at L is dropped (p = 0 there)
        const bool fold = ax == 0 && g.freesurf;
        if (on_node) {
            st->first[ax] = base;
            st->cnt[ax] = 1;
            st->w[ax][0] = (fold && base == g.L[0]) ? 0.0f : 1.0f;
        } else {
            st->first[ax] = base - g.ri + 1;
            st->cnt[ax] = 2 * g.ri;
            double wd[kMaxTaps] = {0};
            for (int k = 0; k < 2 * g.ri; k++) {
                const double u = (st->first[ax] + k) - x;
                const double sinc = std::sin(M_PI * u) / (M_PI * u);
                const double q = u / g.ri;
                const double arg = 1.0 - q * q;
                const double win = arg > 0.0 ? std::cyl_bessel_i(0.0, kaiser_b * std::sqrt(arg)) / i0b : 0.0;
                wd[k] = sinc * win;
            }
            if (fold) {
                for (int k = 0; k < 2 * g.ri; k++) {
                    const int node = st->first[ax] + k;
                    if (node >= g.L[0]) continue;
                    const int km = 2 * g.L[0] - node - st->first[ax];
                    if (km >= 2 * g.ri) return false;
                    wd[km] -= wd[k];
                    wd[k] = 0.0;
                }
                const int k0 = g.L[0] - st->first[ax];
                if (k0 >= 0 && k0 < 2 * g.ri) wd[k0] = 0.0;
            }
            for (int k = 0; k < 2 * g.ri; k++) st->w[ax][k] = (float)wd[k];
        }
    }
    return true;
}

TimeWeights time_weights(int it, int dr, int nsamp)
{
    TimeWeights tw{};
    tw.nsamp = nsamp;
    if (it % dr == 0) {                 // on a stored sample: that sample alone
        tw.first = it / dr;
        tw.w[0] = 1.0f;
        return tw;
    }
    const double x = (double)it / (double)dr;
    const int base = (int)std::floor(x);
    tw.first = base - kTimeR + 1;
    const double i0b = std::cyl_bessel_i(0.0, kTimeB);
    for (int q = 0; q < 2 * kTimeR; q++) {
        const double u = (tw.first + q) - x;
        const double sinc = std::sin(M_PI * u) / (M_PI * u);
        const double r = u / kTimeR;
        const double arg = 1.0 - r * r;
        const double win = arg > 0.0 ? std::cyl_bessel_i(0.0, kTimeB * std::sqrt(arg)) / i0b : 0.0;
        tw.w[q] = (float)(sinc * win);
    }
    return tw;
}

void set_layout(Grid &g, const int n[3])
{
    g.px = (g.ne[0] + 7) / 8 * 8;
    g.ntot = (long long)g.px * g.ne[1] * g.ne[2];
    g.nphys = (long long)n[0] * n[1] * n[2];
    g.S = 2 * g.nb + 1;
    // slab arrays compress their axis to S; the y slab (3D) keeps the padded
    // row pitch px so that 4 consecutive z nodes form an aligned float4
    g.slab_n[0] = (long long)g.S * g.ne[1] * g.ne[2];
    g.slab_n[1] = (long long)g.ne[0] * g.S * g.ne[2];
    g.slab_n[2] = g.ndim == 3 ? (long long)g.px * g.ne[1] * g.S : 0;
}

}  // namespace smi
